"""Host-side helpers of the benchmark: the k_zc traffic guard, the clock
sampler's parsing of nvidia-smi records, and the named workloads."""
import os

import numpy as np

import bench


def test_traffic_follows_the_captured_source_only(monkeypatch):
    src = os.path.join(bench.ROOT, "paper_2009_12505_gb300", "csrc", "hfx_zc.cu")
    monkeypatch.setattr(bench, "ZC_CAPTURED_SHA", bench.source_digest(src))
    t = bench.zc_traffic(1e12)
    assert t == bench.ZC_BYTES_PER_TENSOR_FLOP * 1e12
    monkeypatch.setattr(bench, "ZC_CAPTURED_SHA", "0000000000000000")
    assert bench.zc_traffic(1e12) is None


def test_source_digest_ignores_comments_only(tmp_path):
    base = "int f(int x) {\n  return x + 1;\n}\n"
    a, b, c = tmp_path / "a.cu", tmp_path / "b.cu", tmp_path / "c.cu"
    a.write_text(base)
    b.write_text("// a comment\n" + base.replace("x + 1;", "x + 1;  /* note */") + "\n\n")
    c.write_text(base.replace("x + 1", "x + 2"))
    assert bench.source_digest(str(a)) == bench.source_digest(str(b))
    assert bench.source_digest(str(a)) != bench.source_digest(str(c))


def test_sample_atoms_and_term_total():
    assert bench.sample_atoms(8) == list(range(8))
    a = bench.sample_atoms(512)
    assert len(a) == 8 and a[0] == 0 and max(a) < 512 and len(set(a)) == 8

    class Fake:   # every atom: 3 + 2 + 1 + 0 surviving terms
        def keys(self, theta, atoms=None):
            return None, np.array([3, 2, 1, 0])
    tot, atoms = bench.oracle_term_total(Fake(), 512, 1e-6)
    assert tot == 6 * 512 and atoms == a


def test_clock_summary_median_max_and_reasons(tmp_path):
    c = bench.ClockSampler(0)
    c.path = os.path.join(tmp_path, "clocks.csv")
    c.proc = object()  # as if sampling had run
    rows = [
        "0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "garbage line",
    ]
    with open(c.path, "w") as f:
        f.write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"] and s["samples"] == 3


def test_named_workloads():
    assert set(bench.WORKLOADS) >= {"si8", "si64", "si8_fullrange", "si8_metal"}
    metal = bench.workload("si8_metal", 0)
    full = bench.workload("si8_fullrange", 0)
    assert metal.cut_D == 24.0 and full.cut_V == 50.0
    assert "metallic D" in bench.workload_desc(metal)
    assert "full-range Coulomb V" in bench.workload_desc(full)
    # ranks draw different cells of the same shape (weak scaling)
    a, b = bench.workload("si8", 0), bench.workload("si8", 1)
    assert a.seed != b.seed
    np.testing.assert_array_equal(a.C.keys, b.C.keys)
    assert not np.array_equal(a.C.data, b.C.data)
