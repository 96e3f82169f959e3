"""The second workload's generators, full-range or metallic cells:
full-range Coulomb V (mu = 0, R_Q up to 50 bohr) and a metallic D whose
off-site magnitude decays polynomially (Sec. III.B).  Checked on CPU: the
envelopes are exactly the stated ones on the same random draws, the tasks
are denser than the insulating, screened baseline, and the oracle still
equals the brute-force four-centre sum on such a cell."""
import math

import numpy as np

import oracle
import refforms
import synth


def _small():
    return synth.custom("pair", 1.0, 6, [[0, 0, 0], [2, 1, 1]], [2, 3], [3, 4])


def test_metallic_d_envelope_on_the_same_draws():
    s = _small()
    ins = synth.gen_D(s, 7.0, seed=3)
    met = synth.gen_D(s, 7.0, seed=3, decay="power")
    assert ins.keys() == met.keys()
    for (i, j, *n), blk in ins.items():
        d = math.sqrt(float(np.sum((s.grid[j] + np.array(n) * s.period - s.grid[i]) ** 2)))
        if d == 0.0:
            np.testing.assert_array_equal(met[(i, j, *n)], blk)
        else:
            ratio = (1.0 + d / 3.0) ** -2 / math.exp(-d / 3.0)
            np.testing.assert_allclose(met[(i, j, *n)], blk * ratio, rtol=1e-14)


def test_full_range_v_is_bare_coulomb_on_the_same_draws():
    s = _small()
    scr = synth.gen_V(s, 9.0, seed=4)
    full = synth.gen_V(s, 9.0, seed=4, mu=0.0)
    for (i, j, *n), blk in scr.items():
        d = math.sqrt(float(np.sum((s.grid[j] + np.array(n) * s.period - s.grid[i]) ** 2)))
        if d == 0.0:
            np.testing.assert_array_equal(full[(i, j, *n)], blk)
        else:
            np.testing.assert_allclose(full[(i, j, *n)], blk / math.erfc(0.11 * d), rtol=1e-13)


def _survivors(wl, theta):
    _, counts = oracle.Oracle.of(wl).keys(theta)
    return int(counts.sum())


def test_second_workload_has_denser_tasks():
    """At the same theta, a metallic D and a full-range V leave more terms
    than the insulating, screened cell with the same cutoffs."""
    cell = synth.si_diamond(1, nao=4, nabf=6)
    base = synth.make_workload(cell, 6.0, 10.0, 10.0, seed=7)
    metal = synth.make_workload(cell, 6.0, 10.0, 10.0, seed=7, d_decay="power")
    full = synth.make_workload(cell, 6.0, 10.0, 10.0, seed=7, mu=0.0)
    theta = 1e-4
    n0 = _survivors(base, theta)
    assert _survivors(metal, theta) > n0
    assert _survivors(full, theta) > n0


def test_oracle_equals_brute_force_on_a_metallic_full_range_cell():
    s = _small()
    wl = synth.make_workload(s, 3.5, 5.5, 5.0, seed=8, mu=0.0, d_decay="power")
    res = oracle.Oracle.of(wl).build(0.0)
    sig = oracle.block_dict(res["keys"], res["data"], res["offs"], wl.system.nao)
    scale = max(np.abs(v).max() for v in sig.values())
    assert scale > 0.01
    for k, v in sig.items():
        b = refforms.brute_sigma(wl, k[0], (k[1], tuple(k[2:])))
        assert np.abs(b - v).max() <= 1e-12 * scale, k
