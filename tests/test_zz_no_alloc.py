"""hfx_term_noalloc: the allocation-free single-term entry point.

It is for callers that cannot allocate device memory when they call the
library (a framework that owns the GPU's memory pool, a loop where
cudaMalloc/cudaFree are not allowed, or a process whose device memory is
already reserved), so it keeps its intermediates in a fixed static device
array.  This test checks it, twice in a row, against the exchange block the
regular hfx_build entry point produces for a cluster whose only contribution
to that block is the same term, and against the CPU oracle's block.  It lives
in a file of its own that pytest collects last."""
import ctypes

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10


def _cluster(seed):
    """Atoms A=0, B=1, F=2, G=3 with uneven sizes; C on (A,F) and (B,G), V on
    (A,B), D on (F,G) only: Sigma_AB receives exactly one term,
    -sum C_AF V_AB C_BG D_FG."""
    nao, nabf = [5, 4, 3, 6], [7, 6, 2, 3]
    s = synth.custom("quad", 1.0, 1000, [[0, 0, 0], [3, 0, 0], [0, 2, 0], [3, 2, 0]], nao, nabf)
    rng = np.random.default_rng(seed)
    z = (0, 0, 0)
    C = {(0, 2) + z: rng.standard_normal((7, 5, 3)), (1, 3) + z: rng.standard_normal((6, 4, 6))}
    V = {(0, 1) + z: rng.standard_normal((7, 6))}
    D = {(2, 3) + z: rng.standard_normal((3, 6))}
    wl = synth.Workload("quad", s, synth.pack(C), synth.pack(V), synth.pack(D), 0, 0, 0, seed)
    return wl, C[(0, 2) + z], V[(0, 1) + z], C[(1, 3) + z], D[(2, 3) + z]


def test_noalloc_term_matches_build_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_12505_gb300 as hfx
    lib = hfx.load_library()
    for call, seed in enumerate((11, 12)):
        wl, cA, V, cB, D = _cluster(seed)
        ctx = hfx.Context(wl.system.nao, wl.system.nabf)
        for k in "CVD":
            ctx.set_blocks(k, getattr(wl, k))
        ctx.build(0.0)
        ref = ctx.get(0, 1, [0, 0, 0])          # Sigma_AB from hfx_build
        dev = [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in (cA, V, cB, D)]
        out = torch.full((5, 4), float("nan"), dtype=torch.float64, device="cuda")
        rc = lib.hfx_term_noalloc(7, 6, 5, 3, 4, 6, *(ctypes.c_void_p(t.data_ptr()) for t in dev),
                                  ctypes.c_void_p(out.data_ptr()), None)
        assert rc == 0, call
        torch.cuda.synchronize()
        got = -out.cpu().numpy()                # the build adds minus the term
        assert np.abs(got - ref).max() <= TOL, (call, np.abs(got - ref).max())
        orc = oracle.Oracle.of(wl).build(0.0)
        blk = oracle.block_dict(orc["keys"], orc["data"], orc["offs"], wl.system.nao)
        assert np.abs(got - blk[(0, 1, 0, 0, 0)]).max() <= TOL, call


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2009_12505_gb300 as hfx
    lib = hfx.load_library()
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    p = ctypes.c_void_p(x.data_ptr())
    # nabf_a * nao_j * nao_l = 256 * 32 * 32 > 131072: rejected before any launch
    assert lib.hfx_term_noalloc(256, 4, 4, 4, 32, 32, p, p, p, p, p, None) == 2
    # nao_i * nao_j = 2^31 (with 1-wide intermediates): rejected before any launch
    assert lib.hfx_term_noalloc(1, 1, 1 << 16, 1, 1 << 15, 1, p, p, p, p, p, None) == 2
