"""The adjoint hfx_grad (dE_X/dC, dE_X/dV with the surviving-term set of the
build frozen) against central finite differences of the CPU oracle with the
same frozen screen, plus the Euler identities of the frozen-screen energy:
E is linear in V and quadratic in C, so sum dV.V = E and sum dC.C = 2E."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def tiny3():
    s = synth.custom("tiny3", 1.0, 5, [[0, 0, 0], [2, 1, 0], [1, 3, 2]], [2, 4, 3], [3, 5, 2])
    return synth.make_workload(s, 3.2, 4.2, 3.0, seed=6)


def gpu_grad(wl, theta, prec="fp64"):
    import paper_2009_12505_gb300 as hfx
    c = hfx.Context(wl.system.nao, wl.system.nabf)
    for k in "CVD":
        c.set_blocks(k, getattr(wl, k))
    ex = c.build(theta, prec)
    dC, dV = c.grad(wl.C.data.size, wl.V.data.size)
    return ex, dC, dV


def oracle_fd(wl, theta, which, idx, h):
    o0 = oracle.Oracle.of(wl)
    norms = {k: o0.maxabs(k) for k in "CVD"}
    vals = []
    for sgn in (1, -1):
        b = getattr(wl, which)
        d = b.data.copy()
        d[idx] += sgn * h
        parts = {k: getattr(wl, k) for k in "CVD"}
        parts[which] = synth.Blocks(b.keys, d, b.offs)
        o = oracle.Oracle(wl.system.nao, wl.system.nabf, parts["C"], parts["V"], parts["D"])
        for k in "CVD":
            o.set_maxabs(k, norms[k])
        vals.append(o.build(theta)["ex"])
    return (vals[0] - vals[1]) / (2 * h)


@pytest.mark.parametrize("make,theta", [(tiny3, 0.0), (tiny3, 2e-2), (synth.ab_shrunk, 1e-3)])
def test_grad_matches_finite_differences(make, theta):
    wl = make()
    ex, dC, dV = gpu_grad(wl, theta)
    rng = np.random.default_rng(5)
    n = 6 if wl.system.natoms > 3 else 12
    for which, g in (("C", dC), ("V", dV)):
        for idx in rng.choice(getattr(wl, which).data.size, n, replace=False):
            fd = oracle_fd(wl, theta, which, int(idx), 1e-3)
            assert abs(g[idx] - fd) <= 1e-8 * max(1.0, abs(fd)), (which, idx, g[idx], fd)


@pytest.mark.parametrize("make,theta", [(synth.si_shrunk, 1e-2), (synth.ab_shrunk, 1e-3)])
def test_grad_euler_identities(make, theta):
    wl = make()
    ex, dC, dV = gpu_grad(wl, theta)
    assert abs(np.dot(dV, wl.V.data) - ex) <= 1e-9 * abs(ex)
    assert abs(np.dot(dC, wl.C.data) - 2 * ex) <= 1e-9 * abs(ex)


def test_grad_deterministic():
    wl = synth.ab_shrunk()
    _, a, b = gpu_grad(wl, 1e-3)
    _, c, d = gpu_grad(wl, 1e-3)
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(b, d)


def test_grad_after_split_build_uses_its_screen():
    """The adjoint of a split-precision build differentiates the same frozen
    set of terms: it agrees with the adjoint after an FP64 build."""
    wl = synth.si_shrunk()
    _, a, b = gpu_grad(wl, 1e-2, "fp64")
    _, c, d = gpu_grad(wl, 1e-2, "ozaki")
    np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(b, d)


def test_autograd_function():
    import paper_2009_12505_gb300 as hfx
    wl = tiny3()
    ctx = hfx.Context(wl.system.nao, wl.system.nabf)
    for k in "CVD":
        ctx.set_blocks(k, getattr(wl, k))
    C = torch.tensor(wl.C.data, device="cuda", requires_grad=True)
    V = torch.tensor(wl.V.data, device="cuda", requires_grad=True)
    D = torch.tensor(wl.D.data, device="cuda")
    E = hfx.ExchangeEnergy.apply(ctx, 0.0, "fp64", 0, C, V, D)
    E.backward()
    ref = oracle.Oracle.of(wl).build(0.0)["ex"]
    assert abs(E.item() - ref) <= 1e-12 * max(1.0, abs(ref))
    _, dC, dV = gpu_grad(wl, 0.0)
    np.testing.assert_allclose(C.grad.cpu().numpy(), dC, rtol=0, atol=1e-13)
    np.testing.assert_allclose(V.grad.cpu().numpy(), dV, rtol=0, atol=1e-13)
