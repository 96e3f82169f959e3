"""GPU parity for the steps next to the build, against oracle/fourier.py:
the density matrix from eigenvectors (Eq. DM_realspace) and Sigma at k
points (Eq. Ham_rs2kspace), both through the C ABI."""
import numpy as np
import pytest

import oracle
import synth
from oracle import fourier
from paper_2009_12505_gb300 import hfx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _eigvecs(nb, nbands, kf, symmetric, seed):
    """Random coefficients; with symmetric k sets (k, -k) C(-k) = conj C(k) and
    equal occupations, so D is real."""
    rng = np.random.default_rng(seed)
    nk = len(kf)
    coef = rng.normal(size=(nk, nb, nbands)) + 1j * rng.normal(size=(nk, nb, nbands))
    occ = rng.uniform(0, 2, (nk, nbands))
    if symmetric:
        for q in range(1, nk, 2):
            coef[q] = np.conj(coef[q - 1])
            occ[q] = occ[q - 1]
    return coef, occ


def _keys(natoms, count, seed):
    rng = np.random.default_rng(seed)
    ks = {(int(rng.integers(natoms)), int(rng.integers(natoms)), *map(int, rng.integers(-2, 3, 3)))
          for _ in range(count)}
    return np.array(sorted(ks), np.int32)


@pytest.mark.parametrize("symmetric", [True, False])
def test_density_matches_oracle(symmetric):
    nao, nabf = [3, 5, 2, 4], [4, 4, 4, 4]
    kf = np.array([[0.1, 0.2, 0.0], [-0.1, -0.2, 0.0], [0.3, 0.0, 0.25], [-0.3, 0.0, -0.25],
                   [0.45, -0.15, 0.05], [-0.45, 0.15, -0.05]])
    coef, occ = _eigvecs(sum(nao), 9, kf, symmetric, seed=3)
    keys = _keys(len(nao), 40, seed=4)
    ctx = hfx.Context(nao, nabf)
    got, maxim = ctx.density_from_eigvecs(kf, coef, occ, keys)
    ref = fourier.density(nao, kf, coef, occ, keys)
    flat = np.concatenate([b.ravel() for b in ref])
    scale = np.abs(flat).max()
    assert got.shape == flat.shape
    np.testing.assert_allclose(got, flat.real, rtol=0, atol=1e-13 * scale)
    im = np.abs(flat.imag).max()
    assert abs(maxim - im) <= 1e-13 * scale
    if symmetric:
        assert im <= 1e-13 * scale


def test_sigma_k_matches_oracle_after_a_build():
    wl = synth.si_shrunk()
    theta = 1e-2
    nao = wl.system.nao
    ctx = hfx.Context(nao, wl.system.nabf)
    for k in "CVD":
        ctx.set_blocks(k, getattr(wl, k))
    ctx.build(theta, "fp64")
    orc = oracle.Oracle.of(wl).build(theta)
    blocks = [orc["data"][orc["offs"][e]:orc["offs"][e + 1]] for e in range(len(orc["keys"]))]
    kf = np.array([[0.0, 0.0, 0.0], [0.25, 0.0, 0.0], [0.1, -0.3, 0.2], [0.5, 0.5, 0.5]])
    got = ctx.sigma_k(kf)
    ref = fourier.sigma_k(nao, orc["keys"], blocks, kf)
    scale = np.abs(ref).max()
    assert scale > 1.0
    # FP64 end to end: 1e-10 of the largest element
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * scale)
    for m in got:   # Sigma(I, J, n) = Sigma(J, I, -n)^T
        np.testing.assert_allclose(m, m.conj().T, rtol=0, atol=1e-10 * scale)


def test_errors():
    ctx = hfx.Context([2, 3], [4, 4])
    with pytest.raises(hfx.HfxError) as e:
        ctx.sigma_k([[0.0, 0.0, 0.0]])
    assert e.value.status == 3  # HFX_E_STATE: no build yet
    coef = np.ones((1, 5, 1), np.complex128)
    with pytest.raises(hfx.HfxError) as e:
        ctx.density_from_eigvecs([[0, 0, 0]], coef, [[1.0]], [[0, 2, 0, 0, 0]])
    assert e.value.status == 1  # HFX_E_ARG: atom 2 does not exist
