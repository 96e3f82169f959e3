"""Pins for the oracle of the steps next to the build (oracle/fourier.py):
Eq. DM_realspace (density matrix from eigenvectors) and Eq. Ham_rs2kspace
(Sigma at k points), against closed forms that do not go through the
oracle's code: a one-orbital chain (Dirichlet kernel, cosine band), a
complete set of occupied orbitals (identity), the sign of each phase, and
discrete orthogonality of a full k grid."""
import numpy as np

from oracle import fourier


def _chain_k(N):
    return np.array([[j / N, 0.0, 0.0] for j in range(N)])


def test_density_of_a_filled_cosine_band_is_the_dirichlet_kernel():
    """One orbital per cell, c = 1, k_j = j / N with j in [-m, m] occupied:
    D(n) = (1/N) sum_{j=-m}^{m} e^{2 pi i j n / N}
         = sin(pi (2m + 1) n / N) / (N sin(pi n / N)),  (2m + 1) / N at n = 0."""
    N, m = 12, 3
    js = np.arange(N)
    kf = _chain_k(N)
    occ = ((js <= m) | (js >= N - m)).astype(float)[:, None]  # j = -m .. m mod N
    coef = np.ones((N, 1, 1), np.complex128)
    keys = [[0, 0, n, 0, 0] for n in range(-5, 6)]
    got = fourier.density([1], kf, coef, occ, keys)
    for (_, _, n, _, _), blk in zip(keys, got):
        ref = (2 * m + 1) / N if n == 0 else np.sin(np.pi * (2 * m + 1) * n / N) / (
            N * np.sin(np.pi * n / N))
        assert abs(blk[0, 0].real - ref) < 1e-14
        assert abs(blk[0, 0].imag) < 1e-14


def test_density_of_a_complete_occupied_set_is_the_identity():
    """Unitary C(k) with every band occupied: sum_b c c* = 1, so the diagonal
    blocks of D(0) are identities and every off-diagonal block vanishes,
    whatever the k points and n."""
    rng = np.random.default_rng(0)
    nao = [2, 3]
    nb, nk = 5, 3
    coef = np.empty((nk, nb, nb), np.complex128)
    for q in range(nk):
        a = rng.normal(size=(nb, nb)) + 1j * rng.normal(size=(nb, nb))
        coef[q], _ = np.linalg.qr(a)
    kf = rng.uniform(-0.5, 0.5, (nk, 3))
    occ = np.ones((nk, nb))
    keys = [[0, 0, 0, 0, 0], [0, 1, 0, 0, 0], [1, 1, 0, 0, 0], [1, 0, 1, 0, -1]]
    got = fourier.density(nao, kf, coef, occ, keys)
    np.testing.assert_allclose(got[0], np.eye(2), atol=1e-14)
    np.testing.assert_allclose(got[1], np.zeros((2, 3)), atol=1e-14)
    np.testing.assert_allclose(got[2], np.eye(3), atol=1e-14)
    # n != 0: (1/nk) sum_q e^{2 pi i k.n} I restricted to an off-diagonal block = 0
    np.testing.assert_allclose(got[3], np.zeros((3, 2)), atol=1e-14)


def test_density_phase_sign():
    """Key (K, L, n) joins sites (K, 0) and (L, n): e^{-i k.(R_K - R_L)} =
    e^{+2 pi i kappa.n}; at kappa = 1/4, n = 1 that is +i."""
    got = fourier.density([1], [[0.25, 0, 0]], np.ones((1, 1, 1)), [[1.0]], [[0, 0, 1, 0, 0]])
    assert abs(got[0][0, 0] - 1j) < 1e-15


def test_sigma_k_of_a_cosine_band():
    """Onsite e0 and hopping t to n = +-1: Sigma(k) = e0 + 2 t cos(2 pi kappa)."""
    e0, t = -0.7, 0.3
    kf = _chain_k(16)
    got = fourier.sigma_k([1], [[0, 0, -1, 0, 0], [0, 0, 0, 0, 0], [0, 0, 1, 0, 0]],
                          [[t], [e0], [t]], kf)
    ref = e0 + 2 * t * np.cos(2 * np.pi * kf[:, 0])
    np.testing.assert_allclose(got[:, 0, 0].real, ref, atol=1e-15)
    np.testing.assert_allclose(got[:, 0, 0].imag, 0, atol=1e-15)


def test_sigma_k_phase_sign():
    """Eq. Ham_rs2kspace uses e^{+i k.R}: one block at n = (0, 1, 0) and
    kappa = (0, 1/4, 0) gives i times the block."""
    blk = np.array([[1.0, 2.0], [3.0, 4.0]])
    got = fourier.sigma_k([2], [[0, 0, 0, 1, 0]], [blk], [[0, 0.25, 0]])
    np.testing.assert_allclose(got[0], 1j * blk, atol=1e-15)


def test_sigma_k_inverts_on_a_full_grid():
    """(1/N) sum_q e^{-2 pi i kappa_q n} Sigma(k_q) recovers Sigma(R_n) for
    |n| < N / 2 (discrete orthogonality)."""
    rng = np.random.default_rng(1)
    nao, N = [2, 1], 8
    keys, blocks = [], []
    for n in range(-2, 3):
        for I, J in ((0, 0), (0, 1), (1, 0), (1, 1)):
            keys.append([I, J, n, 0, 0])
            blocks.append(rng.normal(size=(nao[I], nao[J])))
    kf = _chain_k(N)
    sk = fourier.sigma_k(nao, keys, blocks, kf)
    off = fourier.basis_offsets(nao)
    for key, blk in zip(keys, blocks):
        I, J, n = key[0], key[1], key[2]
        back = sum(np.exp(-2j * np.pi * kf[q, 0] * n) * sk[q] for q in range(N)) / N
        np.testing.assert_allclose(back[off[I]:off[I + 1], off[J]:off[J + 1]], blk, atol=1e-13)


def test_sigma_k_is_hermitian_for_a_hermitian_lattice_sum():
    """Sigma(I, J, n) = Sigma(J, I, -n)^T makes every Sigma(k) Hermitian."""
    rng = np.random.default_rng(2)
    nao = [2, 3]
    blocks = {}
    for n in (-1, 0, 1):
        for I in range(2):
            for J in range(2):
                if (J, I, -n) in blocks:
                    blocks[(I, J, n)] = blocks[(J, I, -n)].T
                else:
                    b = rng.normal(size=(nao[I], nao[J]))
                    blocks[(I, J, n)] = b + b.T if (I == J and n == 0) else b
    assert len(blocks) == 12
    keys = [[I, J, n, 0, 0] for (I, J, n) in blocks]
    sk = fourier.sigma_k(nao, keys, list(blocks.values()), [[0.1, 0, 0], [0.37, 0, 0], [-0.2, 0, 0]])
    assert np.abs(sk).max() > 0.1
    for m in sk:
        np.testing.assert_allclose(m, m.conj().T, atol=1e-14)
