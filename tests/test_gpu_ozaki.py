"""The split-precision tensor-core product (tcgen05, bf16 digit slices).

* one digit per operand on integer inputs |x| <= 63 reproduces the exact
  integer product (shared-memory descriptors, TMEM layout, exact f32 group
  sums up to K = 640);
* with k digits the error obeys the truncation bound
  |C - AB| <= K * 2^(ea + eb) * c * 2^(-7k) elementwise (ea, eb row scales)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (200, 100, 640), (77, 13, 45), (300, 190, 96)])
def test_integer_product_exact(M, N, K):
    import paper_2009_12505_gb300 as hfx
    rng = np.random.default_rng(M * 1000 + N + K)
    A = rng.integers(-63, 64, size=(M, K)).astype(np.float64)
    B = rng.integers(-63, 64, size=(K, N)).astype(np.float64)
    C = hfx.hfx.selftest_ozaki(A, B, 1)
    ref = (A.astype(np.int64) @ B.astype(np.int64)).astype(np.float64)
    np.testing.assert_array_equal(C, ref)


def _row_scale(X):
    m = np.abs(X).max(axis=1)
    e = np.where(m > 0, np.floor(np.log2(np.where(m > 0, m, 1))) + 2, -1000)
    return e


@pytest.mark.parametrize("k", [2, 3, 4, 5, 6])
def test_ozaki_error_bound(k):
    import paper_2009_12505_gb300 as hfx
    rng = np.random.default_rng(k)
    M, N, K = 150, 90, 600
    # rows with very different magnitudes, like V and C blocks at different distances
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-8, 2, size=(M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-8, 2, size=(1, N)))
    C = hfx.hfx.selftest_ozaki(A, B, k)
    ref = A @ B
    ea, eb = _row_scale(A), _row_scale(B.T)
    bound = K * np.ldexp(1.0, (ea[:, None] + eb[None, :] - 7 * k).astype(int)) * 4
    assert np.all(np.abs(C - ref) <= bound + 1e-300)
    if k == 6:
        rel = np.abs(C - ref).max() / np.abs(ref).max()
        assert rel < 1e-11
