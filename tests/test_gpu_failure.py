"""Failure detection on the GPU without a fault: a bounded device wait that
nothing satisfies expires, the kernel reports HFX_E_TIMEOUT through its error
word and returns, and the CUDA context stays usable for a normal build."""
import numpy as np
import pytest

import oracle
import synth
from gpu_common import compare_full, gpu_build
from paper_2009_12505_gb300 import hfx

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HFX_E_TIMEOUT = 6


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("limit", [1000, 2_000_000])
def test_bounded_wait_expires(limit):
    rc, waited = hfx.selftest_timeout(limit)
    assert rc == HFX_E_TIMEOUT
    # the wait gave up after about `limit` clocks, not before
    assert limit <= waited < limit + 1_000_000


def test_bad_limit_rejected():
    rc, _ = hfx.selftest_timeout(0)
    assert rc == 1  # HFX_E_ARG


def test_context_usable_after_expiry():
    rc, _ = hfx.selftest_timeout(10_000)
    assert rc == HFX_E_TIMEOUT
    wl = synth.si_shrunk()
    ref = oracle.Oracle.of(wl).build(1e-2)
    for prec, tol in (("fp64", 1e-10), ("ozaki", 1e-8)):
        _, g = gpu_build(wl, 1e-2, prec, 6 if prec == "ozaki" else 0)
        compare_full(wl, 1e-2, g, ref, tol)
    assert np.isfinite(g["ex"])
