"""Helpers shared by the GPU parity tests."""
import numpy as np

import oracle
import paper_2009_12505_gb300 as hfx


def gpu_build(wl, theta, prec="fp64", nslices=0, ctx=None):
    c = ctx or hfx.Context(wl.system.nao, wl.system.nabf)
    if ctx is None:
        for k in "CVD":
            c.set_blocks(k, getattr(wl, k))
    ex = c.build(theta, prec, nslices)
    return c, {"keys": c.keys(), "offs": c.offsets(), "data": c.sigma(), "ex": ex,
               "stats": c.stats()}


def as_dict(res, nao):
    return oracle.block_dict(res["keys"], res["data"], res["offs"], nao)


def compare_full(wl, theta, gpu, orc_res, tol):
    """Exact key set and survivor counts; max |dSigma| <= tol; |dE_X| small."""
    np.testing.assert_array_equal(gpu["keys"], orc_res["keys"])
    np.testing.assert_array_equal(np.array(gpu["stats"]["survivors"]), orc_res["counts"])
    np.testing.assert_array_equal(gpu["offs"], orc_res["offs"])
    err = float(np.abs(gpu["data"] - orc_res["data"]).max()) if gpu["data"].size else 0.0
    assert err <= tol, err
    return err
