"""Thin ctypes binding of libhfx (include/hfx.h): argument marshalling only.

Every step of the build runs in the CUDA library.  Arrays may be numpy
arrays (host) or torch CUDA tensors (device, passed by data pointer).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

HFX_FP64, HFX_BF16X3, HFX_OZAKI = 0, 1, 2
_PREC = {"fp64": HFX_FP64, "bf16x3": HFX_BF16X3, "ozaki": HFX_OZAKI}
_STATUS = {0: "HFX_OK", 1: "HFX_E_ARG", 2: "HFX_E_SHAPE", 3: "HFX_E_STATE", 4: "HFX_E_NOMEM",
           5: "HFX_E_CUDA", 6: "HFX_E_TIMEOUT", 7: "HFX_E_NOTFOUND"}

_lock = threading.Lock()
_lib = None


class HfxError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Stats(ctypes.Structure):
    _fields_ = [("version", ctypes.c_int32), ("prec", ctypes.c_int32), ("theta", ctypes.c_double),
                ("n_sigma_blocks", ctypes.c_int64), ("n_work_items", ctypes.c_int64),
                ("n_active_abg", ctypes.c_int64), ("survivors", ctypes.c_int64 * 4),
                ("canonical_flops", ctypes.c_double), ("executed_flops", ctypes.c_double),
                ("ms_screen", ctypes.c_double), ("ms_contract", ctypes.c_double),
                ("ms_reduce", ctypes.c_double), ("ms_total", ctypes.c_double),
                ("n_waves", ctypes.c_int64), ("scratch_bytes", ctypes.c_int64),
                ("kernel_ms", ctypes.c_double * 8), ("kernel_flops", ctypes.c_double * 8),
                ("n_launches", ctypes.c_int64), ("mirror", ctypes.c_int32),
                ("nslices", ctypes.c_int32), ("kernel_tensor_flops", ctypes.c_double * 8),
                ("canonical_flops_piece", ctypes.c_double * 4), ("canonical_flops_y", ctypes.c_double),
                ("kernel_unpadded_flops", ctypes.c_double * 8),
                ("zc_dt_max_over_avg", ctypes.c_double), ("eps_eri", ctypes.c_double),
                ("n_eri_removed", ctypes.c_int64)]

KERNELS = ["screen", "Y", "Dstage", "Q", "v1_DFG", "v3_DAG", "v2_DFB", "v4_DAB"]


def build_library(force: bool = False, verbose: bool = False) -> str:
    return _build.build(force=force, verbose=verbose)


def load_library():
    """Build (if stale) and load libhfx; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build()
        lib = ctypes.CDLL(path)
        P, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        S = ctypes.c_int
        sig = {
            "hfx_create": (S, [P, i32, P, P, i32, P, P, P, P]),
            "hfx_set_C": (S, [P, i32, i32, P, P]),
            "hfx_set_V": (S, [P, i32, i32, P, P]),
            "hfx_set_D": (S, [P, i32, i32, P, P]),
            "hfx_set_many": (S, [P, ctypes.c_char, i64, P, P, P, ctypes.c_int]),
            "hfx_clear": (S, [P, ctypes.c_char]),
            "hfx_build": (S, [P, f64, ctypes.c_int, i32, P]),
            "hfx_H_count": (S, [P, P]),
            "hfx_H_keys": (S, [P, P]),
            "hfx_H_offsets": (S, [P, P]),
            "hfx_get_H": (S, [P, i32, i32, P, P]),
            "hfx_get_H_all": (S, [P, P, ctypes.c_int]),
            "hfx_grad": (S, [P, P, P]),
            "hfx_stats": (S, [P, P]),
            "hfx_last_error": (ctypes.c_char_p, [P]),
            "hfx_term_noalloc": (S, [i32, i32, i32, i32, i32, i32, P, P, P, P, P, P]),
            "hfx_set_shard": (S, [P, P, i32]),
            "hfx_set_eri_screen": (S, [P, f64]),
            "hfx_get_H_fixed": (S, [P, P, ctypes.c_int]),
            "hfx_set_H_fixed": (S, [P, P, ctypes.c_int, P]),
            "hfx_selftest_ozaki": (S, [i32, i32, i32, P, P, P, i32]),
            "hfx_selftest_timeout": (S, [i64, P]),
            "hfx_probe_fp64": (S, [P, P]),
            "hfx_build_batch": (S, [P, i32, P, ctypes.c_int, i32, P]),
            "hfx_density_from_eigvecs": (S, [P, i32, P, i32, P, P, i64, P, P, P]),
            "hfx_sigma_k": (S, [P, i32, P, P]),
            "hfx_destroy": (None, [P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def selftest_ozaki(A, B, nslices: int):
    """C = A @ B (host FP64) through the split-precision tensor-core product."""
    lib = load_library()
    A = np.ascontiguousarray(A, np.float64)
    B = np.ascontiguousarray(B, np.float64)
    M, K = A.shape
    K2, N = B.shape
    assert K == K2
    C = np.zeros((M, N), np.float64)
    rc = lib.hfx_selftest_ozaki(M, N, K, _p(A), _p(B), _p(C), int(nslices))
    if rc != 0:
        raise HfxError(rc, "hfx_selftest_ozaki failed")
    return C


def build_batch(contexts, thetas, prec: str = "ozaki", nslices: int = 0):
    """hfx_build_batch over Context objects; returns the E_X of every cell."""
    lib = load_library()
    n = len(contexts)
    hs = (ctypes.c_void_p * max(n, 1))(*[c._h.value for c in contexts])
    th = np.ascontiguousarray(thetas, np.float64)
    ex = np.zeros(max(n, 1), np.float64)
    rc = lib.hfx_build_batch(hs, n, _p(th), _PREC[prec], int(nslices), _p(ex))
    if rc != 0:
        msgs = [lib.hfx_last_error(c._h).decode() for c in contexts]
        raise HfxError(rc, "; ".join(m for m in msgs if m) or "hfx_build_batch failed")
    return ex[:n]


def selftest_timeout(limit_cycles: int):
    """Run the bounded-wait expiry self-test; returns (status, cycles waited).
    HFX_E_TIMEOUT (6) is the expected status."""
    lib = load_library()
    w = ctypes.c_int64(0)
    rc = lib.hfx_selftest_timeout(int(limit_cycles), ctypes.byref(w))
    return int(rc), int(w.value)


def probe_fp64():
    """(DFMA TFLOP/s, FP64 tensor-core TFLOP/s) measured on the current device."""
    lib = load_library()
    a, b = ctypes.c_double(), ctypes.c_double()
    rc = lib.hfx_probe_fp64(ctypes.byref(a), ctypes.byref(b))
    if rc != 0:
        raise HfxError(rc, "hfx_probe_fp64 failed")
    return a.value, b.value


def term_noalloc(cA, V, cB, D, out, stream=None):
    """hfx_term_noalloc on device tensors: out[i][j] = sum cA[a][i][k] V[a][b] cB[b][j][l] D[k][l].

    cA (nabf_a, nao_i, nao_k), V (nabf_a, nabf_b), cB (nabf_b, nao_j, nao_l),
    D (nao_k, nao_l), out (nao_i, nao_j): contiguous float64 CUDA tensors."""
    lib = load_library()
    pa, ni, nk = cA.shape
    pb, nj, nl = cB.shape
    st = None if stream is None else ctypes.c_void_p(int(stream))
    rc = lib.hfx_term_noalloc(pa, pb, ni, nk, nj, nl, _p(cA), _p(V), _p(cB), _p(D), _p(out), st)
    if rc != 0:
        raise HfxError(rc, "hfx_term_noalloc failed")
    return out


class ExchangeEnergy:
    """torch.autograd.Function wrapper: E_X(C, V) with D fixed.

    ``apply(ctx, theta, prec, nslices, C, V, D)`` with C, V, D the packed
    block data (CUDA float64 tensors, key-sorted layout of ``ctx``'s keys)
    returns E_X as a 0-d tensor; backward returns dE_X/dC and dE_X/dV from
    hfx_grad with the surviving-term set of the forward build."""

    _fn = None

    @classmethod
    def apply(cls, ctx, theta, prec, nslices, C, V, D):
        import torch
        if cls._fn is None:
            class _Fn(torch.autograd.Function):
                @staticmethod
                def forward(fctx, hctx, theta_, prec_, nsl_, C_, V_, D_):
                    for k, t in (("C", C_), ("V", V_), ("D", D_)):
                        keys, offs = hctx._layout[k]
                        hctx.set_many(k, keys, t.detach().contiguous(), offs, on_device=True)
                    ex = hctx.build(theta_, prec_, nsl_)
                    fctx.hctx = hctx
                    fctx.shapes = (C_.numel(), V_.numel())
                    return torch.tensor(ex, dtype=torch.float64, device=C_.device)

                @staticmethod
                def backward(fctx, gout):
                    nC, nV = fctx.shapes
                    dC, dV = fctx.hctx.grad(nC, nV)
                    dev = gout.device
                    return (None, None, None, None, torch.from_numpy(dC).to(dev) * gout,
                            torch.from_numpy(dV).to(dev) * gout, None)
            cls._fn = _Fn
        return cls._fn.apply(ctx, theta, prec, nslices, C, V, D)


class Context:
    """One periodic system.  nao/nabf are per-atom sizes."""

    def __init__(self, nao, nabf, stream=None, lattice=None, pos=None):
        self._lib = load_library()
        nao = np.ascontiguousarray(nao, np.int32)
        nabf = np.ascontiguousarray(nabf, np.int32)
        natoms = nao.shape[0]
        self.nao, self.nabf = nao, nabf
        species = np.arange(natoms, dtype=np.int32)
        lat = None if lattice is None else np.ascontiguousarray(lattice, np.float64).reshape(9)
        ps = None if pos is None else np.ascontiguousarray(pos, np.float64).reshape(-1)
        h = ctypes.c_void_p()
        st = None if stream is None else ctypes.c_void_p(int(stream))
        rc = self._lib.hfx_create(_p(lat), natoms, _p(ps), _p(species), natoms, _p(nao), _p(nabf),
                                  st, ctypes.byref(h))
        if rc != 0:
            raise HfxError(rc, "hfx_create failed")
        self._h = h
        self._layout = {}

    def _check(self, rc):
        if rc != 0:
            raise HfxError(rc, self._lib.hfx_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.hfx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_block(self, which: str, i: int, j: int, n, blk):
        fn = {"C": self._lib.hfx_set_C, "V": self._lib.hfx_set_V, "D": self._lib.hfx_set_D}[which]
        nn = np.ascontiguousarray(n, np.int32)
        b = np.ascontiguousarray(blk, np.float64)
        if not (0 <= i < len(self.nao) and 0 <= j < len(self.nao)):
            raise HfxError(1, "atom index out of range")
        need = {"C": self.nabf[i] * self.nao[i] * self.nao[j], "V": self.nabf[i] * self.nabf[j],
                "D": self.nao[i] * self.nao[j]}[which]
        if b.size != need or nn.size != 3:
            raise HfxError(2, f"block has {b.size} values, the {which} block needs {need}")
        self._check(fn(self._h, i, j, _p(nn), _p(b)))

    def set_many(self, which: str, keys, data, offs, on_device: bool = False):
        k = np.ascontiguousarray(keys, np.int32).reshape(-1, 5)
        o = np.ascontiguousarray(offs, np.int64)
        d = data if on_device else np.ascontiguousarray(data, np.float64)
        n_data = d.numel() if hasattr(d, "numel") else d.size
        if o.shape[0] != k.shape[0] + 1 or (k.shape[0] and (o[0] < 0 or o[-1] > n_data)):
            raise HfxError(2, "offsets do not match the keys or exceed the data")
        self._check(self._lib.hfx_set_many(self._h, which.encode(), k.shape[0], _p(k), _p(d),
                                           _p(o), 1 if on_device else 0))

    def set_blocks(self, which: str, blocks, on_device: bool = False):
        """blocks: object with keys/data/offs (e.g. synth.Blocks)."""
        self.set_many(which, blocks.keys, blocks.data, blocks.offs, on_device)
        self._layout[which] = (np.ascontiguousarray(blocks.keys, np.int32),
                               np.ascontiguousarray(blocks.offs, np.int64))

    def clear(self, which: str):
        self._check(self._lib.hfx_clear(self._h, which.encode()))

    def build(self, theta: float, prec="fp64", nslices: int = 0) -> float:
        ex = ctypes.c_double()
        p = _PREC[prec] if isinstance(prec, str) else int(prec)
        self._check(self._lib.hfx_build(self._h, float(theta), p, int(nslices), ctypes.byref(ex)))
        return ex.value

    def count(self) -> int:
        n = ctypes.c_int64()
        self._check(self._lib.hfx_H_count(self._h, ctypes.byref(n)))
        return n.value

    def keys(self) -> np.ndarray:
        n = self.count()
        out = np.zeros((n, 5), np.int32)
        self._check(self._lib.hfx_H_keys(self._h, _p(out)))
        return out

    def offsets(self) -> np.ndarray:
        out = np.zeros(self.count() + 1, np.int64)
        self._check(self._lib.hfx_H_offsets(self._h, _p(out)))
        return out

    def sigma(self, out=None, on_device: bool = False):
        """All Sigma blocks packed at offsets(); a numpy array, or fills ``out``."""
        if out is None:
            out = np.zeros(int(self.offsets()[-1]), np.float64)
            on_device = False
        self._check(self._lib.hfx_get_H_all(self._h, _p(out), 1 if on_device else 0))
        return out

    def get(self, i: int, j: int, n) -> np.ndarray:
        out = np.zeros((int(self.nao[i]), int(self.nao[j])), np.float64)
        nn = np.ascontiguousarray(n, np.int32)
        self._check(self._lib.hfx_get_H(self._h, i, j, _p(nn), _p(out)))
        return out

    def set_eri_screen(self, eps_eri):
        """Cauchy-Schwarz ERI screen at eps_eri for the next builds (None or a
        negative value: off)."""
        self._check(self._lib.hfx_set_eri_screen(self._h, -1.0 if eps_eri is None
                                                 else float(eps_eri)))

    def set_shard(self, owner, rank: int):
        """Contract only the pairs of central atoms with owner[a] == rank (None: all)."""
        if owner is None:
            self._check(self._lib.hfx_set_shard(self._h, None, 0))
            return
        o = np.ascontiguousarray(owner, np.int32)
        if o.shape[0] != len(self.nao):
            raise HfxError(1, "owner needs one rank per atom")
        self._check(self._lib.hfx_set_shard(self._h, _p(o), int(rank)))

    def sigma_fixed(self, out=None, on_device: bool = False) -> np.ndarray:
        """The Sigma accumulators, (nelem, 2) int64 (units 2^-32, 2^-64); into
        ``out`` (a host array, or a CUDA int64 tensor with on_device) if given."""
        if out is None:
            out = np.zeros((int(self.offsets()[-1]), 2), np.int64)
            on_device = False
        self._check(self._lib.hfx_get_H_fixed(self._h, _p(out), 1 if on_device else 0))
        return out

    def set_sigma_fixed(self, words, on_device: bool = False) -> float:
        """Load summed accumulators (host array, or CUDA int64 tensor with
        on_device) and recompute Sigma and E_X; returns E_X."""
        w = words if on_device else np.ascontiguousarray(words, np.int64)
        ex = ctypes.c_double()
        self._check(self._lib.hfx_set_H_fixed(self._h, _p(w), 1 if on_device else 0,
                                              ctypes.byref(ex)))
        return ex.value

    def grad(self, nC: int, nV: int):
        dC = np.zeros(nC, np.float64)
        dV = np.zeros(nV, np.float64)
        self._check(self._lib.hfx_grad(self._h, _p(dC), _p(dV)))
        return dC, dV

    def density_from_eigvecs(self, kfrac, coef, occ, keys):
        """Real-space density-matrix blocks for keys (n, 5) from eigenvectors
        coef (nk, nbasis, nbands) complex and occupations occ (nk, nbands) at
        fractional k points kfrac (nk, 3).  Returns (packed blocks in key
        order, largest |imaginary part| dropped)."""
        kf = np.ascontiguousarray(np.asarray(kfrac, np.float64).reshape(-1, 3))
        c = np.asarray(coef, np.complex128)
        nk, nbasis, nbands = c.shape
        cc = np.ascontiguousarray(np.stack([c.real, c.imag], axis=-1))
        f = np.ascontiguousarray(np.asarray(occ, np.float64).reshape(nk, nbands))
        k = np.ascontiguousarray(np.asarray(keys, np.int32).reshape(-1, 5))
        nat = len(self.nao)
        ok = (k[:, 0] >= 0) & (k[:, 0] < nat) & (k[:, 1] >= 0) & (k[:, 1] < nat)
        # keys with atoms out of range are rejected by the library (HFX_E_ARG)
        size = int(sum(int(self.nao[a]) * int(self.nao[b]) for a, b in k[ok][:, :2].tolist()))
        out = np.zeros(max(size, 1), np.float64)
        mi = ctypes.c_double(0.0)
        self._check(self._lib.hfx_density_from_eigvecs(self._h, nk, _p(kf), nbands, _p(cc), _p(f),
                                                        k.shape[0], _p(k), _p(out),
                                                        ctypes.byref(mi)))
        return out[:size], mi.value

    def sigma_k(self, kfrac) -> np.ndarray:
        """The last build's Sigma at fractional k points: complex (nk, nb, nb)."""
        kf = np.ascontiguousarray(np.asarray(kfrac, np.float64).reshape(-1, 3))
        nb = int(np.sum(self.nao))
        out = np.zeros((kf.shape[0], nb, nb, 2), np.float64)
        self._check(self._lib.hfx_sigma_k(self._h, kf.shape[0], _p(kf), _p(out)))
        return out[..., 0] + 1j * out[..., 1]

    def stats(self) -> dict:
        s = Stats()
        self._check(self._lib.hfx_stats(self._h, ctypes.byref(s)))
        d = {f: getattr(s, f) for f, _ in Stats._fields_}
        d["survivors"] = list(s.survivors)
        d["kernel_ms"] = dict(zip(KERNELS, list(s.kernel_ms)))
        d["kernel_flops"] = dict(zip(KERNELS, list(s.kernel_flops)))
        d["kernel_tensor_flops"] = dict(zip(KERNELS, list(s.kernel_tensor_flops)))
        d["kernel_unpadded_flops"] = dict(zip(KERNELS, list(s.kernel_unpadded_flops)))
        d["canonical_flops_piece"] = list(s.canonical_flops_piece)
        d["canonical_flops_y"] = s.canonical_flops_y
        return d
