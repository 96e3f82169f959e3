"""CPU oracle for the screened periodic LRI exchange build (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use this package.  The library under ``paper_2009_12505_gb300`` never
imports it, and it imports nothing from the library.

The arithmetic lives in ``hfx_oracle.c`` (plain FP64 C, Algorithm 1 loop order,
C((VC)D) multiplication order per term).  This module compiles it with gcc and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hfx_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle (gcc -O3 -fopenmp -ffp-contract=off) if stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
            lib.orc_create.restype = P
            lib.orc_create.argtypes = [i32, P, P] + [i64, P, P, P] * 3
            lib.orc_destroy.argtypes = [P]
            lib.orc_keys.restype = i64
            lib.orc_keys.argtypes = [P, f64, i32, i32, P, i64, P, P]
            lib.orc_blocks.restype = ctypes.c_int
            lib.orc_blocks.argtypes = [P, f64, i64, P, P, P, ctypes.c_int, P]
            lib.orc_ex.restype = f64
            lib.orc_ex.argtypes = [P, i64, P, P, P]
            lib.orc_maxabs.argtypes = [P, ctypes.c_char, P]
            lib.orc_set_maxabs.argtypes = [P, ctypes.c_char, P]
            lib.orc_set_eri.argtypes = [P, f64]
            lib.orc_eri_sq.argtypes = [P, P]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Oracle:
    """Oracle over one block set.  ``C``, ``V``, ``D`` are objects with
    ``keys`` (n,5) int32, ``data`` float64 and ``offs`` (n+1,) int64."""

    def __init__(self, nao, nabf, C, V, D):
        self._lib = _load()
        self.nao = np.ascontiguousarray(nao, np.int32)
        self.nabf = np.ascontiguousarray(nabf, np.int32)
        self._keep = []
        args = [ctypes.c_int32(len(self.nao)), _ptr(self.nao), _ptr(self.nabf)]
        self.counts_blocks = {}
        for name, b in (("C", C), ("V", V), ("D", D)):
            k = np.ascontiguousarray(b.keys, np.int32)
            d = np.ascontiguousarray(b.data, np.float64)
            o = np.ascontiguousarray(b.offs, np.int64)
            self._keep += [k, d, o]
            self.counts_blocks[name] = k.shape[0]
            args += [ctypes.c_int64(k.shape[0]), _ptr(k), _ptr(d), _ptr(o)]
        self._h = self._lib.orc_create(*args)

    @classmethod
    def of(cls, wl):
        return cls(wl.system.nao, wl.system.nabf, wl.C, wl.V, wl.D)

    def close(self):
        if self._h:
            self._lib.orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def keys(self, theta: float, atoms=None, extra: bool = False):
        """Sigma key set at theta (sorted) and surviving terms per variant
        (ABFs on (I,J), (I,L), (K,J), (K,L)); ``atoms`` = (first, end) limits
        the central atoms.  With ``extra`` also returns {"active_abg",
        "canonical_flops"} (Algorithm 3 count, 2 flops per multiply-add)."""
        a0, a1 = (0, 0) if atoms is None else atoms
        counts = np.zeros(4, np.int64)
        ex = np.zeros(2, np.int64)
        n = self._lib.orc_keys(self._h, float(theta), a0, a1, None, 0, _ptr(counts), _ptr(ex))
        keys = np.zeros((n, 5), np.int32)
        self._lib.orc_keys(self._h, float(theta), a0, a1, _ptr(keys), n, _ptr(counts), _ptr(ex))
        if extra:
            return keys, counts, {"active_abg": int(ex[0]), "canonical_flops": 2.0 * float(ex[1])}
        return keys, counts

    def blocks(self, theta: float, keys, nthreads: int = 0, terms: bool = False):
        """Sigma blocks for the given keys: (data, offs) packed in key order,
        plus the surviving terms per block when ``terms``."""
        keys = np.ascontiguousarray(np.asarray(keys, np.int32).reshape(-1, 5))
        n = keys.shape[0]
        sizes = self.nao[keys[:, 0]].astype(np.int64) * self.nao[keys[:, 1]]
        out = np.zeros(int(sizes.sum()), np.float64)
        offs = np.zeros(n + 1, np.int64)
        nterms = np.zeros(n, np.int64)
        rc = self._lib.orc_blocks(self._h, float(theta), n, _ptr(keys), _ptr(out), _ptr(offs),
                                  int(nthreads), _ptr(nterms))
        if rc != 0:
            raise ValueError("oracle work buffers cover nao <= 64 and nabf <= 128")
        return (out, offs, nterms) if terms else (out, offs)

    def ex(self, keys, data, offs) -> float:
        keys = np.ascontiguousarray(keys, np.int32)
        data = np.ascontiguousarray(data, np.float64)
        offs = np.ascontiguousarray(offs, np.int64)
        return float(self._lib.orc_ex(self._h, keys.shape[0], _ptr(keys), _ptr(data),
                                      _ptr(offs)))

    def build(self, theta: float, nthreads: int = 0):
        """Full build: dict with keys, data, offs, counts (per variant) and ex."""
        keys, counts = self.keys(theta)
        data, offs = self.blocks(theta, keys, nthreads)
        return {"keys": keys, "data": data, "offs": offs, "counts": counts,
                "ex": self.ex(keys, data, offs)}

    def set_maxabs(self, which: str, vals) -> None:
        """Use these block upper limits in the screen (frozen surviving set)."""
        v = np.ascontiguousarray(vals, np.float64)
        assert v.shape[0] == self.counts_blocks[which]
        self._keep.append(v)
        self._lib.orc_set_maxabs(self._h, which.encode()[0:1], _ptr(v))

    def set_eri(self, eps_eri):
        """Turn on the Cauchy-Schwarz ERI screen at eps_eri (Eq. CS-ERI): a
        term also needs sqrt(Q_AF) sqrt(Q_BG) > eps_eri; None turns it off."""
        self._lib.orc_set_eri(self._h, -1.0 if eps_eri is None else float(eps_eri))

    def eri_sq(self) -> np.ndarray:
        """sqrt(max(Q, 0)) per C block (key order) of the ERI screen."""
        out = np.zeros(self.counts_blocks["C"], np.float64)
        self._lib.orc_eri_sq(self._h, _ptr(out))
        return out

    def maxabs(self, which: str) -> np.ndarray:
        out = np.zeros(self.counts_blocks[which], np.float64)
        self._lib.orc_maxabs(self._h, which.encode()[0:1], _ptr(out))
        return out


def block_dict(keys, data, offs, nao):
    """{key tuple: 2-D block} view of a packed Sigma result."""
    out = {}
    for e, k in enumerate(np.asarray(keys)):
        kt = tuple(int(x) for x in k)
        out[kt] = data[offs[e]:offs[e + 1]].reshape(int(nao[kt[0]]), int(nao[kt[1]]))
    return out
