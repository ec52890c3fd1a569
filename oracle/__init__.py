"""Python handle on the plain FP64 CPU oracle (``xamg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU leg of
the benchmark use it to check and time the CUDA library.  The library itself
never imports this package.

The oracle follows the paper's method step by step (multi-RHS SpMM, classical
AMG with Chebyshev order-2 smoothing as a V(1,1) preconditioner, coarsest
direct solve, PCG and BiCGStab with per-column status); the readings it takes
where the paper is silent are listed in the header of ``xamg_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "xamg_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")

DEFAULTS = dict(theta=0.25, max_coarse=64, max_levels=25, cheb_steps=2, power_iters=20,
                lo_frac=0.3, hi_safety=1.1, max_dense=4096)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, no vendor code)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu99", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_spmm.argtypes = [C.c_int, C.c_int, _i32p, _i32p, _f64p, C.c_int, _f64p, _f64p]
        L.orc_spmm.restype = C.c_int
        L.orc_setup.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double, C.c_int, C.c_int,
                                C.c_int, C.c_int, C.c_double, C.c_double, C.c_int,
                                C.POINTER(C.c_int)]
        L.orc_setup.restype = C.c_void_p
        L.orc_free.argtypes = [C.c_void_p]
        L.orc_nlev.argtypes = [C.c_void_p]
        L.orc_nlev.restype = C.c_int
        L.orc_level_sizes.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_int),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        L.orc_level_csr.argtypes = [C.c_void_p, C.c_int, C.c_int, _i32p, _i32p, _f64p]
        L.orc_level_cf.argtypes = [C.c_void_p, C.c_int, _i32p]
        L.orc_level_dinv.argtypes = [C.c_void_p, C.c_int, _f64p]
        L.orc_level_cheb.argtypes = [C.c_void_p, C.c_int, _f64p]
        L.orc_coarse_lu.argtypes = [C.c_void_p, _f64p, _i32p]
        L.orc_cheb_smooth.argtypes = [C.c_void_p, C.c_int, C.c_int, _f64p, _f64p, C.c_int,
                                      C.c_void_p]
        L.orc_cheb_smooth.restype = C.c_int
        L.orc_vcycle.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p]
        L.orc_vcycle.restype = C.c_int
        L.orc_vcycle_prec.argtypes = [C.c_void_p, C.c_int, C.c_int, _f64p, _f64p]
        L.orc_vcycle_prec.restype = C.c_int
        _f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
        L.orc_spmm_f.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, _f32p, _f32p]
        L.orc_spmm_f.restype = C.c_int
        L.orc_bf16_bits.argtypes = [C.c_float]
        L.orc_bf16_bits.restype = C.c_uint16
        for name in ("orc_pcg_prec", "orc_bicgstab_prec", "orc_rbicgstab_prec", "orc_pbicgstab_prec"):
            f = getattr(L, name)
            f.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, _f64p, _f64p, C.c_double, C.c_int,
                          _i32p, _f64p, _i32p]
            f.restype = C.c_int
        for name in ("orc_pcg", "orc_bicgstab"):
            f = getattr(L, name)
            f.argtypes = [C.c_void_p, C.c_int, _f64p, _f64p, C.c_double, C.c_int, _i32p, _f64p,
                          _i32p]
            f.restype = C.c_int
        L.orc_lu_factor.argtypes = [C.c_int, _f64p, _i32p]
        L.orc_lu_factor.restype = C.c_int
        L.orc_lu_solve.argtypes = [C.c_int, _f64p, _i32p, C.c_int, _f64p]
        L.orc_splitmix_uniform.argtypes = [C.c_uint64]
        L.orc_splitmix_uniform.restype = C.c_double
        _lib = L
    return _lib


def _csr_args(A):
    return (np.ascontiguousarray(A.rowptr, dtype=np.int32), np.ascontiguousarray(A.col, dtype=np.int32),
            np.ascontiguousarray(A.val, dtype=np.float64))


def spmm(A, X: np.ndarray, ncols: int | None = None) -> np.ndarray:
    """Y = A X for an n x m row-major block (m >= 1)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    if X.ndim == 1:
        X = X[:, None]
    rp, ci, v = _csr_args(A)
    Y = np.empty((A.n, X.shape[1]), dtype=np.float64)
    rc = lib().orc_spmm(A.n, X.shape[0] if ncols is None else ncols, rp, ci, v, X.shape[1], X, Y)
    if rc != 0:
        raise ValueError(f"orc_spmm failed: {rc}")
    return Y


@dataclass
class Level:
    n: int
    A: tuple          # (rowptr, col, val)
    P: tuple | None   # n x n_next
    R: tuple | None
    cf: np.ndarray | None
    dinv: np.ndarray
    cheb: np.ndarray | None  # lo, hi, lambda_hat, gershgorin


class Hierarchy:
    """The oracle's frozen AMG hierarchy (owned C object plus copies of its parts)."""

    def __init__(self, A, **params):
        p = dict(DEFAULTS)
        p.update(params)
        rp, ci, v = _csr_args(A)
        err = C.c_int(0)
        self._h = lib().orc_setup(A.n, rp, ci, v, p["theta"], p["max_coarse"], p["max_levels"],
                                  p["cheb_steps"], p["power_iters"], p["lo_frac"], p["hi_safety"],
                                  p["max_dense"], C.byref(err))
        if not self._h:
            raise RuntimeError(f"oracle setup failed: {err.value}")
        self.params = p
        self.n = A.n

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_free(self._h)
            self._h = None

    @property
    def nlev(self) -> int:
        return lib().orc_nlev(self._h)

    def level(self, l: int) -> Level:
        L = lib()
        n = C.c_int(); na = C.c_int64(); npn = C.c_int64()
        L.orc_level_sizes(self._h, l, C.byref(n), C.byref(na), C.byref(npn))
        n = n.value

        def get(which, rows, nnz):
            rp = np.empty(rows + 1, np.int32); ci = np.empty(max(nnz, 1), np.int32)
            vv = np.empty(max(nnz, 1), np.float64)
            L.orc_level_csr(self._h, l, which, rp, ci, vv)
            return rp, ci[:nnz], vv[:nnz]

        A = get(0, n, na.value)
        dinv = np.empty(n, np.float64)
        L.orc_level_dinv(self._h, l, dinv)
        if l + 1 < self.nlev:
            P = get(1, n, npn.value)
            nc = C.c_int(); d1 = C.c_int64(); d2 = C.c_int64()
            L.orc_level_sizes(self._h, l + 1, C.byref(nc), C.byref(d1), C.byref(d2))
            R = get(2, nc.value, npn.value)
            cf = np.empty(n, np.int32)
            L.orc_level_cf(self._h, l, cf)
            ch = np.empty(4, np.float64)
            L.orc_level_cheb(self._h, l, ch)
        else:
            P = R = cf = ch = None
        return Level(n, A, P, R, cf, dinv, ch)

    def coarse_lu(self):
        lv = self.level(self.nlev - 1)
        lu = np.empty(lv.n * lv.n, np.float64); piv = np.empty(lv.n, np.int32)
        lib().orc_coarse_lu(self._h, lu, piv)
        return lu.reshape(lv.n, lv.n), piv

    def cheb_smooth(self, l: int, B: np.ndarray, X0: np.ndarray | None = None, want_residual=True):
        B = np.ascontiguousarray(B, dtype=np.float64)
        m = B.shape[1]
        X = np.zeros_like(B) if X0 is None else np.ascontiguousarray(X0, dtype=np.float64).copy()
        R = np.empty_like(B) if want_residual else None
        rc = lib().orc_cheb_smooth(self._h, l, m, B, X, 1 if X0 is None else 0,
                                   R.ctypes.data if want_residual else None)
        if rc != 0:
            raise RuntimeError(f"orc_cheb_smooth failed: {rc}")
        return X, R

    def vcycle(self, B: np.ndarray) -> np.ndarray:
        B = np.ascontiguousarray(B, dtype=np.float64)
        X = np.empty_like(B)
        rc = lib().orc_vcycle(self._h, B.shape[1], B, X)
        if rc != 0:
            raise RuntimeError(f"orc_vcycle failed: {rc}")
        return X

    def vcycle_prec(self, prec: int, B: np.ndarray) -> np.ndarray:
        """One V-cycle with the preconditioner precision prec (0 FP64, 1 FP32, 2 bf16 A)."""
        B = np.ascontiguousarray(B, dtype=np.float64)
        X = np.empty_like(B)
        rc = lib().orc_vcycle_prec(self._h, prec, B.shape[1], B, X)
        if rc != 0:
            raise RuntimeError(f"orc_vcycle_prec failed: {rc}")
        return X

    def spmm_f(self, l: int, which: int, X: np.ndarray, bf16: bool = False) -> np.ndarray:
        """FP32 product of level l's operator (0 A, 1 P, 2 R) with an FP32 block."""
        X = np.ascontiguousarray(X, dtype=np.float32)
        rows = self.level(l).n if which != 2 else self.level(l + 1).n
        Y = np.empty((rows, X.shape[1]), dtype=np.float32)
        rc = lib().orc_spmm_f(self._h, l, which, 1 if bf16 else 0, X.shape[1], X, Y)
        if rc != 0:
            raise RuntimeError(f"orc_spmm_f failed: {rc}")
        return Y

    def _solve(self, fn, B, tol, maxit, prec=None, X0=None):
        B = np.ascontiguousarray(B, dtype=np.float64)
        m = B.shape[1]
        X = np.empty_like(B) if X0 is None else np.ascontiguousarray(X0, dtype=np.float64).copy()
        it = np.zeros(m, np.int32); rr = np.zeros(m, np.float64); st = np.zeros(m, np.int32)
        if prec is None:
            rc = fn(self._h, m, B, X, tol, maxit, it, rr, st)
        else:
            rc = fn(self._h, prec, 0 if X0 is None else 1, m, B, X, tol, maxit, it, rr, st)
        if rc < 0:
            raise RuntimeError(f"oracle solve failed: {rc}")
        return SolveResult(X, it, rr, st, rc)

    def pcg(self, B, tol=1e-8, maxit=200, prec=0, X0=None):
        """PCG; with prec 1 (FP32) or 2 (bf16 A) the preconditioner is the
        reduced-precision V-cycle and the iteration is flexible PCG; X0 is an
        optional initial guess."""
        if prec or X0 is not None:
            return self._solve(lib().orc_pcg_prec, B, tol, maxit, prec, X0)
        return self._solve(lib().orc_pcg, B, tol, maxit)

    def bicgstab(self, B, tol=1e-8, maxit=200, prec=0, X0=None, variant="classical"):
        """BiCGStab; variant "reordered" (two dot-product groups per iteration,
        recurrences for rho and |r|) or "pipelined" (auxiliary products so that
        each dot-product group overlaps one operator application)."""
        if variant == "reordered":
            return self._solve(lib().orc_rbicgstab_prec, B, tol, maxit, prec, X0)
        if variant == "pipelined":
            return self._solve(lib().orc_pbicgstab_prec, B, tol, maxit, prec, X0)
        if prec or X0 is not None:
            return self._solve(lib().orc_bicgstab_prec, B, tol, maxit, prec, X0)
        return self._solve(lib().orc_bicgstab, B, tol, maxit)


@dataclass
class SolveResult:
    X: np.ndarray
    iters: np.ndarray
    relres: np.ndarray
    status: np.ndarray
    rc: int


def lu_factor(A: np.ndarray):
    a = np.ascontiguousarray(A, dtype=np.float64).copy()
    piv = np.empty(a.shape[0], np.int32)
    rc = lib().orc_lu_factor(a.shape[0], a.reshape(-1), piv)
    if rc != 0:
        raise RuntimeError("singular")
    return a, piv


def lu_solve(lu: np.ndarray, piv: np.ndarray, B: np.ndarray) -> np.ndarray:
    b = np.ascontiguousarray(B, dtype=np.float64).copy()
    if b.ndim == 1:
        b = b[:, None]
    lib().orc_lu_solve(lu.shape[0], np.ascontiguousarray(lu).reshape(-1), piv, b.shape[1], b.reshape(-1))
    return b


def bf16_bits(f: float) -> int:
    """bf16 bits of an FP32 value, round to nearest even."""
    return int(lib().orc_bf16_bits(f))


def splitmix_uniform(i: int) -> float:
    return lib().orc_splitmix_uniform(i)
