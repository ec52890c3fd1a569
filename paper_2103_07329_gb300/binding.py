"""Thin ctypes binding of the C ABI in ``include/xamg_gpu.h``.

Argument marshalling only: every step of the solve phase runs in the CUDA
library.  Device blocks are passed as torch CUDA tensors (float64,
contiguous, n x m row-major); streams as ``torch.cuda.Stream`` or raw handles.
If the compiled library is missing this module raises at import time instead
of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

OK = 0
ERR_INVALID_ARG = -1
ERR_CUDA = -2
ERR_OOM = -3
ERR_NONFINITE = -4
ERR_TIMEOUT = -5
ERR_SETUP = -6
NOT_CONVERGED = 1
BREAKDOWN = 2
PCG = 0
BICGSTAB = 1
BICGSTAB_REORDERED = 2
BICGSTAB_PIPELINED = 3
PREC_FP64 = 0
PREC_FP32 = 1
PREC_BF16 = 2
MAX_RHS = 32

# every entry point declared in include/xamg_gpu.h
EXPORTS = [
    "xamg_strerror", "xamg_amg_params_default", "xamg_solve_opts_default",
    "xamg_setup_hierarchy", "xamg_destroy", "xamg_hier_save", "xamg_hier_load", "xamg_hier_info",
    "xamg_level_info",
    "xamg_level_export", "xamg_coarse_export", "xamg_workspace_bytes", "xamg_solve",
    "xamg_solve_host", "xamg_level_spmm", "xamg_level_spmm_precond", "xamg_set_index16",
    "xamg_index16_info", "xamg_set_tail", "xamg_tail_info", "xamg_smooth", "xamg_vcycle", "xamg_vcycle_precond",
    "xamg_coarse_solve",
    "xamg_coldot", "xamg_timing_enable", "xamg_timing_read", "xamg_kernel_launches",
    "xamg_coldot_noalloc",
    "xamg_net_param_count", "xamg_net_create", "xamg_net_destroy", "xamg_net_set_params",
    "xamg_net_get_params", "xamg_net_forward", "xamg_net_loss_grad", "xamg_net_train_step",
    "xamg_net_predict_x0", "xamg_conv3d_bf16", "xamg_conv3d_bf16_wgrad",
    "xamg_autotune", "xamg_set_split", "xamg_set_graphs", "xamg_batch_opts_default", "xamg_batch_create", "xamg_batch_destroy", "xamg_batch_info",
    "xamg_batch_solve",
]


class XamgError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: {strerror(code)} ({code})")
        self.code = code


class CsrT(C.Structure):
    _fields_ = [("n", C.c_int32), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class AmgParamsT(C.Structure):
    _fields_ = [("theta", C.c_double), ("max_coarse", C.c_int32), ("max_levels", C.c_int32),
                ("cheb_steps", C.c_int32), ("power_iters", C.c_int32),
                ("cheb_lo_frac", C.c_double), ("cheb_hi_safety", C.c_double),
                ("max_dense", C.c_int32), ("nthreads", C.c_int32), ("device_upload", C.c_int32)]


class SolveOptsT(C.Structure):
    _fields_ = [("method", C.c_int32), ("precond", C.c_int32), ("x0_given", C.c_int32),
                ("stream", C.c_void_p), ("workspace", C.c_void_p), ("workspace_bytes", C.c_size_t)]


class AdamT(C.Structure):
    _fields_ = [("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float)]


class BatchOptsT(C.Structure):
    _fields_ = [("autotune", C.c_int32), ("use_graph", C.c_int32)]


class NetLossT(C.Structure):
    _fields_ = [("kind", C.c_int32), ("sample_weight", C.c_void_p)]


LOSS_MSE = 0
LOSS_ENERGY = 1


class StatsT(C.Structure):
    _fields_ = [("iters", C.c_void_p), ("relres", C.c_void_p), ("status", C.c_void_p),
                ("iterations", C.c_int32), ("vcycles", C.c_int32)]


_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"CUDA library {LIB_PATH} is not built; run "
                          "`python -m paper_2103_07329_gb300.build` (nvcc, sm_103a)")
    try:  # let the library share torch's CUDA runtime when torch is present
        import torch  # noqa: F401
    except Exception:
        pass
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "xamg_strerror": ([C.c_int], C.c_char_p),
        "xamg_amg_params_default": ([C.POINTER(AmgParamsT)], None),
        "xamg_solve_opts_default": ([C.POINTER(SolveOptsT)], None),
        "xamg_setup_hierarchy": ([C.POINTER(CsrT), C.POINTER(AmgParamsT), C.POINTER(vp)], C.c_int),
        "xamg_destroy": ([vp], C.c_int),
        "xamg_hier_save": ([vp, vp, C.c_size_t, C.POINTER(C.c_size_t)], C.c_int),
        "xamg_hier_load": ([vp, C.c_size_t, C.POINTER(vp)], C.c_int),
        "xamg_hier_info": ([vp, C.POINTER(i32), C.POINTER(dbl)], C.c_int),
        "xamg_level_info": ([vp, i32, C.POINTER(i32), C.POINTER(i64), C.POINTER(i64)], C.c_int),
        "xamg_level_export": ([vp, i32, vp, vp, vp, vp, vp, vp, vp, vp], C.c_int),
        "xamg_coarse_export": ([vp, C.POINTER(i32), vp, vp], C.c_int),
        "xamg_workspace_bytes": ([vp, i32, i32, i32, C.POINTER(C.c_size_t)], C.c_int),
        "xamg_solve": ([vp, vp, vp, i32, dbl, i32, C.POINTER(SolveOptsT), C.POINTER(StatsT)], C.c_int),
        "xamg_solve_host": ([vp, vp, vp, i32, dbl, i32, C.POINTER(SolveOptsT), C.POINTER(StatsT)],
                            C.c_int),
        "xamg_level_spmm": ([vp, i32, i32, vp, vp, i32, vp], C.c_int),
        "xamg_level_spmm_precond": ([vp, i32, i32, i32, vp, vp, i32, vp], C.c_int),
        "xamg_set_index16": ([vp, i32], C.c_int),
        "xamg_index16_info": ([vp, i32, C.POINTER(i32)], C.c_int),
        "xamg_set_tail": ([vp, i64, dbl, i32], C.c_int),
        "xamg_tail_info": ([vp, i32, C.POINTER(i32)], C.c_int),
        "xamg_smooth": ([vp, i32, vp, vp, vp, i32, i32, vp], C.c_int),
        "xamg_vcycle": ([vp, vp, vp, i32, vp], C.c_int),
        "xamg_vcycle_precond": ([vp, i32, vp, vp, i32, vp], C.c_int),
        "xamg_coarse_solve": ([vp, vp, vp, i32, vp], C.c_int),
        "xamg_coldot": ([vp, vp, i64, i32, vp, vp], C.c_int),
        "xamg_coldot_noalloc": ([vp, vp, i64, i32, vp, vp], C.c_int),
        "xamg_timing_enable": ([vp, i32], C.c_int),
        "xamg_kernel_launches": ([], C.c_int64),
        "xamg_timing_read": ([vp, i32, i32, C.POINTER(i64), C.POINTER(dbl), C.POINTER(dbl),
                              C.POINTER(dbl)], C.c_int),
        "xamg_net_param_count": ([], C.c_int64),
        "xamg_net_create": ([i32, i32, C.POINTER(vp)], C.c_int),
        "xamg_net_destroy": ([vp], None),
        "xamg_net_set_params": ([vp, vp], C.c_int),
        "xamg_net_get_params": ([vp, vp], C.c_int),
        "xamg_net_forward": ([vp, vp, vp, i32, vp], C.c_int),
        "xamg_net_loss_grad": ([vp, vp, vp, i32, C.POINTER(NetLossT), C.POINTER(C.c_float), vp, vp],
                               C.c_int),
        "xamg_net_train_step": ([vp, vp, vp, i64, vp, i32, C.POINTER(NetLossT), C.POINTER(AdamT),
                                 C.POINTER(C.c_float), vp], C.c_int),
        "xamg_net_predict_x0": ([vp, vp, vp, dbl, vp, i32, vp], C.c_int),
        "xamg_conv3d_bf16": ([vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, i32, vp], C.c_int),
        "xamg_conv3d_bf16_wgrad": ([vp, vp, vp, vp, vp, i32, i32, i32, i32, vp], C.c_int),
        "xamg_autotune": ([vp, i32, i32, vp, C.POINTER(i32), C.POINTER(i32)], C.c_int),
        "xamg_set_split": ([vp, i32, i32, i32, i32, i32], C.c_int),
        "xamg_set_graphs": ([vp, i32], C.c_int),
        "xamg_batch_opts_default": ([C.POINTER(BatchOptsT)], None),
        "xamg_batch_create": ([vp, vp, i32, C.POINTER(BatchOptsT), C.POINTER(vp)], C.c_int),
        "xamg_batch_destroy": ([vp], C.c_int),
        "xamg_batch_info": ([vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i64)], C.c_int),
        "xamg_batch_solve": ([vp, vp, vp, dbl, i32, vp, vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def lib():
    return _load()


def strerror(code: int) -> str:
    return _load().xamg_strerror(code).decode()


def _check(rc: int, what: str, allow_positive=False) -> int:
    if rc < 0 or (rc > 0 and not allow_positive):
        raise XamgError(rc, what)
    return rc


def _ptr(t) -> int:
    """Device address of a torch CUDA tensor (float64, contiguous) or an int."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            return torch.cuda.current_stream().cuda_stream
        except Exception:
            return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def amg_params(**kw) -> AmgParamsT:
    p = AmgParamsT()
    _load().xamg_amg_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise TypeError(f"unknown AMG parameter {k}")
        setattr(p, k, v)
    return p


class SolveStats:
    def __init__(self, m):
        self.iters = np.zeros(m, np.int32)
        self.relres = np.zeros(m, np.float64)
        self.status = np.zeros(m, np.int32)
        self.iterations = 0
        self.vcycles = 0
        self.rc = 0

    def struct(self) -> StatsT:
        return StatsT(self.iters.ctypes.data, self.relres.ctypes.data, self.status.ctypes.data, 0, 0)


class Hierarchy:
    """Handle on the library's frozen AMG hierarchy (``xamg_setup_hierarchy``)."""

    def __init__(self, A, **params):
        L = _load()
        self._keep = (np.ascontiguousarray(A.rowptr, np.int32), np.ascontiguousarray(A.col, np.int32),
                      np.ascontiguousarray(A.val, np.float64))
        rp, ci, v = self._keep
        csr = CsrT(A.n, int(rp[-1]), rp.ctypes.data, ci.ctypes.data, v.ctypes.data)
        prm = amg_params(**params)
        h = C.c_void_p()
        rc = L.xamg_setup_hierarchy(C.byref(csr), C.byref(prm), C.byref(h))
        self._keep = None
        _check(rc, "xamg_setup_hierarchy")
        self._h = h
        self.n = A.n
        self.on_device = bool(prm.device_upload)

    def save(self) -> bytes:
        """xamg_hier_save: the frozen hierarchy as bytes."""
        L = _load()
        n = C.c_size_t()
        _check(L.xamg_hier_save(self._h, None, 0, C.byref(n)), "xamg_hier_save")
        buf = C.create_string_buffer(n.value)
        _check(L.xamg_hier_save(self._h, buf, n.value, C.byref(n)), "xamg_hier_save")
        return buf.raw[:n.value]

    @classmethod
    def load(cls, blob: bytes) -> "Hierarchy":
        """xamg_hier_load: a hierarchy from the bytes of save()."""
        L = _load()
        buf = C.create_string_buffer(bytes(blob), len(blob))
        h = C.c_void_p()
        _check(L.xamg_hier_load(buf, len(blob), C.byref(h)), "xamg_hier_load")
        self = cls.__new__(cls)
        self._h = h
        n = C.c_int32()
        na = C.c_int64()
        npn = C.c_int64()
        _check(L.xamg_level_info(h, 0, C.byref(n), C.byref(na), C.byref(npn)), "xamg_level_info")
        self.n = n.value
        # graphs are on by default; re-enabling them changes nothing and is
        # accepted only by a hierarchy on the device
        self.on_device = L.xamg_set_graphs(h, 1) == 0
        return self

    def close(self):
        if getattr(self, "_h", None):
            _load().xamg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def levels(self) -> int:
        n = C.c_int32()
        _check(_load().xamg_hier_info(self._h, C.byref(n), None), "xamg_hier_info")
        return n.value

    @property
    def op_complexity(self) -> float:
        oc = C.c_double()
        _check(_load().xamg_hier_info(self._h, None, C.byref(oc)), "xamg_hier_info")
        return oc.value

    def level_info(self, l: int):
        n = C.c_int32(); na = C.c_int64(); npn = C.c_int64()
        _check(_load().xamg_level_info(self._h, l, C.byref(n), C.byref(na), C.byref(npn)),
               "xamg_level_info")
        return n.value, na.value, npn.value

    def level_export(self, l: int):
        n, na, npn = self.level_info(l)
        rp = np.empty(n + 1, np.int32); ci = np.empty(max(na, 1), np.int32); v = np.empty(max(na, 1))
        prp = np.empty(n + 1, np.int32); pci = np.empty(max(npn, 1), np.int32)
        pv = np.empty(max(npn, 1)); cf = np.zeros(n, np.int32); ch = np.empty(4)
        _check(_load().xamg_level_export(self._h, l, rp.ctypes.data, ci.ctypes.data, v.ctypes.data,
                                         prp.ctypes.data, pci.ctypes.data, pv.ctypes.data,
                                         cf.ctypes.data, ch.ctypes.data), "xamg_level_export")
        last = l + 1 == self.levels
        return dict(n=n, A=(rp, ci[:na], v[:na]),
                    P=None if last else (prp, pci[:npn], pv[:npn]),
                    cf=None if last else cf, cheb=None if last else ch)

    def coarse_export(self):
        nc = C.c_int32()
        _check(_load().xamg_coarse_export(self._h, C.byref(nc), None, None), "xamg_coarse_export")
        lu = np.empty(nc.value * nc.value); piv = np.empty(nc.value, np.int32)
        _check(_load().xamg_coarse_export(self._h, C.byref(nc), lu.ctypes.data, piv.ctypes.data),
               "xamg_coarse_export")
        return lu.reshape(nc.value, nc.value), piv

    def workspace_bytes(self, m: int, method: int = PCG, precond: int = PREC_FP64) -> int:
        b = C.c_size_t()
        _check(_load().xamg_workspace_bytes(self._h, m, method, precond, C.byref(b)),
               "xamg_workspace_bytes")
        return b.value

    def _opts(self, method, stream, workspace, precond=PREC_FP64, x0_given=False):
        o = SolveOptsT()
        _load().xamg_solve_opts_default(C.byref(o))
        o.method = method
        o.precond = precond
        o.x0_given = 1 if x0_given else 0
        o.stream = _stream(stream)
        if workspace is not None:
            o.workspace = _ptr(workspace)
            o.workspace_bytes = workspace.numel() * workspace.element_size()
        return o

    def solve(self, B, X, tol=1e-8, maxit=200, method=PCG, stream=None, workspace=None,
              precond=PREC_FP64, x0_given=False) -> SolveStats:
        """xamg_solve on device blocks B, X (torch float64 CUDA tensors, n x m);
        with x0_given, X holds the initial guess on entry."""
        m = B.shape[1] if B.dim() == 2 else 1
        st = SolveStats(m)
        s = st.struct()
        o = self._opts(method, stream, workspace, precond, x0_given)
        rc = _load().xamg_solve(self._h, _ptr(B), _ptr(X), m, tol, maxit, C.byref(o), C.byref(s))
        _check(rc, "xamg_solve", allow_positive=True)
        st.iterations, st.vcycles, st.rc = s.iterations, s.vcycles, rc
        return st

    def solve_host(self, B: np.ndarray, X: np.ndarray, tol=1e-8, maxit=200, method=PCG,
                   stream=None, precond=PREC_FP64, x0_given=False) -> SolveStats:
        """xamg_solve_host on host arrays (float64, C order, n x m)."""
        assert B.flags.c_contiguous and X.flags.c_contiguous and B.dtype == np.float64
        m = B.shape[1]
        st = SolveStats(m)
        s = st.struct()
        o = self._opts(method, stream, None, precond, x0_given)
        rc = _load().xamg_solve_host(self._h, B.ctypes.data, X.ctypes.data, m, tol, maxit,
                                     C.byref(o), C.byref(s))
        _check(rc, "xamg_solve_host", allow_positive=True)
        st.iterations, st.vcycles, st.rc = s.iterations, s.vcycles, rc
        return st

    def spmm(self, level: int, which: int, X, Y, stream=None):
        m = X.shape[1]
        _check(_load().xamg_level_spmm(self._h, level, which, _ptr(X), _ptr(Y), m, _stream(stream)),
               "xamg_level_spmm")

    def spmm_precond(self, precond: int, level: int, which: int, X, Y, stream=None):
        """xamg_level_spmm_precond: the reduced-precision product of the
        V-cycle (FP64 blocks in and out, FP32 inside)."""
        m = X.shape[1]
        _check(_load().xamg_level_spmm_precond(self._h, precond, level, which, _ptr(X), _ptr(Y), m,
                                               _stream(stream)), "xamg_level_spmm_precond")

    def set_tail(self, max_elems: int = 131072, wait_limit_s: float = 2.0, extra_arrivals: int = 0):
        """xamg_set_tail: the fused coarse tail of the V-cycle (0 turns it off)."""
        _check(_load().xamg_set_tail(self._h, max_elems, wait_limit_s, extra_arrivals), "xamg_set_tail")

    def tail_info(self, m: int) -> int:
        """xamg_tail_info: first level of the fused tail for pad(m) columns, or -1."""
        f = C.c_int32()
        _check(_load().xamg_tail_info(self._h, m, C.byref(f)), "xamg_tail_info")
        return f.value

    def set_index16(self, on: bool = True):
        """xamg_set_index16: 16-bit column indices of the reduced-precision products on or off."""
        _check(_load().xamg_set_index16(self._h, 1 if on else 0), "xamg_set_index16")

    def index16_info(self, level: int) -> int:
        """xamg_index16_info: bit mask of level's operators (A 1, P 2, R 4) with 16-bit indices."""
        mk = C.c_int32()
        _check(_load().xamg_index16_info(self._h, level, C.byref(mk)), "xamg_index16_info")
        return mk.value

    def smooth(self, level: int, B, X, R=None, x_zero=True, stream=None):
        m = B.shape[1]
        _check(_load().xamg_smooth(self._h, level, _ptr(B), _ptr(X), _ptr(R), 1 if x_zero else 0, m,
                                   _stream(stream)), "xamg_smooth")

    def vcycle(self, B, X, stream=None):
        _check(_load().xamg_vcycle(self._h, _ptr(B), _ptr(X), B.shape[1], _stream(stream)),
               "xamg_vcycle")

    def vcycle_precond(self, precond, B, X, stream=None):
        _check(_load().xamg_vcycle_precond(self._h, precond, _ptr(B), _ptr(X), B.shape[1],
                                           _stream(stream)), "xamg_vcycle_precond")

    def coarse_solve(self, B, X, stream=None):
        _check(_load().xamg_coarse_solve(self._h, _ptr(B), _ptr(X), B.shape[1], _stream(stream)),
               "xamg_coarse_solve")

    def autotune(self, m: int, precond: int = PREC_FP32, stream=None):
        """xamg_autotune: time every row split of each level's products on
        blocks of pad(m) columns of precision `precond` and keep the fastest;
        returns (products tuned, products that chose a split other than the
        first candidate)."""
        t = C.c_int32(); w = C.c_int32()
        _check(_load().xamg_autotune(self._h, m, precond, _stream(stream), C.byref(t), C.byref(w)),
               "xamg_autotune")
        return t.value, w.value

    def set_split(self, m: int, precond: int, level: int, which: int, candidate: int):
        """xamg_set_split: force tuning candidate `candidate` (-1: the default
        rule) for operator `which` of `level` on pad(m)-column blocks."""
        _check(_load().xamg_set_split(self._h, m, precond, level, which, candidate), "xamg_set_split")

    def set_graphs(self, on: bool = True):
        """xamg_set_graphs: CUDA graphs of the steady PCG iteration on or off."""
        _check(_load().xamg_set_graphs(self._h, 1 if on else 0), "xamg_set_graphs")

    def timing_enable(self, on: bool = True):
        _check(_load().xamg_timing_enable(self._h, 1 if on else 0), "xamg_timing_enable")

    def timing_read(self, level: int, which: int):
        n = C.c_int64(); ms = C.c_double(); fl = C.c_double(); by = C.c_double()
        _check(_load().xamg_timing_read(self._h, level, which, C.byref(n), C.byref(ms), C.byref(fl),
                                        C.byref(by)), "xamg_timing_read")
        return dict(launches=n.value, ms=ms.value, flops=fl.value, bytes=by.value)


def kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(_load().xamg_kernel_launches())


def coldot(U, V, out, stream=None):
    """xamg_coldot: out[j] = sum_i U[i, j] V[i, j] on device tensors."""
    n, m = U.shape
    _check(_load().xamg_coldot(_ptr(U), _ptr(V), n, m, _ptr(out), _stream(stream)), "xamg_coldot")


def coldot_noalloc(U, V, out, stream=None):
    """xamg_coldot_noalloc: the same column dots as ``coldot`` for callers that
    must not allocate device memory during the call; the partial sums go to a
    fixed 256 KiB array inside the library.  Calls that overlap on the GPU race
    on that array."""
    n, m = U.shape
    _check(_load().xamg_coldot_noalloc(_ptr(U), _ptr(V), n, m, _ptr(out), _stream(stream)),
           "xamg_coldot_noalloc")


# ---- learned initial guess ----

def net_param_count() -> int:
    return int(_load().xamg_net_param_count())


def _bits(t):
    """Device address of a bf16 tensor passed as its uint16 bit patterns."""
    return None if t is None else _ptr(t)


def conv3d_bf16(x, w, bias=None, mask=None, relu=False, adjoint=False, stream=None):
    """xamg_conv3d_bf16 on channels-last bf16 tensors x [batch, N, N, N, c];
    w: float32 CUDA tensor [cout, 27, cin]. Returns the bf16 output tensor."""
    import torch
    batch, N = x.shape[0], x.shape[1]
    cout, _, cin = w.shape
    cres = cin if adjoint else cout
    out = torch.empty((batch, N, N, N, cres), dtype=torch.bfloat16, device=x.device)
    _check(_load().xamg_conv3d_bf16(_bits(x), _bits(mask), _ptr(w), _ptr(bias), _bits(out), batch, N,
                                    cin, cout, 1 if relu else 0, 1 if adjoint else 0,
                                    _stream(stream)), "xamg_conv3d_bf16")
    return out


def conv3d_bf16_wgrad(x, g, act=None, stream=None):
    """xamg_conv3d_bf16_wgrad: (dW [cout, 27, cin], db [cout]) as float32 CUDA tensors."""
    import torch
    batch, N, cin, cout = x.shape[0], x.shape[1], x.shape[-1], g.shape[-1]
    dw = torch.empty((cout, 27, cin), dtype=torch.float32, device=x.device)
    db = torch.empty(cout, dtype=torch.float32, device=x.device)
    _check(_load().xamg_conv3d_bf16_wgrad(_bits(x), _bits(g), _bits(act), _ptr(dw), _ptr(db), batch,
                                          N, cin, cout, _stream(stream)), "xamg_conv3d_bf16_wgrad")
    return dw, db


class Net:
    """Handle on the library's warm-start network (``xamg_net_create``)."""

    def __init__(self, N: int, max_batch: int):
        h = C.c_void_p()
        _check(_load().xamg_net_create(N, max_batch, C.byref(h)), "xamg_net_create")
        self._h = h
        self.N = N
        self.max_batch = max_batch
        self.nparams = net_param_count()

    def close(self):
        if getattr(self, "_h", None):
            _load().xamg_net_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, np.float32)
        assert p.size == self.nparams
        _check(_load().xamg_net_set_params(self._h, p.ctypes.data), "xamg_net_set_params")

    def get_params(self) -> np.ndarray:
        p = np.empty(self.nparams, np.float32)
        _check(_load().xamg_net_get_params(self._h, p.ctypes.data), "xamg_net_get_params")
        return p

    def forward(self, inp, out, stream=None):
        """inp: float32 CUDA [batch, N^3, 2]; out: float32 CUDA [batch, N^3]."""
        _check(_load().xamg_net_forward(self._h, _ptr(inp), _ptr(out), inp.shape[0], _stream(stream)),
               "xamg_net_forward")

    def loss_grad(self, inp, target, loss=LOSS_MSE, weight=None, stream=None):
        """(loss, flat float32 gradient) on one batch; weight: float32 CUDA [batch] or None."""
        g = np.empty(self.nparams, np.float32)
        lv = C.c_float()
        lo = NetLossT(loss, _ptr(weight))
        _check(_load().xamg_net_loss_grad(self._h, _ptr(inp), _ptr(target), inp.shape[0], C.byref(lo),
                                          C.byref(lv), g.ctypes.data, _stream(stream)),
               "xamg_net_loss_grad")
        return float(lv.value), g

    def train_step(self, inp, target, idx, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, loss=LOSS_MSE,
                   weight=None, stream=None, want_loss=True):
        """One Adam step on samples idx (int32 CUDA) of inp/target; weight:
        float32 CUDA [nsamples] or None."""
        opt = AdamT(lr, beta1, beta2, eps)
        lo = NetLossT(loss, _ptr(weight))
        lv = C.c_float()
        _check(_load().xamg_net_train_step(self._h, _ptr(inp), _ptr(target), inp.shape[0], _ptr(idx),
                                           idx.shape[0], C.byref(lo), C.byref(opt),
                                           C.byref(lv) if want_loss else None, _stream(stream)),
               "xamg_net_train_step")
        return float(lv.value) if want_loss else None

    def predict_x0(self, B, logk, X0, out_scale: float, stream=None):
        """X0 (float64 CUDA n x m) from B (float64 CUDA n x m) and logk (float32 CUDA n)."""
        _check(_load().xamg_net_predict_x0(self._h, _ptr(B), _ptr(logk), out_scale, _ptr(X0), B.shape[1],
                                           _stream(stream)), "xamg_net_predict_x0")


# ---- batched solve of many independent systems ----

class Batch:
    """Handle on ``xamg_batch_create``: the hierarchies (``Hierarchy``, on the
    device) of independent systems and their column counts; solves them
    together with ``solve``."""

    def __init__(self, hiers, ms, autotune: bool = True, use_graph: bool = True):
        L = _load()
        n = len(hiers)
        hs = (C.c_void_p * n)(*[h.handle.value for h in hiers])
        marr = (C.c_int32 * n)(*[int(m) for m in ms])
        o = BatchOptsT()
        L.xamg_batch_opts_default(C.byref(o))
        o.autotune = 1 if autotune else 0
        o.use_graph = 1 if use_graph else 0
        b = C.c_void_p()
        _check(L.xamg_batch_create(hs, marr, n, C.byref(o), C.byref(b)), "xamg_batch_create")
        self._h = b
        self._hiers = list(hiers)   # the hierarchies must outlive the batch
        self.ms = [int(m) for m in ms]

    def close(self):
        if getattr(self, "_h", None):
            _load().xamg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def info(self):
        a = C.c_int32(); t = C.c_int32(); w = C.c_int32(); by = C.c_int64()
        _check(_load().xamg_batch_info(self._h, C.byref(a), C.byref(t), C.byref(w), C.byref(by)),
               "xamg_batch_info")
        return dict(launches_per_iteration=a.value, ops_tuned=t.value, ops_wide=w.value,
                    workspace_bytes=by.value)

    def solve(self, Bs, Xs, tol=1e-8, maxit=200, stream=None):
        """xamg_batch_solve on lists of device blocks (torch float64 CUDA,
        n_s x m_s); returns one SolveStats per system (rc: the batch's code)."""
        n = len(self.ms)
        assert len(Bs) == n and len(Xs) == n
        bp = (C.c_void_p * n)(*[_ptr(B) for B in Bs])
        xp = (C.c_void_p * n)(*[_ptr(X) for X in Xs])
        stats = [SolveStats(m) for m in self.ms]
        arr = (StatsT * n)(*[st.struct() for st in stats])
        rc = _load().xamg_batch_solve(self._h, bp, xp, tol, maxit, _stream(stream), arr)
        _check(rc, "xamg_batch_solve", allow_positive=True)
        for st, a in zip(stats, arr):
            st.iterations, st.vcycles, st.rc = a.iterations, a.vcycles, rc
        return stats
