"""Python binding of the C ABI in include/leja.h (argument marshalling only).

PyTorch provides device memory and streams; every compute step runs in libleja.so's kernels.
Device arrays are torch CUDA tensors; host arrays are NumPy arrays.
"""
from __future__ import annotations

import ctypes
import dataclasses

import numpy as np

from . import _ffi
from ._ffi import (LL_EST_HUTCHINSON, LL_EST_HUTCHPP, LL_F32, LL_F64, LL_KERNEL_AUTO, LL_KERNEL_BAND, LL_KERNEL_GATHER, LL_KERNEL_TMA,  # noqa: F401
                   LL_PREC_DF64, LL_PREC_F32_MIXED, LL_PREC_F64, LL_PROBE_GAUSSIAN, LL_PROBE_RADEMACHER, LL_STREAM_G, LL_STREAM_POWER, LL_STREAM_S,
                   LL_SVAL_CENTER, LL_SVAL_HALF_LMAX)

PRECISIONS = {"f64": LL_PREC_F64, "df64": LL_PREC_DF64, "f32": LL_PREC_F32_MIXED}
PROBE_KINDS = {"rademacher": LL_PROBE_RADEMACHER, "gaussian": LL_PROBE_GAUSSIAN}
STEP_KERNELS = {"auto": LL_KERNEL_AUTO, "gather": LL_KERNEL_GATHER, "tma": LL_KERNEL_TMA, "band": LL_KERNEL_BAND}
ESTIMATORS = {"hutchpp": LL_EST_HUTCHPP, "hutchinson": LL_EST_HUTCHINSON}


class LejaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_ffi.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.name = _ffi.STATUS_NAMES.get(status, str(status))


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


class Handle:
    """Owns an ll_handle (device workspace and kept forward state) on the current device."""

    def __init__(self):
        self._lib = _ffi.load()
        h = ctypes.c_void_p()
        st = self._lib.ll_create(ctypes.byref(h))
        if st != 0:
            raise LejaError(st, "ll_create failed")
        self.ptr = h

    def check(self, st: int):
        if st != 0:
            msg = self._lib.ll_last_error(self.ptr)
            raise LejaError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ptr", None):
            self._lib.ll_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_step_config(self, kernel: str = "auto", threads_per_block: int = 0, rows_per_thread: int = 0):
        """Step kernel of ll_apply_poly and ll_logdet_backward on this handle."""
        self.check(self._lib.ll_set_step_config(self.ptr, STEP_KERNELS[kernel], threads_per_block, rows_per_thread))

    def set_adjoint_fusion(self, mode: str = "auto"):
        """The backward's gradient contraction fused into its reverse steps: "auto" (timed per
        shape), "on" or "off" (ll_set_adjoint_fusion)."""
        self.check(self._lib.ll_set_adjoint_fusion(self.ptr, FUSE_MODES[mode]))

    def set_keep_budget(self, nbytes: int = 0):
        """Device memory the forward may keep for the backward (0 = half the free memory)."""
        self.check(self._lib.ll_set_keep_budget(self.ptr, int(nbytes)))

    def trim(self):
        """Free the handle's device workspace (the kept forward state with it)."""
        self.check(self._lib.ll_trim_workspace(self.ptr))

    def debug_inject(self, what: str = "none"):
        """Test hook: "stall" makes the TMA step kernel's first-tile waits run out (LL_ERR_TIMEOUT)."""
        self.check(self._lib.ll_debug_inject(self.ptr, {"none": _ffi.LL_INJECT_NONE, "stall": _ffi.LL_INJECT_STALL}[what]))

    def info(self) -> dict:
        inf = _ffi.ll_info()
        self.check(self._lib.ll_get_info(self.ptr, ctypes.byref(inf)))
        return {f: getattr(inf, f) for f, _ in _ffi.ll_info._fields_}


@dataclasses.dataclass
class DeviceCSR:
    """A CSR matrix resident on the GPU (int32 indices; float64 or float32 values)."""

    n: int
    rowptr: object
    colind: object
    values: object

    @staticmethod
    def from_host(csr, dtype: str = "f64", device: str = "cuda") -> "DeviceCSR":
        torch = _torch()
        vt = torch.float64 if dtype == "f64" else torch.float32
        return DeviceCSR(n=int(csr.n),
                         rowptr=torch.as_tensor(np.asarray(csr.rowptr, dtype=np.int32)).to(device),
                         colind=torch.as_tensor(np.asarray(csr.colind, dtype=np.int32)).to(device),
                         values=torch.as_tensor(np.asarray(csr.values)).to(device=device, dtype=vt))

    @property
    def nnz(self) -> int:
        return int(self.colind.shape[0])

    def c(self) -> _ffi.ll_csr:
        torch = _torch()
        assert self.rowptr.dtype == torch.int32 and self.colind.dtype == torch.int32
        assert self.rowptr.is_contiguous() and self.colind.is_contiguous() and self.values.is_contiguous()
        dt = LL_F64 if self.values.dtype == torch.float64 else LL_F32
        return _ffi.ll_csr(self.n, self.nnz, self.rowptr.data_ptr(), self.colind.data_ptr(),
                           self.values.data_ptr(), dt)


def host_csr_struct(csr) -> tuple[_ffi.ll_csr, tuple]:
    """ll_csr over host NumPy arrays (kept alive by the returned tuple)."""
    rp = np.ascontiguousarray(csr.rowptr, dtype=np.int32)
    ci = np.ascontiguousarray(csr.colind, dtype=np.int32)
    va = np.ascontiguousarray(csr.values)
    dt = LL_F64 if va.dtype == np.float64 else LL_F32
    s = _ffi.ll_csr(int(csr.n), int(ci.shape[0]), rp.ctypes.data, ci.ctypes.data, va.ctypes.data, dt)
    return s, (rp, ci, va)


DD_SCHEMES = {"auto": _ffi.LL_DD_AUTO, "table_q": _ffi.LL_DD_TABLE_Q}
GRAM_METHODS = {"auto": _ffi.LL_GRAM_AUTO, "tensor": _ffi.LL_GRAM_TENSOR, "dfloat": _ffi.LL_GRAM_DFLOAT}
FUSE_MODES = {"auto": _ffi.LL_FUSE_AUTO, "on": _ffi.LL_FUSE_ON, "off": _ffi.LL_FUSE_OFF}
REORDERS = {"auto": _ffi.LL_REORDER_AUTO, "none": _ffi.LL_REORDER_NONE, "degree": _ffi.LL_REORDER_DEGREE}


def options(degree: int = 40, probes: int = 30, seed: int = 0, probe_kind: str = "rademacher",
            precision: str = "df64", sval_mode: int = LL_SVAL_CENTER, keep_for_backward: bool = False,
            rows_per_thread: int = 0, threads_per_block: int = 0, ckpt_stride: int = 0,
            use_graph: bool = True, timeout_cycles: int = 0, step_kernel: str = "auto",
            estimator: str = "hutchpp", tol: float = 0.0, dd_scheme: str = "auto",
            qr_gram: str = "auto", reorder: str = "auto") -> _ffi.ll_options:
    o = _ffi.ll_options()
    _ffi.load().ll_default_options(ctypes.byref(o))
    o.degree = degree
    o.probes = probes
    o.seed = seed
    o.probe_kind = PROBE_KINDS[probe_kind]
    o.precision = PRECISIONS[precision]
    o.sval_mode = sval_mode
    o.keep_for_backward = int(keep_for_backward)
    o.rows_per_thread = rows_per_thread
    o.threads_per_block = threads_per_block
    o.ckpt_stride = ckpt_stride
    o.use_graph = int(use_graph)
    o.timeout_cycles = timeout_cycles
    o.step_kernel = STEP_KERNELS[step_kernel]
    o.estimator = ESTIMATORS[estimator]
    o.tol = tol
    o.dd_scheme = DD_SCHEMES[dd_scheme]
    o.qr_gram = GRAM_METHODS[qr_gram]
    o.reorder = REORDERS[reorder]
    return o


# ------------------------------------------------------------------------------ host pieces

def ll_leja_points(count: int) -> np.ndarray:
    out = np.zeros(count, dtype=np.float64)
    st = _ffi.load().ll_leja_points(count, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != 0:
        raise LejaError(st, "ll_leja_points")
    return out


def ll_divided_differences(lmin: float, lmax: float, degree: int, sval_mode: int = LL_SVAL_CENTER):
    out = np.zeros(degree + 1, dtype=np.float64)
    terms = ctypes.c_int(0)
    st = _ffi.load().ll_divided_differences(_ffi.ll_bounds(lmin, lmax), degree, sval_mode,
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(terms))
    if st != 0:
        raise LejaError(st, "ll_divided_differences")
    return out, terms.value


def ll_divided_differences_q(lmin: float, lmax: float, degree: int) -> np.ndarray:
    """The Newton coefficients by the divided-difference table in binary128 on the host."""
    out = np.zeros(degree + 1, dtype=np.float64)
    st = _ffi.load().ll_divided_differences_q(_ffi.ll_bounds(lmin, lmax), degree,
                                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    if st != 0:
        raise LejaError(st, "ll_divided_differences_q")
    return out


# ---------------------------------------------------------------------------- device pieces

def ll_gershgorin(h: Handle, A: DeviceCSR, stream=None) -> tuple[float, float]:
    out = _ffi.ll_bounds()
    a = A.c()
    h.check(h._lib.ll_gershgorin(h.ptr, ctypes.byref(a), ctypes.byref(out), _stream_ptr(stream)))
    return out.lmin, out.lmax


def ll_power_lmax(h: Handle, A: DeviceCSR, iters: int = 20, seed: int = 0, stream=None) -> float:
    out = ctypes.c_double()
    a = A.c()
    h.check(h._lib.ll_power_lmax(h.ptr, ctypes.byref(a), iters, seed, ctypes.byref(out), _stream_ptr(stream)))
    return out.value


def ll_power_lmax_noalloc(A: DeviceCSR, iters: int = 20, seed: int = 0, stream=None) -> float:
    """ll_power_lmax without any device allocation and without a handle, for callers that
    cannot allocate device memory (their memory belongs to another allocator, or they cannot
    afford cudaMalloc's implicit synchronisation). At most 262,144 rows; calls share one
    library-owned scratch array, so calls that overlap on the GPU must be serialised."""
    out = ctypes.c_double()
    a = A.c()
    st = _ffi.load().ll_power_lmax_noalloc(ctypes.byref(a), iters, seed, ctypes.byref(out), _stream_ptr(stream))
    if st != 0:
        raise LejaError(st, "ll_power_lmax_noalloc")
    return out.value


def ll_probes(h: Handle, kind: str, seed: int, stream_id: int, n: int, cols: int, stream=None):
    torch = _torch()
    out = torch.empty((n, cols), dtype=torch.float64, device="cuda")
    h.check(h._lib.ll_probes(h.ptr, PROBE_KINDS[kind], seed, stream_id, n, cols, out.data_ptr(), cols,
                             _stream_ptr(stream)))
    return out


def ll_apply_poly(h: Handle, A: DeviceCSR, lmin: float, lmax: float, degree: int, V, precision: str = "f64",
                  stream=None):
    torch = _torch()
    assert V.dtype == torch.float64 and V.is_cuda and V.dim() == 2 and V.stride(1) == 1
    n, b = V.shape
    out = torch.empty((n, b), dtype=torch.float64, device=V.device)
    a = A.c()
    h.check(h._lib.ll_apply_poly(h.ptr, ctypes.byref(a), _ffi.ll_bounds(lmin, lmax), degree, PRECISIONS[precision],
                                 V.data_ptr(), V.stride(0), b, out.data_ptr(), b, _stream_ptr(stream)))
    return out


def ll_apply_poly_tol(h: Handle, A: DeviceCSR, lmin: float, lmax: float, degree: int, tol: float, V,
                      precision: str = "f64", stream=None):
    """Algorithm 2 with its stopping rule, column by column: (PV, final degree of every column)."""
    torch = _torch()
    assert V.dtype == torch.float64 and V.is_cuda and V.dim() == 2 and V.stride(1) == 1
    n, b = V.shape
    out = torch.empty((n, b), dtype=torch.float64, device=V.device)
    deg = (ctypes.c_int * max(b, 1))()
    a = A.c()
    h.check(h._lib.ll_apply_poly_tol(h.ptr, ctypes.byref(a), _ffi.ll_bounds(lmin, lmax), degree, tol,
                                     PRECISIONS[precision], V.data_ptr(), V.stride(0), b, out.data_ptr(), b, deg,
                                     _stream_ptr(stream)))
    return out, np.array(deg[:b], dtype=np.int64)


def ll_stop_degrees(h: Handle, pass_: int) -> np.ndarray:
    """Final degree of every column of pass 1 or 2 of the last forward."""
    cnt = ctypes.c_int()
    h.check(h._lib.ll_stop_degrees(h.ptr, pass_, None, 0, ctypes.byref(cnt)))
    buf = (ctypes.c_int * max(cnt.value, 1))()
    h.check(h._lib.ll_stop_degrees(h.ptr, pass_, buf, cnt.value, None))
    return np.array(buf[:cnt.value], dtype=np.int64)


def ll_logdet_forward(h: Handle, A: DeviceCSR, lmin: float, lmax: float, opts: _ffi.ll_options, stream=None) -> float:
    est = ctypes.c_double()
    a = A.c()
    h.check(h._lib.ll_logdet_forward(h.ptr, ctypes.byref(a), _ffi.ll_bounds(lmin, lmax), ctypes.byref(opts),
                                     ctypes.byref(est), _stream_ptr(stream)))
    return est.value


def ll_logdet_forward_host(h: Handle, csr, lmin: float, lmax: float, opts: _ffi.ll_options, stream=None) -> float:
    est = ctypes.c_double()
    a, keep = host_csr_struct(csr)
    h.check(h._lib.ll_logdet_forward_host(h.ptr, ctypes.byref(a), _ffi.ll_bounds(lmin, lmax), ctypes.byref(opts),
                                          ctypes.byref(est), _stream_ptr(stream)))
    del keep
    return est.value


def ll_logdet_backward(h: Handle, A: DeviceCSR, grad_output: float = 1.0, stream=None, through_qr: bool = False):
    """Gradient of the kept forward estimate with respect to the stored values: with Q and G'
    frozen, or (through_qr) with the derivative through the sketch's QR as well."""
    torch = _torch()
    g = torch.empty(A.nnz, dtype=torch.float64, device="cuda")
    a = A.c()
    fn = h._lib.ll_logdet_backward_qr if through_qr else h._lib.ll_logdet_backward
    h.check(fn(h.ptr, ctypes.byref(a), grad_output, g.data_ptr(), _stream_ptr(stream)))
    return g


def ll_param_grad(h: Handle, grad_values, dvalues, stream=None) -> np.ndarray:
    """sum_e grad_values[e] * dvalues[p, e] for every parameter p (dvalues: (nparams, nnz) FP64
    CUDA tensor of d a_e / d theta_p)."""
    torch = _torch()
    assert grad_values.dtype == torch.float64 and dvalues.dtype == torch.float64
    dv = dvalues.contiguous()
    if dv.dim() == 1:
        dv = dv[None, :]
    npar, nnz = dv.shape
    out = np.zeros(npar, dtype=np.float64)
    h.check(h._lib.ll_param_grad(h.ptr, grad_values.data_ptr(), dv.data_ptr(), nnz, nnz, npar,
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_ptr(stream)))
    return out


def ll_kept_basis(h: Handle, stream=None):
    """(Q, G') of the last forward with keep_for_backward, as FP64 torch tensors (copies)."""
    torch = _torch()
    n = ctypes.c_int64()
    kq = ctypes.c_int()
    kg = ctypes.c_int()
    h.check(h._lib.ll_kept_basis(h.ptr, None, 0, ctypes.byref(n), ctypes.byref(kq), ctypes.byref(kg), None))
    out = torch.empty((n.value, kq.value + kg.value), dtype=torch.float64, device="cuda")
    h.check(h._lib.ll_kept_basis(h.ptr, out.data_ptr(), kq.value + kg.value, None, None, None, _stream_ptr(stream)))
    return out[:, :kq.value], out[:, kq.value:]


def ll_logdet_batched(h: Handle, mats: list, bounds: list, opts: _ffi.ll_options, degrees=None, stream=None):
    """Independent estimates of several device CSR matrices (matrix i uses seed + i) with one
    persistent launch per pass."""
    count = len(mats)
    arr = (_ffi.ll_csr * count)(*[A.c() for A in mats])
    barr = (_ffi.ll_bounds * count)(*[_ffi.ll_bounds(lo, hi) for lo, hi in bounds])
    deg = None
    if degrees is not None:
        deg = (ctypes.c_int * count)(*[int(x) for x in degrees])
    out = np.zeros(count, dtype=np.float64)
    h.check(h._lib.ll_logdet_batched(h.ptr, arr, barr, count, ctypes.byref(opts), deg,
                                     out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _stream_ptr(stream)))
    return out


def ll_logdet_sweep(h: Handle, O: DeviceCSR, D, thetas, bounds: list, opts: _ffi.ll_options, degrees=None,
                    stream=None):
    """log det(diag(D) + theta O) for every theta of `thetas` (one block pass pair over all of them,
    the same probes for each). O: device CSR; D: CUDA FP64 tensor of n values; bounds: (lmin, lmax)
    of each theta's matrix; degrees: one per theta, or None for opts.degree."""
    torch = _torch()
    t = len(thetas)
    if not (isinstance(D, torch.Tensor) and D.is_cuda and D.dtype == torch.float64 and D.is_contiguous()
            and D.numel() == O.n):
        raise ValueError("D must be a contiguous CUDA float64 tensor of n values")
    if len(bounds) != t or (degrees is not None and len(degrees) != t):
        raise ValueError("one bound pair (and degree) per theta")
    th = np.ascontiguousarray(thetas, dtype=np.float64)
    barr = (_ffi.ll_bounds * t)(*[_ffi.ll_bounds(lo, hi) for lo, hi in bounds])
    deg = None
    if degrees is not None:
        deg = (ctypes.c_int * t)(*[int(x) for x in degrees])
    out = np.zeros(t, dtype=np.float64)
    h.check(h._lib.ll_logdet_sweep(h.ptr, ctypes.byref(O.c()), D.data_ptr(), t,
                                   th.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), barr, deg,
                                   ctypes.byref(opts), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   _stream_ptr(stream)))
    return out


def logdet_leja(A: DeviceCSR, bounds: tuple[float, float], degree: int, probes: int, seed: int,
                precision: str = "df64", probe_kind: str = "rademacher", handle: Handle | None = None) -> float:
    """logdet_leja(csr, bounds, degree, probes, seed) -> estimate (Algorithm 3)."""
    h = handle or Handle()
    return ll_logdet_forward(h, A, bounds[0], bounds[1],
                             options(degree=degree, probes=probes, seed=seed, precision=precision, probe_kind=probe_kind))


def ll_gram(h: Handle, X, Z=None, method: str = "auto", kx: int | None = None, stream=None):
    """X^T Z (X^T X when Z is None) by CholeskyQR2's Gram kernels (method "auto", "tensor" or
    "dfloat"). X is a CUDA float64 tensor n x kx, or a float32 tensor n x 2 ld holding a
    double-float block in the library's column-pair layout (then kx gives its width). Z: a CUDA
    float64 tensor n x kz or None. Returns a kx x kz (kx x kx) float64 tensor."""
    torch = _torch()
    n = X.shape[0]
    if X.dtype == torch.float64:
        kx, ldx, lay = X.shape[1], X.stride(0), LL_PREC_F64
    else:
        ldx, lay = X.shape[1] // 2, LL_PREC_DF64
    kz, ldz = (0, 0) if Z is None else (Z.shape[1], Z.stride(0))
    out = torch.empty((kx, kx if Z is None else kz), dtype=torch.float64, device="cuda")
    h.check(h._lib.ll_gram(h.ptr, lay, X.data_ptr(), ldx, kx, 0 if Z is None else Z.data_ptr(), ldz, kz, n,
                           GRAM_METHODS[method], out.data_ptr(), _stream_ptr(stream)))
    return out


def df64_block(x, ld: int | None = None):
    """The library's double-float column-pair layout of a float64 array x (n x k, host): a float32
    array n x 2 ld (ld even, >= k) whose 16 bytes of columns (2q, 2q+1) per row are
    (hi_2q, hi_2q+1, lo_2q, lo_2q+1), hi = float32(x), lo = float32(x - hi); pad columns zero."""
    x = np.asarray(x, dtype=np.float64)
    n, k = x.shape
    ld = ld or (k + (k & 1))
    hi = x.astype(np.float32)
    lo = (x - hi.astype(np.float64)).astype(np.float32)
    out = np.zeros((n, ld // 2, 4), dtype=np.float32)
    hp = np.zeros((n, ld), dtype=np.float32)
    lp = np.zeros((n, ld), dtype=np.float32)
    hp[:, :k], lp[:, :k] = hi, lo
    out[:, :, 0], out[:, :, 1] = hp[:, 0::2], hp[:, 1::2]
    out[:, :, 2], out[:, :, 3] = lp[:, 0::2], lp[:, 1::2]
    return out.reshape(n, 2 * ld)
