"""Thin ctypes binding of libfv (include/fv.h), same names as the C ABI.

Argument marshalling only: every step of the solver runs in the CUDA library.
Arrays are numpy (host) or torch CUDA tensors (device, zero copy, on the
handle's stream).  There is no fallback: if libfv.so is missing or cannot be
loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfv.so")

FV_OK, FV_EINVAL, FV_ENOMEM, FV_ECUDA, FV_ENONFINITE, FV_ETIMEOUT = range(6)
FV_FP64, FV_FP32_DEV = 0, 1
FV_BC_WALL, FV_BC_TRANSMISSIVE = 0, 1
FV_XFACE_GL, FV_XFACE_OR = 0, 1
FV_TILING_AUTO, FV_TILING_TILE, FV_TILING_STRIP = 0, 1, 2
STATUS_NAMES = {0: "FV_OK", 1: "FV_EINVAL", 2: "FV_ENOMEM", 3: "FV_ECUDA",
                4: "FV_ENONFINITE", 5: "FV_ETIMEOUT"}


class fv_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("x0", C.c_double), ("y0", C.c_double),
                ("dx", C.c_double), ("dy", C.c_double)]


class fv_eos(C.Structure):
    _fields_ = [("rho0", C.c_double), ("k0", C.c_double), ("gamma", C.c_double),
                ("g", C.c_double), ("eps_gas", C.c_double)]


class fv_bc(C.Structure):
    _fields_ = [("side", C.c_int32 * 4), ("solid", C.POINTER(C.c_uint8))]


class fv_diag(C.Structure):
    _fields_ = [("t", C.c_double), ("steps", C.c_int64), ("dt_next", C.c_double),
                ("mass", C.c_double), ("status", C.c_int32)]


class fv_adjoint_spec(C.Structure):
    _fields_ = [("nsteps", C.c_int32), ("cfl", C.c_double), ("ngauges", C.c_int32),
                ("gauges", C.POINTER(C.c_int64)), ("target", C.POINTER(C.c_double)),
                ("checkpoint_every", C.c_int32), ("m_series", C.POINTER(C.c_double)),
                ("nheights", C.c_int32), ("height_id", C.POINTER(C.c_int32)),
                ("dL_dh", C.POINTER(C.c_double))]


class fv_adjoint_info(C.Structure):
    _fields_ = [("loss", C.c_double), ("t", C.c_double), ("checkpoints", C.c_int32),
                ("recomputed_steps", C.c_int32), ("forward_ms", C.c_double),
                ("reverse_ms", C.c_double)]


class FvError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


if not os.path.exists(LIB_PATH):
    raise ImportError(f"libfv.so not built at {LIB_PATH}; run paper_1806_04960_gb300/build.py")
_lib = C.CDLL(LIB_PATH)
_H = C.c_void_p
_D = C.POINTER(C.c_double)
_lib.fv_create.argtypes = [C.POINTER(fv_grid), C.POINTER(fv_eos), C.POINTER(fv_bc), C.c_int,
                           C.c_void_p, C.POINTER(_H)]
_lib.fv_set_state.argtypes = [_H, C.c_void_p, C.c_int]
_lib.fv_step.argtypes = [_H, C.c_int32, C.c_double, _D]
_lib.fv_get_state.argtypes = [_H, C.c_void_p, C.c_int]
_lib.fv_step_timed.argtypes = [_H, C.c_int32, C.c_double, _D, _D]
_lib.fv_get_levels.argtypes = [_H, C.POINTER(C.c_int32)]
_lib.fv_get_diag.argtypes = [_H, C.POINTER(fv_diag)]
_lib.fv_destroy.argtypes = [_H]
_lib.fv_destroy.restype = None
_lib.fv_last_error.restype = C.c_char_p
_lib.fv_version.restype = C.c_char_p
for _f in ("fv_create", "fv_set_state", "fv_step", "fv_step_timed", "fv_get_state",
           "fv_get_levels", "fv_get_diag"):
    getattr(_lib, _f).restype = C.c_int

_lib.fv_host_xface.argtypes = [_D, _D, _D, _D, _D]
_lib.fv_host_yface.argtypes = [_D, _D, _D, _D, _D]
_lib.fv_host_xface.restype = C.c_int
_lib.fv_host_xface_or.argtypes = [_D, _D, _D, _D, _D]
_lib.fv_host_xface_or.restype = C.c_int
_lib.fv_host_cell_ops.argtypes = [_D]
_lib.fv_host_cell_ops_first_order.argtypes = [_D]
_lib.fv_host_cell_ops_first_order.restype = C.c_int
_lib.fv_step_static.argtypes = [C.POINTER(fv_grid), C.POINTER(fv_eos), C.POINTER(C.c_int32),
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p, _D]
_lib.fv_step_static.restype = C.c_int
_B = C.c_void_p
_lib.fv_batch_create.argtypes = [C.c_int32, C.POINTER(fv_grid), C.POINTER(fv_eos), C.POINTER(fv_bc),
                                 C.c_int, C.c_void_p, C.POINTER(_B)]
_lib.fv_batch_set_state.argtypes = [_B, C.c_int32, C.c_void_p, C.c_int]
_lib.fv_batch_step.argtypes = [_B, C.c_int32, C.c_double]
_lib.fv_batch_step_timed.argtypes = [_B, C.c_int32, C.c_double, _D]
_lib.fv_batch_tune.argtypes = [_B, C.c_double, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_int32)]
_lib.fv_batch_set_launch.argtypes = [_B, C.c_int32, C.c_int32, C.c_int32]
_lib.fv_batch_get_state.argtypes = [_B, C.c_int32, C.c_void_p, C.c_int]
_lib.fv_batch_get_diag.argtypes = [_B, C.c_int32, C.POINTER(fv_diag)]
_lib.fv_batch_size.argtypes = [_B]
_lib.fv_batch_size.restype = C.c_int32
_lib.fv_batch_destroy.argtypes = [_B]
_lib.fv_batch_destroy.restype = None
for _f in ("fv_batch_create", "fv_batch_set_state", "fv_batch_step", "fv_batch_step_timed",
           "fv_batch_get_state", "fv_batch_get_diag", "fv_batch_tune", "fv_batch_set_launch"):
    getattr(_lib, _f).restype = C.c_int
_lib.fv_host_cell_ops.restype = C.c_int
_lib.fv_host_yface.restype = C.c_int
_lib.fv_adjoint.argtypes = [_H, C.POINTER(fv_adjoint_spec), C.c_void_p, C.c_int,
                            C.POINTER(fv_adjoint_info)]
_lib.fv_adjoint.restype = C.c_int
_lib.fv_set_partition.argtypes = [_H, C.c_int32, C.c_int32]
_lib.fv_part_halo_bytes.argtypes = [_H, C.POINTER(C.c_int64)]
_lib.fv_part_rate.argtypes = [_H, C.c_void_p]
_lib.fv_part_set_rate.argtypes = [_H, C.c_void_p, C.c_int32]
_lib.fv_part_pack.argtypes = [_H, C.c_int32, C.c_void_p]
_lib.fv_part_unpack.argtypes = [_H, C.c_int32, C.c_void_p]
for _f in ("fv_set_partition", "fv_part_halo_bytes", "fv_part_rate", "fv_part_set_rate",
           "fv_part_pack", "fv_part_unpack", "fv_step_frozen", "fv_device_rcp"):
    getattr(_lib, _f).restype = C.c_int
_lib.fv_step_frozen.argtypes = [_H, C.c_int32, _D, C.POINTER(C.c_int32), C.c_int32,
                                C.POINTER(C.c_int64), _D]
_lib.fv_step_frozen.restype = C.c_int
_lib.fv_device_rcp.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]
_lib.fv_device_rcp.restype = C.c_int
_lib.fv_measure_fma_peak.argtypes = [C.c_int32, C.c_int32, _D, _D]
_lib.fv_measure_fma_peak.restype = C.c_int
_lib.fv_set_order.argtypes = [_H, C.c_int32]
_lib.fv_set_order.restype = C.c_int
_lib.fv_set_xface.argtypes = [_H, C.c_int32]
_lib.fv_set_xface.restype = C.c_int
_lib.fv_host_face_f32.argtypes = [C.c_int, _D, _D, _D, C.c_int, _D, _D]
_lib.fv_host_face_f32.restype = C.c_int
_lib.fv_set_strip_height.argtypes = [_H, C.c_int32]
_lib.fv_set_strip_height.restype = C.c_int
_lib.fv_tune.argtypes = [_H, C.POINTER(C.c_int32)]
_lib.fv_tune.restype = C.c_int
_lib.fv_set_tiling.argtypes = [_H, C.c_int32]
_lib.fv_set_tiling.restype = C.c_int
_lib.fv_host_yface_o1.argtypes = [_D, _D, C.c_double, _D, C.c_double, C.c_double, C.c_double,
                                  _D, _D]
_lib.fv_host_yface_o1.restype = C.c_int
_lib.fv_host_adjoint_step.argtypes = [C.POINTER(fv_grid), C.POINTER(fv_eos), C.POINTER(C.c_int32),
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                      C.c_void_p, C.c_int]
_lib.fv_host_adjoint_step.restype = C.c_int
_lib.fv_host_height_step.argtypes = [C.POINTER(fv_grid), C.POINTER(fv_eos), C.POINTER(C.c_int32),
                                     C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                     C.c_void_p, C.c_int, C.c_void_p, C.c_int]
_lib.fv_host_height_step.restype = C.c_int
_lib.fv_host_adj_check.argtypes = [C.c_int, _D, _D, _D, _D, _D, _D]
_lib.fv_host_adj_check.restype = C.c_int

ABI_SYMBOLS = ("fv_create", "fv_set_state", "fv_step", "fv_step_timed", "fv_get_state",
               "fv_get_levels",
               "fv_get_diag", "fv_destroy", "fv_last_error", "fv_version", "fv_host_xface",
               "fv_host_yface", "fv_host_cell_ops", "fv_host_cell_ops_first_order", "fv_host_adj_check", "fv_step_static", "fv_batch_create",
               "fv_batch_set_state", "fv_batch_step", "fv_batch_step_timed", "fv_batch_get_state",
               "fv_batch_get_diag", "fv_batch_size", "fv_batch_destroy", "fv_adjoint",
               "fv_host_adjoint_step", "fv_set_order", "fv_host_yface_o1",
               "fv_host_xface_or", "fv_set_xface", "fv_set_tiling", "fv_host_face_f32",
               "fv_set_strip_height", "fv_tune", "fv_host_height_step", "fv_batch_tune",
               "fv_batch_set_launch", "fv_measure_fma_peak", "fv_set_partition",
               "fv_part_halo_bytes", "fv_part_rate", "fv_part_set_rate", "fv_part_pack",
               "fv_part_unpack", "fv_step_frozen", "fv_device_rcp")


def _check(st):
    if st != FV_OK:
        raise FvError(st, _lib.fv_last_error().decode())


def fv_version() -> str:
    return _lib.fv_version().decode()


def fv_last_error() -> str:
    return _lib.fv_last_error().decode()


def _ptr(x):
    """(address, on_device) of a contiguous float64 numpy array or torch tensor."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise ValueError("state arrays must be C-contiguous float64")
        return x.ctypes.data, 0
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous():
            raise ValueError("state tensors must be contiguous float64")
        return x.data_ptr(), 1 if x.is_cuda else 0
    raise TypeError(f"unsupported array type {type(x)}")


def _host_face(fun, qm, qp, model):
    m = np.ascontiguousarray(model, dtype=np.float64)
    a = np.ascontiguousarray(qm, dtype=np.float64)
    b = np.ascontiguousarray(qp, dtype=np.float64)
    Dm, Dp = np.zeros(4), np.zeros(4)
    P = lambda x: x.ctypes.data_as(_D)
    _check(fun(P(m), P(a), P(b), P(Dm), P(Dp)) and FV_EINVAL)
    return Dm, Dp


def fv_host_xface(qm, qp, model):
    """Host evaluation of the kernels' x-face fluctuations (D-, D+)."""
    return _host_face(_lib.fv_host_xface, qm, qp, model)


def fv_host_xface_or(qm, qp, model):
    """Host evaluation of the kernels' Osher-Romberg x-face fluctuations."""
    return _host_face(_lib.fv_host_xface_or, qm, qp, model)


def fv_host_yface(qm, qp, model):
    """Host evaluation of the kernels' y-face fluctuations (D-, D+)."""
    return _host_face(_lib.fv_host_yface, qm, qp, model)


def fv_host_face_f32(which: int, qm, qp, model, paired: bool = True):
    """Host evaluation of an FP32 face solver (which = 0: x, 1: y) in the
    paired form of the FP32 kernels or in the scalar form (fv_host_face_f32)."""
    m = np.ascontiguousarray(model, dtype=np.float64)
    a = np.ascontiguousarray(qm, dtype=np.float64)
    b = np.ascontiguousarray(qp, dtype=np.float64)
    Dm, Dp = np.zeros(4), np.zeros(4)
    P = lambda x: x.ctypes.data_as(_D)
    _check(_lib.fv_host_face_f32(int(which), P(m), P(a), P(b), int(bool(paired)), P(Dm), P(Dp))
           and FV_EINVAL)
    return Dm, Dp


HOST_ADJ_SIZES = {0: (8, 8), 1: (8, 8), 2: (29, 22), 3: (23, 8)}


def fv_host_adj_check(which: int, model, k, x, lout=None):
    """Host value (and, with lout, reverse derivative d<lout, out>/dx) of one
    per-face or per-cell building block of the kernels (see fv_model_host.h)."""
    nin, nout = HOST_ADJ_SIZES[which]
    m = np.ascontiguousarray(model, dtype=np.float64)
    kk = np.ascontiguousarray(np.zeros(6) if k is None else k, dtype=np.float64)
    xi = np.ascontiguousarray(x, dtype=np.float64)
    assert xi.size == nin
    out = np.zeros(nout)
    P = lambda a: a.ctypes.data_as(_D)
    if lout is None:
        _check(_lib.fv_host_adj_check(which, P(m), P(kk), P(xi), None, P(out), None) and FV_EINVAL)
        return out
    lo = np.ascontiguousarray(lout, dtype=np.float64)
    assert lo.size == nout
    lin = np.zeros(nin)
    _check(_lib.fv_host_adj_check(which, P(m), P(kk), P(xi), P(lo), P(out), P(lin)) and FV_EINVAL)
    return out, lin


def fv_host_yface_o1(fa, aEa, fb, aEb, ya, dy, model):
    """Host evaluation of the kernels' first-order y face (D-, D+)."""
    m = np.ascontiguousarray(model, dtype=np.float64)
    a = np.ascontiguousarray(fa, dtype=np.float64)
    b = np.ascontiguousarray(fb, dtype=np.float64)
    Dm, Dp = np.zeros(4), np.zeros(4)
    P = lambda x: x.ctypes.data_as(_D)
    _check(_lib.fv_host_yface_o1(P(m), P(a), float(aEa), P(b), float(aEb), float(ya), float(dy),
                                 P(Dm), P(Dp)) and FV_EINVAL)
    return Dm, Dp


def fv_set_order(h, order: int) -> None:
    _check(_lib.fv_set_order(h, int(order)))


def fv_set_xface(h, solver: int) -> None:
    _check(_lib.fv_set_xface(h, int(solver)))


def fv_set_tiling(h, tiling: int) -> None:
    _check(_lib.fv_set_tiling(h, int(tiling)))


def fv_set_strip_height(h, rows: int) -> None:
    _check(_lib.fv_set_strip_height(h, int(rows)))


def fv_tune(h) -> int:
    rows = C.c_int32(0)
    _check(_lib.fv_tune(h, C.byref(rows)))
    return rows.value


def fv_host_cell_ops(first_order: bool = False) -> dict:
    """Operation counts of one cell-update of the kernels (see fv_model_host.h);
    first_order: a cell that the order switch advances at first order."""
    out = np.zeros(5)
    f = _lib.fv_host_cell_ops_first_order if first_order else _lib.fv_host_cell_ops
    _check(f(out.ctypes.data_as(_D)) and FV_EINVAL)
    names = ("add", "mul", "div", "sqrt", "cmp")
    d = {k: int(v) for k, v in zip(names, out)}
    d["flops"] = d["add"] + d["mul"] + d["div"] + d["sqrt"]
    return d


def _dev_addr(x) -> int:
    """Device address of a contiguous CUDA tensor (any dtype)."""
    if not (getattr(x, "is_cuda", False) and x.is_contiguous()):
        raise ValueError("expected a contiguous CUDA tensor")
    return x.data_ptr()


def fv_set_partition(h, own_lo: int, own_hi: int) -> None:
    _check(_lib.fv_set_partition(h, int(own_lo), int(own_hi)))


def fv_part_halo_bytes(h) -> int:
    n = C.c_int64(0)
    _check(_lib.fv_part_halo_bytes(h, C.byref(n)))
    return n.value


def fv_part_rate(h, rate_dev) -> None:
    _check(_lib.fv_part_rate(h, C.c_void_p(_dev_addr(rate_dev))))


def fv_part_set_rate(h, rates_dev) -> None:
    """Adopt the largest of the device doubles in ``rates_dev``."""
    _check(_lib.fv_part_set_rate(h, C.c_void_p(_dev_addr(rates_dev)), int(rates_dev.numel())))


def fv_part_pack(h, side: int, buf_dev) -> None:
    _check(_lib.fv_part_pack(h, int(side), C.c_void_p(_dev_addr(buf_dev))))


def fv_part_unpack(h, side: int, buf_dev) -> None:
    _check(_lib.fv_part_unpack(h, int(side), C.c_void_p(_dev_addr(buf_dev))))


def fv_step_frozen(h, dt, K, gauges=None):
    """len(dt) steps with the given dt (n,) and levels K (n, nx) (fv_step_frozen);
    returns alpha rho at the gauges after each step, (n, ngauges)."""
    dt = np.ascontiguousarray(dt, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.int32)
    n = dt.size
    g = np.ascontiguousarray([] if gauges is None else gauges, dtype=np.int64)
    m = np.zeros((max(n, 1), max(g.size, 1)))
    _check(_lib.fv_step_frozen(h, n, dt.ctypes.data_as(_D), K.ctypes.data_as(C.POINTER(C.c_int32)),
                               g.size, g.ctypes.data_as(C.POINTER(C.c_int64)) if g.size else None,
                               m.ctypes.data_as(_D) if g.size else None))
    return m[:n, :g.size]


def fv_device_rcp(x_dev, out_dev, stream: int = 0) -> None:
    """The FP64 device reciprocal at the doubles of x_dev (fv_device_rcp)."""
    _check(_lib.fv_device_rcp(C.c_void_p(_dev_addr(x_dev)), C.c_void_p(_dev_addr(out_dev)),
                              int(x_dev.numel()), C.c_void_p(stream)))


def fv_measure_fma_peak(kind: int, reps: int = 3):
    """Measured FMA peak of the current device: kind 0 FP32 FFMA, 1 FP32
    FFMA2, 2 FP64 DFMA.  Returns (TFLOP/s, fastest launch in ms)."""
    tf, ms = C.c_double(0.0), C.c_double(0.0)
    _check(_lib.fv_measure_fma_peak(int(kind), int(reps), C.byref(tf), C.byref(ms)))
    return tf.value, ms.value


def fv_create(grid: fv_grid, eos: fv_eos, bc: fv_bc, prec: int, stream: int = 0):
    h = _H()
    _check(_lib.fv_create(C.byref(grid), C.byref(eos), C.byref(bc), int(prec),
                          C.c_void_p(stream), C.byref(h)))
    return h


def fv_set_state(h, q) -> None:
    p, dev = _ptr(q)
    _check(_lib.fv_set_state(h, C.c_void_p(p), dev))


def fv_step(h, n: int, cfl: float, want_time: bool = False):
    if want_time:
        t = C.c_double(0.0)
        _check(_lib.fv_step(h, int(n), float(cfl), C.byref(t)))
        return t.value
    _check(_lib.fv_step(h, int(n), float(cfl), None))
    return None


def fv_step_timed(h, n: int, cfl: float):
    """(kernel_ms, total_ms) of n steps, timed with CUDA events on the stream."""
    k, t = C.c_double(0.0), C.c_double(0.0)
    _check(_lib.fv_step_timed(h, int(n), float(cfl), C.byref(k), C.byref(t)))
    return k.value, t.value


def fv_get_state(h, out) -> None:
    p, dev = _ptr(out)
    _check(_lib.fv_get_state(h, C.c_void_p(p), dev))


def fv_get_levels(h, nx: int) -> np.ndarray:
    K = np.zeros(nx, dtype=np.int32)
    _check(_lib.fv_get_levels(h, K.ctypes.data_as(C.POINTER(C.c_int32))))
    return K


def fv_get_diag(h) -> fv_diag:
    d = fv_diag()
    _check(_lib.fv_get_diag(h, C.byref(d)))
    return d


def fv_adjoint(h, nsteps: int, cfl: float, gauges, target, grad_out, checkpoint_every: int = 0,
               want_series: bool = False, height_id=None, nheights: int | None = None):
    """Gradient of the gauge loss (see fv.h) after ``nsteps`` steps with respect
    to the handle's current state, written to ``grad_out`` (4, ny, nx) float64
    (numpy or CUDA tensor), and with ``height_id`` ((ny, nx) int32, see
    ``cases.height_ids``) with respect to the obstacle heights.  Returns
    (fv_adjoint_info, m series (nsteps, ngauges) or None, dL/dh (nheights) or
    None)."""
    g = np.ascontiguousarray(gauges, dtype=np.int64)
    t = np.ascontiguousarray(target, dtype=np.float64)
    if t.size != int(nsteps) * g.size:
        raise ValueError("target must hold nsteps x ngauges values")
    series = np.zeros((int(nsteps), g.size)) if want_series else None
    hid, dh, nh = None, None, 0
    if height_id is not None:
        hid = np.ascontiguousarray(height_id, dtype=np.int32)
        nh = int(hid.max()) + 1 if nheights is None else int(nheights)
        dh = np.zeros(max(nh, 1))
    spec = fv_adjoint_spec(int(nsteps), float(cfl), int(g.size),
                           g.ctypes.data_as(C.POINTER(C.c_int64)), t.ctypes.data_as(_D),
                           int(checkpoint_every),
                           series.ctypes.data_as(_D) if want_series else None, nh,
                           hid.ctypes.data_as(C.POINTER(C.c_int32)) if nh > 0 else None,
                           dh.ctypes.data_as(_D) if nh > 0 else None)
    info = fv_adjoint_info()
    p, dev = _ptr(grad_out)
    _check(_lib.fv_adjoint(h, C.byref(spec), C.c_void_p(p), dev, C.byref(info)))
    return info, series, (dh[:nh] if height_id is not None else None)


def fv_destroy(h) -> None:
    _lib.fv_destroy(h)


class Solver:
    """Convenience wrapper: one handle for one case (see cases.Case)."""

    def __init__(self, case, prec: int = FV_FP64, stream: int | None = None):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:  # pragma: no cover
                stream = 0
        self.case = case
        self.prec = prec
        self.stream = stream
        self.grid = fv_grid(case.nx, case.ny, case.x0, case.y0, case.dx, case.dy)
        self.eos = fv_eos(case.rho0, case.k0, case.gamma, case.g, case.eps)
        self._solid = np.ascontiguousarray(case.solid, dtype=np.uint8)
        self.bc = fv_bc((C.c_int32 * 4)(*case.sides),
                        self._solid.ctypes.data_as(C.POINTER(C.c_uint8)))
        self.h = fv_create(self.grid, self.eos, self.bc, prec, stream)

    def set_state(self, q) -> None:
        if isinstance(q, np.ndarray):
            q = np.ascontiguousarray(q, dtype=np.float64)
        fv_set_state(self.h, q)

    def set_order(self, order: int) -> None:
        """Scheme of the following steps: 2 (default) or 1 (fv_set_order)."""
        fv_set_order(self.h, order)

    def set_xface(self, solver: int) -> None:
        """x-face viscosity: FV_XFACE_GL (default) or FV_XFACE_OR (fv_set_xface)."""
        fv_set_xface(self.h, solver)

    def set_tiling(self, tiling: int) -> None:
        """Step-kernel staging: FV_TILING_AUTO (default), FV_TILING_TILE or
        FV_TILING_STRIP (fv_set_tiling); the results are bitwise the same."""
        fv_set_tiling(self.h, tiling)

    def set_strip_height(self, rows: int) -> None:
        """Rows per strip of the strip kernel, 0 = built-in choice (fv_set_strip_height)."""
        fv_set_strip_height(self.h, rows)

    def tune(self) -> int:
        """Time the strip heights on the current state and keep the fastest
        (fv_tune); returns the chosen height."""
        return fv_tune(self.h)

    def step(self, n: int, cfl: float | None = None, want_time: bool = False):
        return fv_step(self.h, n, self.case.cfl if cfl is None else cfl, want_time)

    def step_timed(self, n: int, cfl: float | None = None):
        return fv_step_timed(self.h, n, self.case.cfl if cfl is None else cfl)

    def get_state(self, out=None):
        if out is None:
            out = np.empty((4, self.case.ny, self.case.nx), dtype=np.float64)
        fv_get_state(self.h, out)
        return out

    def levels(self) -> np.ndarray:
        return fv_get_levels(self.h, self.case.nx)

    def adjoint(self, nsteps: int, gauges, target, cfl: float | None = None,
                checkpoint_every: int = 0, grad=None, want_series: bool = False):
        """Gauge-loss gradient with respect to the current state (fv_adjoint);
        the handle advances by ``nsteps``.  Returns (grad, info, series)."""
        if grad is None:
            grad = np.empty((4, self.case.ny, self.case.nx), dtype=np.float64)
        info, series, _ = fv_adjoint(self.h, nsteps, self.case.cfl if cfl is None else cfl,
                                     gauges, target, grad, checkpoint_every, want_series)
        return grad, info, series

    def adjoint_heights(self, nsteps: int, gauges, target, height_id, cfl: float | None = None,
                        checkpoint_every: int = 0, grad=None, want_series: bool = False):
        """``adjoint`` plus the derivative with respect to the obstacle heights
        named by ``height_id`` (``cases.height_ids``; raising the obstacles, see
        fv.h).  Returns (grad, dL/dh (nheights), info, series)."""
        if grad is None:
            grad = np.empty((4, self.case.ny, self.case.nx), dtype=np.float64)
        info, series, dh = fv_adjoint(self.h, nsteps, self.case.cfl if cfl is None else cfl,
                                      gauges, target, grad, checkpoint_every, want_series,
                                      height_id=height_id)
        return grad, dh, info, series

    def record_free_run(self, nsteps: int, cfl: float | None = None):
        """Advance nsteps one at a time, recording the dt and levels each step
        used (the values fv_adjoint holds; input of step_frozen)."""
        cfl = self.case.cfl if cfl is None else cfl
        dts = np.zeros(nsteps)
        Ks = np.zeros((nsteps, self.case.nx), dtype=np.int32)
        fv_step(self.h, 0, cfl)
        for k in range(nsteps):
            Ks[k] = self.levels()
            dts[k] = self.diag().dt_next
            fv_step(self.h, 1, cfl)
        return dts, Ks

    def step_frozen(self, dt, K, gauges=None):
        """Steps with the given dt and levels (fv_step_frozen); returns the
        gauges' alpha rho after each step."""
        return fv_step_frozen(self.h, dt, K, gauges)

    def diag(self) -> fv_diag:
        return fv_get_diag(self.h)

    def close(self) -> None:
        if self.h:
            fv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Ensemble of independent cases advanced together (fv_batch_*)."""

    def __init__(self, case_list, prec: int = FV_FP64, stream: int | None = None):
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
            except ImportError:  # pragma: no cover
                stream = 0
        self.cases = list(case_list)
        n = len(self.cases)
        self._solids = [np.ascontiguousarray(c.solid, dtype=np.uint8) for c in self.cases]
        grids = (fv_grid * n)(*[fv_grid(c.nx, c.ny, c.x0, c.y0, c.dx, c.dy) for c in self.cases])
        eos = (fv_eos * n)(*[fv_eos(c.rho0, c.k0, c.gamma, c.g, c.eps) for c in self.cases])
        bcs = (fv_bc * n)(*[fv_bc((C.c_int32 * 4)(*c.sides), s.ctypes.data_as(C.POINTER(C.c_uint8)))
                            for c, s in zip(self.cases, self._solids)])
        self.b = _B()
        _check(_lib.fv_batch_create(n, grids, eos, bcs, int(prec), C.c_void_p(stream),
                                    C.byref(self.b)))

    def set_state(self, dom: int, q) -> None:
        if isinstance(q, np.ndarray):
            q = np.ascontiguousarray(q, dtype=np.float64)
        p, dev = _ptr(q)
        _check(_lib.fv_batch_set_state(self.b, int(dom), C.c_void_p(p), dev))

    def step(self, n: int, cfl: float) -> None:
        _check(_lib.fv_batch_step(self.b, int(n), float(cfl)))

    def step_timed(self, n: int, cfl: float) -> float:
        t = C.c_double(0.0)
        _check(_lib.fv_batch_step_timed(self.b, int(n), float(cfl), C.byref(t)))
        return t.value

    def set_launch(self, rows: int, order: int, persistent: int) -> None:
        """Fix the strip height, work order and launch form (fv_batch_set_launch)."""
        _check(_lib.fv_batch_set_launch(self.b, int(rows), int(order), int(persistent)))

    def tune(self, cfl: float) -> tuple:
        """Pick the fastest strip height, work order and launch form
        (fv_batch_tune); returns (rows, order, persistent)."""
        rows, order, pers = C.c_int32(0), C.c_int32(0), C.c_int32(0)
        _check(_lib.fv_batch_tune(self.b, float(cfl), C.byref(rows), C.byref(order),
                                  C.byref(pers)))
        return rows.value, order.value, pers.value

    def get_state(self, dom: int, out=None):
        c = self.cases[dom]
        if out is None:
            out = np.empty((4, c.ny, c.nx), dtype=np.float64)
        p, dev = _ptr(out)
        _check(_lib.fv_batch_get_state(self.b, int(dom), C.c_void_p(p), dev))
        return out

    def diag(self, dom: int) -> fv_diag:
        d = fv_diag()
        _check(_lib.fv_batch_get_diag(self.b, int(dom), C.byref(d)))
        return d

    def size(self) -> int:
        return int(_lib.fv_batch_size(self.b))

    def close(self) -> None:
        if self.b:
            _lib.fv_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def gauge_loss_function():
    """torch.autograd.Function computing the gauge loss of fv_adjoint from an
    initial state tensor; backward returns grad_output * dL/dQ0.

    Usage: L = gauge_loss_function().apply(q0, solver, nsteps, cfl, gauges,
    target) with q0 a (4, ny, nx) float64 CUDA tensor.  The forward call runs
    the steps and the reverse sweep together (fv_adjoint) and keeps the
    gradient; the solver's state is advanced by nsteps."""
    import torch

    class GaugeLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, q0, solver, nsteps, cfl, gauges, target):
            q0c = q0.detach().contiguous()
            solver.set_state(q0c)
            grad = torch.empty_like(q0c)
            info, _, _ = fv_adjoint(solver.h, nsteps, cfl, gauges, target, grad)
            ctx.save_for_backward(grad)
            return torch.tensor(info.loss, dtype=q0.dtype, device=q0.device)

        @staticmethod
        def backward(ctx, gout):
            (grad,) = ctx.saved_tensors
            return gout * grad, None, None, None, None, None

    return GaugeLoss
