"""ctypes binding of librdc (``include/rdc.h``): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the model: all work runs in librdc's CUDA kernels.  Host arrays
may be NumPy arrays or CPU torch tensors (for bfloat16); device pointers and
streams are plain integers (``tensor.data_ptr()``, ``stream.cuda_stream``).

The library must have been built (``paper_1901_06535_gb300.build.build()``);
importing this module without it raises immediately -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

RDC_OK = 0
RDC_EINVAL = 1
RDC_ENOMEM = 2
RDC_ECUDA = 3
RDC_ENONFINITE = 4
RDC_ETIMEOUT = 5
RDC_EUNSTABLE_WARN = 6
RDC_EUNSUPPORTED = 7

RDC_F32 = 0
RDC_F64 = 1
RDC_F32_BF16STORE = 2
RDC_F32_F16STORE = 3

RDC_DTYPE_F32 = 0
RDC_DTYPE_F64 = 1
RDC_DTYPE_BF16 = 2
RDC_DTYPE_F16 = 3

RDC_DIFFUSION_ONLY = 1
RDC_REACTION_ONLY = 2
RDC_STOCH_ROUND = 4

PRECISION_NAMES = {"f32": RDC_F32, "f64": RDC_F64, "bf16": RDC_F32_BF16STORE,
                   "f16": RDC_F32_F16STORE}


class rdc_grid(ctypes.Structure):
    _fields_ = [("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class rdc_params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("f", ctypes.c_double),
                ("q", ctypes.c_double), ("Du", ctypes.c_double),
                ("dt", ctypes.c_double), ("dx", ctypes.c_double),
                ("precision", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("k_block", ctypes.c_int32), ("round_seed", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rdc_view(ctypes.Structure):
    _fields_ = [("u", ctypes.c_void_p), ("v", ctypes.c_void_p),
                ("phi", ctypes.c_void_p), ("pitch_bytes", ctypes.c_size_t),
                ("phi_pitch_bytes", ctypes.c_size_t), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("elem_bytes", ctypes.c_int32), ("steps_done", ctypes.c_int64),
                ("launches", ctypes.c_int64), ("stream", ctypes.c_void_p),
                ("unstable", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("stability_rho", ctypes.c_double)]


class rdc_launch_shape(ctypes.Structure):
    _fields_ = [("bx", ctypes.c_int32), ("rows", ctypes.c_int32),
                ("tx", ctypes.c_int32), ("ty", ctypes.c_int32),
                ("nthreads", ctypes.c_int32), ("k", ctypes.c_int32),
                ("variant", ctypes.c_int32), ("krows", ctypes.c_int32)]


class rdc_batch_info(ctypes.Structure):
    _fields_ = [("ngrids", ctypes.c_int32), ("slots", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("k", ctypes.c_int32),
                ("rows", ctypes.c_int32), ("krows", ctypes.c_int32),
                ("graphs", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("total_cells", ctypes.c_double), ("launches", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64), ("cells_stepped", ctypes.c_double),
                ("tuned_gcups", ctypes.c_double), ("stream", ctypes.c_void_p)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class rdc_division_report(ctypes.Structure):
    _fields_ = [("checked", ctypes.c_uint64 * 3), ("mismatches", ctypes.c_uint64 * 3),
                ("first_bad", ctypes.c_uint32 * 3), ("reserved", ctypes.c_uint32)]

    def as_dict(self):
        return {"checked": list(self.checked), "mismatches": list(self.mismatches),
                "first_bad": list(self.first_bad)}


class RdcError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = f"{where}: {rdc_status_str(status)}"
        last = rdc_last_error()
        if last:
            msg += f" [{last}]"
        super().__init__(msg)


_LIB = None
_LOCK = threading.Lock()

# C signatures: name -> (restype, argtypes)
_P = ctypes.c_void_p
_SIGS = {
    "rdc_params_default": (ctypes.c_int, [ctypes.POINTER(rdc_params)]),
    "rdc_create": (ctypes.c_int, [rdc_grid, ctypes.POINTER(rdc_params), _P, _P, ctypes.POINTER(_P)]),
    "rdc_create_f64phi": (ctypes.c_int, [rdc_grid, ctypes.POINTER(rdc_params), _P, _P, ctypes.POINTER(_P)]),
    "rdc_create_ext": (ctypes.c_int, [rdc_grid, ctypes.POINTER(rdc_params), ctypes.POINTER(_P),
                                      ctypes.POINTER(_P), _P, ctypes.c_size_t, _P, ctypes.POINTER(_P)]),
    "rdc_destroy": (None, [_P]),
    "rdc_set_phi": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "rdc_reset_rest": (ctypes.c_int, [_P]),
    "rdc_set_step_index": (ctypes.c_int, [_P, ctypes.c_int64]),
    "rdc_seed": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double]),
    "rdc_set_state": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
    "rdc_step": (ctypes.c_int, [_P, ctypes.c_int64]),
    "rdc_read": (ctypes.c_int, [_P, _P, _P, ctypes.c_int32]),
    "rdc_check": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "rdc_probe": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P]),
    "rdc_get_rows": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_size_t]),
    "rdc_put_rows": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, _P, _P, ctypes.c_size_t]),
    "rdc_sync": (ctypes.c_int, [_P]),
    "rdc_rest_state": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                      ctypes.POINTER(ctypes.c_double)]),
    "rdc_stability": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_double)]),
    "rdc_get_view": (ctypes.c_int, [_P, ctypes.POINTER(rdc_view)]),
    "rdc_get_shape": (ctypes.c_int, [_P, ctypes.POINTER(rdc_launch_shape)]),
    "rdc_set_shape": (ctypes.c_int, [_P, ctypes.POINTER(rdc_launch_shape)]),
    "rdc_step_noalloc": (ctypes.c_int, [rdc_grid, ctypes.POINTER(rdc_params), _P, _P, _P, _P, _P,
                                        ctypes.c_size_t, ctypes.c_int64, _P,
                                        ctypes.POINTER(ctypes.c_int64)]),
    "rdc_batch_create": (ctypes.c_int, [ctypes.c_int32, _P, ctypes.POINTER(rdc_params), _P, _P,
                                        ctypes.POINTER(_P)]),
    "rdc_batch_add": (ctypes.c_int, [_P, rdc_grid, ctypes.POINTER(rdc_params), _P,
                                     ctypes.POINTER(ctypes.c_int32)]),
    "rdc_batch_remove": (ctypes.c_int, [_P, ctypes.c_int32]),
    "rdc_batch_destroy": (None, [_P]),
    "rdc_batch_seed": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                      ctypes.c_double, ctypes.c_double]),
    "rdc_batch_set_state": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32]),
    "rdc_batch_set_step_index": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int64]),
    "rdc_batch_step": (ctypes.c_int, [_P, _P, ctypes.c_int32, ctypes.c_int64]),
    "rdc_batch_check": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "rdc_batch_read": (ctypes.c_int, [_P, ctypes.c_int32, _P, _P, ctypes.c_int32]),
    "rdc_batch_sync": (ctypes.c_int, [_P]),
    "rdc_batch_set_config": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            ctypes.c_int32]),
    "rdc_batch_get_info": (ctypes.c_int, [_P, ctypes.POINTER(rdc_batch_info)]),
    "rdc_batch_get_grid": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(rdc_grid)]),
    "rdc_batch_stability": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]),
    "rdc_batch_tune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(rdc_batch_info)]),
    "rdc_tune": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.POINTER(rdc_launch_shape),
                                ctypes.POINTER(ctypes.c_double)]),
    "rdc_snap_segment": (ctypes.c_int, [ctypes.c_double] * 5 +
                         [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    "rdc_draw_line": (ctypes.c_int, [_P] + [ctypes.c_double] * 7),
    "rdc_fill_phi": (ctypes.c_int, [_P, ctypes.c_double]),
    "rdc_read_phi": (ctypes.c_int, [_P, _P, ctypes.c_int32]),
    "rdc_render": (ctypes.c_int, [_P, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                  ctypes.c_double, _P, ctypes.c_int32]),
    "rdc_timelapse_record": (ctypes.c_int, [_P, ctypes.c_int32]),
    "rdc_check_division": (ctypes.c_int, [ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64,
                                          ctypes.POINTER(rdc_division_report)]),
    "rdc_stoch_round_sample": (ctypes.c_int, [ctypes.c_int32, ctypes.c_uint32, ctypes.c_int64,
                                              ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                              _P, _P, _P]),
    "rdc_philox_sample": (ctypes.c_int, [ctypes.c_int32, _P, _P, _P]),
    "rdc_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "rdc_last_error": (ctypes.c_char_p, []),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded librdc (raises if it has not been built)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(
                    f"librdc.so is not built at {path}; call "
                    "paper_1901_06535_gb300.build.build() (needs nvcc)")
            L = ctypes.CDLL(path)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
        return _LIB


def exported_symbols():
    return list(_SIGS)


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------

def _host_ptr(a, what: str):
    """(pointer, dtype code, shape) of a C-contiguous host array or tensor."""
    if a is None:
        return None, None, None
    if hasattr(a, "data_ptr") and hasattr(a, "is_contiguous"):   # torch tensor
        import torch
        if a.is_cuda:
            raise ValueError(f"{what}: expected a host tensor")
        if not a.is_contiguous():
            raise ValueError(f"{what}: tensor must be contiguous")
        codes = {torch.float32: RDC_DTYPE_F32, torch.float64: RDC_DTYPE_F64,
                 torch.bfloat16: RDC_DTYPE_BF16, torch.float16: RDC_DTYPE_F16}
        if a.dtype not in codes:
            raise ValueError(f"{what}: unsupported dtype {a.dtype}")
        return a.data_ptr(), codes[a.dtype], tuple(a.shape)
    a = np.asarray(a)
    if not a.flags.c_contiguous:
        raise ValueError(f"{what}: array must be C-contiguous")
    codes = {np.dtype(np.float32): RDC_DTYPE_F32, np.dtype(np.float64): RDC_DTYPE_F64,
             np.dtype(np.float16): RDC_DTYPE_F16}
    if a.dtype not in codes:
        raise ValueError(f"{what}: unsupported dtype {a.dtype}")
    return a.ctypes.data, codes[a.dtype], a.shape


def _check_cells(shape, width: int, height: int, what: str):
    """A host array handed to the library must hold exactly one value per
    cell (the library reads or writes width * height of them)."""
    if shape is not None and int(np.prod(shape)) != width * height:
        raise ValueError(f"{what}: {tuple(shape)} holds {int(np.prod(shape))} values, "
                         f"the grid has {height} x {width} cells")


def _same_code(cu, cv, what: str):
    if cu is not None and cv is not None and cu != cv:
        raise ValueError(f"{what} must have the same dtype")
    return cu if cu is not None else cv


CUDA_STREAM_LEGACY = 0x1


def _stream(stream):
    """None -> NULL (a library-owned stream).  0, torch's handle for the
    default stream, maps to cudaStreamLegacy so that the work stays ordered
    with it instead of silently going to a private stream."""
    if stream is None:
        return None
    s = int(stream)
    return CUDA_STREAM_LEGACY if s == 0 else s


def _chk(rc: int, where: str, allow=()):
    if rc != RDC_OK and rc not in allow:
        raise RdcError(rc, where)
    return rc


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------

def rdc_status_str(rc: int) -> str:
    return lib().rdc_status_str(int(rc)).decode()


def rdc_last_error() -> str:
    return lib().rdc_last_error().decode()


def rdc_params_default(**overrides) -> rdc_params:
    p = rdc_params()
    _chk(lib().rdc_params_default(ctypes.byref(p)), "rdc_params_default")
    fields = {f for f, _ in p._fields_}
    for k, v in overrides.items():
        if k not in fields:
            raise TypeError(f"rdc_params has no field {k!r}")
        if k == "precision" and isinstance(v, str):
            v = PRECISION_NAMES[v]
        if k == "round_seed":
            v = ctypes.c_int32(int(v) & 0xFFFFFFFF).value   # an unsigned 32-bit key
        setattr(p, k, v)
    return p


def rdc_create(width: int, height: int, params: rdc_params, phi=None, stream=None):
    """Returns an opaque handle (int).  phi: H x W float32 (or float64, which
    routes to rdc_create_f64phi) host array, or None for uniform phi_active."""
    h = _P()
    g = rdc_grid(int(width), int(height))
    if phi is None:
        rc = lib().rdc_create(g, ctypes.byref(params), None, _stream(stream), ctypes.byref(h))
        _chk(rc, "rdc_create")
        return h.value
    ptr, code, shape = _host_ptr(phi, "phi")
    if shape != (height, width):
        raise ValueError(f"phi shape {shape} != ({height}, {width})")
    if code == RDC_DTYPE_F32:
        rc = lib().rdc_create(g, ctypes.byref(params), ptr, _stream(stream), ctypes.byref(h))
    elif code == RDC_DTYPE_F64:
        rc = lib().rdc_create_f64phi(g, ctypes.byref(params), ptr, _stream(stream), ctypes.byref(h))
    else:
        raise ValueError("phi must be float32 or float64")
    _chk(rc, "rdc_create")
    return h.value


def rdc_create_f64phi(width: int, height: int, params: rdc_params, phi, stream=None):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    return rdc_create(width, height, params, phi, stream)


def rdc_create_ext(width: int, height: int, params: rdc_params, dev_u, dev_v, dev_phi,
                   pitch_bytes: int, stream=None):
    """dev_u, dev_v: pairs of device pointers (ints); dev_phi a device pointer."""
    h = _P()
    U = (_P * 2)(*[int(x) for x in dev_u])
    V = (_P * 2)(*[int(x) for x in dev_v])
    rc = lib().rdc_create_ext(rdc_grid(int(width), int(height)), ctypes.byref(params), U, V,
                              int(dev_phi), int(pitch_bytes), _stream(stream), ctypes.byref(h))
    _chk(rc, "rdc_create_ext")
    return h.value


def rdc_destroy(h) -> None:
    if h:
        lib().rdc_destroy(h)


def rdc_set_phi(h, phi) -> int:
    ptr, code, shape = _host_ptr(phi, "phi")
    view = rdc_get_view(h)
    _check_cells(shape, view.width, view.height, "phi")
    return _chk(lib().rdc_set_phi(h, ptr, code), "rdc_set_phi")


def rdc_reset_rest(h) -> int:
    return _chk(lib().rdc_reset_rest(h), "rdc_reset_rest")


def rdc_set_step_index(h, n: int) -> int:
    return _chk(lib().rdc_set_step_index(h, int(n)), "rdc_set_step_index")


def rdc_batch_set_step_index(b, idx: int, n: int) -> int:
    return _chk(lib().rdc_batch_set_step_index(b, int(idx), int(n)), "rdc_batch_set_step_index")


def rdc_seed(h, cx: float, cy: float, r: float, value: float) -> int:
    return _chk(lib().rdc_seed(h, float(cx), float(cy), float(r), float(value)), "rdc_seed")


def rdc_set_state(h, u=None, v=None) -> int:
    pu, cu, su = _host_ptr(u, "u")
    pv, cv, sv = _host_ptr(v, "v")
    code = _same_code(cu, cv, "u and v")
    if code is None:
        return RDC_OK
    view = rdc_get_view(h)
    _check_cells(su, view.width, view.height, "u")
    _check_cells(sv, view.width, view.height, "v")
    return _chk(lib().rdc_set_state(h, pu, pv, code), "rdc_set_state")


def rdc_step(h, n: int) -> int:
    return _chk(lib().rdc_step(h, int(n)), "rdc_step")


def rdc_read(h, u_out=None, v_out=None):
    """Fills caller-owned host arrays (same dtype); returns the status
    (RDC_OK or RDC_ENONFINITE)."""
    pu, cu, su = _host_ptr(u_out, "u_out")
    pv, cv, sv = _host_ptr(v_out, "v_out")
    code = _same_code(cu, cv, "u_out and v_out")
    if code is None:
        code = RDC_DTYPE_F64
    else:
        view = rdc_get_view(h)
        _check_cells(su, view.width, view.height, "u_out")
        _check_cells(sv, view.width, view.height, "v_out")
    return _chk(lib().rdc_read(h, pu, pv, code), "rdc_read", allow=(RDC_ENONFINITE,))


def rdc_check(h):
    """(status, first_bad_flat_index or -1)."""
    fb = ctypes.c_int64(-1)
    rc = _chk(lib().rdc_check(h, ctypes.byref(fb)), "rdc_check", allow=(RDC_ENONFINITE,))
    return rc, fb.value


def rdc_probe(h, cells) -> np.ndarray:
    """u at the given flat cell indices (any shape), as a flat float64 array."""
    c = np.ascontiguousarray(cells, dtype=np.int64).ravel()
    out = np.empty(c.size, dtype=np.float64)
    _chk(lib().rdc_probe(h, c.size, c.ctypes.data, out.ctypes.data), "rdc_probe")
    return out


def _rows_buf(x, nbytes: int, elem_bytes: int, name: str):
    """Address of a row buffer: an int (device or host pointer), an object
    with data_ptr() (a torch tensor), or a C-contiguous numpy array of the
    storage element size holding at least nbytes."""
    if x is None:
        return None
    if isinstance(x, (int, np.integer)):
        return int(x)
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous or x.dtype.itemsize != elem_bytes or x.nbytes < nbytes:
            raise ValueError(f"{name}: need a C-contiguous array of {elem_bytes}-byte elements "
                             f"holding {nbytes} bytes")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    raise TypeError(f"{name}: pointer, numpy array or tensor expected")


def _rows_call(fn, h, row0, nrows, u, v, pitch_bytes, what):
    view = rdc_get_view(h)
    row = int(pitch_bytes) or view.width * view.elem_bytes
    need = max(int(nrows) - 1, 0) * row + view.width * view.elem_bytes if nrows > 0 else 0
    pu = _rows_buf(u, need, view.elem_bytes, "u")
    pv = _rows_buf(v, need, view.elem_bytes, "v")
    _chk(fn(h, int(row0), int(nrows), pu, pv, int(pitch_bytes)), what)
    if isinstance(u, np.ndarray) or isinstance(v, np.ndarray):
        rdc_sync(h)  # a host array is complete (get) or free to reuse (put) on return


def rdc_get_rows(h, row0: int, nrows: int, u_dst=None, v_dst=None, pitch_bytes: int = 0):
    """Copies rows [row0, row0 + nrows) of the current u and v into u_dst and
    v_dst (storage type; pitch_bytes 0 = packed rows).  Buffers are pointers
    (ints), tensors, or numpy arrays (then the call waits for the copy)."""
    _rows_call(lib().rdc_get_rows, h, row0, nrows, u_dst, v_dst, pitch_bytes, "rdc_get_rows")


def rdc_put_rows(h, row0: int, nrows: int, u_src=None, v_src=None, pitch_bytes: int = 0):
    """Writes rows [row0, row0 + nrows) of the current u and v from u_src and
    v_src (the layout of rdc_get_rows)."""
    _rows_call(lib().rdc_put_rows, h, row0, nrows, u_src, v_src, pitch_bytes, "rdc_put_rows")


def rdc_sync(h) -> int:
    return _chk(lib().rdc_sync(h), "rdc_sync")


def rdc_rest_state(phi: float, f: float, q: float) -> float:
    out = ctypes.c_double()
    _chk(lib().rdc_rest_state(float(phi), float(f), float(q), ctypes.byref(out)), "rdc_rest_state")
    return out.value


def rdc_stability(h):
    """(status, rho) with status RDC_OK or RDC_EUNSTABLE_WARN."""
    rho = ctypes.c_double()
    rc = _chk(lib().rdc_stability(h, ctypes.byref(rho)), "rdc_stability",
              allow=(RDC_EUNSTABLE_WARN,))
    return rc, rho.value


def rdc_get_view(h) -> rdc_view:
    v = rdc_view()
    _chk(lib().rdc_get_view(h, ctypes.byref(v)), "rdc_get_view")
    return v


def rdc_check_division(q: float = 0.002, n_random: int = 1 << 26, seed: int = 1) -> dict:
    """Exhaustive device check of the FP32 division used by the kernels
    (see include/rdc.h); returns checked / mismatches / first_bad per part."""
    rep = rdc_division_report()
    _chk(lib().rdc_check_division(float(q), int(n_random), int(seed), ctypes.byref(rep)),
         "rdc_check_division")
    return rep.as_dict()


def rdc_stoch_round_sample(precision, seed: int, step: int, row: int, col0: int, x):
    """Rounds each float32 x[i] as the step kernels round the new u and v of
    cell (col0 + i, row) writing state `step` under RDC_STOCH_ROUND with key
    `seed`; returns (u, v) float32 arrays (widened back from 16 bits)."""
    if isinstance(precision, str):
        precision = PRECISION_NAMES[precision]
    x = np.ascontiguousarray(x, dtype=np.float32).ravel()
    u = np.empty_like(x)
    v = np.empty_like(x)
    _chk(lib().rdc_stoch_round_sample(int(precision), int(seed) & 0xFFFFFFFF, int(step),
                                      int(row), int(col0), int(x.size),
                                      x.ctypes.data, u.ctypes.data, v.ctypes.data),
         "rdc_stoch_round_sample")
    return u, v


def rdc_philox_sample(ctr, key):
    """Philox4x32-10 on the device, as the step kernels compute it: ctr is an
    (n, 4) array of counters, key an (n, 2) array of keys (32-bit words);
    returns the (n, 4) uint32 outputs."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32).reshape(-1, 4)
    k = np.ascontiguousarray(key, dtype=np.uint32).reshape(-1, 2)
    if c.shape[0] != k.shape[0]:
        raise ValueError("one key per counter")
    out = np.empty_like(c)
    _chk(lib().rdc_philox_sample(int(c.shape[0]), c.ctypes.data, k.ctypes.data,
                                 out.ctypes.data), "rdc_philox_sample")
    return out


def rdc_step_noalloc(width: int, height: int, params: rdc_params, u_in: int, v_in: int,
                     phi: int, u_out: int, v_out: int, pitch_bytes: int, n: int,
                     stream=None, check: bool = True):
    """Allocation-free stepping of caller-owned device buffers (pointers as
    ints).  Returns (status, first_bad); with check=False the health check is
    skipped and the call stays asynchronous."""
    fb = ctypes.c_int64(-1)
    s = _stream(stream)
    rc = lib().rdc_step_noalloc(rdc_grid(int(width), int(height)), ctypes.byref(params),
                                int(u_in), int(v_in), int(phi), int(u_out), int(v_out),
                                int(pitch_bytes), int(n), None if s == CUDA_STREAM_LEGACY else s,
                                ctypes.byref(fb) if check else None)
    _chk(rc, "rdc_step_noalloc", allow=(RDC_ENONFINITE,))
    return rc, fb.value


RDC_WIDTH_PERMEABLE = 2
RDC_WIDTH_SEMIPERMEABLE = 3
RDC_WIDTH_IMPERMEABLE = 8
RDC_SNAP_DEGREES = 15.0


def rdc_snap_segment(x0, y0, x1, y1, snap_deg=RDC_SNAP_DEGREES):
    a = ctypes.c_double()
    b = ctypes.c_double()
    _chk(lib().rdc_snap_segment(float(x0), float(y0), float(x1), float(y1), float(snap_deg),
                                ctypes.byref(a), ctypes.byref(b)), "rdc_snap_segment")
    return a.value, b.value


def rdc_draw_line(h, x0, y0, x1, y1, width, value, snap_deg=0.0) -> int:
    return _chk(lib().rdc_draw_line(h, float(x0), float(y0), float(x1), float(y1), float(width),
                                    float(value), float(snap_deg)), "rdc_draw_line")


def rdc_read_phi(h, dtype=np.float64) -> np.ndarray:
    view = rdc_get_view(h)
    out = np.empty((view.height, view.width), dtype=dtype)
    ptr, code, _ = _host_ptr(out, "out")
    _chk(lib().rdc_read_phi(h, ptr, code), "rdc_read_phi")
    return out


def rdc_fill_phi(h, value) -> int:
    return _chk(lib().rdc_fill_phi(h, float(value)), "rdc_fill_phi")


RDC_RENDER_SNAPSHOT = 0
RDC_RENDER_TIMELAPSE = 1


def rdc_render(h, what: int = RDC_RENDER_SNAPSHOT, u_scale: float = 1.0, v_scale: float = 1.0,
               phi_threshold: float = 0.07575, out=None):
    """RGBA8 image as an (H, W, 4) uint8 array (a new host array unless `out`
    -- a host array or a CUDA tensor -- is given)."""
    view = rdc_get_view(h)
    if out is None:
        out = np.empty((view.height, view.width, 4), dtype=np.uint8)
    on_dev = 1 if (hasattr(out, "is_cuda") and out.is_cuda) else 0
    if hasattr(out, "data_ptr"):                       # torch tensor, host or device
        ok = out.is_contiguous()
        nbytes = out.numel() * out.element_size()
        ptr = out.data_ptr()
    else:
        out = np.asarray(out)
        ok = out.flags.c_contiguous
        nbytes = out.nbytes
        ptr = out.ctypes.data
    if not ok or nbytes != view.width * view.height * 4:
        raise ValueError(f"out: must be a contiguous buffer of {view.height} x {view.width} "
                         f"x 4 bytes, got {nbytes} bytes")
    _chk(lib().rdc_render(h, int(what), float(u_scale), float(v_scale), float(phi_threshold),
                          ptr, on_dev), "rdc_render")
    return out


def rdc_timelapse_record(h, reset: bool = False) -> int:
    return _chk(lib().rdc_timelapse_record(h, int(bool(reset))), "rdc_timelapse_record")


def rdc_tune(h, reps: int = 3):
    """(shape dict, best GCUPS measured)."""
    sh = rdc_launch_shape()
    g = ctypes.c_double()
    _chk(lib().rdc_tune(h, int(reps), ctypes.byref(sh), ctypes.byref(g)), "rdc_tune")
    return {f: getattr(sh, f) for f, _ in sh._fields_}, g.value


def rdc_get_shape(h) -> rdc_launch_shape:
    s = rdc_launch_shape()
    _chk(lib().rdc_get_shape(h, ctypes.byref(s)), "rdc_get_shape")
    return s


def rdc_set_shape(h, bx: int, rows: int, tx: int, ty: int, nthreads: int, k: int,
                  variant: int = 0, krows: int = 256) -> int:
    s = rdc_launch_shape(bx, rows, tx, ty, nthreads, k, variant, krows)
    return _chk(lib().rdc_set_shape(h, ctypes.byref(s)), "rdc_set_shape")


# ---------------------------------------------------------------------------
# batches
# ---------------------------------------------------------------------------

def rdc_batch_create(grids, params, phis=None, stream=None):
    """grids: list of (width, height); params: list of rdc_params (one per
    grid; for an empty batch a single rdc_params); phis: None or a list of
    host float32 maps / None.  Returns a handle."""
    n = len(grids)
    G = (rdc_grid * max(n, 1))(*[rdc_grid(int(w), int(h)) for w, h in grids])
    plist = list(params) if n > 0 else [params[0] if isinstance(params, (list, tuple)) else params]
    P = (rdc_params * len(plist))(*plist)
    keep = []
    if phis is None:
        phi_arr = None
    else:
        arr = (_P * n)()
        for i, ph in enumerate(phis):
            if ph is None:
                arr[i] = None
            else:
                a = np.ascontiguousarray(ph, dtype=np.float32)
                keep.append(a)
                arr[i] = a.ctypes.data
        phi_arr = arr
    h = _P()
    rc = lib().rdc_batch_create(n, G, P, phi_arr, _stream(stream), ctypes.byref(h))
    _chk(rc, "rdc_batch_create")
    return h.value


def rdc_batch_add(b, width: int, height: int, params: rdc_params, phi=None) -> int:
    idx = ctypes.c_int32(-1)
    ptr = None
    if phi is not None:
        a = np.ascontiguousarray(phi, dtype=np.float32)
        if a.shape != (height, width):
            raise ValueError("phi shape mismatch")
        ptr = a.ctypes.data
    rc = lib().rdc_batch_add(b, rdc_grid(int(width), int(height)), ctypes.byref(params), ptr,
                             ctypes.byref(idx))
    _chk(rc, "rdc_batch_add")
    return idx.value


def rdc_batch_remove(b, idx: int) -> int:
    return _chk(lib().rdc_batch_remove(b, int(idx)), "rdc_batch_remove")


def rdc_batch_destroy(b) -> None:
    if b:
        lib().rdc_batch_destroy(b)


def rdc_batch_seed(b, idx: int, cx: float, cy: float, r: float, value: float) -> int:
    return _chk(lib().rdc_batch_seed(b, int(idx), float(cx), float(cy), float(r), float(value)),
                "rdc_batch_seed")


def rdc_batch_get_grid(b, idx: int):
    """(width, height) of grid idx."""
    g = rdc_grid()
    _chk(lib().rdc_batch_get_grid(b, int(idx), ctypes.byref(g)), "rdc_batch_get_grid")
    return g.width, g.height


def rdc_batch_stability(b, idx: int):
    """(status, rho) of grid idx: status RDC_OK or RDC_EUNSTABLE_WARN."""
    rho = ctypes.c_double()
    rc = _chk(lib().rdc_batch_stability(b, int(idx), ctypes.byref(rho)), "rdc_batch_stability",
              allow=(RDC_EUNSTABLE_WARN,))
    return rc, rho.value


def rdc_batch_set_state(b, idx: int, u=None, v=None) -> int:
    pu, cu, su = _host_ptr(u, "u")
    pv, cv, sv = _host_ptr(v, "v")
    code = _same_code(cu, cv, "u and v")
    if code is None:
        return RDC_OK
    w, h = rdc_batch_get_grid(b, idx)
    _check_cells(su, w, h, "u")
    _check_cells(sv, w, h, "v")
    return _chk(lib().rdc_batch_set_state(b, int(idx), pu, pv, code), "rdc_batch_set_state")


def rdc_batch_step(b, idx=None, n: int = 1) -> int:
    if idx is None:
        return _chk(lib().rdc_batch_step(b, None, 0, int(n)), "rdc_batch_step")
    a = np.ascontiguousarray(idx, dtype=np.int32)
    return _chk(lib().rdc_batch_step(b, a.ctypes.data, len(a), int(n)), "rdc_batch_step")


def rdc_batch_check(b, idx: int):
    fb = ctypes.c_int64(-1)
    rc = _chk(lib().rdc_batch_check(b, int(idx), ctypes.byref(fb)), "rdc_batch_check",
              allow=(RDC_ENONFINITE,))
    return rc, fb.value


def rdc_batch_read(b, idx: int, u_out=None, v_out=None) -> int:
    pu, cu, su = _host_ptr(u_out, "u_out")
    pv, cv, sv = _host_ptr(v_out, "v_out")
    code = _same_code(cu, cv, "u_out and v_out")
    if code is None:
        code = RDC_DTYPE_F64
    else:
        w, h = rdc_batch_get_grid(b, idx)
        _check_cells(su, w, h, "u_out")
        _check_cells(sv, w, h, "v_out")
    return _chk(lib().rdc_batch_read(b, int(idx), pu, pv, code), "rdc_batch_read",
                allow=(RDC_ENONFINITE,))


def rdc_batch_sync(b) -> int:
    return _chk(lib().rdc_batch_sync(b), "rdc_batch_sync")


def rdc_batch_set_config(b, k: int, rows: int, krows: int, graphs: bool = True) -> int:
    return _chk(lib().rdc_batch_set_config(b, int(k), int(rows), int(krows), int(bool(graphs))),
                "rdc_batch_set_config")


def rdc_batch_get_info(b) -> rdc_batch_info:
    info = rdc_batch_info()
    _chk(lib().rdc_batch_get_info(b, ctypes.byref(info)), "rdc_batch_get_info")
    return info


def rdc_batch_tune(b, reps: int = 3) -> rdc_batch_info:
    info = rdc_batch_info()
    _chk(lib().rdc_batch_tune(b, int(reps), ctypes.byref(info)), "rdc_batch_tune")
    return info
