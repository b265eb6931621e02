"""GB300 (sm_103a) time-stepper for the two-variable Oregonator
reaction-diffusion model (Eq. 1 and Table 1 of the RDCSim paper).

The compute path is librdc, hand-written CUDA behind the C ABI in
``include/rdc.h``; ``_capi`` binds it with ctypes under the same names, and
``Sim`` is a small convenience wrapper.  PyTorch is optional here: it is used
by callers for device memory and streams only.
"""
from __future__ import annotations

import numpy as np

from ._capi import (  # noqa: F401  (re-exported C-ABI names)
    RDC_DIFFUSION_ONLY, RDC_DTYPE_BF16, RDC_DTYPE_F16, RDC_DTYPE_F32, RDC_DTYPE_F64,
    RDC_ECUDA, RDC_EINVAL, RDC_ENOMEM, RDC_ENONFINITE, RDC_ETIMEOUT, RDC_EUNSTABLE_WARN,
    RDC_EUNSUPPORTED, RDC_F32, RDC_F32_BF16STORE,
    RDC_F32_F16STORE, RDC_F64, RDC_OK, RDC_REACTION_ONLY, PRECISION_NAMES, RdcError,
    lib, rdc_check, rdc_create, rdc_create_ext, rdc_create_f64phi, rdc_destroy,
    rdc_get_shape, rdc_get_view, rdc_last_error, rdc_params, rdc_params_default,
    rdc_probe, rdc_read, rdc_reset_rest, rdc_rest_state, rdc_seed, rdc_set_phi,
    rdc_set_shape, rdc_set_state, rdc_stability, rdc_status_str, rdc_step, rdc_step_noalloc,
    rdc_sync, rdc_batch_add, rdc_batch_check, rdc_batch_create, rdc_batch_destroy,
    rdc_batch_get_grid, rdc_batch_get_info, rdc_batch_read, rdc_batch_remove, rdc_batch_seed,
    rdc_batch_set_config, rdc_batch_set_state, rdc_batch_step, rdc_batch_sync, rdc_batch_tune,
    RDC_RENDER_SNAPSHOT, RDC_RENDER_TIMELAPSE, rdc_render, rdc_timelapse_record, rdc_tune,
    RDC_SNAP_DEGREES, RDC_WIDTH_IMPERMEABLE, RDC_WIDTH_PERMEABLE, RDC_WIDTH_SEMIPERMEABLE,
    rdc_draw_line, rdc_fill_phi, rdc_read_phi, rdc_snap_segment, rdc_check_division,
    rdc_division_report, RDC_STOCH_ROUND, rdc_stoch_round_sample, rdc_set_step_index,
    rdc_batch_set_step_index, rdc_philox_sample, rdc_batch_stability, rdc_get_rows,
    rdc_put_rows)


class Sim:
    """One simulation on the current CUDA device.

    >>> s = Sim(256, 256, precision="f32")
    >>> s.seed(127.5, 127.5, 6, 0.8); s.step(1000); u, v = s.read()
    """

    def __init__(self, width: int, height: int, phi=None, precision="f32",
                 stream=None, **params):
        p = rdc_params_default(**params)
        if isinstance(precision, str):
            precision = PRECISION_NAMES[precision]
        p.precision = int(precision)
        self.params = p
        self.width, self.height = int(width), int(height)
        self.handle = rdc_create(width, height, p, phi, stream)

    def close(self):
        if getattr(self, "handle", None):
            rdc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def seed(self, cx, cy, r, value=0.8):
        rdc_seed(self.handle, cx, cy, r, value)

    def step(self, n: int):
        rdc_step(self.handle, n)

    def read(self, dtype=np.float64, check: bool = True):
        u = np.empty((self.height, self.width), dtype=dtype)
        v = np.empty_like(u)
        rc = rdc_read(self.handle, u, v)
        if check and rc != RDC_OK:
            raise RdcError(rc, "Sim.read")
        return u, v

    def set_state(self, u=None, v=None):
        rdc_set_state(self.handle, u, v)

    def set_phi(self, phi):
        rdc_set_phi(self.handle, phi)

    def probe(self, cells):
        return rdc_probe(self.handle, cells)

    def sync(self):
        rdc_sync(self.handle)

    def shape(self):
        s = rdc_get_shape(self.handle)
        return {k: getattr(s, k) for k, _ in s._fields_}

    def set_shape(self, **kw):
        cur = self.shape()
        cur.update(kw)
        rdc_set_shape(self.handle, cur["bx"], cur["rows"], cur["tx"], cur["ty"],
                      cur["nthreads"], cur["k"], cur["variant"], cur["krows"])

    def view(self):
        return rdc_get_view(self.handle)
