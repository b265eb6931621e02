"""Checkpoint/resume and out-of-bounds checks on the device path.

* Resume: state read back (in the storage type) and written into a new
  simulation continues exactly like an uninterrupted run.
* Canaries: every step kernel runs on caller-owned planes (rdc_create_ext)
  surrounded by NaN canaries -- padding columns inside the row pitch and whole
  rows above and below each plane; after many steps with every kernel variant
  the canaries are intact, i.e. no kernel wrote outside [0, W) x [0, H)."""
from __future__ import annotations

import numpy as np
import pytest

from tests.helpers import PREC

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16", "f64"])
def test_checkpoint_resume_bitwise(gpu, prec):
    import torch
    W, H = 190, 123
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16,
           "f64": torch.float64}[prec]
    p = gpu.rdc_params_default(precision=PREC[prec], k_block=3)
    a = gpu.rdc_create(W, H, p)
    try:
        gpu.rdc_seed(a, 95.0, 60.0, 9.0, 0.8)
        gpu.rdc_step(a, 40)
        u = torch.empty((H, W), dtype=tdt)
        v = torch.empty((H, W), dtype=tdt)
        gpu.rdc_read(a, u, v)                     # checkpoint in the storage type
        gpu.rdc_step(a, 55)
        ref = np.empty((H, W))
        gpu.rdc_read(a, ref, None)
    finally:
        gpu.rdc_destroy(a)
    b = gpu.rdc_create(W, H, p)
    try:
        gpu.rdc_set_state(b, u, v)                # resume
        gpu.rdc_step(b, 55)
        got = np.empty((H, W))
        gpu.rdc_read(b, got, None)
    finally:
        gpu.rdc_destroy(b)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_checkpoint_resume_stochastic_rounding(gpu, prec):
    """With RDC_STOCH_ROUND the random stream follows the step index: restoring
    the state and the saved index continues bit for bit; without the index
    the resumed run draws other bits."""
    import torch
    W, H = 150, 97
    tdt = {"bf16": torch.bfloat16, "f16": torch.float16}[prec]
    p = gpu.rdc_params_default(precision=PREC[prec], k_block=4, flags=gpu.RDC_STOCH_ROUND,
                               round_seed=77)
    a = gpu.rdc_create(W, H, p)
    try:
        gpu.rdc_seed(a, 70.0, 50.0, 8.0, 0.8)
        gpu.rdc_step(a, 41)
        u = torch.empty((H, W), dtype=tdt)
        v = torch.empty((H, W), dtype=tdt)
        gpu.rdc_read(a, u, v)
        saved = gpu.rdc_get_view(a).steps_done
        gpu.rdc_step(a, 30)
        ref = np.empty((H, W))
        gpu.rdc_read(a, ref, None)
    finally:
        gpu.rdc_destroy(a)
    assert saved == 41
    outs = {}
    for restore in (True, False):
        b = gpu.rdc_create(W, H, p)
        try:
            gpu.rdc_set_state(b, u, v)
            if restore:
                gpu.rdc_set_step_index(b, saved)
            gpu.rdc_step(b, 30)
            got = np.empty((H, W))
            gpu.rdc_read(b, got, None)
            outs[restore] = got
        finally:
            gpu.rdc_destroy(b)
    assert np.array_equal(outs[True], ref)
    assert not np.array_equal(outs[False], ref)


def test_batch_checkpoint_resume_stochastic_rounding(gpu):
    """A stochastically rounded grid of a batch resumes bit for bit from its
    state and step index."""
    W, H = 120, 80
    p = gpu.rdc_params_default(precision=2, k_block=4, flags=gpu.RDC_STOCH_ROUND, round_seed=9)
    b = gpu.rdc_batch_create([(W, H), (64, 64)], [p, p])
    try:
        gpu.rdc_batch_seed(b, 0, 60.0, 40.0, 7.0, 0.8)
        gpu.rdc_batch_step(b, None, 25)
        u = np.empty((H, W), dtype=np.float32)
        v = np.empty((H, W), dtype=np.float32)
        gpu.rdc_batch_read(b, 0, u, v)         # BF16 values are exact in float32
        gpu.rdc_batch_step(b, [0], 18)
        ref = np.empty((H, W))
        gpu.rdc_batch_read(b, 0, ref, None)
        # restore grid 1's slot from grid 0's checkpoint: a different grid index
        gpu.rdc_batch_remove(b, 1)
        j = gpu.rdc_batch_add(b, W, H, p)
        gpu.rdc_batch_set_state(b, j, u, v)
        gpu.rdc_batch_set_step_index(b, j, 25)
        gpu.rdc_batch_step(b, [j], 18)
        got = np.empty((H, W))
        gpu.rdc_batch_read(b, j, got, None)
    finally:
        gpu.rdc_batch_destroy(b)
    assert np.array_equal(got, ref)


SHAPES = [dict(k=1, bx=32, rows=3), dict(k=1, bx=256, rows=1), dict(k=4, variant=0, krows=7),
          dict(k=6, variant=0, krows=100), dict(k=3, variant=1, tx=16, ty=8, nthreads=64),
          dict(k=8, variant=1, tx=40, ty=24, nthreads=128)]


@pytest.mark.parametrize("prec", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("W,H", [(37, 29), (130, 67), (1, 5)])
def test_no_writes_outside_the_grid(gpu, prec, W, H):
    import torch
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16, "f64": torch.float64}[prec]
    esz = torch.tensor([], dtype=tdt).element_size()
    pitch = ((W + 7) // 8) * 8 + 8                  # at least 8 padding columns
    pad_rows = 2
    dev = torch.device("cuda")

    def plane(dtype):
        t = torch.full((H + 2 * pad_rows, pitch), float("nan"), dtype=dtype, device=dev)
        return t

    us = [plane(tdt) for _ in range(2)]
    vs = [plane(tdt) for _ in range(2)]
    phid = torch.float64 if prec == "f64" else torch.float32
    phi = plane(phid)
    phi[pad_rows:pad_rows + H, :W] = 0.054
    inner = lambda t: t[pad_rows:pad_rows + H]       # noqa: E731
    p = gpu.rdc_params_default(precision=PREC[prec])
    h = gpu.rdc_create_ext(W, H, p, [inner(t).data_ptr() for t in us],
                           [inner(t).data_ptr() for t in vs], inner(phi).data_ptr(),
                           pitch * esz, torch.cuda.current_stream().cuda_stream)
    try:
        gpu.rdc_reset_rest(h)
        gpu.rdc_seed(h, W / 2, H / 2, max(1.0, min(W, H) / 3), 0.8)
        for sh in SHAPES:
            s = gpu.rdc_get_shape(h)
            cur = {f: getattr(s, f) for f, _ in s._fields_}
            cur.update(sh)
            gpu.rdc_set_shape(h, cur["bx"], cur["rows"], cur["tx"], cur["ty"], cur["nthreads"],
                              cur["k"], cur["variant"], cur["krows"])
            gpu.rdc_step(h, 2 * cur["k"] + 1)
        assert gpu.rdc_check(h)[0] == gpu.RDC_OK
        torch.cuda.synchronize()
    finally:
        gpu.rdc_destroy(h)
    for t in us + vs + [phi]:
        host = t.float().cpu()
        assert torch.isnan(host[:pad_rows]).all() and torch.isnan(host[pad_rows + H:]).all()
        assert torch.isnan(host[:, W:]).all()
