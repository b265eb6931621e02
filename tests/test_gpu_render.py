"""Colour-map and timelapse outputs (§3.1) on the GPU, byte for byte against
the oracle's definition, on seeded synthetic states (never GPU output)."""
from __future__ import annotations

import numpy as np
import pytest

import rdc_inputs as ri
from tests.helpers import PREC, round_to_storage

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["f32", "bf16", "f64"])
def test_render_snapshot_matches_oracle(gpu, orc, prec):
    c = ri.and_gate(131, 77, arm=40, out_len=20)
    H, W = c.phi.shape
    rng = np.random.default_rng(12)
    u = rng.uniform(-0.2, 1.3, size=(H, W))
    v = rng.uniform(-0.1, 0.6, size=(H, W))
    u[3, :8] = np.array([127.5, 128.5, 0.0, 255.0, 254.5, 1.5, 2.5, 63.75]) / 255.0
    p = gpu.rdc_params_default(precision=PREC[prec])
    phi_in = c.phi if prec == "f64" else c.phi.astype(np.float32)
    h = gpu.rdc_create(W, H, p, phi_in)
    try:
        gpu.rdc_set_state(h, u, v)
        img = gpu.rdc_render(h, gpu.RDC_RENDER_SNAPSHOT, 1.0, 2.0, 0.07575)
    finally:
        gpu.rdc_destroy(h)
    # the oracle renders the stored values (rounded to the storage type, then FP32)
    us = round_to_storage(u, prec).astype(np.float32)
    vs = round_to_storage(v, prec).astype(np.float32)
    phi_s = phi_in.astype(np.float64)
    ref = orc.render(us, vs, phi_s, 1.0, 2.0, thr=0.07575)
    assert np.array_equal(img, ref)


def test_timelapse_matches_oracle(gpu, orc):
    H, W = 45, 70
    rng = np.random.default_rng(3)
    states = [rng.uniform(0.0, 1.0, size=(H, W)).astype(np.float32) for _ in range(5)]
    phi = np.full((H, W), 0.054, dtype=np.float32)
    phi[:, 30:33] = 0.2
    p = gpu.rdc_params_default(precision=0)
    h = gpu.rdc_create(W, H, p, phi)
    tl = None
    try:
        for k, s in enumerate(states):
            gpu.rdc_set_state(h, s, s)
            gpu.rdc_timelapse_record(h, reset=(k == 2))
            tl = orc.timelapse(s, None if k in (0, 2) else tl)
        img = gpu.rdc_render(h, gpu.RDC_RENDER_TIMELAPSE, 1.0, 1.0, 0.1)
    finally:
        gpu.rdc_destroy(h)
    ref = orc.render(states[-1], states[-1], phi.astype(np.float64), 1.0, 1.0, thr=0.1, tl=tl)
    assert np.array_equal(img, ref)


def test_render_into_device_buffer(gpu):
    import torch
    W, H = 64, 32
    p = gpu.rdc_params_default(precision=0)
    h = gpu.rdc_create(W, H, p)
    try:
        gpu.rdc_seed(h, 20, 10, 5, 0.8)
        host = gpu.rdc_render(h)
        dev = torch.empty((H, W, 4), dtype=torch.uint8, device="cuda")
        gpu.rdc_render(h, out=dev)
        gpu.rdc_sync(h)
        assert np.array_equal(dev.cpu().numpy(), host)
        assert host[10, 20, 0] == 204 and host[0, 0, 0] == 1   # 0.8 * 255 = 204; u* * 255 ~ 0.55
    finally:
        gpu.rdc_destroy(h)


@pytest.mark.parametrize("prec", ["f32", "bf16", "f64"])
@pytest.mark.parametrize("W,H", [(1000, 600), (1001, 7), (3, 5)])
def test_render_device_buffer_any_alignment(gpu, prec, W, H):
    """The same bytes into a 16-byte aligned device buffer (vector stores
    when W is a multiple of 4) and into one 4 bytes off (pixel stores), as
    into host memory."""
    import torch
    p = gpu.rdc_params_default(precision=PREC[prec])
    h = gpu.rdc_create(W, H, p)
    try:
        gpu.rdc_seed(h, W / 3, H / 2, max(1.0, min(W, H) / 4), 0.8)
        gpu.rdc_step(h, 7)
        host = gpu.rdc_render(h, gpu.RDC_RENDER_SNAPSHOT, 1.0, 3.0, 0.054)
        raw = torch.zeros(H * W * 4 + 16, dtype=torch.uint8, device="cuda")
        for off in (0, 4):
            dev = raw[off:off + H * W * 4].view(H, W, 4)
            gpu.rdc_render(h, gpu.RDC_RENDER_SNAPSHOT, 1.0, 3.0, 0.054, out=dev)
            gpu.rdc_sync(h)
            assert np.array_equal(dev.cpu().numpy(), host), off
    finally:
        gpu.rdc_destroy(h)


@pytest.mark.parametrize("thr", [0.1, float(np.float32(0.1)) + 1e-12, 0.125,
                                 float(np.nextafter(np.float32(0.2), np.float32(0))),
                                 -np.inf, np.inf, 1e300, 1e-300])
def test_render_threshold_is_an_fp64_comparison(gpu, orc, thr):
    """G = 255 exactly where phi >= thr in FP64, for float phi values on both
    sides of thresholds that are and are not float values."""
    W, H = 16, 4
    f = np.float32
    vals = [f(0.1), np.nextafter(f(0.1), f(0)), np.nextafter(f(0.1), f(1)), f(0.125),
            np.nextafter(f(0.125), f(0)), f(0.2), np.nextafter(f(0.2), f(0)), f(0.054)]
    phi = np.resize(np.array(vals, dtype=np.float32), (H, W))
    p = gpu.rdc_params_default(precision=0)
    h = gpu.rdc_create(W, H, p, phi)
    try:
        img = gpu.rdc_render(h, gpu.RDC_RENDER_SNAPSHOT, 1.0, 1.0, thr)
        u = np.empty((H, W), dtype=np.float32)
        v = np.empty((H, W), dtype=np.float32)
        gpu.rdc_read(h, u, v)
    finally:
        gpu.rdc_destroy(h)
    ref = orc.render(u, v, phi.astype(np.float64), 1.0, 1.0, thr=thr)
    assert np.array_equal(img, ref)
    assert np.array_equal(img[..., 1] == 255, phi.astype(np.float64) >= thr)


LINES = [  # (x0, y0, x1, y1, width, value, snap)
    (10.0, 12.5, 120.0, 12.5, 2.0, 0.2, 0.0),
    (20.0, 30.0, 90.0, 80.0, 3.0, 0.0975, 15.0),
    (60.7, 5.2, 61.9, 70.3, 8.0, 0.2, 15.0),
    (-10.0, 40.0, 200.0, 44.0, 3.0, 0.054, 0.0),
    (130.0, 70.0, 130.0, 70.0, 5.0, 0.2, 0.0),
]


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_draw_lines_match_oracle(gpu, orc, prec):
    W, H = 140, 90
    p = gpu.rdc_params_default(precision=PREC[prec])
    h = gpu.rdc_create(W, H, p)
    ref = np.full((H, W), 0.054)
    try:
        gpu.rdc_fill_phi(h, 0.054)
        for (x0, y0, x1, y1, w, val, snap) in LINES:
            gpu.rdc_draw_line(h, x0, y0, x1, y1, w, val, snap)
            orc.draw_line(ref, x0, y0, x1, y1, w, val, snap)
        phi = gpu.rdc_read_phi(h)
    finally:
        gpu.rdc_destroy(h)
    expect = ref if prec == "f64" else ref.astype(np.float32).astype(np.float64)
    assert np.array_equal(phi, expect)
    assert (phi == expect.max()).sum() > 100
