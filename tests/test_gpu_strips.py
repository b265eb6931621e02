"""Row strips on the GPU: rdc_get_rows / rdc_put_rows and StripGrid.

StripGrid steps one grid as several simulations of row strips on one device,
exchanging halo rows of u and v with rdc_get_rows straight into the
neighbour's planes.  Its result must equal one simulation of the whole grid
bit for bit in every storage type, at k = 1 and with temporal blocking,
for ragged strip heights and step counts that are not a multiple of the halo.
"""
from __future__ import annotations

import numpy as np
import pytest

from paper_1901_06535_gb300.strips import StripGrid

pytestmark = pytest.mark.gpu


def _phi(W, H):
    phi = np.full((H, W), 0.054, dtype=np.float32)
    phi[:, W // 3:W // 3 + 4] = 0.0975          # a passive column crossing every strip
    phi[H // 2, :] = 0.0975                       # and a passive row
    return phi


def _seeds(W, H, n, seed):
    rng = np.random.default_rng(seed)
    # centres on a 1/8 grid: shifting them by whole rows is exact
    return [(rng.integers(0, 8 * W) / 8.0, rng.integers(0, 8 * H) / 8.0,
             float(rng.integers(3, 9)), 0.8) for _ in range(n)]


def _whole(gpu, W, H, phi, seeds, steps, prec, k):
    s = gpu.Sim(W, H, phi=phi, precision=prec, k_block=k)
    for d in seeds:
        s.seed(*d)
    s.step(steps)
    out = s.read()
    s.close()
    return out


CASES = [  # W, H, strips, halo, k_block, steps, storage
    (130, 67, 2, 1, 1, 40, "f32"),
    (130, 67, 3, 4, 4, 50, "f32"),
    (257, 129, 4, 6, 6, 61, "f32"),
    (257, 129, 3, 8, 5, 45, "bf16"),
    (200, 97, 2, 4, 4, 33, "f16"),
    (100, 60, 3, 4, 4, 30, "f64"),
    (64, 41, 5, 8, 8, 27, "f32"),
]


@pytest.mark.parametrize("W,H,n,halo,k,steps,prec", CASES)
def test_strip_grid_equals_whole_grid(gpu, W, H, n, halo, k, steps, prec):
    phi = _phi(W, H)
    seeds = _seeds(W, H, 4, W * H + n)
    seeds.append((W / 2.0, (H // n) - 0.5, 6.0, 0.8))   # on the first cut
    ref_u, ref_v = _whole(gpu, W, H, phi, seeds, steps, prec, k)
    with StripGrid(W, H, n, phi=phi, halo=halo, precision=prec, k_block=k) as g:
        for d in seeds:
            g.seed(*d)
        g.step(steps)
        u, v = g.read()
    assert np.array_equal(u, ref_u) and np.array_equal(v, ref_v)
    assert np.abs(ref_u - ref_u[0, 0]).max() > 0.1      # a wave is moving


def test_strip_grid_full_size(gpu):
    """8192^2 with 200 disks (the single-grid workload's set-up) as four
    strips at k = 5, against the whole grid."""
    W = H = 8192
    rng = np.random.default_rng(7)
    seeds = [(rng.integers(0, 8 * W) / 8.0, rng.integers(0, 8 * H) / 8.0,
              float(rng.integers(4, 11)), 0.8) for _ in range(200)]
    ref_u, ref_v = _whole(gpu, W, H, None, seeds, 60, "f32", 5)
    with StripGrid(W, H, 4, halo=5, precision="f32", k_block=5) as g:
        for d in seeds:
            g.seed(*d)
        g.step(60)
        u, v = g.read()
    assert np.array_equal(u, ref_u) and np.array_equal(v, ref_v)


def test_strip_grid_refuses_stochastic_rounding(gpu):
    with pytest.raises(ValueError):
        StripGrid(64, 64, 2, precision="bf16", flags=gpu.RDC_STOCH_ROUND, round_seed=3)


def test_get_put_rows_round_trip(gpu):
    W, H = 77, 53
    s = gpu.Sim(W, H, precision="f32")
    s.seed(30.0, 20.0, 9.0, 0.8)
    s.step(25)
    u, v = s.read(dtype=np.float32)
    # packed rows into host arrays
    gu = np.empty((7, W), np.float32)
    gv = np.empty((7, W), np.float32)
    gpu.rdc_get_rows(s.handle, 11, 7, gu, gv)
    assert np.array_equal(gu, u[11:18]) and np.array_equal(gv, v[11:18])
    # pitched rows, one plane only
    wide = np.full((7, W + 9), -1.0, np.float32)
    gpu.rdc_get_rows(s.handle, 40, 7, wide, None, pitch_bytes=(W + 9) * 4)
    assert np.array_equal(wide[:, :W], u[40:47]) and np.all(wide[:, W:] == -1.0)
    # device buffers (tensors), then write rows back elsewhere
    import torch
    du = torch.empty((3, W), dtype=torch.float32, device="cuda")
    dv = torch.empty((3, W), dtype=torch.float32, device="cuda")
    gpu.rdc_get_rows(s.handle, 0, 3, du, dv)
    gpu.rdc_put_rows(s.handle, 50, 3, du, dv)
    s.sync()
    u2, v2 = s.read(dtype=np.float32)
    assert np.array_equal(u2[50:53], u[0:3]) and np.array_equal(v2[50:53], v[0:3])
    assert np.array_equal(u2[:50], u[:50]) and np.array_equal(v2[:50], v[:50])
    # host rows in
    gpu.rdc_put_rows(s.handle, 20, 2, np.full((2, W), 0.25, np.float32), None)
    u3, v3 = s.read(dtype=np.float32)
    assert np.all(u3[20:22] == 0.25) and np.array_equal(v3, v2)
    gpu.rdc_get_rows(s.handle, 5, 0, None, None)      # nothing to copy
    for bad in ((50, 4, 0), (-1, 2, 0), (0, -1, 0), (0, 2, W * 4 - 4)):
        with pytest.raises(gpu.RdcError):
            gpu.rdc_get_rows(s.handle, bad[0], bad[1], gu, gv, pitch_bytes=bad[2])
    s.close()


@pytest.mark.parametrize("prec", ["bf16", "f16", "f64"])
def test_get_rows_storage_types(gpu, prec):
    """Rows come out in the storage type, bit for bit as rdc_read widens them."""
    W, H = 40, 24
    s = gpu.Sim(W, H, precision=prec)
    s.seed(20.0, 12.0, 6.0, 0.8)
    s.step(15)
    u, _ = s.read()
    view = s.view()
    dt = {2: np.uint16, 8: np.float64}[view.elem_bytes]
    raw = np.empty((4, W), dt)
    gpu.rdc_get_rows(s.handle, 6, 4, raw, None)
    if prec == "f64":
        got = raw
    elif prec == "bf16":
        got = (raw.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
    else:
        got = raw.view(np.float16).astype(np.float64)
    assert np.array_equal(got, u[6:10])
    s.close()
