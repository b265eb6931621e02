"""rdc_step_noalloc: stepping caller-owned device buffers without any device
allocation, for callers that cannot allocate (inside CUDA-graph stream
capture, hosts that own all device memory through their own pool, loops that
cannot afford cudaMalloc's implicit synchronisation).

Checked against the handle API (rdc_create + rdc_step + rdc_read) on the same
initial state, bit for bit -- the tolerance the GPU tests use between two CUDA
paths of one precision -- on two calls in a row, the second continuing from
the first one's output.  This file is collected last on purpose."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W, H = 300, 170
SEEDS = [(150.0, 85.0, 9.0, 0.8), (30.0, 20.0, 5.0, 1.0)]


def _reference_states(pkg, prec, k, n1, n2):
    """Initial state and the states after n1 and n1 + n2 steps, through the
    handle API."""
    import torch
    npdt = {0: np.float32, 1: np.float64}[prec]
    p = pkg.rdc_params_default(precision=prec, k_block=k)
    h = pkg.rdc_create(W, H, p)
    out = []
    try:
        for s in SEEDS:
            pkg.rdc_seed(h, *s)
        for n in (0, n1, n2):
            pkg.rdc_step(h, n)
            u = np.empty((H, W), dtype=npdt)
            v = np.empty((H, W), dtype=npdt)
            assert pkg.rdc_read(h, u, v) == pkg.RDC_OK
            out.append((torch.from_numpy(u), torch.from_numpy(v)))
    finally:
        pkg.rdc_destroy(h)
    return out


@pytest.mark.parametrize("prec,k", [(0, 1), (0, 4), (1, 3)], ids=["f32-k1", "f32-k4", "f64-k3"])
def test_noalloc_matches_handle_api_on_two_calls(gpu, prec, k):
    import torch
    dt = {0: torch.float32, 1: torch.float64}[prec]
    esz = 4 if prec == 0 else 8
    pitch = 304                                   # elements; rows of 1216 / 2432 bytes
    dev = torch.device("cuda")
    n1, n2 = 37, 20
    (u0, v0), (u1r, v1r), (u2r, v2r) = _reference_states(gpu, prec, k, n1, n2)

    def dev_plane(src=None):
        t = torch.zeros((H, pitch), dtype=dt, device=dev)
        if src is not None:
            t[:, :W] = src.to(dev)
        return t

    u_in, v_in = dev_plane(u0), dev_plane(v0)
    phi = torch.full((H, pitch), 0.054, dtype=dt, device=dev)
    u_a, v_a, u_b, v_b = dev_plane(), dev_plane(), dev_plane(), dev_plane()
    p = gpu.rdc_params_default(precision=prec, k_block=k)
    stream = torch.cuda.current_stream().cuda_stream
    args = (W, H, p)

    # a first call sets up the scratch address and loads the kernels
    gpu.rdc_step_noalloc(*args, u_in.data_ptr(), v_in.data_ptr(), phi.data_ptr(),
                         u_a.data_ptr(), v_a.data_ptr(), pitch * esz, n1, stream)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]

    rc, bad = gpu.rdc_step_noalloc(*args, u_in.data_ptr(), v_in.data_ptr(), phi.data_ptr(),
                                   u_a.data_ptr(), v_a.data_ptr(), pitch * esz, n1, stream)
    assert rc == gpu.RDC_OK and bad == -1
    rc, bad = gpu.rdc_step_noalloc(*args, u_a.data_ptr(), v_a.data_ptr(), phi.data_ptr(),
                                   u_b.data_ptr(), v_b.data_ptr(), pitch * esz, n2, stream)
    assert rc == gpu.RDC_OK and bad == -1
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0      # nothing was allocated

    assert torch.equal(u_a[:, :W].cpu(), u1r) and torch.equal(v_a[:, :W].cpu(), v1r)
    assert torch.equal(u_b[:, :W].cpu(), u2r) and torch.equal(v_b[:, :W].cpu(), v2r)
    assert not torch.equal(u2r, u1r)                  # the second call did advance


def test_noalloc_health_flag_is_reset_between_calls(gpu):
    import torch
    dev = torch.device("cuda")
    pitch = 304
    us = gpu.rdc_rest_state(0.054, 1.4, 0.002)
    good = torch.full((H, pitch), us, dtype=torch.float32, device=dev)
    bad = good.clone()
    bad[11, 7] = float("nan")
    v = torch.full((H, pitch), us, dtype=torch.float32, device=dev)
    phi = torch.full((H, pitch), 0.054, dtype=torch.float32, device=dev)
    uo = torch.empty_like(good)
    vo = torch.empty_like(good)
    p = gpu.rdc_params_default(precision=0)
    s = torch.cuda.current_stream().cuda_stream
    rc, idx = gpu.rdc_step_noalloc(W, H, p, bad.data_ptr(), v.data_ptr(), phi.data_ptr(),
                                   uo.data_ptr(), vo.data_ptr(), pitch * 4, 2, s)
    assert rc == gpu.RDC_ENONFINITE and 0 <= idx < W * H
    rc, idx = gpu.rdc_step_noalloc(W, H, p, good.data_ptr(), v.data_ptr(), phi.data_ptr(),
                                   uo.data_ptr(), vo.data_ptr(), pitch * 4, 2, s)
    assert rc == gpu.RDC_OK and idx == -1


def test_noalloc_refuses_grids_beyond_the_static_scratch(gpu):
    import torch
    n = 4096                                            # 2 x 64 MiB of FP32 scratch needed
    t = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = gpu.rdc_params_default(precision=0)
    with pytest.raises(gpu.RdcError) as e:
        gpu.rdc_step_noalloc(n, n, p, t.data_ptr(), t.data_ptr() + 16, t.data_ptr() + 32,
                             t.data_ptr() + 48, t.data_ptr() + 64, n * 4, 5)
    assert e.value.status == gpu.RDC_EUNSUPPORTED
