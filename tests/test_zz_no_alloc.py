"""rdc_step_noalloc: stepping caller-owned device buffers without any device
allocation, for callers that cannot allocate (applications whose device
memory comes from their own pool, loops that cannot afford the implicit device
synchronisation of cudaMalloc and cudaFree).

Checked against the handle API (rdc_create + rdc_step + rdc_read) on the same
initial state, bit for bit -- the tolerance the GPU tests use between two CUDA
paths of one precision -- on two calls in a row, the second continuing from
the first one's output, in every storage type.  This file is collected last
on purpose."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W, H = 300, 170
SEEDS = [(150.0, 85.0, 9.0, 0.8), (30.0, 20.0, 5.0, 1.0)]


def _reference_states(pkg, prec, k, n1, n2, W=W, H=H):
    """Initial state and the states after n1 and n1 + n2 steps, through the
    handle API (16-bit states read back as float32, which is exact)."""
    import torch
    npdt = np.float64 if prec == 1 else np.float32
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


def _torch_types(prec):
    import torch
    st = {0: torch.float32, 1: torch.float64, 2: torch.bfloat16, 3: torch.float16}[prec]
    return st, (torch.float64 if prec == 1 else torch.float32)


@pytest.mark.parametrize("prec,k", [(0, 1), (0, 4), (1, 3), (2, 4), (3, 1), (2, 1), (3, 6)],
                         ids=["f32-k1", "f32-k4", "f64-k3", "bf16-k4", "f16-k1", "bf16-k1",
                              "f16-k6"])
def test_noalloc_matches_handle_api_on_two_calls(gpu, prec, k):
    import torch
    dt, phidt = _torch_types(prec)
    esz = torch.empty(0, dtype=dt).element_size()
    pitch = 304                                   # elements; rows of 608 / 1216 / 2432 bytes
    dev = torch.device("cuda")
    n1, n2 = 37, 20
    (u0, v0), (u1r, v1r), (u2r, v2r) = _reference_states(gpu, prec, k, n1, n2)

    def dev_plane(src=None):
        t = torch.zeros((H, pitch), dtype=dt, device=dev)
        if src is not None:
            t[:, :W] = src.to(dev).to(dt)         # exact: the values are of the storage type
        return t

    u_in, v_in = dev_plane(u0), dev_plane(v0)
    phi = torch.full((H, pitch), 0.054, dtype=phidt, device=dev)
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

    rd = u1r.dtype
    assert torch.equal(u_a[:, :W].cpu().to(rd), u1r) and torch.equal(v_a[:, :W].cpu().to(rd), v1r)
    assert torch.equal(u_b[:, :W].cpu().to(rd), u2r) and torch.equal(v_b[:, :W].cpu().to(rd), v2r)
    assert not torch.equal(u2r, u1r)                  # the second call did advance


@pytest.mark.parametrize("k,n", [(1, 1), (4, 4), (6, 6), (2, 1)],
                         ids=["k1-n1", "k4-n4", "k6-n6", "k2-n1"])
def test_noalloc_single_launch_takes_grids_beyond_the_scratch(gpu, k, n):
    """A call of one launch keeps no intermediate state, so a 2048 x 2048
    FP32 grid (two planes would be 256 bytes over the scratch array) runs, twice
    in a row, and equals the handle API bit for bit."""
    import torch
    Wb = Hb = 2048
    p = gpu.rdc_params_default(precision=0, k_block=k)
    h = gpu.rdc_create(Wb, Hb, p)
    ref = []
    try:
        gpu.rdc_seed(h, 1000.0, 900.0, 9.0, 0.8)
        for _ in range(3):
            u = np.empty((Hb, Wb), dtype=np.float32)
            v = np.empty((Hb, Wb), dtype=np.float32)
            assert gpu.rdc_read(h, u, v) == gpu.RDC_OK
            ref.append((torch.from_numpy(u), torch.from_numpy(v)))
            gpu.rdc_step(h, n)
    finally:
        gpu.rdc_destroy(h)
    dev = torch.device("cuda")
    planes = [ref[0][0].to(dev), ref[0][1].to(dev)] + [torch.empty((Hb, Wb), device=dev)
                                                        for _ in range(4)]
    phi = torch.full((Hb, Wb), 0.054, device=dev)
    s = torch.cuda.current_stream().cuda_stream
    for c in range(2):
        ui, vi, uo, vo = planes[2 * c], planes[2 * c + 1], planes[2 * c + 2], planes[2 * c + 3]
        rc, bad = gpu.rdc_step_noalloc(Wb, Hb, p, ui.data_ptr(), vi.data_ptr(), phi.data_ptr(),
                                       uo.data_ptr(), vo.data_ptr(), Wb * 4, n, s)
        assert rc == gpu.RDC_OK and bad == -1
        assert torch.equal(uo.cpu(), ref[c + 1][0]) and torch.equal(vo.cpu(), ref[c + 1][1])


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
    """Five launches on a 4096 x 4096 FP32 grid would need 2 x 64 MiB of
    scratch: refused before anything is enqueued (the buffers are real and
    large enough, so nothing could go out of bounds even if it were not)."""
    import torch
    n = 4096
    t = [torch.zeros((n, n), dtype=torch.float32, device="cuda") for _ in range(5)]
    p = gpu.rdc_params_default(precision=0)
    with pytest.raises(gpu.RdcError) as e:
        gpu.rdc_step_noalloc(n, n, p, *(x.data_ptr() for x in t), n * 4, 5)
    assert e.value.status == gpu.RDC_EUNSUPPORTED
    assert torch.count_nonzero(t[3]) == 0 and torch.count_nonzero(t[4]) == 0
