"""Stochastic rounding to 16-bit storage (RDC_STOCH_ROUND) on the GPU.

* The device's Philox4x32-10 reproduces the generator's published
  known-answer vectors and equals the oracle's on random counters and keys.
* The device rounding of a value, for any cell, step and key, equals the
  oracle's (its own Philox4x32-10 and rounding rule, written separately),
  bit for bit.
* The rounding is a function of (key, column, row, step) only: every launch
  configuration, k_block, batch and split of the steps gives the same bits.
* It removes the stagnation of round-to-nearest: a cosine mode of the
  diffusion-only model, whose per-step change is far below half a storage
  spacing, stays frozen under round-to-nearest but decays at the closed-form
  rate (1 + dt Du lambda)^n under stochastic rounding.
* The 256² single-disk workload's front arrival times stay within 1 % of the FP64 oracle."""
from __future__ import annotations

import numpy as np
import pytest

import rdc_inputs as ri
from tests.helpers import PREC, gpu_run, orc_run

pytestmark = pytest.mark.gpu

SR = 4


def _values(rng, n):
    mag = np.exp(rng.uniform(np.log(1e-6), np.log(6e4), n)).astype(np.float32)
    x = mag * rng.choice(np.array([-1, 1], dtype=np.float32), n)
    x[:8] = [0.0, -0.0, 0.3, 0.5, 65504.0, 65510.0, 1e-7, -2.5e-5]
    # the edges of FP16's normal range and values just inside and outside them
    tiny = np.float32(2.0 ** -14)
    x[8:16] = [tiny, np.nextafter(tiny, np.float32(0)), np.nextafter(tiny, np.float32(1)),
               -tiny, 65503.0, -65503.99, np.float32(65472.5), np.float32(3.3e38)]
    return x


def test_device_philox_known_answers(gpu, orc):
    from tests.oracle_pins import philox_kat
    kat = philox_kat()
    ctr = np.array([c for c, _, _ in kat], dtype=np.uint32)
    key = np.array([k for _, k, _ in kat], dtype=np.uint32)
    want = np.array([o for _, _, o in kat], dtype=np.uint32)
    assert np.array_equal(gpu.rdc_philox_sample(ctr, key), want)
    rng = np.random.default_rng(11)
    ctr = rng.integers(0, 2**32, (4096, 4), dtype=np.uint64).astype(np.uint32)
    key = rng.integers(0, 2**32, (4096, 2), dtype=np.uint64).astype(np.uint32)
    got = gpu.rdc_philox_sample(ctr, key)
    ref = np.array([orc.philox4x32_10([int(x) for x in c], [int(x) for x in k])
                    for c, k in zip(ctr, key)], dtype=np.uint32)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
@pytest.mark.parametrize("seed,step,row,col0", [(0, 1, 0, 0), (7, 12345, 3, 1),
                                                (0xFFFFFFFF, (3 << 32) + 5, 4095, 77),
                                                (123456789, 2**40 + 1, 1, 2**20)])
def test_device_rounding_matches_oracle(gpu, orc, fmt, seed, step, row, col0):
    rng = np.random.default_rng(step % 1000 + row)
    x = _values(rng, 20000)
    u, v = gpu.rdc_stoch_round_sample(fmt, seed, step, row, col0, x)
    ou, ov = orc.round_stoch_cells(x, seed, step, row, col0, fmt)
    assert np.array_equal(u.view(np.uint32), ou.view(np.uint32))
    assert np.array_equal(v.view(np.uint32), ov.view(np.uint32))
    # u and v of one cell use different words: they disagree somewhere
    inexact = u != x
    assert np.any(u[inexact] != v[inexact])


def _seeds(W, H):
    return [(W * 0.3, H * 0.4, 5.0, 0.8), (W * 0.7, H * 0.6, 4.0, 0.8), (1.0, H - 2.0, 3.0, 0.8)]


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_rounding_is_the_same_for_every_launch(gpu, prec):
    W, H, n = 203, 117, 24
    s = _seeds(W, H)
    ref, vref, _ = gpu_run(gpu, W, H, seeds=s, n=n, prec=prec, flags=SR, round_seed=5, k=1)
    runs = {
        "k4": dict(k=4),
        "k6 rows 7": dict(k=6, shape=dict(k=6, variant=0, krows=7)),
        "k5 streamed": dict(k=5, shape=dict(k=5, variant=0, krows=16)),
        "k7 streamed rows 5": dict(k=7, shape=dict(k=7, variant=0, krows=5)),
        "k3 streamed": dict(k=3, shape=dict(k=3, variant=0, krows=32)),
        "k2 streamed": dict(k=2, shape=dict(k=2, variant=0, krows=64)),
        "k3 tile": dict(k=3, shape=dict(k=3, variant=1, tx=16, ty=8, nthreads=64)),
        "k8 tile": dict(k=8, shape=dict(k=8, variant=1, tx=40, ty=24, nthreads=128)),
        "k1 rows 3": dict(k=1, shape=dict(rows=3, bx=64)),
        "split 5+7+12": dict(k=4, chunks=[5, 7, 12]),
    }
    for name, kw in runs.items():
        u, v, _ = gpu_run(gpu, W, H, seeds=s, n=n, prec=prec, flags=SR, round_seed=5, **kw)
        assert np.array_equal(u, ref) and np.array_equal(v, vref), name
    # a different key and round-to-nearest give different states
    u2, _, _ = gpu_run(gpu, W, H, seeds=s, n=n, prec=prec, flags=SR, round_seed=6, k=1)
    urn, _, _ = gpu_run(gpu, W, H, seeds=s, n=n, prec=prec, flags=0, k=1)
    assert not np.array_equal(u2, ref) and not np.array_equal(urn, ref)


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_nan_cells_are_stored_alike_by_every_launch(gpu, prec):
    """A state holding NaN (and an infinity): the single step and the
    streamed kernels store the same bits (non-finite values round to nearest;
    the NaN spreads), and the health check reports it."""
    W, H, n = 96, 40, 12
    p = gpu.rdc_params_default(precision=PREC[prec], flags=SR, round_seed=9)
    us = gpu.rdc_rest_state(0.054, 1.4, 0.002)
    u = np.full((H, W), us, dtype=np.float32)
    v = u.copy()
    u[20, 30] = np.nan
    u[5, 70] = np.inf
    v[33, 10] = np.nan
    outs = []
    for k in (1, 4, 5):
        u_out, v_out, ex = gpu_run(gpu, W, H, n=n, prec=prec, flags=SR, round_seed=9, k=k,
                                   state=(u, v), dtype=np.float32)
        assert ex["status"] == gpu.RDC_ENONFINITE
        outs.append((u_out.view(np.uint32), v_out.view(np.uint32)))
    for o in outs[1:]:
        assert np.array_equal(o[0], outs[0][0]) and np.array_equal(o[1], outs[0][1])
    assert np.isnan(outs[0][0].view(np.float32)).sum() > 1


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_test_modes_with_stochastic_rounding(gpu, prec):
    """Diffusion-only and reaction-only with SR: the tile kernel (k > 1) and
    the single step agree."""
    W, H, n = 90, 61, 10
    s = _seeds(W, H)
    for flags in (1, 2):
        a, _, _ = gpu_run(gpu, W, H, seeds=s, n=n, prec=prec, flags=flags | SR, round_seed=3, k=1)
        b, _, _ = gpu_run(gpu, W, H, seeds=s, n=n, prec=prec, flags=flags | SR, round_seed=3,
                          k=5, shape=dict(k=5, variant=1, tx=32, ty=16, nthreads=128))
        assert np.array_equal(a, b), flags


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_batch_with_stochastic_rounding_equals_solo(gpu, prec):
    sizes = [(130, 67), (64, 64), (33, 100)]
    params = [gpu.rdc_params_default(precision=PREC[prec], flags=SR, round_seed=11 + i, k_block=4)
              for i in range(len(sizes))]
    b = gpu.rdc_batch_create(sizes, params)
    try:
        for i, (W, H) in enumerate(sizes):
            for d in _seeds(W, H):
                gpu.rdc_batch_seed(b, i, *d)
        gpu.rdc_batch_step(b, [0, 2], 9)
        gpu.rdc_batch_step(b, None, 14)
        counts = [23, 14, 23]
        for i, (W, H) in enumerate(sizes):
            u = np.empty((H, W))
            gpu.rdc_batch_read(b, i, u, None)
            us, _, _ = gpu_run(gpu, W, H, seeds=_seeds(W, H), n=counts[i], prec=prec, flags=SR,
                               round_seed=11 + i, k=1)
            assert np.array_equal(u, us), i
    finally:
        gpu.rdc_batch_destroy(b)


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_stochastic_rounding_follows_the_diffusion_decay(gpu, prec):
    """u = 0.5 + A cos(pi k (j + 1/2) / W) under diffusion only.  Each step
    changes u by about 7e-6, far below half a storage spacing at 0.5 (2e-3
    for BF16, 2.4e-4 for FP16): round-to-nearest freezes the mode, while the
    stochastically rounded mode decays like the exact recurrence,
    A_n = A (1 + dt Du lambda_k)^n, lambda_k = -(4/dx^2) sin^2(pi k / 2W)."""
    W, H, kx, A, n = 256, 64, 8, 0.1, 10000
    j = np.arange(W)
    mode = np.cos(np.pi * kx * (j + 0.5) / W)
    u0 = np.tile(0.5 + A * mode, (H, 1)).astype(np.float32)
    v0 = np.full((H, W), 0.5, dtype=np.float32)
    dt, Du, dx = 1e-3, 0.45, 0.25
    lam = -(4 / dx**2) * np.sin(np.pi * kx / (2 * W)) ** 2
    want = A * (1 + dt * Du * lam) ** n            # ~ 0.5 A

    def amplitude(u):
        prof = u.mean(axis=0) - 0.5
        return 2.0 / W * float(np.dot(prof, mode))

    a0 = amplitude(u0.astype(np.float64))
    u_rn, _, _ = gpu_run(gpu, W, H, n=n, prec=prec, flags=1, state=(u0, v0), k=4)
    u_sr, _, _ = gpu_run(gpu, W, H, n=n, prec=prec, flags=1 | SR, round_seed=1, state=(u0, v0),
                         k=4)
    a_rn, a_sr = amplitude(u_rn), amplitude(u_sr)
    print(f"[{prec}] amplitude: start {a0:.5f}, RN {a_rn:.5f}, SR {a_sr:.5f}, exact {want:.5f}")
    assert abs(a_rn - a0) < 0.02 * A                 # frozen (stagnation)
    assert abs(a_sr - want) < 0.03 * A               # decays as the exact recurrence
    assert abs(a_sr - a0) > 0.3 * A


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_arrival_times_256_single_disk_stochastic(gpu, orc, om, prec, record_property):
    W = H = 256
    seeds = [(127.5, 127.5, 6.0, 0.8)]
    probes = ri.axis_probes(W, H, (20, 40, 60))
    n = 4700
    ref = orc_run(orc, om, W, H, seeds=seeds, n=n, probes=probes)
    _, _, ex = gpu_run(gpu, W, H, seeds=seeds, n=n, prec=prec, flags=SR, round_seed=2,
                       probes=probes)
    t_ref, t = ref["t_arr"], ex["t_arr"]
    assert np.all(t_ref > 0) and np.all(t > 0), (t_ref, t)
    rel = np.abs(t - t_ref) / t_ref
    record_property("arrival_rel_err", rel.tolist())
    print(f"[{prec} SR] arrival times {t.tolist()} vs oracle {t_ref.tolist()}: rel {rel.tolist()}")
    assert np.all(rel <= 0.01), (prec, t_ref, t, rel)


def test_tuning_keeps_the_stochastic_bits(gpu):
    """rdc_tune times candidate shapes on the spare buffers: the state, the
    step index and hence the random stream are unchanged, and the tuned
    shape gives the bits of single steps."""
    W, H, n = 260, 190, 21
    s = _seeds(W, H)
    ref, _, _ = gpu_run(gpu, W, H, seeds=s, n=n, prec="bf16", flags=SR, round_seed=4, k=1)
    p = gpu.rdc_params_default(precision=PREC["bf16"], flags=SR, round_seed=4)
    h = gpu.rdc_create(W, H, p)
    try:
        for d in s:
            gpu.rdc_seed(h, *d)
        gpu.rdc_step(h, 5)
        gpu.rdc_tune(h, 2)
        assert gpu.rdc_get_view(h).steps_done == 5
        gpu.rdc_step(h, n - 5)
        u = np.empty((H, W))
        gpu.rdc_read(h, u, None)
    finally:
        gpu.rdc_destroy(h)
    assert np.array_equal(u, ref)
