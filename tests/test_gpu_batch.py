"""Batches of independent grids: every grid's result equals the same grid run
alone (bit for bit), whatever the subset, the launch configuration, graphs
on or off, and after grids join and leave; FP64 batches equal the oracle."""
from __future__ import annotations

import numpy as np
import pytest

import rdc_inputs as ri
from tests.helpers import PREC

pytestmark = pytest.mark.gpu

# uneven sizes, ragged against every vector width and item shape
SIZES = [(130, 67), (257, 129), (64, 64), (1, 1), (33, 300), (500, 20), (128, 128)]


def _grid_setup(i, W, H):
    rng = np.random.default_rng(100 + i)
    eps = float(rng.uniform(0.02, 0.03))
    phi = float(rng.uniform(0.05, 0.08))
    disks = [(float(rng.uniform(0, W)), float(rng.uniform(0, H)), float(rng.integers(1, 7)), 0.8)
             for _ in range(int(rng.integers(1, 4)))]
    return eps, phi, disks


def _solo(pkg, W, H, eps, phi, disks, n, prec, k=1):
    p = pkg.rdc_params_default(precision=PREC[prec], eps=eps, k_block=k)
    dt = np.float64 if prec == "f64" else np.float32
    h = pkg.rdc_create(W, H, p, np.full((H, W), phi, dtype=dt))
    try:
        for d in disks:
            pkg.rdc_seed(h, *d)
        pkg.rdc_step(h, n)
        u = np.empty((H, W))
        v = np.empty((H, W))
        pkg.rdc_read(h, u, v)
    finally:
        pkg.rdc_destroy(h)
    return u, v


def _make_batch(pkg, prec, k=1, sizes=SIZES):
    grids, params, phis, setups = [], [], [], []
    for i, (W, H) in enumerate(sizes):
        eps, phi, disks = _grid_setup(i, W, H)
        grids.append((W, H))
        params.append(pkg.rdc_params_default(precision=PREC[prec], eps=eps, k_block=k))
        phis.append(np.full((H, W), phi, dtype=np.float32))
        setups.append((eps, phi, disks))
    b = pkg.rdc_batch_create(grids, params, phis)
    for i, (_, _, disks) in enumerate(setups):
        for d in disks:
            pkg.rdc_batch_seed(b, i, *d)
    return b, setups


def _read(pkg, b, i, W, H):
    u = np.empty((H, W))
    v = np.empty((H, W))
    assert pkg.rdc_batch_read(b, i, u, v) == pkg.RDC_OK
    return u, v


@pytest.mark.parametrize("prec", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("k", [1, 3, 4, 5, 6, 8])
def test_batch_equals_solo(gpu, prec, k):
    n = 2 * k + 5 if k > 1 else 13
    b, setups = _make_batch(gpu, prec, k)
    try:
        gpu.rdc_batch_step(b, None, n)
        for i, (W, H) in enumerate(SIZES):
            eps, _, disks = setups[i]
            # the phi map is float32 in the batch: round it the same way solo
            phi32 = float(np.float32(setups[i][1]))
            u, v = _read(gpu, b, i, W, H)
            us, vs = _solo(gpu, W, H, eps, phi32, disks, n, prec, k=1)
            assert np.array_equal(u, us) and np.array_equal(v, vs), (i, W, H)
    finally:
        gpu.rdc_batch_destroy(b)


def test_batch_f64_equals_oracle(gpu, orc, om):
    sizes = [(40, 23), (17, 64), (5, 5)]
    b, setups = _make_batch(gpu, "f64", 2, sizes)
    try:
        n = 45
        gpu.rdc_batch_step(b, None, n)
        for i, (W, H) in enumerate(sizes):
            eps, phi, disks = setups[i]
            phi_map = np.full((H, W), float(np.float32(phi)))
            u0, v0 = orc.rest_field(phi_map)
            for (cx, cy, r, val) in disks:
                orc.seed_disk(u0, cx, cy, r, val)
            ref = orc.run(phi_map, u0, v0, n, params=om.Params(eps=eps))
            u, v = _read(gpu, b, i, W, H)
            assert np.array_equal(u, ref["u"]) and np.array_equal(v, ref["v"]), i
    finally:
        gpu.rdc_batch_destroy(b)


def test_batch_subsets_and_graphs(gpu):
    """Stepping subsets in any order, with or without graphs, leaves each grid
    where its own step count says."""
    b, setups = _make_batch(gpu, "f32", 4)
    try:
        counts = [0] * len(SIZES)
        plan = [([0, 2, 4], 9), (None, 4), ([1, 6], 7), ([3], 1), ([5, 0], 12), (None, 3)]
        for j, (sub, n) in enumerate(plan):
            gpu.rdc_batch_set_config(b, 4, 8 if j % 2 else 16, 32 + 16 * j, graphs=(j % 3 != 1))
            gpu.rdc_batch_step(b, sub, n)
            for i in (range(len(SIZES)) if sub is None else sub):
                counts[i] += n
        # the same plan twice more: graph replays
        for sub, n in plan[:2]:
            gpu.rdc_batch_step(b, sub, n)
            for i in (range(len(SIZES)) if sub is None else sub):
                counts[i] += n
        info = gpu.rdc_batch_get_info(b)
        assert info.graph_launches >= 1
        for i, (W, H) in enumerate(SIZES):
            eps, phi, disks = setups[i]
            u, v = _read(gpu, b, i, W, H)
            us, vs = _solo(gpu, W, H, eps, float(np.float32(phi)), disks, counts[i], "f32")
            assert np.array_equal(u, us) and np.array_equal(v, vs), (i, counts[i])
    finally:
        gpu.rdc_batch_destroy(b)


def test_two_batches_on_two_streams(gpu):
    """Two batches stepped concurrently on their own streams (each batch's
    work queue is its own): every grid equals the same grid run alone."""
    import torch
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    made = []
    try:
        for st, k in ((s1, 6), (s2, 5)):
            grids, params, phis, setups = [], [], [], []
            for i, (W, H) in enumerate(SIZES):
                eps, phi, disks = _grid_setup(i, W, H)
                grids.append((W, H))
                params.append(gpu.rdc_params_default(precision=0, eps=eps, k_block=k))
                phis.append(np.full((H, W), phi, dtype=np.float32))
                setups.append((eps, phi, disks))
            b = gpu.rdc_batch_create(grids, params, phis, stream=st.cuda_stream)
            made.append((b, setups))
            for i, (_, _, disks) in enumerate(setups):
                for d in disks:
                    gpu.rdc_batch_seed(b, i, *d)
        for _ in range(6):                  # interleaved, no host sync between
            for b, _ in made:
                gpu.rdc_batch_step(b, None, 11)
        torch.cuda.synchronize()
        for b, setups in made:
            for i, (W, H) in enumerate(SIZES):
                eps, phi, disks = setups[i]
                u, v = _read(gpu, b, i, W, H)
                us, vs = _solo(gpu, W, H, eps, float(np.float32(phi)), disks, 66, "f32")
                assert np.array_equal(u, us) and np.array_equal(v, vs), (i, W, H)
    finally:
        for b, _ in made:
            gpu.rdc_batch_destroy(b)


def test_batch_tune_keeps_state(gpu):
    b, setups = _make_batch(gpu, "f32", 1)
    try:
        gpu.rdc_batch_step(b, None, 6)
        before = [_read(gpu, b, i, W, H) for i, (W, H) in enumerate(SIZES)]
        info = gpu.rdc_batch_tune(b, 2)
        assert info.tuned_gcups > 0 and 1 <= info.k <= 8
        after = [_read(gpu, b, i, W, H) for i, (W, H) in enumerate(SIZES)]
        for (u0, v0), (u1, v1) in zip(before, after):
            assert np.array_equal(u0, u1) and np.array_equal(v0, v1)
        gpu.rdc_batch_step(b, None, 11)
        for i, (W, H) in enumerate(SIZES):
            eps, phi, disks = setups[i]
            u, _ = _read(gpu, b, i, W, H)
            us, _ = _solo(gpu, W, H, eps, float(np.float32(phi)), disks, 17, "f32")
            assert np.array_equal(u, us)
    finally:
        gpu.rdc_batch_destroy(b)


def test_batch_add_remove(gpu):
    p = gpu.rdc_params_default(precision=0, k_block=2)
    b = gpu.rdc_batch_create([], [p])
    try:
        a = gpu.rdc_batch_add(b, 100, 50, p)
        c = gpu.rdc_batch_add(b, 64, 200, p)
        gpu.rdc_batch_seed(b, a, 50, 25, 6, 0.8)
        gpu.rdc_batch_step(b, None, 10)
        gpu.rdc_batch_remove(b, a)
        d = gpu.rdc_batch_add(b, 80, 80, p)       # reuses the freed slot
        assert d == a
        gpu.rdc_batch_seed(b, d, 40, 40, 5, 0.8)
        gpu.rdc_batch_seed(b, c, 32, 100, 5, 0.8)
        gpu.rdc_batch_step(b, None, 9)
        u, _ = _read(gpu, b, d, 80, 80)
        us, _ = _solo(gpu, 80, 80, p.eps, 0.054, [(40, 40, 5, 0.8)], 9, "f32")
        assert np.array_equal(u, us)
        u, _ = _read(gpu, b, c, 64, 200)
        # grid c: 10 steps, seed, 9 steps
        p1 = gpu.rdc_params_default(precision=0)
        h = gpu.rdc_create(64, 200, p1)
        try:
            gpu.rdc_step(h, 10)
            gpu.rdc_seed(h, 32, 100, 5, 0.8)
            gpu.rdc_step(h, 9)
            ref = np.empty((200, 64))
            gpu.rdc_read(h, ref, None)
        finally:
            gpu.rdc_destroy(h)
        assert np.array_equal(u, ref)
        info = gpu.rdc_batch_get_info(b)
        assert info.ngrids == 2 and info.slots == 2
    finally:
        gpu.rdc_batch_destroy(b)


def test_batch_sweep_workload_small(gpu):
    """A scaled-down parameter sweep (sizes 128/256, phi ~ U[0.05, 0.08],
    eps ~ U[0.02, 0.03], 1-8 disks): tuned batch equals solo runs."""
    spec = ri.sweep_batch(seed=4, n_grids=12, sizes=(128, 256))
    grids = [(n, n) for n in spec.sizes]
    params = [gpu.rdc_params_default(precision=0, eps=e) for e in spec.eps]
    phis = [np.full((n, n), ph, dtype=np.float32) for n, ph in zip(spec.sizes, spec.phi)]
    b = gpu.rdc_batch_create(grids, params, phis)
    try:
        for i, disks in enumerate(spec.disks):
            for (cx, cy, r) in disks:
                gpu.rdc_batch_seed(b, i, cx, cy, r, 0.8)
        gpu.rdc_batch_tune(b, 2)
        gpu.rdc_batch_step(b, None, 50)
        for i in (0, 5, 11):
            n = spec.sizes[i]
            u, _ = _read(gpu, b, i, n, n)
            us, _ = _solo(gpu, n, n, spec.eps[i], float(np.float32(spec.phi[i])),
                          [(cx, cy, r, 0.8) for (cx, cy, r) in spec.disks[i]], 50, "f32")
            assert np.array_equal(u, us)
    finally:
        gpu.rdc_batch_destroy(b)


def test_sweep_grid_that_crosses_the_pole(gpu, orc, om):
    """Grid 257 of the 512-grid sweep (256 x 256, eps = 0.02004, phi = 0.070)
    overshoots past the pole u = -q in the wave tail: the FP64 oracle reports
    it at step 419.  The FP64 GPU path is bit-identical, so its health flag
    must be clear after 418 steps and raised after 419."""
    spec = ri.sweep_batch(seed=4, n_grids=512)
    i = 257
    n = spec.sizes[i]
    phi = np.full((n, n), float(np.float32(spec.phi[i])))
    u0, v0 = orc.rest_field(phi)
    for (cx, cy, r) in spec.disks[i]:
        orc.seed_disk(u0, cx, cy, r, 0.8)
    ref = orc.run(phi, u0, v0, 500, params=om.Params(eps=spec.eps[i]))
    assert ref["status"] == om.ENONFINITE
    bad_step = ref["bad_step"]
    p = gpu.rdc_params_default(precision=1, eps=spec.eps[i], k_block=1)
    h = gpu.rdc_create(n, n, p, phi)
    try:
        for (cx, cy, r) in spec.disks[i]:
            gpu.rdc_seed(h, cx, cy, r, 0.8)
        gpu.rdc_step(h, bad_step - 1)
        assert gpu.rdc_check(h) == (0, -1)
        gpu.rdc_step(h, 1)
        rc, idx = gpu.rdc_check(h)
        assert rc == gpu.RDC_ENONFINITE and idx == ref["bad_index"]
    finally:
        gpu.rdc_destroy(h)
