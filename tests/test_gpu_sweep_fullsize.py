"""Parity of the 512-grid parameter sweep at its full size (sizes from
{128, 256, 512, 1024}^2, 188 M cells, per-grid eps and phi, 1-8 disks each) in
the launch shapes the benchmark times: all grids stepped together by the
batched kernels, then sampled grids compared with the FP64 oracle run on the
same whole grid.  The bound is the early-pointwise one: a few FP32 roundings
of the largest state value per step, times the steps, with a safety factor."""
from __future__ import annotations

import numpy as np
import pytest

import rdc_inputs as ri

pytestmark = pytest.mark.gpu

STEPS = 60
TOL = 1e-5


def _sample(spec):
    idx = {0, 1, 2, 511}
    for size in (128, 256, 512, 1024):
        idx.add(next(i for i, n in enumerate(spec.sizes) if n == size))
    return sorted(idx)


@pytest.mark.parametrize("k,krows", [(6, 128), (4, 128)])
def test_sweep_fullsize_sampled_grids(gpu, orc, om, k, krows, record_property):
    spec = ri.sweep_batch(seed=4, n_grids=512)
    grids = [(n, n) for n in spec.sizes]
    params = [gpu.rdc_params_default(precision=0, eps=e) for e in spec.eps]
    phis = [np.full((n, n), ph, dtype=np.float32) for n, ph in zip(spec.sizes, spec.phi)]
    b = gpu.rdc_batch_create(grids, params, phis)
    got = {}
    try:
        for i, disks in enumerate(spec.disks):
            for (cx, cy, r) in disks:
                gpu.rdc_batch_seed(b, i, cx, cy, r, ri.SEED_VALUE)
        gpu.rdc_batch_set_config(b, k, 16, krows, True)
        gpu.rdc_batch_step(b, None, STEPS)
        for i in _sample(spec):
            n = spec.sizes[i]
            assert gpu.rdc_batch_check(b, i)[0] == gpu.RDC_OK, i
            u = np.empty((n, n))
            v = np.empty((n, n))
            gpu.rdc_batch_read(b, i, u, v)
            got[i] = (u, v)
    finally:
        gpu.rdc_batch_destroy(b)
    worst = {}
    for i, (u, v) in got.items():
        n = spec.sizes[i]
        phi = np.full((n, n), float(np.float32(spec.phi[i])))
        u0, v0 = orc.rest_field(phi)
        for (cx, cy, r) in spec.disks[i]:
            orc.seed_disk(u0, cx, cy, r, ri.SEED_VALUE)
        ref = orc.run(phi, u0, v0, STEPS, params=om.Params(eps=spec.eps[i]), nthreads=4)
        assert ref["status"] == om.OK
        worst[i] = float(max(np.max(np.abs(u - ref["u"])), np.max(np.abs(v - ref["v"]))))
    record_property("sweep_maxabs", worst)
    assert max(worst.values()) <= TOL, worst
