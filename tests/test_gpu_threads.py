"""Separate handles used from several host threads at once.

The C ABI promises that distinct handles may be used from distinct threads
(a handle itself is not thread-safe).  Each case below creates its own
simulation or batch, stimulates it, steps it and reads it back; the cases run
first one after another, then all at once from a thread pool (ctypes releases
the interpreter lock during each library call, so the calls overlap), twice.
Every concurrent result must equal the sequential one bit for bit.  The cases
cover every kernel family: the single step, the streamed and shared-memory
temporally blocked kernels (two of them above 48 KB of shared memory, whose
attribute the library raises once per device), stochastic rounding, FP64 and
a batch.
"""
from __future__ import annotations

import concurrent.futures

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W, H, STEPS = 300, 200, 120


def _sim_case(gpu, precision, shape=None, **params):
    def run():
        s = gpu.Sim(W, H, precision=precision, **params)
        if shape:
            s.set_shape(**shape)
        s.seed(W / 3.0, H / 2.0, 9.0, 0.8)
        s.seed(2 * W / 3.0 + 0.25, H / 3.0, 6.0, 0.8)
        s.step(STEPS)
        out = s.read()
        s.close()
        return out
    return run


def _batch_case(gpu):
    def run():
        grids = [(96, 64), (130, 70), (64, 64)]
        ps = [gpu.rdc_params_default(k_block=4) for _ in grids]
        b = gpu.rdc_batch_create(grids, ps)
        for i, (w, h) in enumerate(grids):
            gpu.rdc_batch_seed(b, i, w / 2.0, h / 2.0, 5.0, 0.8)
        gpu.rdc_batch_step(b, None, STEPS)
        out = []
        for i, (w, h) in enumerate(grids):
            u = np.empty((h, w))
            v = np.empty_like(u)
            gpu.rdc_batch_read(b, i, u, v)
            out.append((u, v))
        gpu.rdc_batch_destroy(b)
        return out
    return run


def _cases(gpu):
    return [
        _sim_case(gpu, "f32", k_block=1),
        _sim_case(gpu, "f32", k_block=5),
        _sim_case(gpu, "bf16", shape=dict(k=4, variant=1, tx=64, ty=64, nthreads=512)),
        _sim_case(gpu, "f32", shape=dict(k=6, variant=1, tx=64, ty=32, nthreads=256)),
        _sim_case(gpu, "f16", flags=gpu.RDC_STOCH_ROUND, round_seed=11),
        _sim_case(gpu, "f64", k_block=1),
        _sim_case(gpu, "f16", k_block=3),
        _batch_case(gpu),
    ]


def _same(a, b):
    if isinstance(a, list):
        return all(_same(x, y) for x, y in zip(a, b)) and len(a) == len(b)
    return all(np.array_equal(x, y) for x, y in zip(a, b))


def test_separate_handles_from_threads_equal_sequential(gpu):
    cases = _cases(gpu)
    ref = [c() for c in cases]
    for _ in range(2):
        with concurrent.futures.ThreadPoolExecutor(max_workers=len(cases)) as ex:
            got = list(ex.map(lambda c: c(), cases))
        for i, (r, g) in enumerate(zip(ref, got)):
            assert _same(r, g), f"case {i} differs when run concurrently"
