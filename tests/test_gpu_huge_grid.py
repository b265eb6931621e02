"""A grid with more than 2^31 cells (65536 x 33000 = 2.16e9 cells, 43 GB of
FP32 state and phi): stimulation, the single-step and streamed kernels, the
health check and probes address cells beyond index 2^31 correctly.  Cells
near the far corner are compared with the oracle on a window cut at the
grid's border (after n steps a cell depends only on cells within n)."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

W, H = 65536, 33000
SEED = (65500.0, 32990.0, 6.0, 0.8)          # near the bottom-right corner


PROBE_ROWS, PROBE_COLS = 20, 60                 # the probed block in the far corner


def _oracle_window(orc, om, n):
    # the window reaches the grid's right and bottom borders; its top and
    # left edges (cut, not borders) lie n + 2 cells beyond the probed block
    i0 = H - PROBE_ROWS - (n + 2)
    j0 = W - PROBE_COLS - (n + 2)
    h, w = H - i0, W - j0
    phi = np.full((h, w), 0.054)
    u, v = orc.rest_field(phi)
    orc.seed_disk(u, SEED[0] - j0, SEED[1] - i0, SEED[2], SEED[3])
    out = orc.run(phi, u, v, n)
    return out["u"], i0, j0


@pytest.mark.parametrize("k", [1, 4])
def test_beyond_2_pow_31_cells(gpu, orc, om, k):
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 60 * 2**30:
        pytest.skip("needs about 45 GB of free device memory")
    n = 8
    p = gpu.rdc_params_default(precision=0, k_block=k)
    h = gpu.rdc_create(W, H, p)
    try:
        gpu.rdc_seed(h, *SEED)
        gpu.rdc_step(h, n)
        assert gpu.rdc_check(h) == (0, -1)
        ref, i0, j0 = _oracle_window(orc, om, n)
        rows = np.arange(H - PROBE_ROWS, H)
        cols = np.arange(W - PROBE_COLS, W)
        ii, jj = np.meshgrid(rows, cols, indexing="ij")
        cells = (ii.astype(np.int64) * W + jj).ravel()
        assert cells.min() > 2**31
        got = gpu.rdc_probe(h, cells).reshape(ii.shape)
    finally:
        gpu.rdc_destroy(h)
    want = ref[ii - i0, jj - j0]
    assert np.max(np.abs(got - want)) < 4e-6
    assert np.max(got) > 0.5                     # the stimulated disk is there


def test_tall_grid_default_shape(gpu, orc, om):
    """A grid taller than 65535 x 64 rows (64 x 4,200,000): the default
    launch shapes (k = 4 streamed steps) and the autotuner's candidates keep
    gridDim.y within its 65535 limit, and the cells near the bottom border
    match the oracle."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < 8 * 2**30:
        pytest.skip("needs about 6 GB of free device memory")
    w, h_rows, n = 64, 4_200_000, 8
    seed = (40.0, h_rows - 12.0, 6.0, 0.8)
    p = gpu.rdc_params_default(precision=0)
    h = gpu.rdc_create(w, h_rows, p)
    try:
        s = gpu.rdc_get_shape(h)
        assert s.k == 4 and s.variant == 0
        assert (h_rows + s.krows - 1) // s.krows <= 65535
        gpu.rdc_seed(h, *seed)
        gpu.rdc_step(h, n)
        assert gpu.rdc_check(h) == (0, -1)
        # the autotuner skips the shapes that would exceed the limit; its
        # timing launches leave the current state alone
        t, gcups = gpu.rdc_tune(h, reps=1)
        assert gcups > 0
        if t["k"] > 1:
            rows_per_cta = t["krows"] if t["variant"] == 0 else t["ty"]
            assert (h_rows + rows_per_cta - 1) // rows_per_cta <= 65535, t
        rows = np.arange(h_rows - PROBE_ROWS, h_rows)
        ii, jj = np.meshgrid(rows, np.arange(w), indexing="ij")
        got = gpu.rdc_probe(h, (ii.astype(np.int64) * w + jj).ravel()).reshape(ii.shape)
    finally:
        gpu.rdc_destroy(h)
    # oracle on the bottom rows: the window's top edge (a cut, not a border)
    # lies n + 2 rows above the probed block
    i0 = h_rows - PROBE_ROWS - (n + 2)
    phi = np.full((h_rows - i0, w), 0.054)
    u, v = orc.rest_field(phi)
    orc.seed_disk(u, seed[0], seed[1] - i0, seed[2], seed[3])
    ref = orc.run(phi, u, v, n)["u"]
    assert np.max(np.abs(got - ref[ii - i0, jj])) < 4e-6
    assert np.max(got) > 0.5
