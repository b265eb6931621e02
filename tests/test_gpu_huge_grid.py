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
