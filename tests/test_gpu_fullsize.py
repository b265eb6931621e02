"""Parity at the benchmark's full size (8192 x 8192, 200 seeded disks) in the
benchmark's launch configuration, on sampled cells.

After n steps a cell depends only on the cells within n of it (five-point
stencil), so the oracle evaluates each sampled cell on a window of radius
n + 1 cut from its own initial state (rest state plus the same disks); where
the window reaches the grid's border it is cut there, and the mirror rule then
applies exactly as on the full grid.  No GPU value is ever an oracle input.
"""
from __future__ import annotations

import numpy as np
import pytest

import rdc_inputs as ri
from tests.helpers import PREC, round_to_storage

pytestmark = pytest.mark.gpu

N = 8192
DISKS = ri.random_disks(3, 200, N, N)


def _samples(rng, k):
    pts = [(0, 0), (0, N - 1), (N - 1, 0), (N - 1, N - 1), (N // 2, N // 2)]
    # cells on or next to disk rims, where the state changes fastest
    for (cx, cy, r) in DISKS[:k]:
        for ang in (0.3, 2.0, 4.1):
            i = int(round(cy + (r + 0.4) * np.sin(ang)))
            j = int(round(cx + (r + 0.4) * np.cos(ang)))
            if 0 <= i < N and 0 <= j < N:
                pts.append((i, j))
    pts += [tuple(x) for x in rng.integers(0, N, size=(k, 2))]
    return pts


def _oracle_cell(orc, i, j, n):
    R = n + 1
    i0, i1 = max(0, i - R), min(N, i + R + 1)
    j0, j1 = max(0, j - R), min(N, j + R + 1)
    h, w = i1 - i0, j1 - j0
    phi = np.full((h, w), ri.PHI_ACTIVE)
    u, v = orc.rest_field(phi)
    for (cx, cy, r) in DISKS:
        if cx + r + 1 < j0 or cx - r - 1 > j1 or cy + r + 1 < i0 or cy - r - 1 > i1:
            continue
        orc.seed_disk(u, cx - j0, cy - i0, r, ri.SEED_VALUE)
    out = orc.run(phi, u, v, n)
    return out["u"][i - i0, j - j0], out["v"][i - i0, j - j0], u[i - i0, j - j0]


@pytest.mark.parametrize("prec,k,n,tol", [("f64", 1, 3, 0.0), ("f64", 3, 3, 0.0),
                                          ("f32", 1, 4, 2e-6), ("f32", 4, 4, 2e-6),
                                          ("f32", 6, 6, 3e-6), ("f32", 0, 12, 5e-6),
                                          ("bf16", 4, 4, 2e-2), ("f16", 1, 4, 5e-3)])
def test_fullsize_sampled(gpu, orc, prec, k, n, tol):
    p = gpu.rdc_params_default(precision=PREC[prec], k_block=k)
    h = gpu.rdc_create(N, N, p)
    try:
        for (cx, cy, r) in DISKS:
            gpu.rdc_seed(h, cx, cy, r, ri.SEED_VALUE)
        rng = np.random.default_rng(7)
        pts = _samples(rng, 40)
        cells = np.array([i * N + j for i, j in pts], dtype=np.int64)
        u0 = gpu.rdc_probe(h, cells)
        gpu.rdc_step(h, n)
        assert gpu.rdc_check(h) == (0, -1)
        u_gpu = gpu.rdc_probe(h, cells)
    finally:
        gpu.rdc_destroy(h)
    worst = 0.0
    for c, (i, j) in enumerate(pts):
        uo, _, u0o = _oracle_cell(orc, i, j, n)
        assert u0[c] == round_to_storage(u0o, prec)        # same initial cell
        worst = max(worst, abs(u_gpu[c] - uo))
        if tol == 0.0:
            assert u_gpu[c] == uo, (i, j, u_gpu[c], uo)
    assert worst <= tol, worst
