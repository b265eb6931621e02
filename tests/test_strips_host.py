"""The row-strip plan of paper_1901_06535_gb300.strips, on the CPU.

The plan's rows and copies are checked as sets, and then driven with the
FP64 oracle as the stepper: every strip is its own grid of the rows it holds
(mirror borders at the cut), the plan's copies fill the halos, and the
strips' own rows must equal the unsplit oracle bit for bit (Eq. 1 couples
rows only through the Laplacian of u).  Also: the row-copy entry points
refuse a NULL simulation without touching a device.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_1901_06535_gb300.strips import strip_plan


@pytest.mark.parametrize("height,n,halo", [(29, 2, 4), (30, 3, 1), (37, 3, 6), (64, 4, 8),
                                           (17, 1, 5), (13, 2, 6)])
def test_plan_rows_and_copies(height, n, halo):
    strips, transfers = strip_plan(height, n, halo)
    owned = [r for s in strips for r in range(s.r0, s.r1)]
    assert owned == list(range(height))                       # a partition, in order
    assert max(s.r1 - s.r0 for s in strips) - min(s.r1 - s.r0 for s in strips) <= 1
    for s in strips:
        assert s.e0 == max(s.r0 - halo, 0) and s.e1 == min(s.r1 + halo, height)
    halo_rows = {(s.index, r) for s in strips for r in range(s.e0, s.e1) if not s.r0 <= r < s.r1}
    filled = set()
    for t in transfers:
        src, dst = strips[t.src], strips[t.dst]
        for k in range(t.nrows):
            g_src = src.e0 + t.src_row + k
            g_dst = dst.e0 + t.dst_row + k
            assert g_src == g_dst                              # the same whole-grid row
            assert src.r0 <= g_src < src.r1                    # sent from the sender's own rows
            assert (t.dst, g_dst) not in filled
            filled.add((t.dst, g_dst))
    assert filled == halo_rows                                 # every halo row, once


@pytest.mark.parametrize("height,n,halo", [(10, 3, 4), (7, 2, 4), (0, 1, 1), (8, 0, 1), (8, 2, 0)])
def test_plan_refuses(height, n, halo):
    with pytest.raises(ValueError):
        strip_plan(height, n, halo)


def _initial(orc, W, H):
    phi = np.full((H, W), 0.054)
    phi[:, W // 2:W // 2 + 3] = 0.0975
    u, v = orc.rest_field(phi)
    orc.seed_disk(u, 10.0, H / 2 - 1.5, 6.0, 0.8)          # across a strip boundary
    orc.seed_disk(u, W - 7.0, 3.0, 4.0, 1.0)
    return phi, u, v


@pytest.mark.parametrize("n,halo,steps", [(2, 1, 23), (3, 4, 50), (4, 6, 61), (3, 5, 7)])
def test_plan_driven_oracle_equals_unsplit(orc, n, halo, steps):
    W, H = 33, 31
    phi, u, v = _initial(orc, W, H)
    ref = orc.run(phi, u, v, steps)
    strips, transfers = strip_plan(H, n, halo)
    su = [u[s.e0:s.e1].copy() for s in strips]
    sv = [v[s.e0:s.e1].copy() for s in strips]
    left = steps
    while left > 0:
        m = min(left, halo)
        for t in transfers:
            rows = slice(t.src_row, t.src_row + t.nrows)
            su[t.dst][t.dst_row:t.dst_row + t.nrows] = su[t.src][rows]
            sv[t.dst][t.dst_row:t.dst_row + t.nrows] = sv[t.src][rows]
        for i, s in enumerate(strips):
            out = orc.run(np.ascontiguousarray(phi[s.e0:s.e1]), su[i], sv[i], m)
            su[i], sv[i] = out["u"], out["v"]
        left -= m
    got_u = np.concatenate([su[i][s.r0 - s.e0:s.r1 - s.e0] for i, s in enumerate(strips)])
    got_v = np.concatenate([sv[i][s.r0 - s.e0:s.r1 - s.e0] for i, s in enumerate(strips)])
    assert np.array_equal(got_u, ref["u"]) and np.array_equal(got_v, ref["v"])


def test_plan_driven_oracle_needs_the_exchange(orc):
    """Control: stepping past the halo without an exchange leaves the strips'
    own rows wrong near the cut (so the equality above tests the copies)."""
    W, H, halo = 33, 31, 2
    phi, u, v = _initial(orc, W, H)
    ref = orc.run(phi, u, v, 12)
    strips, _ = strip_plan(H, 2, halo)
    s = strips[0]
    out = orc.run(np.ascontiguousarray(phi[s.e0:s.e1]), u[s.e0:s.e1].copy(),
                  v[s.e0:s.e1].copy(), 12)
    assert not np.array_equal(out["u"][:s.r1 - s.e0], ref["u"][s.r0:s.r1])


def test_row_copies_refuse_null_sim(librdc):
    L = librdc.lib()
    buf = (ctypes.c_float * 64)()
    for fn in (L.rdc_get_rows, L.rdc_put_rows):
        assert fn(None, 0, 1, buf, buf, 0) == librdc.RDC_EINVAL
        assert fn(None, 0, 0, None, None, 0) == librdc.RDC_EINVAL


def test_strip_grid_refuses_before_touching_the_device(librdc):
    """Stochastic rounding and a halo wider than a strip are refused before
    any simulation is created (no device needed)."""
    from paper_1901_06535_gb300.strips import StripGrid
    with pytest.raises(ValueError):
        StripGrid(64, 64, 2, precision="bf16", flags=librdc.RDC_STOCH_ROUND, round_seed=3)
    with pytest.raises(ValueError):
        StripGrid(64, 10, 3, halo=4)                 # strips of 3 and 4 rows
    with pytest.raises(ValueError):
        StripGrid(64, 64, 2, phi=np.zeros((63, 64), np.float32))
