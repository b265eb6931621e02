"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds geometry and random draws only -- excitability (phi) maps,
stimulus disks, probe positions, batch and session descriptions.  It holds
none of the model's arithmetic (no reaction term, no Laplacian, no rest
state), so that the CUDA path and the oracle can both consume its outputs
without sharing any of the method.

Conventions: a grid is H rows x W columns, row-major; cell (i, j) has its
centre at x = j, y = i; a disk is (cx, cy, r) in those units.  Random draws
use NumPy's PCG64 ``default_rng(seed)``.

The workloads stand in for the paper's hand-drawn circuits (§4): the paper
uses no dataset, and its figures are not available, so every geometry here is
synthetic, built from the written description of each circuit.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Table 1 values used as map levels.
PHI_ACTIVE = 0.054
PHI_PASSIVE_PAPER = 0.0975
PHI_PASSIVE_STRONG = 0.2     # the strongly inhibiting background used by the workloads
SEED_VALUE = 0.8


# ---------------------------------------------------------------------------
# geometry primitives
# ---------------------------------------------------------------------------

def _centres(W: int, H: int):
    y, x = np.mgrid[0:H, 0:W]
    return x.astype(np.float64), y.astype(np.float64)


def capsule_mask(W: int, H: int, x0: float, y0: float, x1: float, y1: float,
                 width: float) -> np.ndarray:
    """Cells whose centre lies within width/2 of the segment (x0,y0)-(x1,y1)."""
    x, y = _centres(W, H)
    dx, dy = x1 - x0, y1 - y0
    L2 = dx * dx + dy * dy
    if L2 == 0.0:
        t = np.zeros_like(x)
    else:
        t = np.clip(((x - x0) * dx + (y - y0) * dy) / L2, 0.0, 1.0)
    px, py = x0 + t * dx, y0 + t * dy
    return (x - px) ** 2 + (y - py) ** 2 <= (0.5 * width) ** 2


def rect_mask(W: int, H: int, x0: float, y0: float, x1: float, y1: float) -> np.ndarray:
    """Cells with x0 <= x < x1 and y0 <= y < y1."""
    x, y = _centres(W, H)
    return (x >= x0) & (x < x1) & (y >= y0) & (y < y1)


def polygon_mask(W: int, H: int, pts) -> np.ndarray:
    """Cells whose centre is inside the polygon (even-odd rule)."""
    x, y = _centres(W, H)
    inside = np.zeros((H, W), dtype=bool)
    n = len(pts)
    for a in range(n):
        xa, ya = pts[a]
        xb, yb = pts[(a + 1) % n]
        cond = (ya > y) != (yb > y)
        with np.errstate(divide="ignore", invalid="ignore"):
            xi = xa + (y - ya) * (xb - xa) / (yb - ya)
        inside ^= cond & (x < xi)
    return inside


def disk_cells(W: int, H: int, cx: float, cy: float, r: float) -> np.ndarray:
    """Boolean mask of (i - cy)^2 + (j - cx)^2 <= r^2 (used by geometry code
    to keep probes and seeds inside channels; not a stimulation step)."""
    x, y = _centres(W, H)
    return (x - cx) ** 2 + (y - cy) ** 2 <= r * r


def uniform_phi(W: int, H: int, phi: float = PHI_ACTIVE, dtype=np.float64) -> np.ndarray:
    return np.full((H, W), phi, dtype=dtype)


# ---------------------------------------------------------------------------
# circuits (§4)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Circuit:
    """A phi map plus where to stimulate it and where to look."""
    phi: np.ndarray
    seeds: dict            # name -> (cx, cy, r)
    probes: dict           # name -> flat cell index
    meta: dict


# Calibrated on the oracle (tests/golden/and_gate_window.txt): a single wave
# crosses a 3-cell band up to phi_gap ~ 0.0901, two colliding waves up to
# ~ 0.0920; 0.091 sits in the middle of that window.
AND_GAP_CELLS = 3
AND_PHI_GAP = 0.091


def and_gate(W: int = 256, H: int = 256, *, channel: float = 16.0,
             gap: float = AND_GAP_CELLS, arm: float = 80.0, out_len: float = 60.0,
             angle_deg: float = 0.0, out_width: float | None = None,
             phi_gap: float | None = AND_PHI_GAP,
             phi_active: float = PHI_ACTIVE,
             phi_passive: float = PHI_PASSIVE_STRONG,
             seed_r: float = 6.0) -> Circuit:
    """Coincidence detector (AND gate, §4.1).

    Two input channels of width ``channel`` run toward a junction from the
    left and the right (``angle_deg`` below the horizontal; 0 = head-on) and
    the output channel runs straight down from the junction.  A band of
    ``gap`` cells of weakly inhibiting substrate (``phi_gap``; a 3-cell
    "semi-permeable" line, §3) separates the junction from the output
    channel, so that (per §4.1) only the collision of two input waves
    opposite the output crosses it.  ``phi_gap=None`` makes the band plain
    background.
    Inputs A and B are stimulated at the far ends of the two arms; the output
    probe sits ``out_len/2`` cells into the output channel.
    """
    x_c = (W - 1) / 2.0
    y_j = H * 0.45
    th = math.radians(angle_deg)
    ddx, ddy = arm * math.cos(th), arm * math.sin(th)
    ax, ay = x_c - ddx, y_j - ddy
    bx, by = x_c + ddx, y_j - ddy
    act = capsule_mask(W, H, ax, ay, x_c, y_j, channel)
    act |= capsule_mask(W, H, bx, by, x_c, y_j, channel)
    y_gap0 = y_j + 0.5 * channel
    y_out0 = y_gap0 + gap
    act &= ~(_centres(W, H)[1] >= y_gap0)           # nothing of the arms below the gap line
    ow = channel if out_width is None else out_width
    act |= rect_mask(W, H, x_c - 0.5 * ow, y_out0, x_c + 0.5 * ow,
                     y_out0 + out_len)
    phi = np.where(act, phi_active, phi_passive).astype(np.float64)
    if phi_gap is not None:
        band = rect_mask(W, H, x_c - 0.5 * ow - gap, y_gap0, x_c + 0.5 * ow + gap, y_out0)
        phi[band] = phi_gap
    # seeds one channel-radius in from each arm's far end, along the arm
    s = 0.5 * channel + 1.0
    seeds = {"A": (ax + s * math.cos(th), ay + s * math.sin(th), seed_r),
             "B": (bx - s * math.cos(th), by + s * math.sin(th), seed_r)}
    py = int(round(y_out0 + 0.5 * out_len))
    px = int(round(x_c))
    probes = {"out": py * W + px,
              "junction": int(round(y_j)) * W + px}
    return Circuit(phi, seeds, probes,
                   {"kind": "and_gate", "channel": channel, "gap": gap,
                    "arm": arm, "out_len": out_len, "angle_deg": angle_deg,
                    "out_width": ow,
                    "phi_active": phi_active,
                    "phi_passive": phi_passive, "y_gap0": y_gap0,
                    "y_out0": y_out0})


# Calibrated on the oracle (tests/golden/diode_calibration.txt): with a
# 24-cell channel and a 1-cell gap, gap levels phi in [0.11, 0.115] with
# points of 4 to 10 cells all pass anode -> cathode and block cathode ->
# anode; (0.11, 8) has a working neighbour on every side.
DIODE_GAP_CELLS = 1
DIODE_TIP_CELLS = 8.0
DIODE_CHANNEL = 24.0
DIODE_PHI_GAP = 0.11


def diode(W: int = 128, H: int = 48, *, channel: float = DIODE_CHANNEL,
          gap: float = DIODE_GAP_CELLS, tip: float = DIODE_TIP_CELLS,
          phi_active: float = PHI_ACTIVE,
          phi_passive: float = PHI_PASSIVE_STRONG,
          phi_gap: float | None = DIODE_PHI_GAP,
          seed_r: float = 6.0, flip: bool = False) -> Circuit:
    """Chemical diode (§4.2).

    A horizontal active channel of width ``channel`` is cut by a passive gap.
    The anode side ends flat at the gap; the cathode side ends in a triangle
    whose point (``tip`` cells long) faces the gap.  Inside the channel's
    bounding box the non-active cells (the gap and the flanks of the point)
    hold ``phi_gap`` (a weaker inhibitor than the background); everything
    else is ``phi_passive``.  By the paper's account a
    wave passes from anode to cathode but not from cathode to anode.  The
    anode is on the left (``flip`` mirrors the map left-right).  Seeds sit at
    the two far ends; probes sit near each end, past the gap.
    """
    y_c = (H - 1) / 2.0
    x_gap0 = W * 0.5 - 0.5 * gap
    x_gap1 = x_gap0 + gap
    half = 0.5 * channel
    act = rect_mask(W, H, 0.0, y_c - half, x_gap0, y_c + half + 1e-9)     # anode, flat end
    cat = rect_mask(W, H, x_gap1 + tip, y_c - half, float(W), y_c + half + 1e-9)
    cat |= polygon_mask(W, H, [(x_gap1 + tip + 0.5, y_c - half - 0.5),
                               (x_gap1 + tip + 0.5, y_c + half + 0.5),
                               (x_gap1, y_c)])
    act |= cat
    phi = np.where(act, phi_active, phi_passive).astype(np.float64)
    if phi_gap is not None:
        box = rect_mask(W, H, x_gap0, y_c - half, x_gap1 + tip + 1.0, y_c + half + 1e-9)
        phi[box & ~act] = phi_gap
    seeds = {"anode": (8.0, y_c, seed_r), "cathode": (W - 9.0, y_c, seed_r)}
    yi = int(round(y_c))
    probes = {"anode_end": yi * W + 4, "cathode_end": yi * W + (W - 5)}
    if flip:
        phi = phi[:, ::-1].copy()
        seeds = {"anode": (W - 1 - 8.0, y_c, seed_r), "cathode": (8.0, y_c, seed_r)}
        probes = {"anode_end": yi * W + (W - 5), "cathode_end": yi * W + 4}
    return Circuit(phi, seeds, probes,
                   {"kind": "diode", "channel": channel, "gap": gap, "tip": tip,
                    "phi_active": phi_active, "phi_passive": phi_passive,
                    "flip": flip})


# ---------------------------------------------------------------------------
# random workloads
# ---------------------------------------------------------------------------

def random_disks(seed: int, n: int, W: int, H: int, rmin: int = 4, rmax: int = 10):
    """n disks with integer radius U{rmin..rmax} and centre U[0,W) x U[0,H)."""
    rng = np.random.default_rng(seed)
    r = rng.integers(rmin, rmax + 1, size=n)
    cx = rng.uniform(0.0, W, size=n)
    cy = rng.uniform(0.0, H, size=n)
    return [(float(a), float(b), float(c)) for a, b, c in zip(cx, cy, r)]


def centre(W: int, H: int):
    """Geometric centre in cell-index units ((W-1)/2, (H-1)/2)."""
    return (W - 1) / 2.0, (H - 1) / 2.0


def axis_probes(W: int, H: int, distances=(20, 40, 60)):
    """Flat indices of cells on the +x axis at the given distances from the
    integer cell nearest the centre."""
    cy = H // 2
    cx = W // 2
    return [cy * W + (cx + d) for d in distances if cx + d < W]


@dataclasses.dataclass
class BatchSpec:
    sizes: list          # N per grid (square N x N)
    phi: list            # uniform phi per grid
    eps: list            # epsilon per grid
    disks: list          # list of disk lists per grid


def sweep_batch(seed: int = 4, n_grids: int = 512, sizes=(128, 256, 512, 1024),
                phi_range=(0.05, 0.08), eps_range=(0.02, 0.03),
                max_disks: int = 8) -> BatchSpec:
    """Parameter sweep of independent square grids of uneven sizes."""
    rng = np.random.default_rng(seed)
    N = rng.choice(np.asarray(sizes), size=n_grids)
    phi = rng.uniform(*phi_range, size=n_grids)
    eps = rng.uniform(*eps_range, size=n_grids)
    disks = []
    for g in range(n_grids):
        k = int(rng.integers(1, max_disks + 1))
        r = rng.integers(4, 11, size=k)
        cx = rng.uniform(0.0, N[g], size=k)
        cy = rng.uniform(0.0, N[g], size=k)
        disks.append([(float(a), float(b), float(c)) for a, b, c in zip(cx, cy, r)])
    return BatchSpec([int(n) for n in N], [float(p) for p in phi],
                     [float(e) for e in eps], disks)


@dataclasses.dataclass
class SessionSpec:
    sid: int
    size: int
    phi: np.ndarray            # size x size float32
    touches: list              # per frame: (cx, cy, r, value)
    arrival: float             # seconds from the start


def diode_sessions(seed: int = 5, n: int = 64, sizes=(512, 1024, 2048), rate: float = 20.0,
                   frames: int = 20, touch_r: float = 6.0) -> list:
    """Interactive sessions: Poisson arrivals at ``rate`` per second, square
    grids of a random size, each a diode channel (see ``diode``) placed at a
    random position and orientation in a phi = 0.2 background; each frame
    starts with a u = 0.8 touch disk at a random point of the channel's anode
    half."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for sid in range(n):
        t += float(rng.exponential(1.0 / rate))
        N = int(rng.choice(np.asarray(sizes)))
        band_h = 48
        c = diode(N, band_h, flip=bool(rng.integers(0, 2)))
        phi = np.full((N, N), PHI_PASSIVE_STRONG, dtype=np.float32)
        y0 = int(rng.integers(0, N - band_h))
        phi[y0:y0 + band_h, :] = c.phi.astype(np.float32)
        ax, ay, _ = c.seeds["anode"]
        vertical = bool(rng.integers(0, 2))
        touches = []
        lo, hi = (4.0, N / 2 - 10.0) if ax < N / 2 else (N / 2 + 10.0, N - 5.0)
        for _ in range(frames):
            x = float(rng.uniform(lo, hi))
            y = float(y0 + ay + rng.uniform(-4, 4))
            touches.append((y, x, touch_r, SEED_VALUE) if vertical else (x, y, touch_r, SEED_VALUE))
        if vertical:
            phi = np.ascontiguousarray(phi.T)
        out.append(SessionSpec(sid, N, phi, touches, t))
    return out
