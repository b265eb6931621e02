"""One grid stepped as row strips with a halo exchange.

In Eq. 1 only the Laplacian of u couples a row to its neighbours (v has no
diffusion term and phi is static).  A grid cut into strips of rows can
therefore be stepped strip by strip: each strip is a simulation of its own
holding its rows plus ``halo`` rows of each neighbour, and after at most
``halo`` steps the neighbours exchange ``halo`` rows of u and v again.  The
strip's cut edge is a mirror border, which corrupts one halo row per step, so
after ``halo`` steps exactly the strip's own rows are still those of the whole
grid (ghost-zone recompute, the exchange a multi-device split of one large
grid needs; the paper runs one device).

``strip_plan`` is the host logic: the rows each strip owns and holds, and the
row copies of one exchange.  ``StripGrid`` runs the strips as simulations on
one device and one stream, copying halo rows with ``rdc_get_rows`` straight
into the neighbour's planes.  Across devices the same copies become
``rdc_get_rows`` into a send buffer and ``rdc_put_rows`` from a receive
buffer around a send/recv pair.
"""
from __future__ import annotations

from dataclasses import dataclass
from fractions import Fraction

import numpy as np

from . import _capi as C


@dataclass(frozen=True)
class Strip:
    """Rows of strip ``index``: it owns [r0, r1) and holds [e0, e1) (whole-grid
    row indices); local row 0 of its simulation is row e0."""
    index: int
    r0: int
    r1: int
    e0: int
    e1: int

    @property
    def rows(self) -> int:
        return self.e1 - self.e0


@dataclass(frozen=True)
class Transfer:
    """One row copy of an exchange: ``nrows`` rows of u and v from local row
    ``src_row`` of strip ``src`` to local row ``dst_row`` of strip ``dst``."""
    src: int
    src_row: int
    dst: int
    dst_row: int
    nrows: int


def strip_plan(height: int, nstrips: int, halo: int):
    """Splits ``height`` rows into ``nstrips`` strips as even as integers allow
    (the first ones one row shorter where the division is ragged) with
    ``halo`` rows from each neighbour; returns (strips, transfers).  Every
    strip must own at least ``halo`` rows, so that the rows it sends are its
    own."""
    height, nstrips, halo = int(height), int(nstrips), int(halo)
    if nstrips < 1 or halo < 1 or height < 1:
        raise ValueError("height, nstrips and halo must be positive")
    bounds = [i * height // nstrips for i in range(nstrips + 1)]
    if min(b - a for a, b in zip(bounds, bounds[1:])) < (halo if nstrips > 1 else 1):
        raise ValueError(f"{nstrips} strips of {height} rows: some strip owns fewer than "
                         f"halo = {halo} rows")
    strips = [Strip(i, bounds[i], bounds[i + 1], max(bounds[i] - halo, 0),
                    min(bounds[i + 1] + halo, height)) for i in range(nstrips)]
    transfers = []
    for up, dn in zip(strips, strips[1:]):
        # the lower strip's first owned rows are the upper strip's bottom halo
        transfers.append(Transfer(dn.index, dn.r0 - dn.e0, up.index, up.r1 - up.e0, halo))
        # the upper strip's last owned rows are the lower strip's top halo
        transfers.append(Transfer(up.index, up.r1 - halo - up.e0, dn.index, 0, halo))
    return strips, transfers


class StripGrid:
    """A W x H grid stepped as ``nstrips`` row strips on the current device.

    The results equal one simulation of the whole grid bit for bit in every
    storage type; stochastic rounding is refused, because its random words
    are keyed by the row index within each strip's simulation.
    """

    def __init__(self, width: int, height: int, nstrips: int, phi=None, halo: int | None = None,
                 precision="f32", stream=None, **params):
        p = C.rdc_params_default(**params)
        if isinstance(precision, str):
            precision = C.PRECISION_NAMES[precision]
        p.precision = int(precision)
        if p.flags & C.RDC_STOCH_ROUND:
            raise ValueError("row strips and stochastic rounding: the random words are keyed "
                             "by the row within a strip, so the split would change them")
        self.params = p
        self.width, self.height = int(width), int(height)
        # default: the steps one launch fuses (4 when k_block = 0 picks the
        # size-dependent default), so that every exchange is followed by one launch
        self.halo = int(halo) if halo else (int(p.k_block) or 4)
        self.strips, self.transfers = strip_plan(self.height, nstrips, self.halo)
        if phi is not None:
            phi = np.asarray(phi)
            if phi.shape != (self.height, self.width):
                raise ValueError(f"phi shape {phi.shape} != ({self.height}, {self.width})")
        self.handles = []
        try:
            for s in self.strips:
                part = None if phi is None else np.ascontiguousarray(phi[s.e0:s.e1])
                self.handles.append(C.rdc_create(self.width, s.rows, p, part, stream))
                if stream is None:
                    # every strip on the first one's stream: the exchange copies
                    # and the steps are then ordered without waits
                    stream = C.rdc_get_view(self.handles[0]).stream
        except Exception:
            self.close()
            raise

    def close(self):
        # the first strip owns the shared stream when the caller gave none
        for h in reversed(getattr(self, "handles", [])):
            C.rdc_destroy(h)
        self.handles = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def seed(self, cx, cy, r, value=0.8):
        """rdc_seed on the whole grid: each strip seeds the disk shifted by its
        first held row.  The shift must be exact in double precision (true of
        every centre on a grid below 2^20 rows with at most 32 fractional bits),
        so that every cell sees the distance the whole grid would compute."""
        for s, h in zip(self.strips, self.handles):
            local = float(cy) - s.e0
            if Fraction(local) != Fraction(float(cy)) - s.e0:
                raise ValueError(f"disk centre row {cy!r} cannot be shifted by {s.e0} exactly")
            C.rdc_seed(h, cx, local, r, value)

    def exchange(self):
        """Copies every strip's halo rows from its neighbours (enqueued on the
        shared stream)."""
        for t in self.transfers:
            dst = C.rdc_get_view(self.handles[t.dst])
            off = t.dst_row * dst.pitch_bytes
            C.rdc_get_rows(self.handles[t.src], t.src_row, t.nrows, dst.u + off, dst.v + off,
                           dst.pitch_bytes)

    def step(self, n: int):
        """n Euler steps of the whole grid: exchanges, then at most ``halo``
        steps of every strip, until n are done."""
        n = int(n)
        if n < 0:
            raise ValueError("n must be >= 0")
        while n > 0:
            m = min(n, self.halo)
            if len(self.handles) > 1:
                self.exchange()
            for h in self.handles:
                C.rdc_step(h, m)
            n -= m

    def read(self, dtype=np.float64, check: bool = True):
        """(u, v) of the whole grid from the strips' own rows.  With check, a
        strip whose health check fails (on any row it holds) raises."""
        u = np.empty((self.height, self.width), dtype=dtype)
        v = np.empty_like(u)
        for s, h in zip(self.strips, self.handles):
            su = np.empty((s.rows, self.width), dtype=dtype)
            sv = np.empty_like(su)
            rc = C.rdc_read(h, su, sv)
            if check and rc != C.RDC_OK:
                raise C.RdcError(rc, f"StripGrid.read (strip {s.index})")
            a, b = s.r0 - s.e0, s.r1 - s.e0
            u[s.r0:s.r1] = su[a:b]
            v[s.r0:s.r1] = sv[a:b]
        return u, v

    def sync(self):
        for h in self.handles:
            C.rdc_sync(h)
