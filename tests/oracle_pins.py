"""Pins of the FP64 oracle: checks against what the model and the mathematics
fix, independent of the oracle's own code.

Each pin takes an ``oracle.Oracle`` and raises AssertionError on failure, so
the same checks run against the real oracle (tests/test_oracle_pins.py) and
against deliberately broken copies of it (tests/test_oracle_mutants.py).

What each pin fixes:
  rest_root            p(u*) = 0 for the cubic obtained by setting Eq. 1's
                       bracket to zero with v = u; checked against
                       numpy.roots (a library routine), not the oracle's
                       bisection.
  rest_fixed_point     a homogeneous field at u = v = u* does not move under
                       the full step (uses the step's own reaction term, so
                       it ties the step to the cubic).
  jacobian             one step of a small perturbation of the rest state
                       equals (I + dt J) applied to it, J the analytic
                       Jacobian of Eq. 1's reaction part (derivatives taken by
                       hand): pins eps scaling, the f v coupling, the sign of
                       every reaction term and the v equation.
  jacobian_with_mode   the same for a cosine-mode perturbation in the full
                       model: I + dt (J + diag(Du lambda_k, 0)) -- pins how
                       diffusion enters the full update.
  cosine_modes         diffusion alone maps cos(pi k (j+1/2)/W) cos(pi l
                       (i+1/2)/H) to (1 + dt Du lambda) times itself with
                       lambda = -(4/dx^2)[sin^2(pi k/2W) + sin^2(pi l/2H)]:
                       the eigenpairs of the five-node Laplacian under
                       zero-flux (cell-centred mirror) borders.
  conservation         diffusion alone conserves sum(u) (the mirror border
                       has zero flux).
  round_stoch          stochastic rounding to BF16/FP16: over all 2^16 random
                       values the mean is exactly x; the results are the two
                       grid neighbours (NumPy float16, bit truncation for
                       BF16) split at the stated threshold.
  philox               Philox4x32-10 reproduces the generator's published
                       known-answer vectors (tests/golden/philox4x32_10_kat.txt:
                       Random123's entries for 10 rounds); besides, it is a
                       bijection in each counter word, every input bit flips
                       about half the output bits, the output is uniform.
  symmetry             a seed invariant under the 8 symmetries of the square
                       stays exactly invariant.
  one_d                rows that are identical stay identical and equal the
                       1-row grid (the y-terms cancel exactly).
  uniform_is_single    a uniform field of any value evolves like one cell.
  spike                diffusion of a single spike on a 3 x 3 grid gives the
                       textbook five-point weights (interior and corner).
  gauss_circle         the number of lattice points in a disk of radius r
                       about a lattice point is Gauss's N(r); an off-centre
                       disk's centroid is its centre (axes not swapped).
  health               a cell at the pole u = -q, or finite left of it, is
                       reported at the right step and index.
"""
from __future__ import annotations

import math
import os

import numpy as np

# Table 1
EPS, F, PHI_A, PHI_P, Q, DU, DT, DX = 0.0243, 1.4, 0.054, 0.0975, 0.002, 0.45, 0.001, 0.25

# Lattice points with i^2 + j^2 <= r^2 (Gauss circle problem), r = 0..10.
GAUSS_N = [1, 5, 13, 29, 49, 81, 113, 149, 197, 253, 317]


def _params(oracle_mod, flags=0, **kw):
    return oracle_mod.Params(flags=flags, **kw)


def cubic_root_numpy(phi, f=F, q=Q):
    r = np.roots([1.0, f + q - 1.0, phi - q - f * q, -phi * q])
    pos = [x.real for x in r if abs(x.imag) < 1e-12 and x.real > 0]
    assert len(pos) == 1, f"expected one positive root, got {r}"
    return pos[0]


def cubic_root_exact(phi, f=F, q=Q):
    """The positive root to 40 digits, coefficients taken exactly from the
    doubles (sympy's arbitrary-precision root finder)."""
    import pytest
    sympy = pytest.importorskip("sympy")
    from fractions import Fraction
    x = sympy.Symbol("x")
    fr = lambda d: sympy.Rational(Fraction(d))  # noqa: E731
    fq, ff, fp = fr(q), fr(f), fr(phi)
    poly = sympy.Poly(x ** 3 + (ff + fq - 1) * x ** 2 + (fp - fq - ff * fq) * x - fp * fq, x)
    roots = [r for r in poly.nroots(n=40) if r.is_real and r > 0]
    assert len(roots) == 1
    return roots[0]


def pin_rest_root(o, om):
    for phi in (0.054, 0.0975, 0.2, 0.05, 0.08, 0.0301):
        us = o.rest_state(phi)
        ref = cubic_root_numpy(phi)
        assert abs(us - ref) <= 4e-15 * ref, (phi, us, ref)
        exact = cubic_root_exact(phi)
        ulp = np.spacing(us)
        assert abs(float(exact - us)) <= 2 * ulp, (phi, us, exact)


def pin_rest_fixed_point(o, om):
    phi = np.full((9, 16), PHI_A)
    u, v = o.rest_field(phi)
    us = u[0, 0]
    r = o.run(phi, u, v, 20000, params=_params(om))
    assert r["status"] == 0
    assert np.max(np.abs(r["u"] - us)) <= 1e-12
    assert np.max(np.abs(r["v"] - us)) <= 1e-12


def analytic_jacobian(u, v, phi, f=F, q=Q, eps=EPS):
    # R(u, v) = u - u^2 - (f v + phi)(u - q)/(u + q)
    dR_du = 1.0 - 2.0 * u - (f * v + phi) * (2.0 * q) / (u + q) ** 2
    dR_dv = -f * (u - q) / (u + q)
    return np.array([[dR_du / eps, dR_dv / eps], [1.0, -1.0]])


def pin_jacobian(o, om):
    for phi in (PHI_A, PHI_P):
        # linearise about a non-rest point as well, so the u^2 and v terms
        # are weighted differently from the rest state
        for (u0, v0) in ((o.rest_state(phi),) * 2, (0.3, 0.1)):
            J = analytic_jacobian(u0, v0, phi)
            A = np.eye(2) + DT * J
            h = 1e-6
            ph = np.full((1, 1), phi)
            cols = []
            for d in ((h, 0.0), (0.0, h)):
                up = o.step(ph, np.full((1, 1), u0 + d[0]), np.full((1, 1), v0 + d[1]))
                um = o.step(ph, np.full((1, 1), u0 - d[0]), np.full((1, 1), v0 - d[1]))
                cols.append([(up[0][0, 0] - um[0][0, 0]) / (2 * h),
                             (up[1][0, 0] - um[1][0, 0]) / (2 * h)])
            num = np.array(cols).T
            assert np.allclose(num, A, rtol=1e-6, atol=1e-7), (phi, u0, v0, num, A)


def pin_jacobian_with_mode(o, om):
    """Full model (reaction + diffusion): a small cosine-mode perturbation of
    the rest state evolves by I + dt (J + diag(Du lambda_k, 0)) -- pins how the
    diffusion term enters the full update."""
    W, H = 12, 7
    phi = PHI_A
    us = o.rest_state(phi)
    J = analytic_jacobian(us, us, phi)
    for (k, l) in ((1, 0), (3, 2), (W - 1, H - 1)):
        m = cosine_mode(W, H, k, l)
        lam = -(4.0 / DX ** 2) * (math.sin(math.pi * k / (2 * W)) ** 2 +
                                  math.sin(math.pi * l / (2 * H)) ** 2)
        A = np.eye(2) + DT * (J + np.array([[DU * lam, 0.0], [0.0, 0.0]]))
        h = 1e-7
        ph = np.full((H, W), phi)
        cols = []
        for d in ((h, 0.0), (0.0, h)):
            up = o.step(ph, us + d[0] * m, us + d[1] * m)
            um = o.step(ph, us - d[0] * m, us - d[1] * m)
            # project the response back onto the mode
            nm = np.sum(m * m)
            cols.append([np.sum((up[0] - um[0]) * m) / (2 * h * nm),
                         np.sum((up[1] - um[1]) * m) / (2 * h * nm)])
        num = np.array(cols).T
        assert np.allclose(num, A, rtol=1e-5, atol=1e-6), (k, l, num, A)


def cosine_mode(W, H, k, l):
    j = np.arange(W)
    i = np.arange(H)
    return np.outer(np.cos(np.pi * l * (i + 0.5) / H), np.cos(np.pi * k * (j + 0.5) / W))


def pin_cosine_modes(o, om):
    W, H = 13, 8
    p = _params(om, flags=om.DIFFUSION_ONLY)
    for (k, l) in ((0, 0), (1, 0), (0, 1), (3, 2), (5, 7), (W - 1, H - 1), (W - 1, 0)):
        m = cosine_mode(W, H, k, l)
        u = 0.5 + 0.25 * m
        lam = -(4.0 / DX ** 2) * (math.sin(math.pi * k / (2 * W)) ** 2 +
                                  math.sin(math.pi * l / (2 * H)) ** 2)
        expect = 0.5 + 0.25 * (1.0 + DT * DU * lam) * m
        u1, _, rc, _ = o.step(np.full((H, W), PHI_A), u, u.copy(), p)
        assert rc == 0
        assert np.max(np.abs(u1 - expect)) <= 1e-13, (k, l, np.max(np.abs(u1 - expect)))


def pin_conservation(o, om):
    rng = np.random.default_rng(11)
    W, H = 31, 17
    u0 = rng.uniform(0.0, 0.8, size=(H, W))
    p = _params(om, flags=om.DIFFUSION_ONLY)
    r = o.run(np.full((H, W), PHI_A), u0, u0.copy(), 1000, params=p)
    s0 = math.fsum(u0.ravel())
    s1 = math.fsum(r["u"].ravel())
    assert abs(s1 - s0) / s0 <= 1e-12, (s0, s1)
    # and the field did diffuse
    assert np.std(r["u"]) < 0.5 * np.std(u0)


def pin_symmetry(o, om):
    N = 40
    phi = np.full((N, N), PHI_A)
    u, v = o.rest_field(phi)
    o.seed_disk(u, (N - 1) / 2, (N - 1) / 2, 6.0, 0.8)
    r = o.run(phi, u, v, 400)
    U = r["u"]
    assert np.array_equal(U, U[::-1, :])
    assert np.array_equal(U, U[:, ::-1])
    assert np.array_equal(U, U.T)
    assert U.max() > 0.3  # a wave was excited


def pin_one_d(o, om):
    W = 64
    phi1 = np.full((1, W), PHI_A)
    u1, v1 = o.rest_field(phi1)
    u1[:, :4] = 0.8
    r1 = o.run(phi1, u1, v1, 600)
    phi5 = np.full((5, W), PHI_A)
    u5, v5 = o.rest_field(phi5)
    u5[:, :4] = 0.8
    r5 = o.run(phi5, u5, v5, 600)
    for i in range(5):
        assert np.array_equal(r5["u"][i], r1["u"][0])
        assert np.array_equal(r5["v"][i], r1["v"][0])
    assert r1["u"][0, 20] > 0.3 or r1["u"][0, 10] > 0.3  # the front travelled


def pin_uniform_is_single(o, om):
    for val in (0.2, 0.6):
        phi = np.full((6, 7), PHI_A)
        u = np.full((6, 7), val)
        v = np.full((6, 7), 0.05)
        r = o.run(phi, u, v, 300)
        r1 = o.run(phi[:1, :1], u[:1, :1], v[:1, :1], 300)
        assert np.all(r["u"] == r1["u"][0, 0]) and np.all(r["v"] == r1["v"][0, 0])


def pin_spike(o, om):
    a = DT * DU / DX ** 2
    p = _params(om, flags=om.DIFFUSION_ONLY)
    # interior spike: centre loses 4a, each of the 4 neighbours gains a
    u = np.zeros((3, 3))
    u[1, 1] = 1.0
    u1, _, _, _ = o.step(np.full((3, 3), PHI_A), u, u.copy(), p)
    exp = np.zeros((3, 3))
    exp[1, 1] = 1.0 - 4 * a
    exp[0, 1] = exp[2, 1] = exp[1, 0] = exp[1, 2] = a
    assert np.max(np.abs(u1 - exp)) <= 1e-15
    # corner spike: the mirror ghosts are the corner itself, so it loses 2a
    u = np.zeros((3, 3))
    u[0, 0] = 1.0
    u1, _, _, _ = o.step(np.full((3, 3), PHI_A), u, u.copy(), p)
    exp = np.zeros((3, 3))
    exp[0, 0] = 1.0 - 2 * a
    exp[0, 1] = exp[1, 0] = a
    assert np.max(np.abs(u1 - exp)) <= 1e-15


def pin_gauss_circle(o, om):
    N = 41
    for r, expect in enumerate(GAUSS_N):
        u = np.zeros((N, N))
        n = o.seed_disk(u, 20.0, 20.0, float(r), 1.0)
        assert n == expect and int(u.sum()) == expect, (r, n, expect)
    # half-integer centre: symmetric under the square's symmetries, and
    # clipped at the border
    u = np.zeros((8, 8))
    o.seed_disk(u, 3.5, 3.5, 2.0, 1.0)
    assert np.array_equal(u, u.T) and np.array_equal(u, u[::-1, ::-1])
    assert int(u.sum()) == 12  # (+-1/2, +-1/2) x4, (+-3/2, +-1/2) x8
    u = np.zeros((5, 5))
    assert o.seed_disk(u, 0.0, 0.0, 1.0, 1.0) == 3
    # an off-centre disk on a non-square grid: x is the column, y the row,
    # and a lattice disk about a lattice point has its centroid at the centre
    u = np.zeros((30, 17))
    n = o.seed_disk(u, 5.0, 12.0, 4.0, 1.0)
    ii, jj = np.nonzero(u)
    assert n == GAUSS_N[4] and ii.mean() == 12.0 and jj.mean() == 5.0


def pin_health(o, om):
    phi = np.full((4, 5), PHI_A)
    u, v = o.rest_field(phi)
    u[2, 3] = -Q            # exactly at the pole
    r = o.run(phi, u, v, 10)
    assert r["status"] == om.ENONFINITE and r["bad_step"] == 1 and r["bad_index"] == 2 * 5 + 3
    # finite but left of the pole: u + q < 0 must be reported too
    u, v = o.rest_field(phi)
    u[1, 4] = -0.01
    r = o.run(phi, u, v, 10)
    assert r["status"] == om.ENONFINITE and r["bad_step"] == 1 and r["bad_index"] == 1 * 5 + 4
    assert np.isfinite(r["u"]).all()
    u, v = o.rest_field(phi)
    r = o.run(phi, u, v, 10)
    assert r["status"] == 0 and r["bad_step"] == -1


def pin_render(o, om):
    """§3.1: red carries u, blue carries v, green marks inhibitive substrate;
    values are clamped to [0, 1] and coded to 0..255 with ties to even."""
    u = np.array([[1.0, 0.0, 0.5, 2.0, -1.0, 127.5 / 255, 128.5 / 255]], dtype=np.float32)
    v = np.array([[0.0, 1.0, 0.25, -3.0, 9.0, 0.0, 0.0]], dtype=np.float32)
    phi = np.array([[0.054, 0.2, 0.0975, 0.054, 0.2, 0.054, 0.054]])
    img = o.render(u, v, phi, 1.0, 1.0, thr=0.07575)
    assert img[0, 0].tolist() == [255, 0, 0, 255]        # pure u -> red
    assert img[0, 1].tolist() == [0, 255, 255, 255]      # v, on substrate
    assert img[0, 2].tolist() == [128, 255, 64, 255]     # 127.5 -> 128, 63.75 -> 64
    assert img[0, 3].tolist() == [255, 0, 0, 255]        # clamped above / below
    assert img[0, 4].tolist() == [0, 255, 255, 255]
    assert img[0, 5, 0] == 128 and img[0, 6, 0] == 128   # ties to even: 127.5, 128.5
    tl = o.timelapse(u)
    tl = o.timelapse(np.zeros_like(u), tl)
    tl = o.timelapse(np.full_like(u, 0.75), tl)
    assert np.array_equal(tl, np.maximum(np.maximum(u, 0), 0.75).astype(np.float32))
    img = o.render(u, v, phi, 1.0, 1.0, thr=0.07575, tl=tl)
    assert (img[..., 2] == 0).all() and img[0, 1, 0] == 191   # 0.75 * 255 = 191.25
    # green where phi >= the threshold: at it, and one double either side
    t = 0.07575
    z = np.zeros((1, 3), dtype=np.float32)
    img = o.render(z, z, np.array([[t, np.nextafter(t, 0.0), np.nextafter(t, 1.0)]]), thr=t)
    assert img[0, :, 1].tolist() == [255, 0, 255]
    # a reset replaces the record whatever it held (larger values included)
    import ctypes
    fp = ctypes.POINTER(ctypes.c_float)
    rec = np.full(u.shape, 5.0, dtype=np.float32)
    uu = np.ascontiguousarray(u, dtype=np.float32)
    o.lib.orc_timelapse(uu.size, uu.ctypes.data_as(fp), rec.ctypes.data_as(fp), 1)
    assert np.array_equal(rec, uu)


def pin_draw(o, om):
    """§3 line presets: a horizontal line centred between rows covers exactly
    `width` rows (2, 3 centred on a row, 8); snapped segments lie on multiples
    of 15 degrees and keep their length; a zero-length line is a disk."""
    for width, yc in ((2, 10.5), (3, 10.0), (8, 10.5)):
        phi = np.zeros((24, 40))
        o.draw_line(phi, 5.0, yc, 30.0, yc, float(width), 1.0)
        rows = np.nonzero(phi[:, 17])[0]
        assert len(rows) == width, (width, rows)
        assert phi[:, :5 - width // 2 - 1].sum() == 0        # ends are rounded caps
        assert phi[:, 30 + width // 2 + 2:].sum() == 0       # the segment ends at x1
    x1, y1 = o.snap_segment(0.0, 0.0, 10.0, 9.4, 15.0)     # 43.2 deg -> 45
    assert abs(x1 - y1) < 1e-12 and abs(np.hypot(x1, y1) - np.hypot(10.0, 9.4)) < 1e-12
    x1, y1 = o.snap_segment(3.0, 4.0, 20.0, 5.0, 15.0)     # 3.4 deg -> 0
    assert y1 == 4.0 and abs(x1 - (3.0 + np.hypot(17.0, 1.0))) < 1e-12
    x1, y1 = o.snap_segment(0.0, 0.0, -1.0, 10.0, 15.0)    # 95.7 deg -> 90
    assert abs(x1) < 1e-12 and abs(y1 - np.hypot(1.0, 10.0)) < 1e-12
    phi = np.zeros((21, 21))
    assert o.draw_line(phi, 10.0, 10.0, 10.0, 10.0, 8.0, 1.0) == GAUSS_N[4]


def pin_round_stoch(o, om):
    from fractions import Fraction
    rng = np.random.default_rng(71)
    # exact unbiasedness over all 2^16 random values
    for fmt, xs in (("bf16", [0.3, -1.7e-20, 3.3e25]), ("f16", [0.3, -12.345, 2.5e-3])):
        for x in xs:
            x32 = np.float32(x)
            total = sum(Fraction(o.round_stoch(x32, r, fmt)) for r in range(65536))
            assert total == Fraction(float(x32)) * 65536, (fmt, x)
    # the two neighbours, split at the threshold
    xs = np.concatenate([rng.uniform(0.01, 900.0, 40) * rng.choice([-1, 1], 40),
                         [9.1e-5, -7.3e-5, 3.3e-5, -1.1e-6]]).astype(np.float32)  # FP16 edges
    for x in xs:
        b = int(np.float32(x).view(np.uint32))
        L = b & 0xFFFF
        lo = float(np.uint32(b & 0xFFFF0000).view(np.float32))
        hi = float(np.uint32((b & 0xFFFF0000) + 0x10000).view(np.float32))
        for r in (0, max(L - 1, 0), L, 65535):
            assert o.round_stoch(x, r, "bf16") == (hi if r < L else lo), (x, r)
        lo16 = np.float16(float(x))
        if abs(float(lo16)) > abs(float(x)):
            lo16 = np.nextafter(lo16, np.float16(0))
        hi16 = np.nextafter(lo16, np.float16(np.copysign(np.inf, float(x))))
        thr = Fraction(abs(float(x)) - abs(float(lo16))) / Fraction(abs(float(hi16)) - abs(float(lo16))) * 65536
        for r in (0, int(thr), int(thr) + 1, 65535):
            if 0 <= r < 65536:
                assert o.round_stoch(x, r, "f16") == float(hi16 if r < thr else lo16), (x, r)
    assert o.round_stoch(65510.0, 0, "f16") == 65504.0
    assert o.round_stoch(65520.0, 65535, "f16") == float("inf")


def philox_kat():
    """(counter, key, output) triples of the published known-answer vectors."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "philox4x32_10_kat.txt")
    out = []
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            assert len(w) == 10, line
            out.append((w[0:4], w[4:6], w[6:10]))
    return out


def pin_philox(o, om):
    kat = philox_kat()
    assert len(kat) == 3
    for ctr, key, want in kat:
        got = [int(x) for x in o.philox4x32_10(ctr, key)]
        assert got == want, (ctr, key, [hex(x) for x in got])
    key = [0x1234567, 0x89ABCDE]
    for word in range(4):
        outs = set()
        for v in range(1024):
            ctr = [5, 6, 7, 8]
            ctr[word] = v * 2654435761 % 2**32
            outs.add(tuple(int(x) for x in o.philox4x32_10(ctr, key)))
        assert len(outs) == 1024, word
    rng = np.random.default_rng(72)
    flips = []
    for t in range(192):
        ctr = [int(x) for x in rng.integers(0, 2**32, 4, dtype=np.uint64)]
        k = [int(x) for x in rng.integers(0, 2**32, 2, dtype=np.uint64)]
        base = o.philox4x32_10(ctr, k)
        c2, k2 = list(ctr), list(k)
        if t < 128:
            c2[t // 32] ^= 1 << (t % 32)
        else:
            k2[(t - 128) // 32] ^= 1 << ((t - 128) % 32)
        other = o.philox4x32_10(c2, k2)
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, other)))
    assert 60.0 < float(np.mean(flips)) < 68.0 and min(flips) > 30, (np.mean(flips), min(flips))
    counts = np.zeros(256)
    for i in range(2048):
        for x in o.philox4x32_10([i, 1, 0, 0], [9, 0]):
            counts[int(x) >> 24] += 1
    exp = counts.sum() / 256
    assert float(((counts - exp) ** 2 / exp).sum()) < 350.0


def pin_round_stoch_cells(o, om):
    """The rounding of a row of cells: with x exactly halfway between two
    BF16 values each draw is a fair coin, so the patterns show that every
    field of the counter (the quad column / 4, the row, both halves of the
    64-bit step) and the key changes the draws, that u and v use different
    bits, that the four cells of a quad use four different words, that a
    cell's bits do not depend on where the row segment starts, and that the
    rounding is unbiased over steps.  (Which bits go to u and which to v is a
    convention the GPU parity test fixes.)"""
    base = int(np.float32(0.3).view(np.uint32)) & 0xFFFF0000
    x0 = np.uint32(base | 0x8000).view(np.float32)            # halfway
    lo = float(np.uint32(base).view(np.float32))
    hi = float(np.uint32(base + 0x10000).view(np.float32))
    x = np.full(64, x0, dtype=np.float32)

    def pattern(seed=5, step=7, row=3, col0=0, n=64):
        u, v = o.round_stoch_cells(x[:n], seed, step, row, col0, "bf16")
        assert set(np.unique(u)) <= {lo, hi} and set(np.unique(v)) <= {lo, hi}
        return u == hi, v == hi

    bu, bv = pattern()
    assert 10 < bu.sum() < 54 and 10 < bv.sum() < 54, (bu.sum(), bv.sum())
    assert not np.array_equal(bu, bv)
    for kw in ({"seed": 6}, {"step": 8}, {"step": 7 + 2 ** 32}, {"row": 4}):
        assert not np.array_equal(pattern(**kw)[0], bu), kw
    quads = bu.reshape(16, 4)
    assert not all(len(set(q)) == 1 for q in quads)           # one word per cell
    assert len({tuple(q) for q in quads}) > 4                 # one call per quad
    su, _ = pattern(col0=4, n=60)
    assert np.array_equal(su, bu[4:])
    draws = [o.round_stoch_cells(x[:1], 5, s, 3, 0, "bf16")[0][0] for s in range(4000)]
    sd = (hi - lo) / 2 / math.sqrt(len(draws))
    assert abs(float(np.mean(draws)) - float(x0)) < 5 * sd


ALL_PINS = [pin_rest_root, pin_rest_fixed_point, pin_jacobian, pin_jacobian_with_mode,
            pin_cosine_modes,
            pin_conservation, pin_symmetry, pin_one_d, pin_uniform_is_single, pin_spike,
            pin_gauss_circle, pin_health, pin_render, pin_draw, pin_round_stoch, pin_philox,
            pin_round_stoch_cells]
