"""Pins of the oracle's stochastic rounding (the RDC_STOCH_ROUND variant of
the storage conversion) and of its Philox4x32-10 generator.

The rounding rule is pinned by what defines it: over all 2^16 random values
the mean result is exactly x (unbiasedness), the two possible results are the
neighbours of x on the target grid (checked against NumPy's float16 and a
bit truncation for bfloat16), the probability of rounding away from zero
grows with the distance to the lower neighbour, and the round-to-nearest
cases.  Philox is pinned by the generator's published known-answer vectors
(tests/golden/philox4x32_10_kat.txt, checked in tests/oracle_pins.py) and by
properties its definition implies: each round is a bijection of the counter
for a fixed key (so distinct counters give distinct outputs), every input bit
affects about half of the output bits after ten rounds, and the output words
are uniform."""
from __future__ import annotations

from fractions import Fraction

import numpy as np
import pytest


def _bf16_neighbours(x: np.float32):
    b = int(np.float32(x).view(np.uint32))
    lo = b & 0xFFFF0000
    hi = lo + 0x10000
    f = lambda bits: float(np.uint32(bits).view(np.float32))  # noqa: E731
    return f(lo), f(hi), b & 0xFFFF


def _xs(rng, n, lo, hi):
    """float32 values with random sign, log-uniform magnitude in [lo, hi)."""
    mag = np.exp(rng.uniform(np.log(lo), np.log(hi), n)).astype(np.float32)
    return mag * rng.choice(np.array([-1, 1], dtype=np.float32), n)


@pytest.mark.parametrize("fmt", ["bf16", "f16"])
def test_stochastic_rounding_is_exactly_unbiased(orc, fmt):
    """sum over r16 = 0..65535 of round(x, r16) == 65536 x exactly, for x
    whose distance to the grid is a multiple of 2^-16 of the spacing (every
    float32 for BF16; every float32 in FP16's normal range)."""
    rng = np.random.default_rng(7)
    xs = _xs(rng, 12, 1e-4, 3e4) if fmt == "f16" else _xs(rng, 12, 1e-30, 1e30)
    r = np.arange(65536, dtype=np.uint32)
    for x in xs:
        vals = [orc.round_stoch(x, int(k), fmt) for k in r[::1]]
        total = sum(Fraction(v) for v in vals)
        assert total == Fraction(float(x)) * 65536, (x, fmt)


def test_bf16_results_are_the_two_grid_neighbours(orc):
    rng = np.random.default_rng(8)
    for x in _xs(rng, 400, 1e-38, 1e38):
        lo, hi, L = _bf16_neighbours(x)
        for r16 in (0, 1, L - 1, L, L + 1, 65535, int(rng.integers(65536))):
            if not 0 <= r16 < 65536:
                continue
            got = orc.round_stoch(x, r16, "bf16")
            want = hi if r16 < L else lo
            assert got == want, (x, r16, got, want)


def test_f16_results_are_the_two_grid_neighbours(orc):
    """Against NumPy's float16: the result is representable, lies on the
    correct side, and is the neighbour away from zero exactly for the
    r16 below 2^16 (|x| - |lo|) / spacing."""
    rng = np.random.default_rng(9)
    for x in _xs(rng, 400, 1e-8, 6e4):
        xf = float(x)
        lo16 = np.float16(xf)
        if abs(float(lo16)) > abs(xf):        # RN went away from zero: step back
            lo16 = np.nextafter(lo16, np.float16(0))
        lo = float(lo16)
        hi = float(np.nextafter(lo16, np.float16(np.copysign(np.inf, xf))))
        if lo == xf:
            assert orc.round_stoch(x, 0, "f16") == xf
            continue
        frac = Fraction(abs(xf) - abs(lo)) / Fraction(abs(hi) - abs(lo))
        thr = frac * 65536
        for r16 in (0, 65535, int(rng.integers(65536)), int(thr), int(thr) + 1):
            if not 0 <= r16 < 65536:
                continue
            got = orc.round_stoch(x, r16, "f16")
            assert got == (hi if r16 < thr else lo), (x, r16)
            assert float(np.float16(got)) == got


def test_round_to_nearest_cases(orc):
    for fmt in ("bf16", "f16"):
        assert np.isnan(orc.round_stoch(float("nan"), 0, fmt))
        assert orc.round_stoch(float("inf"), 0, fmt) == float("inf")
        assert orc.round_stoch(-float("inf"), 12345, fmt) == -float("inf")
        assert orc.round_stoch(0.0, 0, fmt) == 0.0
        assert np.signbit(orc.round_stoch(-0.0, 0, fmt))
    assert orc.round_stoch(65504.0, 0, "f16") == 65504.0
    assert orc.round_stoch(65510.0, 0, "f16") == 65504.0          # below the midpoint
    assert orc.round_stoch(65520.0, 65535, "f16") == float("inf")  # the tie goes up
    assert orc.round_stoch(-70000.0, 0, "f16") == -float("inf")
    big = float(np.uint32(0x7F7FFFFF).view(np.float32))             # largest float
    assert orc.round_stoch(big, 0, "bf16") == float("inf")          # carries into inf
    assert orc.round_stoch(big, 65535, "bf16") == float(np.uint32(0x7F7F0000).view(np.float32))


def test_round_probability_grows_with_the_distance(orc):
    """The count of r16 rounding away from zero equals 2^16 times the
    fraction, so it is monotonic in x between two grid values."""
    lo = 0.5
    sp = 2.0 ** -8           # BF16 spacing on [0.5, 1)
    counts = []
    for k in (1, 1000, 20000, 40000, 65535):
        x = np.float32(lo + sp * k / 65536)
        up = sum(orc.round_stoch(x, r, "bf16") > lo for r in range(0, 65536, 7))
        counts.append(up)
    assert counts == sorted(counts) and counts[0] < counts[-1]


def test_philox_is_a_bijection_in_each_counter_word(orc):
    key = [0x12345678, 0x9ABCDEF0]
    for word in range(4):
        outs = set()
        for v in range(4096):
            ctr = [7, 11, 13, 17]
            ctr[word] = v * 2654435761 % 2**32
            outs.add(tuple(orc.philox4x32_10(ctr, key)))
        assert len(outs) == 4096, word


def test_philox_avalanche(orc):
    """Flipping one input bit flips close to half of the 128 output bits."""
    rng = np.random.default_rng(10)
    flips = []
    for _ in range(300):
        ctr = [int(x) for x in rng.integers(0, 2**32, 4, dtype=np.uint64)]
        key = [int(x) for x in rng.integers(0, 2**32, 2, dtype=np.uint64)]
        base = orc.philox4x32_10(ctr, key)
        bit = int(rng.integers(0, 192))
        c2, k2 = list(ctr), list(key)
        if bit < 128:
            c2[bit // 32] ^= 1 << (bit % 32)
        else:
            k2[(bit - 128) // 32] ^= 1 << ((bit - 128) % 32)
        other = orc.philox4x32_10(c2, k2)
        flips.append(sum(bin(int(a) ^ int(b)).count("1") for a, b in zip(base, other)))
    m = float(np.mean(flips))
    assert 60.0 < m < 68.0, m
    assert min(flips) > 30


def test_philox_output_is_uniform(orc):
    """Chi-square of the top byte of each word over sequential counters."""
    counts = np.zeros(256)
    n = 0
    for i in range(8192):
        w = orc.philox4x32_10([i, 3, 0, 0], [42, 0])
        for x in w:
            counts[int(x) >> 24] += 1
            n += 1
    exp = n / 256
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 350.0, chi2        # 255 degrees of freedom: p ~ 1e-4 at 350


def test_cells_use_the_documented_words(orc):
    """round_stoch_cells: counter (col // 4, row, step low, step high), key
    (seed, 0); word col % 4, top 16 bits for u, low 16 bits for v."""
    x = np.float32(0.3)
    seed, step, row = 99, (5 << 32) + 17, 4
    u, v = orc.round_stoch_cells(np.full(8, x), seed, step, row, 6, "bf16")
    for i, col in enumerate(range(6, 14)):
        w = orc.philox4x32_10([col // 4, row, step & 0xFFFFFFFF, step >> 32], [seed, 0])
        word = int(w[col % 4])
        assert u[i] == np.float32(orc.round_stoch(x, word >> 16, "bf16"))
        assert v[i] == np.float32(orc.round_stoch(x, word & 0xFFFF, "bf16"))
