"""Each plausible mistake planted in a copy of the oracle (on the CPU) must
fail at least one pin: a dropped term, a wrong sign, a wrong index, a wrong
border rule, a transposed or swapped operand.  The real oracle is never
modified; every mutant is compiled to a temporary library."""
from __future__ import annotations

import os

import pytest

import oracle
from tests import oracle_pins as P

SRC = os.path.join(os.path.dirname(oracle.__file__), "rdc_oracle.c")

# (name, original text, replacement)
MUTANTS = [
    ("ratio_inverted", "(c - q) / (c + q)", "(c + q) / (c - q)"),
    ("ratio_sign", "(c - q) / (c + q)", "(c + q) / (c + q)"),
    ("phi_sign", "(f * vc + phi[k])", "(f * vc - phi[k])"),
    ("fv_dropped", "(f * vc + phi[k])", "(phi[k])"),
    ("eps_multiplies", "du = R / eps + Du * lap;", "du = R * eps + Du * lap;"),
    ("Du_dropped", "du = R / eps + Du * lap;", "du = R / eps + lap;"),
    ("quadratic_sign", "(c - c * c)", "(c + c * c)"),
    ("quadratic_dropped", "(c - c * c)", "(c)"),
    ("v_sign", "vc + dt * (c - vc)", "vc + dt * (vc - c)"),
    ("v_uses_new_u", "v1[k] = vc + dt * (c - vc);", "v1[k] = vc + dt * (un - vc);"),
    ("dt_dropped", "const double un = c + dt * du;", "const double un = c + du * 0.01;"),
    ("centre_weight", "- 4.0 * c)", "- 3.0 * c)"),
    ("dx_not_squared", "1.0 / (p->dx * p->dx)", "1.0 / p->dx"),
    ("south_wraps", "(i < H - 1) ? i + 1 : H - 1", "(i < H - 1) ? i + 1 : 0"),
    ("east_vertex_mirror", "(j < W - 1) ? j + 1 : W - 1", "(j < W - 1) ? j + 1 : W - 2"),
    ("north_index_swapped", "u[(int64_t)in * W + j]", "u[(int64_t)i * W + jw]"),
    ("south_uses_north", "u[(int64_t)is * W + j]", "u[(int64_t)in * W + j]"),
    ("rows_cols_transposed", "const double e = u[(int64_t)i * W + je];",
     "const double e = u[(int64_t)(je < H ? je : H - 1) * W + i % W];"),
    ("rest_a1_sign", "const double a1 = (phi - q) - f * q;", "const double a1 = (phi + q) - f * q;"),
    ("rest_a0_dropped", "const double a0 = -(phi * q);", "const double a0 = 0.0 * q;"),
    ("seed_strict", "if (dy * dy + dx * dx <= r2)", "if (dy * dy + dx * dx < r2)"),
    ("seed_axes_swapped", "double dy = (double)i - cy;", "double dy = (double)i - cx;"),
    ("health_no_pole", "|| (u + q) <= 0.0;", "|| 0;"),
    ("stoch_threshold_le", "((double)r16 < ldexp(frac, 16))", "((double)r16 <= ldexp(frac, 16))"),
    ("stoch_bf16_precision", "const int mant = fmt == 0 ? 7 : 10;",
     "const int mant = fmt == 0 ? 8 : 10;"),
    ("stoch_f16_subnormal_edge", "const int emin = fmt == 0 ? -126 : -14;",
     "const int emin = fmt == 0 ? -126 : -13;"),
    ("stoch_round_down_only", "? lo + sp : lo;", "? lo : lo;"),
    ("philox_key_dropped", "^ c[1] ^ k0;", "^ c[1];"),
    ("philox_one_round", "round < 10; ++round", "round < 1; ++round"),
    ("philox_word_reused", "^ c[3] ^ k1;", "^ c[1] ^ k1;"),
    ("philox_wrong_multiplier", "0xD2511F53u * (uint64_t)c[0]", "0xD2511F55u * (uint64_t)c[0]"),
    ("philox_hi_lo_swapped",
     "const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;\n        const uint32_t n3 = (uint32_t)p0;",
     "const uint32_t n2 = (uint32_t)p0 ^ c[3] ^ k1;\n        const uint32_t n3 = (uint32_t)(p0 >> 32);"),
    ("philox_key_bumped_first", "uint32_t k0 = key[0], k1 = key[1];",
     "uint32_t k0 = key[0] + 0x9E3779B9u, k1 = key[1] + 0xBB67AE85u;"),
    ("render_red_from_v", "out[4 * k + 0] = r;", "out[4 * k + 0] = b;"),
    ("render_green_strict", "(phi[k] >= thr) ? 255 : 0", "(phi[k] > thr) ? 255 : 0"),
    ("render_no_upper_clamp", "if (y > 1.0f) y = 1.0f;", ""),
    ("render_truncates", "lrintf(255.0f * y)", "(long)(255.0f * y)"),
    ("timelapse_minimum", "u[k] > tl[k]", "u[k] < tl[k]"),
    ("timelapse_no_reset", "(reset || u[k] > tl[k])", "(u[k] > tl[k])"),
    ("snap_floor", "round(a / snap) * snap", "floor(a / snap) * snap"),
    ("snap_length_dropped", "*x1o = x0 + len * cos(r);", "*x1o = x0 + cos(r);"),
    ("draw_segment_unbounded", "if (t > 1.0) t = 1.0;", ""),
    ("draw_full_width", "const double h = 0.5 * width;", "const double h = width;"),
    ("draw_strict", "if (dx * dx + dy * dy <= half2) {", "if (dx * dx + dy * dy < half2) {"),
    ("draw_axes_swapped", "const double x = (double)j, y = (double)i;",
     "const double x = (double)i, y = (double)j;"),
    ("stoch_cells_one_word", "w[col % 4]", "w[0]"),
    ("stoch_cells_quad_dropped", "(uint32_t)(col / 4), (uint32_t)row", "0u, (uint32_t)row"),
    ("stoch_cells_row_dropped", "(uint32_t)(col / 4), (uint32_t)row,", "(uint32_t)(col / 4), 0u,"),
    ("stoch_cells_step_high_dropped", "(uint32_t)(s >> 32)}", "0u}"),
    ("stoch_cells_v_reuses_u_bits", "word & 0xFFFFu", "word >> 16"),
    ("stoch_cells_key_dropped", "{seed, 0u}", "{0u, 0u}"),
]


def _pins_fail(o) -> list[str]:
    """The first pin the mutant fails (one is enough), or none."""
    for pin in P.ALL_PINS:
        try:
            pin(o, oracle)
        except (AssertionError, ValueError):
            return [pin.__name__]
    return []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught(name, old, new, tmp_path):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor not found: {old!r}"
    mutated = src.replace(old, new)
    path = tmp_path / "mut.c"
    path.write_text(mutated)
    lib = oracle.compile_oracle(str(path), str(tmp_path / f"lib{name}.so"), openmp=False)
    failed = _pins_fail(oracle.Oracle(lib))
    assert failed, f"mutant {name} passed every pin"
