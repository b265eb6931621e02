"""Calibrates the §4 circuit geometries on the FP64 oracle and writes the
records kept next to this script.

The paper's circuit figures are not available (§4.1, §4.2 give only the
mechanism), so the free geometric parameters of ``rdc_inputs.and_gate`` and
``rdc_inputs.diode`` were chosen here, on the oracle alone:

  and_gate_window.txt   largest phi of the 3-cell gap band that a single
                        input wave still crosses, and the same for two
                        colliding waves, by bisection; the AND window lies
                        between them and rdc_inputs.AND_PHI_GAP sits inside.
  diode_calibration.txt forward (anode -> cathode) and backward passage for
                        a grid of gap-phi levels and point lengths.

Usage:  python tests/golden/calibrate_circuits.py [--quick]
Runs only oracle/ and rdc_inputs (geometry, no model arithmetic).
"""
from __future__ import annotations

import itertools
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import rdc_inputs as ri  # noqa: E402

THREADS = os.cpu_count() or 1


def _arrives(orc, c, fire, probe, steps):
    u, v = orc.rest_field(c.phi)
    for name in fire:
        cx, cy, r = c.seeds[name]
        orc.seed_disk(u, cx, cy, r, ri.SEED_VALUE)
    t = orc.run(c.phi, u, v, steps, nthreads=THREADS, probes=[c.probes[probe]])["t_arr"][0]
    return t


def and_window(orc, iters=9, steps=9000):
    def passes(pg, fire):
        c = ri.and_gate(160, 128, arm=50, out_len=40, phi_gap=pg)
        return _arrives(orc, c, fire, "out", steps) > 0

    def crit(fire, lo=0.07, hi=0.10):
        assert passes(lo, fire) and not passes(hi, fire)
        for _ in range(iters):
            mid = 0.5 * (lo + hi)
            if passes(mid, fire):
                lo = mid
            else:
                hi = mid
        return lo, hi

    return crit(["A"]), crit(["A", "B"])


def diode_table(orc, steps=14000):
    rows = []
    for pg, tip in itertools.product([0.0975, 0.10, 0.105, 0.11, 0.115, 0.12],
                                     [2.0, 4.0, 6.0, 8.0, 10.0, 14.0]):
        c = ri.diode(128, 48, gap=1, tip=tip, phi_gap=pg)
        f = _arrives(orc, c, ["anode"], "cathode_end", steps)
        b = _arrives(orc, c, ["cathode"], "anode_end", steps)
        rows.append((pg, tip, f, b))
    return rows


def main():
    quick = "--quick" in sys.argv
    orc = oracle.load()
    single, pair = and_window(orc, iters=5 if quick else 9)
    with open(os.path.join(HERE, "and_gate_window.txt"), "w") as f:
        f.write("# AND gate (rdc_inputs.and_gate(160, 128, arm=50, out_len=40)), FP64 oracle,\n")
        f.write("# 3-cell gap band; bisection bracket [passes, blocked] of the band's phi\n")
        f.write(f"single_input  {single[0]:.6f} {single[1]:.6f}\n")
        f.write(f"two_inputs    {pair[0]:.6f} {pair[1]:.6f}\n")
        f.write(f"chosen        {ri.AND_PHI_GAP:.6f}\n")
    rows = diode_table(orc)
    with open(os.path.join(HERE, "diode_calibration.txt"), "w") as f:
        f.write("# diode (rdc_inputs.diode(128, 48, gap=1)), FP64 oracle, 14000 steps;\n")
        f.write("# arrival step at the far probe, -1 = never; columns: phi_gap tip fwd back\n")
        for pg, tip, fw, bw in rows:
            tag = "diode" if fw > 0 and bw < 0 else ""
            f.write(f"{pg:.4f} {tip:5.1f} {fw:9.1f} {bw:9.1f} {tag}\n")
        f.write(f"chosen {ri.DIODE_PHI_GAP:.4f} {ri.DIODE_TIP_CELLS:.1f}\n")


if __name__ == "__main__":
    main()
