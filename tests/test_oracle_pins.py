"""The FP64 oracle against what the model and the mathematics fix (CPU only)."""
from __future__ import annotations

import numpy as np
import pytest

from tests import oracle_pins as P


@pytest.mark.parametrize("pin", P.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(pin, orc, om):
    pin(orc, om)


def test_thread_count_invariance(orc):
    N = 48
    phi = np.full((N, N + 5), P.PHI_A)
    u, v = orc.rest_field(phi)
    orc.seed_disk(u, 20.0, 17.0, 7.0, 0.8)
    a = orc.run(phi, u, v, 300, nthreads=1)
    b = orc.run(phi, u, v, 300, nthreads=4)
    assert np.array_equal(a["u"], b["u"]) and np.array_equal(a["v"], b["v"])


def test_arrival_interpolation_rule(orc):
    """t_arr brackets the first step whose u reaches theta, interpolated
    linearly between the two steps around the crossing."""
    N = 64
    phi = np.full((N, N), P.PHI_A)
    u, v = orc.rest_field(phi)
    orc.seed_disk(u, 31.5, 31.5, 5.0, 0.8)
    probe = 31 * N + 31 + 12
    r = orc.run(phi, u, v, 1500, probes=[probe], theta=0.3)
    t = r["t_arr"][0]
    assert t > 0
    n = int(np.ceil(t))
    a = orc.run(phi, u, v, n - 1)["u"].ravel()[probe]
    b = orc.run(phi, u, v, n)["u"].ravel()[probe]
    assert a < 0.3 <= b
    assert t == pytest.approx((n - 1) + (0.3 - a) / (b - a), abs=1e-12)


def test_stability_reading_phi02(orc, om):
    """At phi = 0.2 forward Euler with dt = 1e-3 is linearly unstable at rest
    (|1 + dt lambda| > 1 for the fast eigenvalue): the homogeneous field does
    not stay at rest to 1e-12, unlike phi = 0.054, but stays bounded."""
    phi = np.full((8, 8), 0.2)
    u, v = orc.rest_field(phi)
    J = P.analytic_jacobian(u[0, 0], v[0, 0], 0.2)
    lam = np.linalg.eigvals(J)
    assert np.max(np.abs(1 + P.DT * lam)) > 1.0
    u[3, 4] += 1e-9
    r = orc.run(phi, u, v, 20000)
    dev = np.max(np.abs(r["u"] - orc.rest_state(0.2)))
    assert 1e-9 < dev < 1e-2
    J54 = P.analytic_jacobian(orc.rest_state(0.054), orc.rest_state(0.054), 0.054)
    assert np.max(np.abs(1 + P.DT * np.linalg.eigvals(J54))) < 1.0


# ---------------------------------------------------------------------------
# the paper's qualitative circuits on the oracle (§4.1, §4.2)
# ---------------------------------------------------------------------------

def _arrival(orc, c, fire, probe, steps):
    import os
    u, v = orc.rest_field(c.phi)
    for name in fire:
        cx, cy, r = c.seeds[name]
        orc.seed_disk(u, cx, cy, r, 0.8)
    return orc.run(c.phi, u, v, steps, nthreads=min(8, os.cpu_count() or 1),
                   probes=[c.probes[probe]])["t_arr"][0]


def test_and_gate_truth_table_oracle(orc):
    """§4.1: a single input does not reach the output (01 -> 0, 10 -> 0),
    two colliding inputs do (11 -> 1); no input, no output."""
    import rdc_inputs as ri
    c = ri.and_gate(160, 128, arm=50, out_len=40)
    steps = 9000
    assert _arrival(orc, c, [], "out", steps) < 0
    assert _arrival(orc, c, ["A"], "out", steps) < 0
    assert _arrival(orc, c, ["B"], "out", steps) < 0
    assert _arrival(orc, c, ["A", "B"], "out", steps) > 0


@pytest.mark.parametrize("flip", [False, True])
def test_diode_direction_oracle(orc, flip):
    """§4.2: a wave passes from the anode (flat side) to the cathode (pointed
    side) and not from the cathode to the anode."""
    import rdc_inputs as ri
    c = ri.diode(flip=flip)
    steps = 12000
    assert _arrival(orc, c, ["anode"], "cathode_end", steps) > 0
    assert _arrival(orc, c, ["cathode"], "anode_end", steps) < 0
