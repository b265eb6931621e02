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
