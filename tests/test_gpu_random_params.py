"""FP64 on the GPU equals the oracle bit for bit across the parameter space,
not only at Table 1: seeded random grid sizes, kinetic parameters (eps, f, q,
Du, dt, dx within the validity limits the C ABI enforces), piecewise phi maps,
seeds, test modes and temporal-blocking depths.  Inputs come from a seeded
generator; expected values only from the oracle."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_CASES = 24


def _case(i):
    rng = np.random.default_rng(9000 + i)
    W = int(rng.integers(1, 48))
    H = int(rng.integers(1, 48))
    q = float(rng.uniform(0.0005, 0.01))
    f = float(rng.uniform(1.0, 3.0)) + 0.01 - q          # f + q > 1
    eps = float(rng.uniform(0.01, 0.1))
    dx = float(rng.uniform(0.1, 1.0))
    dt = float(rng.uniform(1e-4, 2e-3))
    Du = float(rng.uniform(0.0, 0.25 * dx * dx / dt))   # explicit diffusion limit
    phi_lo = q * (1 + f) * 1.2 + 0.01                      # positive rest state
    phi = np.full((H, W), phi_lo + float(rng.uniform(0.0, 0.05)))
    if W > 3 and H > 3:                                    # a passive band
        j0 = int(rng.integers(0, W - 2))
        phi[:, j0:j0 + 2] = phi_lo + 0.1
    seeds = [(float(rng.uniform(0, W)), float(rng.uniform(0, H)),
              float(rng.uniform(0.5, 6.0)), float(rng.choice([0.8, 1.0])))
             for _ in range(int(rng.integers(1, 4)))]
    flags = int(rng.choice([0, 0, 1, 2]))
    k = int(rng.choice([1, 1, 2, 3, 4, 6, 8]))
    n = int(rng.integers(1, 40))
    return dict(W=W, H=H, q=q, f=f, eps=eps, dx=dx, dt=dt, Du=Du, phi=phi, seeds=seeds,
                flags=flags, k=k, n=n)


@pytest.mark.parametrize("i", range(N_CASES))
def test_f64_random_parameters_bitwise(gpu, orc, om, i):
    c = _case(i)
    W, H = c["W"], c["H"]
    p = gpu.rdc_params_default(precision=1, eps=c["eps"], f=c["f"], q=c["q"], Du=c["Du"],
                               dt=c["dt"], dx=c["dx"], flags=c["flags"], k_block=c["k"])
    h = gpu.rdc_create(W, H, p, c["phi"])
    try:
        for s in c["seeds"]:
            gpu.rdc_seed(h, *s)
        gpu.rdc_step(h, c["n"])
        u = np.empty((H, W))
        v = np.empty((H, W))
        gpu.rdc_read(h, u, v)
    finally:
        gpu.rdc_destroy(h)
    params = om.Params(eps=c["eps"], f=c["f"], q=c["q"], Du=c["Du"], dt=c["dt"], dx=c["dx"],
                       flags=c["flags"])
    u0, v0 = orc.rest_field(c["phi"], f=c["f"], q=c["q"])
    for (cx, cy, r, val) in c["seeds"]:
        orc.seed_disk(u0, cx, cy, r, val)
    ref = orc.run(c["phi"], u0, v0, c["n"], params=params)
    assert ref["status"] == om.OK
    assert np.array_equal(u, ref["u"]), (i, c["k"], c["flags"])
    assert np.array_equal(v, ref["v"]), (i, c["k"], c["flags"])


def _gpu(pkg, c, prec, k):
    W, H = c["W"], c["H"]
    p = pkg.rdc_params_default(precision=prec, eps=c["eps"], f=c["f"], q=c["q"], Du=c["Du"],
                               dt=c["dt"], dx=c["dx"], flags=c["flags"], k_block=k)
    h = pkg.rdc_create(W, H, p, c["phi"].astype(np.float32))
    try:
        for s in c["seeds"]:
            pkg.rdc_seed(h, *s)
        pkg.rdc_step(h, c["n"] + 13)
        u = np.empty((H, W))
        v = np.empty((H, W))
        pkg.rdc_read(h, u, v)
    finally:
        pkg.rdc_destroy(h)
    return u, v


@pytest.mark.parametrize("prec", [0, 2])
@pytest.mark.parametrize("i", range(N_CASES))
def test_fp32_random_parameters_kblock_bitwise(gpu, prec, i):
    """FP32 compute (FP32 and BF16 storage): the case's temporal-blocking depth
    gives the bits of single steps for random parameters too."""
    c = _case(i)
    a, av = _gpu(gpu, c, prec, 1)
    b, bv = _gpu(gpu, c, prec, max(2, c["k"]))
    assert np.array_equal(a, b) and np.array_equal(av, bv), (i, c["k"])
