"""Helpers shared by the parity tests: run the same seeded workload through the
CUDA path (C ABI) and through the FP64 oracle."""
from __future__ import annotations

import numpy as np

PREC = {"f32": 0, "f64": 1, "bf16": 2, "f16": 3}


def round_sig(x, bits: int):
    """Round-to-nearest-even of doubles to ``bits`` significant bits (normal
    range only), computed exactly in double arithmetic."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.rint(np.ldexp(m, bits)), e - bits)


def round_to_storage(x, prec: str):
    """Values after a single RN-even rounding to the storage type of prec."""
    x = np.asarray(x, dtype=np.float64)
    if prec == "f64":
        return x.copy()
    if prec == "f32":
        return x.astype(np.float32).astype(np.float64)
    return round_sig(x, {"bf16": 8, "f16": 11}[prec])


def gpu_run(pkg, W, H, phi=None, seeds=(), n=0, prec="f64", flags=0, k=1,
            shape=None, state=None, probes=None, theta=0.3, dtype=np.float64,
            round_seed=0, chunks=None):
    """Runs n steps on the GPU; returns (u, v, extra) as host arrays.

    With ``probes`` (flat indices) it steps one at a time and returns the
    arrival time of each probe (same interpolation rule as the oracle) in
    extra["t_arr"].  ``chunks`` splits the steps into several rdc_step calls.
    """
    p = pkg.rdc_params_default(precision=PREC[prec], flags=flags, k_block=k,
                               round_seed=round_seed)
    if phi is not None:
        phi = np.ascontiguousarray(phi, dtype=np.float64 if prec == "f64" else np.float32)
    h = pkg.rdc_create(W, H, p, phi)
    extra = {}
    try:
        if shape:
            s = pkg.rdc_get_shape(h)
            cur = {f: getattr(s, f) for f, _ in s._fields_}
            cur.update(shape)
            pkg.rdc_set_shape(h, cur["bx"], cur["rows"], cur["tx"], cur["ty"],
                              cur["nthreads"], cur["k"], cur["variant"], cur["krows"])
        if state is not None:
            pkg.rdc_set_state(h, *state)
        for (cx, cy, r, val) in seeds:
            pkg.rdc_seed(h, cx, cy, r, val)
        if probes is None and chunks:
            for c in chunks:                      # n steps as several calls
                pkg.rdc_step(h, c)
        elif probes is None:
            pkg.rdc_step(h, n)
        else:
            pr = np.asarray(probes, dtype=np.int64)
            prev = pkg.rdc_probe(h, pr)
            t = np.where(prev >= theta, 0.0, -1.0)
            for step in range(1, n + 1):
                pkg.rdc_step(h, 1)
                cur = pkg.rdc_probe(h, pr)
                hit = (t < 0) & (cur >= theta)
                t[hit] = (step - 1) + (theta - prev[hit]) / (cur[hit] - prev[hit])
                prev = cur
            extra["t_arr"] = t
        u = np.empty((H, W), dtype=dtype)
        v = np.empty((H, W), dtype=dtype)
        extra["status"] = pkg.rdc_read(h, u, v)
        extra["view"] = pkg.rdc_get_view(h)
    finally:
        pkg.rdc_destroy(h)
    return u, v, extra


def orc_run(orc, om, W, H, phi=None, seeds=(), n=0, flags=0, state=None,
            probes=None, theta=0.3, nthreads=None):
    import os
    if phi is None:
        phi = np.full((H, W), 0.054)
    phi = np.asarray(phi, dtype=np.float64)
    if state is None:
        u, v = orc.rest_field(phi)
    else:
        u = np.array(state[0], dtype=np.float64)
        v = np.array(state[1], dtype=np.float64)
    for (cx, cy, r, val) in seeds:
        orc.seed_disk(u, cx, cy, r, val)
    nt = nthreads or min(16, os.cpu_count() or 1)
    return orc.run(phi, u, v, n, params=om.Params(flags=flags), nthreads=nt,
                   probes=probes, theta=theta)
