"""The AND-gate workload at full size: 1024 x 1024, 20000 Euler steps, two
16-cell input channels meeting head-on, a 3-cell semi-permeable band before
the output channel, phi = 0.2 elsewhere, u = 0.8 input disks (§4.1).

FP64 on the GPU is bit-identical to the oracle (tests/test_gpu_parity.py), so
its truth table here is the oracle's; FP32 must give the same table and an
output arrival within 1 % of FP64.  BF16 storage is run and reported."""
from __future__ import annotations

import numpy as np
import pytest

import rdc_inputs as ri
from tests.helpers import PREC, gpu_run

pytestmark = pytest.mark.gpu

N, STEPS, SAMPLE = 1024, 20000, 50


def _circuit():
    return ri.and_gate(N, N, arm=150, out_len=80)


def _max_at_output(pkg, c, fire, prec, flags=0, round_seed=0):
    """Largest u seen at the output probe, sampled every SAMPLE steps."""
    phi = c.phi if prec == "f64" else c.phi.astype(np.float32)
    p = pkg.rdc_params_default(precision=PREC[prec], k_block=0 if prec != "f64" else 1,
                               flags=flags, round_seed=round_seed)
    h = pkg.rdc_create(N, N, p, phi)
    best = -1.0
    try:
        for name in fire:
            pkg.rdc_seed(h, *c.seeds[name], 0.8)
        for _ in range(STEPS // SAMPLE):
            pkg.rdc_step(h, SAMPLE)
            best = max(best, float(pkg.rdc_probe(h, [c.probes["out"]])[0]))
        assert pkg.rdc_check(h)[0] == pkg.RDC_OK
    finally:
        pkg.rdc_destroy(h)
    return best


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_andgate_1024_truth_table(gpu, prec):
    c = _circuit()
    out = {tuple(f): _max_at_output(gpu, c, f, prec) > 0.3
           for f in ([], ["A"], ["B"], ["A", "B"])}
    assert out == {(): False, ("A",): False, ("B",): False, ("A", "B"): True}, out


def test_andgate_1024_output_arrival_f32_vs_f64(gpu, record_property):
    c = _circuit()
    seeds = [(*c.seeds["A"], 0.8), (*c.seeds["B"], 0.8)]
    t = {}
    for prec in ("f64", "f32"):
        phi = c.phi if prec == "f64" else c.phi.astype(np.float32)
        _, _, ex = gpu_run(gpu, N, N, phi=phi, seeds=seeds, n=STEPS, prec=prec, k=1,
                           probes=[c.probes["out"]])
        t[prec] = float(ex["t_arr"][0])
    record_property("t_out", t)
    assert t["f64"] > 0 and abs(t["f32"] - t["f64"]) <= 0.01 * t["f64"], t


def test_andgate_1024_bf16_reported(gpu, record_property):
    """BF16 storage on the same circuit: reported, not gated (the gate's
    window is about 2 % of the band's phi; BF16 shifts fronts by ~1 %)."""
    c = _circuit()
    table = {"".join(f) or "-": bool(_max_at_output(gpu, c, f, "bf16") > 0.3)
             for f in ([], ["A"], ["B"], ["A", "B"])}
    record_property("bf16_truth_table", table)
    print("bf16 AND truth table at 1024^2:", table)


@pytest.mark.parametrize("prec", ["bf16", "f16"])
def test_andgate_1024_stochastic_rounding_truth_table(gpu, prec, record_property):
    """16-bit storage with stochastic rounding (RDC_STOCH_ROUND) on the same
    circuit, three keys: the AND truth table holds for each.  (BF16 with
    round-to-nearest loses it: v stagnates and the colliding fronts do not
    cross the band; the runs are deterministic for a given key.)"""
    c = _circuit()
    tables = {}
    for seed in (1, 2, 3):
        tables[seed] = {"".join(f) or "-": bool(_max_at_output(gpu, c, f, prec, flags=4,
                                                               round_seed=seed) > 0.3)
                        for f in ([], ["A"], ["B"], ["A", "B"])}
    record_property(f"{prec}_stochastic_truth_tables", tables)
    print(f"{prec} + stochastic rounding AND truth tables at 1024^2:", tables)
    for seed, t in tables.items():
        assert t == {"-": False, "A": False, "B": False, "AB": True}, (seed, t)


def test_andgate_1024_maxabs_1000_reported(gpu, record_property):
    """Pointwise max-abs of u against FP64 after 1000 steps of the 1024²
    AND-gate workload (both inputs fired), for each reduced mode: reported,
    with a sanity bound.  FP64 on the GPU is the oracle's result bit for bit (tested
    elsewhere), so it stands in for the oracle at this size."""
    c = _circuit()
    seeds = [(*c.seeds["A"], 0.8), (*c.seeds["B"], 0.8)]
    ref, _, _ = gpu_run(gpu, N, N, phi=c.phi, seeds=seeds, n=1000, prec="f64", k=1)
    out = {}
    for name, prec, flags in (("f32", "f32", 0), ("f16", "f16", 0), ("bf16", "bf16", 0),
                              ("bf16_stoch", "bf16", 4), ("f16_stoch", "f16", 4)):
        u, _, _ = gpu_run(gpu, N, N, phi=c.phi.astype(np.float32), seeds=seeds, n=1000,
                          prec=prec, k=4, flags=flags, round_seed=1 if flags else 0)
        out[name] = float(np.max(np.abs(u - ref)))
    record_property("andgate_1024_maxabs_u_1000", out)
    print("1024² AND gate: max-abs of u vs FP64 after 1000 steps:", {k: f"{v:.2e}" for k, v in out.items()})
    assert out["f32"] < 0.05 and all(v < 0.9 for v in out.values())
