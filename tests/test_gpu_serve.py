"""Continuous-batching serving loop: sessions arriving while others run are
admitted as memory frees up, their frames share batched launches, and every
session's final state equals the same session run alone, bit for bit."""
from __future__ import annotations

import numpy as np
import pytest

import rdc_inputs as ri

pytestmark = pytest.mark.gpu


def _sessions(serve, n, seed=5, frames=6):
    rng = np.random.default_rng(seed)
    out = []
    for sid in range(n):
        N = int(rng.choice([64, 128, 192]))
        c = ri.diode(N, N // 2 if N > 64 else 48)
        H, W = c.phi.shape
        touches = []
        for f in range(frames):
            if f % 2 == 0:
                cx, cy, r = c.seeds["anode"]
                touches.append((float(cx + rng.uniform(-2, 2)), float(cy), 4.0, 0.8))
            else:
                touches.append(None)
        out.append(serve.Session(sid, W, H, phi=c.phi.astype(np.float32), frames=frames,
                                 touches=touches))
    return out


def _alone(pkg, s, steps, precision=0, flags=0):
    p = pkg.rdc_params_default(precision=precision, flags=flags,
                               round_seed=s.round_seed if flags else 0)
    h = pkg.rdc_create(s.width, s.height, p, s.phi)
    try:
        for f in range(s.frames):
            t = s.touches[f]
            if t is not None:
                pkg.rdc_seed(h, *t)
            pkg.rdc_step(h, steps)
        u = np.empty((s.height, s.width))
        v = np.empty((s.height, s.width))
        pkg.rdc_read(h, u, v)
    finally:
        pkg.rdc_destroy(h)
    return u, v


def test_serving_mix_equals_alone(gpu):
    from paper_1901_06535_gb300 import serve
    sessions = _sessions(serve, 10)
    # a budget that fits only a few sessions at once: the rest wait to be admitted
    budget = 3 * max(s.state_bytes(0) for s in sessions)
    srv = serve.Server(precision=0, k_block=2, steps_per_frame=20, memory_budget=budget)
    finals = {}
    orig_leave = srv._leave

    def leave(s):
        finals[s.sid] = srv.read(s)
        orig_leave(s)

    srv._leave = leave
    try:
        arrivals = [0.002 * i for i in range(len(sessions))]
        wall, st = serve.run_workload(sessions, arrivals, srv)
    finally:
        srv.close()
    assert st["frames"] == sum(s.frames for s in sessions)
    assert 1 <= st["peak_sessions"] <= 3
    assert st["p50_ms"] > 0 and st["p99_ms"] >= st["p50_ms"]
    for s in sessions:
        u, v = finals[s.sid]
        ua, va = _alone(gpu, s, 20)
        assert np.array_equal(u, ua) and np.array_equal(v, va), s.sid


def test_serving_overlapping_arrivals(gpu):
    """All sessions at once, generous budget: many share each tick."""
    from paper_1901_06535_gb300 import serve
    sessions = _sessions(serve, 12, seed=9, frames=4)
    srv = serve.Server(precision=0, k_block=4, steps_per_frame=16)
    finals = {}
    orig_leave = srv._leave

    def leave(s):
        finals[s.sid] = srv.read(s)
        orig_leave(s)

    srv._leave = leave
    try:
        wall, st = serve.run_workload(sessions, [0.0] * len(sessions), srv)
    finally:
        srv.close()
    assert st["peak_sessions"] == len(sessions)
    assert st["ticks"] < st["frames"]          # frames were batched together
    for s in sessions[:4]:
        u, _ = finals[s.sid]
        ua, _ = _alone(gpu, s, 16)
        assert np.array_equal(u, ua)


def test_serving_eviction_mid_stream(gpu):
    """A session dropped while its frame is in flight frees its memory; the
    remaining sessions finish with the same bits as alone."""
    from paper_1901_06535_gb300 import serve
    sessions = _sessions(serve, 6, seed=21, frames=5)
    srv = serve.Server(precision=0, k_block=2, steps_per_frame=12)
    finals = {}
    orig_leave = srv._leave

    def leave(s):
        if s.done_frames >= s.frames:
            finals[s.sid] = srv.read(s)
        orig_leave(s)

    srv._leave = leave
    try:
        for s in sessions:
            srv.arrive(s)
        srv.tick()                                  # all six frames in flight
        used_before = srv.used
        assert srv.evict(sessions[2].sid)           # dropped mid-stream
        assert srv.used < used_before and sessions[2].sid not in srv.active
        while not srv.idle():
            srv.poll()
            if not srv.tick():
                srv.torch.cuda.synchronize()
        st = srv.stats()
    finally:
        srv.close()
    assert st["evicted"] == 1 and sessions[2].sid not in finals
    for s in sessions:
        if s.sid == sessions[2].sid:
            continue
        u, v = finals[s.sid]
        ua, va = _alone(gpu, s, 12)
        assert np.array_equal(u, ua) and np.array_equal(v, va), s.sid


def test_serving_stochastic_rounding_mix_equals_alone(gpu):
    """BF16 storage with stochastic rounding, one key per session: the mix
    gives each session the bits it gets alone (the rounding depends only on
    the session's key, the cell and the step)."""
    from paper_1901_06535_gb300 import serve
    sessions = _sessions(serve, 8, seed=31, frames=4)
    for s in sessions:
        s.round_seed = 1000 + s.sid
    srv = serve.Server(precision=2, k_block=4, steps_per_frame=14, flags=4)
    finals = {}
    orig_leave = srv._leave

    def leave(s):
        finals[s.sid] = srv.read(s)
        orig_leave(s)

    srv._leave = leave
    try:
        serve.run_workload(sessions, [0.001 * i for i in range(len(sessions))], srv)
    finally:
        srv.close()
    for s in sessions:
        u, v = finals[s.sid]
        ua, va = _alone(gpu, s, 14, precision=2, flags=4)
        assert np.array_equal(u, ua) and np.array_equal(v, va), s.sid


def test_serving_size_classes_equal_alone(gpu):
    """Sessions split over three size classes (each its own batch and
    stream, stepping concurrently): every session equals its solo run."""
    from paper_1901_06535_gb300 import serve
    sessions = _sessions(serve, 9, seed=41, frames=5)
    srv = serve.Server(precision=0, k_block=6, steps_per_frame=18, lane_cells=(4000, 10000))
    finals = {}
    lanes = {}
    orig_leave = srv._leave

    def leave(s):
        finals[s.sid] = srv.read(s)
        lanes[s.sid] = s.lane
        orig_leave(s)

    srv._leave = leave
    try:
        serve.run_workload(sessions, [0.0005 * i for i in range(len(sessions))], srv)
    finally:
        srv.close()
    assert len(set(lanes.values())) >= 2, lanes
    for s in sessions:
        u, v = finals[s.sid]
        ua, va = _alone(gpu, s, 18)
        assert np.array_equal(u, ua) and np.array_equal(v, va), s.sid


def test_serving_bench_configuration_mix_equals_alone(gpu):
    """The serving benchmark's configuration: diode sessions of 512², 1024² and
    2048² (at least one of each), k = 6, 50-step frames with a touch before
    each, Poisson arrivals, half of the clients asking at 60 frames per second:
    every session's final state equals its solo run bit for bit."""
    from paper_1901_06535_gb300 import serve
    specs = ri.diode_sessions(seed=5, n=9, frames=4, rate=200.0)
    assert {s.size for s in specs} == {512, 1024, 2048}
    sessions = [serve.Session(s.sid, s.size, s.size, phi=s.phi, frames=4, touches=s.touches,
                              frame_period=(1.0 / 60.0 if s.sid % 2 else 0.0))
                for s in specs]
    srv = serve.Server(precision=0, k_block=6, steps_per_frame=50)
    finals = {}
    orig_leave = srv._leave

    def leave(s):
        finals[s.sid] = srv.read(s)
        orig_leave(s)

    srv._leave = leave
    try:
        wall, st = serve.run_workload(sessions, [s.arrival for s in specs], srv)
    finally:
        srv.close()
    assert st["frames"] == 4 * len(sessions) and st["peak_sessions"] >= 3
    for s in sessions:
        u, v = finals[s.sid]
        ua, va = _alone(gpu, s, 50)
        assert np.array_equal(u, ua) and np.array_equal(v, va), (s.sid, s.width)
