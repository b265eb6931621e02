"""Host logic of the serving loop on the CPU: the library calls and CUDA
streams/events are replaced by fakes that record what the server asks for, so
admission by memory, the per-size-class batches, tick grouping, eviction and
the completion path are checked without a GPU.  (The GPU tests check that
each served session equals its solo run bit for bit.)"""
from __future__ import annotations

import sys
import types

import pytest

from paper_1901_06535_gb300 import serve


class FakeC:
    """Stands in for the ctypes binding: batches are lists of slots."""
    RDC_F32, RDC_F64 = 0, 1

    def __init__(self):
        self.batches = {}
        self.steps = []          # (batch id, sorted slots, n)
        self.seeds = []          # (batch id, slot)
        self.next_id = 1

    def rdc_params_default(self, **kw):
        return types.SimpleNamespace(k_block=kw.get("k_block", 0), eps=0.0243, **{
            k: v for k, v in kw.items() if k != "k_block"})

    def rdc_batch_create(self, grids, params, stream=None):
        b = self.next_id
        self.next_id += 1
        self.batches[b] = {"slots": {}, "stream": stream, "config": None}
        return b

    def rdc_batch_set_config(self, b, k, rows, krows, graphs):
        self.batches[b]["config"] = (k, rows, krows, graphs)

    def rdc_batch_add(self, b, w, h, p, phi):
        slots = self.batches[b]["slots"]
        slot = next(i for i in range(len(slots) + 1) if i not in slots)
        slots[slot] = (w, h)
        return slot

    def rdc_batch_remove(self, b, slot):
        del self.batches[b]["slots"][slot]

    def rdc_batch_seed(self, b, slot, *touch):
        assert slot in self.batches[b]["slots"]
        self.seeds.append((b, slot))

    def rdc_batch_step(self, b, slots, n):
        assert all(s in self.batches[b]["slots"] for s in slots)
        self.steps.append((b, tuple(sorted(slots)), n))

    def rdc_batch_read(self, b, slot, u, v):
        assert slot in self.batches[b]["slots"]

    def rdc_batch_destroy(self, b):
        del self.batches[b]


class FakeEvent:
    pending = []             # events not yet "completed" by the test

    def __init__(self):
        self.done = False

    def record(self, stream):
        self.stream = stream
        FakeEvent.pending.append(self)

    def query(self):
        return self.done


def _fake_torch():
    streams = iter(range(100, 200))

    class Stream:
        def __init__(self):
            self.cuda_stream = next(streams)

    cuda = types.SimpleNamespace(Stream=Stream, Event=FakeEvent,
                                 mem_get_info=lambda: (1 << 40, 1 << 40),
                                 synchronize=lambda: None)
    return types.SimpleNamespace(cuda=cuda)


@pytest.fixture
def fakes(monkeypatch):
    c = FakeC()
    monkeypatch.setattr(serve, "C", c)
    monkeypatch.setitem(sys.modules, "torch", _fake_torch())
    FakeEvent.pending = []
    return c


def _complete_all():
    for ev in FakeEvent.pending:
        ev.done = True
    FakeEvent.pending = []


def _session(sid, n, frames=2, touch=True):
    return serve.Session(sid, n, n, frames=frames,
                         touches=[(n / 2, n / 2, 3.0, 0.8) if touch else None] * frames)


def test_size_classes(fakes):
    srv = serve.Server(steps_per_frame=50)
    assert len(srv.lanes) == 3 and len({ln.stream.cuda_stream for ln in srv.lanes}) == 3
    # thresholds 2^19 and 2^21 cells: 724² and 1448² are just below them
    for n, lane in ((512, 0), (724, 0), (725, 1), (1024, 1), (1448, 1), (1449, 2), (2048, 2),
                    (1, 0)):
        assert srv._lane_of(_session(0, n)) == lane, n
    one = serve.Server(lane_cells=())
    assert len(one.lanes) == 1 and one._lane_of(_session(0, 4096)) == 0


def test_shared_stream_when_given(fakes):
    st = types.SimpleNamespace(cuda_stream=7)
    srv = serve.Server(stream=st)
    assert all(ln.stream is st for ln in srv.lanes)
    assert all(fakes.batches[ln.batch]["stream"] == 7 for ln in srv.lanes)


def test_tick_groups_by_class_and_completes(fakes):
    srv = serve.Server(steps_per_frame=20, k_block=6)
    sessions = [_session(0, 512), _session(1, 2048), _session(2, 512), _session(3, 1024)]
    for s in sessions:
        srv.arrive(s)
    assert srv.tick() == 4
    # one batched step per size class, each over that class's sessions only
    by_batch = {b: slots for b, slots, n in fakes.steps}
    lane_batch = [ln.batch for ln in srv.lanes]
    assert by_batch[lane_batch[0]] == tuple(sorted([sessions[0].slot, sessions[2].slot]))
    assert by_batch[lane_batch[1]] == (sessions[3].slot,)
    assert by_batch[lane_batch[2]] == (sessions[1].slot,)
    assert all(n == 20 for _, _, n in fakes.steps) and len(fakes.seeds) == 4
    assert srv.tick() == 0                      # every session has a frame in flight
    _complete_all()
    assert srv.poll() == 4
    assert all(s.done_frames == 1 for s in sessions)
    assert srv.tick() == 4                      # second frames
    _complete_all()
    srv.poll()
    assert srv.idle() and srv.used == 0
    assert all(not b["slots"] for b in fakes.batches.values())
    st = srv.stats()
    assert st["frames"] == 8 and st["ticks"] == 2 and st["peak_sessions"] == 4
    assert st["cells_stepped"] == 2 * 20 * (2 * 512 ** 2 + 2048 ** 2 + 1024 ** 2)
    srv.close()
    assert not fakes.batches


def test_admission_by_memory(fakes):
    s = [_session(i, 512, frames=1) for i in range(3)]
    srv = serve.Server(memory_budget=2 * s[0].state_bytes(0))
    for x in s:
        srv.arrive(x)
    assert set(srv.active) == {0, 1} and [w.sid for w in srv.waiting] == [2]
    srv.tick()
    _complete_all()
    srv.poll()                                  # 0 and 1 finish and leave; 2 is admitted
    assert set(srv.active) == {2} and not srv.waiting
    assert srv.used == s[2].state_bytes(0)


def test_evict_in_flight_and_waiting(fakes):
    s = [_session(i, 256, frames=3, touch=False) for i in range(3)]
    srv = serve.Server(memory_budget=2 * s[0].state_bytes(0))
    for x in s:
        srv.arrive(x)
    srv.tick()
    assert srv.evict(0)                         # in flight: its frame is dropped
    assert 0 not in srv.active and srv.evicted == 1
    assert set(srv.active) == {1, 2}            # the waiting session took its memory
    assert not srv.evict(99)
    _complete_all()
    srv.poll()
    assert all(f.sid != 0 for f in srv.completed)
    assert srv.evict(2) and srv.evicted == 2
    assert not fakes.seeds                      # no touches were requested


def test_run_workload_drives_to_completion(fakes, monkeypatch):
    # events complete as soon as they are polled once
    monkeypatch.setattr(FakeEvent, "query", lambda self: True)
    sessions = [_session(i, (256, 1024, 2048)[i % 3], frames=3) for i in range(7)]
    srv = serve.Server(steps_per_frame=10)
    wall, st = serve.run_workload(sessions, [0.0] * 7, srv, poll_sleep=0.0)
    assert st["frames"] == 21 and srv.idle() and wall >= 0
    assert st["p99_ms"] >= st["p50_ms"] >= 0


def test_fixed_frame_rate_requests(fakes):
    """A client asking at a fixed rate: its next frame becomes pending only at
    its due time (counted from admission), and a frame's latency counts from
    that due time, not from when the server launched it."""
    import time
    s = _session(0, 256, frames=3)
    s.frame_period = 0.02
    srv = serve.Server(steps_per_frame=5)
    srv.arrive(s)
    assert srv.tick() == 1                      # frame 0 is due at admission
    _complete_all()
    srv.poll()
    assert srv.tick() == 0 and srv.next_due() == pytest.approx(s.admitted_at + 0.02)
    assert not srv.idle()                       # a request is scheduled
    time.sleep(0.025)
    assert srv.tick() == 1                      # frame 1 is due now
    assert srv.completed[0].requested == s.admitted_at
    _complete_all()
    srv.poll()
    assert srv.completed[1].requested == pytest.approx(s.admitted_at + 0.02)
    time.sleep(0.02)
    srv.tick()
    _complete_all()
    srv.poll()
    assert srv.idle() and len(srv.completed) == 3


def test_evict_drops_scheduled_requests(fakes):
    s = _session(0, 256, frames=5)
    s.frame_period = 10.0
    srv = serve.Server()
    srv.arrive(s)
    srv.tick()
    _complete_all()
    srv.poll()
    assert srv.next_due() is not None
    assert srv.evict(0)
    assert srv.next_due() is None and srv.idle()


def test_lane_depth_limits_queued_batches(fakes):
    """With lane_depth 1 a size class launches its next batch only after the
    one on its stream completes; the sessions that became ready meanwhile go
    out together."""
    s = [_session(i, 256, frames=2) for i in range(3)]
    srv = serve.Server(steps_per_frame=5, lane_depth=1)
    srv.arrive(s[0])
    assert srv.tick() == 1
    srv.arrive(s[1])
    srv.arrive(s[2])
    assert srv.tick() == 0                      # the class's stream is busy
    _complete_all()
    srv.poll()
    assert srv.tick() == 3                      # one batch: s0's second frame, s1, s2
    assert fakes.steps[-1][1] == tuple(sorted(x.slot for x in s))
