"""Interactive serving loop with continuous batching.

Many interactive sessions (one grid each, as a user of the paper's app would
have on a tablet, §3) share one GPU.  Each session asks for frames: apply a
touch (catalytic stimulation, §2), then advance ``steps_per_frame`` Euler
steps (the paper's "render rate", §2).  The server

  * keeps every admitted session's state on the device (a slot of one of a
    few batches, one per size class, each with its own CUDA stream, so that
    small sessions' frames do not queue behind large ones);
  * admits waiting sessions whenever the device-memory budget and the session
    slots allow, and frees a session's memory when it leaves;
  * every tick gathers all sessions that have a pending frame and no frame in
    flight, applies their touches and advances them with one batched launch
    sequence per size class (a session arriving while others are on the GPU
    joins the next tick, so its work overlaps theirs on the device);
  * detects completion with CUDA events and records each frame's latency from
    request to completion.  A client either asks for its next frame as soon as
    the last one is done, or at a fixed frame rate (``frame_period``); a frame
    due while the previous one is still on the GPU waits for it, and its
    latency counts from the moment it was due.

Admission and departure never wait for the device: the library takes a
session's memory from a stream-ordered pool and enqueues its initialisation
behind the frames in flight, and the phi maps are copied from page-locked
host memory (``prepare``), so the loop keeps polling every size class while
sessions come and go.

All arithmetic runs in librdc; this module only schedules.  A session's
result is bit-identical to running it alone (tests/test_gpu_serve.py).
"""
from __future__ import annotations

import collections
import dataclasses
import gc
import heapq
import time

import numpy as np

from . import _capi as C


@dataclasses.dataclass
class Session:
    sid: int
    width: int
    height: int
    phi: np.ndarray | None = None          # H x W float32 map, or None (uniform)
    eps: float | None = None
    round_seed: int = 0                     # key of the stochastic rounding (flags RDC_STOCH_ROUND)
    frames: int = 10                        # frames the session will request
    touches: list = dataclasses.field(default_factory=list)  # per frame (cx, cy, r, value) or None
    frame_period: float = 0.0               # seconds between the client's frame requests
                                            # (0: the next one as soon as the last is done)
    # filled in by the server
    lane: int = -1
    slot: int = -1
    done_frames: int = 0
    arrival: float = 0.0
    admitted_at: float = 0.0

    def state_bytes(self, precision: int) -> int:
        esz = {C.RDC_F32: 4, C.RDC_F64: 8}.get(precision, 2)
        psz = 8 if precision == C.RDC_F64 else 4
        pitch = (self.width + 63) // 64 * 64
        return pitch * self.height * (4 * esz + psz)


@dataclasses.dataclass
class Frame:
    sid: int
    index: int
    requested: float
    completed: float = 0.0

    @property
    def latency(self) -> float:
        return self.completed - self.requested


class _Lane:
    """One size class: a batch of its sessions and the stream it runs on."""

    def __init__(self, params, k_block: int, graphs: bool, stream):
        self.stream = stream
        self.batch = C.rdc_batch_create([], [params], stream=stream.cuda_stream)
        C.rdc_batch_set_config(self.batch, max(1, k_block), 8, 64, graphs)


class Server:
    def __init__(self, precision=C.RDC_F32, k_block: int = 6, steps_per_frame: int = 50,
                 memory_budget: int | None = None, max_sessions: int = 1 << 30,
                 stream=None, graphs: bool = False, flags: int = 0,
                 lane_cells: tuple = (1 << 19, 1 << 21), lane_depth: int = 2):
        """k_block: Euler steps per batched launch (6 measured best for the
        p99 frame latency of the 64-session diode workload with three size
        classes: 1.6-1.7 ms; 8: 1.6-1.8; 4 and 5: 3.1-3.4); flags: 0 or RDC_STOCH_ROUND (16-bit storage), for every
        session.  lane_cells: upper cell counts of the size classes (a last
        class takes the rest); each class has its own batch and stream, or
        all share `stream` when one is given.  lane_depth: batched frames a
        size class may have queued on its stream at once (one running, the
        next waiting); sessions that become ready meanwhile join the
        following launch, so batches grow with the load instead of the
        stream filling with many small launches."""
        import torch
        self.torch = torch
        self.precision = precision
        self.flags = int(flags)
        self.steps = int(steps_per_frame)
        self.params = C.rdc_params_default(precision=precision, k_block=k_block, flags=self.flags)
        self.lane_cells = tuple(int(c) for c in lane_cells)
        self.lanes = []
        for _ in range(len(self.lane_cells) + 1):
            st = stream if stream is not None else torch.cuda.Stream()
            self.lanes.append(_Lane(self.params, k_block, graphs, st))
        if memory_budget is None:
            free, _ = torch.cuda.mem_get_info()
            memory_budget = int(free * 0.8)
        self.budget = int(memory_budget)
        self.used = 0
        self.max_sessions = int(max_sessions)
        self.waiting: collections.deque[Session] = collections.deque()
        self.active: dict[int, Session] = {}
        self.pending: dict[int, Frame] = {}      # sid -> requested frame not yet launched
        self.scheduled: list = []                # heap of (due time, sid, frame index)
        self.inflight: list = []                 # (event, [frames], lane)
        self.lane_depth = max(1, int(lane_depth))
        self.completed: list[Frame] = []
        self.ticks = 0
        self.cells_stepped = 0.0
        self.peak_sessions = 0
        self.evicted = 0

    # -- sessions -------------------------------------------------------------
    def prepare(self, sessions):
        """Copies the sessions' phi maps into page-locked host memory (before
        they arrive), so that admitting a session copies its map to the device
        asynchronously instead of staging it through the host."""
        torch = self.torch
        if not hasattr(torch, "from_numpy"):
            return
        for s in sessions:
            if s.phi is not None and getattr(s, "_pinned", None) is None:
                t = torch.from_numpy(np.ascontiguousarray(s.phi, dtype=np.float32)).pin_memory()
                s._pinned = t
                s.phi = t.numpy()

    def arrive(self, s: Session, now: float | None = None):
        s.arrival = time.perf_counter() if now is None else now
        self.waiting.append(s)
        self._admit()

    def _admit(self):
        while self.waiting and len(self.active) < self.max_sessions:
            s = self.waiting[0]
            need = s.state_bytes(self.precision)
            if self.used + need > self.budget:
                break
            p = C.rdc_params_default(precision=self.precision, k_block=self.params.k_block,
                                     flags=self.flags,
                                     round_seed=s.round_seed if self.flags else 0)
            if s.eps is not None:
                p.eps = s.eps
            s.lane = self._lane_of(s)
            s.slot = C.rdc_batch_add(self.lanes[s.lane].batch, s.width, s.height, p, s.phi)
            s.admitted_at = time.perf_counter()
            self.used += need
            self.waiting.popleft()
            self.active[s.sid] = s
            self.peak_sessions = max(self.peak_sessions, len(self.active))
            self._request(s)

    def _lane_of(self, s: Session) -> int:
        cells = s.width * s.height
        for i, c in enumerate(self.lane_cells):
            if cells <= c:
                return i
        return len(self.lane_cells)

    def _request(self, s: Session):
        """The session's next frame: pending at once, or at its due time when
        the client asks at a fixed rate (counted from admission)."""
        if s.done_frames >= s.frames:
            return
        now = time.perf_counter()
        if s.frame_period <= 0.0:
            self.pending[s.sid] = Frame(s.sid, s.done_frames, now)
            return
        due = s.admitted_at + s.done_frames * s.frame_period
        if due <= now:
            self.pending[s.sid] = Frame(s.sid, s.done_frames, due)
        else:
            heapq.heappush(self.scheduled, (due, s.sid, s.done_frames))

    def _release_due(self):
        """Moves the frames whose due time has come to the pending set."""
        now = time.perf_counter()
        while self.scheduled and self.scheduled[0][0] <= now:
            due, sid, idx = heapq.heappop(self.scheduled)
            if sid in self.active:
                self.pending[sid] = Frame(sid, idx, due)

    def next_due(self) -> float | None:
        """perf_counter time of the next scheduled frame request, if any."""
        return self.scheduled[0][0] if self.scheduled else None

    def _leave(self, s: Session):
        C.rdc_batch_remove(self.lanes[s.lane].batch, s.slot)
        self.used -= s.state_bytes(self.precision)
        del self.active[s.sid]
        self._admit()

    # -- the loop -------------------------------------------------------------
    def tick(self) -> int:
        """Launches one batched frame for every session with a pending
        request and none in flight, one launch sequence per size class.
        Returns the number of sessions stepped."""
        self._release_due()
        busy = {f.sid for _, fs, _ in self.inflight for f in fs}
        depth: dict[int, int] = {}
        for _, _, li in self.inflight:
            depth[li] = depth.get(li, 0) + 1
        ready = [sid for sid in self.pending if sid not in busy
                 and depth.get(self.active[sid].lane, 0) < self.lane_depth]
        if not ready:
            return 0
        by_lane: dict[int, list[int]] = {}
        for sid in ready:
            by_lane.setdefault(self.active[sid].lane, []).append(sid)
        for li, sids in sorted(by_lane.items()):
            lane = self.lanes[li]
            frames = []
            slots = []
            for sid in sids:
                s = self.active[sid]
                f = self.pending.pop(sid)
                t = s.touches[f.index] if f.index < len(s.touches) else None
                if t is not None:
                    C.rdc_batch_seed(lane.batch, s.slot, *t)
                slots.append(s.slot)
                frames.append(f)
                self.cells_stepped += s.width * s.height * self.steps
            C.rdc_batch_step(lane.batch, slots, self.steps)
            ev = self.torch.cuda.Event()
            ev.record(lane.stream)
            self.inflight.append((ev, frames, li))
        self.ticks += 1
        return len(ready)

    def poll(self) -> int:
        """Completes finished frames; returns how many completed."""
        n = 0
        still = []
        for ev, frames, li in self.inflight:
            if ev.query():
                now = time.perf_counter()
                for f in frames:
                    if f.sid not in self.active:      # evicted while in flight
                        continue
                    f.completed = now
                    self.completed.append(f)
                    s = self.active[f.sid]
                    s.done_frames += 1
                    n += 1
                    if s.done_frames >= s.frames:
                        self._leave(s)
                    else:
                        self._request(s)
            else:
                still.append((ev, frames, li))
        self.inflight = still
        return n

    def evict(self, sid: int) -> bool:
        """Drops a session at once (a client that went away): its pending or
        in-flight frame is discarded and its memory freed; the other
        sessions are unaffected.  Returns False if the session is unknown."""
        if sid in self.pending:
            del self.pending[sid]
        if any(x[1] == sid for x in self.scheduled):
            self.scheduled = [x for x in self.scheduled if x[1] != sid]
            heapq.heapify(self.scheduled)
        for _, frames, _ in self.inflight:
            frames[:] = [f for f in frames if f.sid != sid]
        if sid in self.active:
            self._leave(self.active[sid])
            self.evicted += 1
            return True
        for s in list(self.waiting):
            if s.sid == sid:
                self.waiting.remove(s)
                self.evicted += 1
                return True
        return False

    def idle(self) -> bool:
        return not (self.waiting or self.active or self.inflight or self.scheduled)

    def read(self, s: Session, dtype=np.float64):
        u = np.empty((s.height, s.width), dtype=dtype)
        v = np.empty_like(u)
        C.rdc_batch_read(self.lanes[s.lane].batch, s.slot, u, v)
        return u, v

    def close(self):
        for lane in self.lanes:
            if lane.batch:
                C.rdc_batch_destroy(lane.batch)
                lane.batch = None

    def stats(self) -> dict:
        lat = np.array([f.latency for f in self.completed]) * 1e3
        return {"frames": len(self.completed),
                "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                "max_ms": float(lat.max()) if len(lat) else None,
                "ticks": self.ticks, "cells_stepped": self.cells_stepped,
                "peak_sessions": self.peak_sessions, "evicted": self.evicted}


def run_workload(sessions, arrivals, server: Server, poll_sleep: float = 50e-6,
                 on_complete=None, time_limit: float = 600.0):
    """Drives a server through a list of sessions arriving at the given times
    (seconds from start).  Returns (wall seconds, stats)."""
    order = sorted(range(len(sessions)), key=lambda i: arrivals[i])
    server.prepare(sessions)
    # the loop allocates many small objects; a garbage-collector pass in the
    # middle of it would hold every completion back, so collect before and
    # after instead
    gc_on = gc.isenabled()
    gc.collect()
    gc.disable()
    try:
        return _drive(server, sessions, arrivals, order, poll_sleep, time_limit)
    finally:
        if gc_on:
            gc.enable()


def _drive(server, sessions, arrivals, order, poll_sleep, time_limit):
    t0 = time.perf_counter()
    nxt = 0
    while True:
        now = time.perf_counter() - t0
        while nxt < len(order) and arrivals[order[nxt]] <= now:
            server.arrive(sessions[order[nxt]])
            nxt += 1
        server.poll()
        launched = server.tick()
        if nxt >= len(order) and server.idle():
            break
        if now > time_limit:
            raise TimeoutError("serving workload did not finish")
        if not launched:
            # nothing to launch: sleep, but no longer than until the next
            # arrival or frame request when no frame is on the GPU
            wait = poll_sleep
            if not server.inflight:
                nexts = [t0 + arrivals[order[nxt]]] if nxt < len(order) else []
                if server.next_due() is not None:
                    nexts.append(server.next_due())
                if nexts:
                    wait = max(poll_sleep, min(nexts) - time.perf_counter())
            time.sleep(min(wait, 1e-3))
    server.torch.cuda.synchronize()
    return time.perf_counter() - t0, server.stats()
