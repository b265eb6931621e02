"""Multi-rank paths on CPU ranks (gloo, world size 2).

1. Row-strip decomposition of one grid: each rank owns a strip of rows and
   steps it with the FP64 oracle on the strip plus one halo row of u from each
   neighbour, exchanged every step (v and phi are local: v does not diffuse,
   Eq. 1, and phi is static).  The gathered result must equal the unsplit
   oracle bit for bit -- the exchange a multi-GPU strip path would need.
2. The same with temporal blocking: K rows of u and v every K steps, the
   halo recomputed (K = 4, 6).
3. The library's strip plan (paper_1901_06535_gb300.strips.strip_plan) on
   three ranks: its copies become send/recv pairs between the ranks that
   hold the strips, and the gathered strips equal the unsplit oracle.
4. The benchmark's rank aggregation: the slowest rank's time and the
   whole-job (weak-scaling) rate.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

W, H, STEPS = 37, 29, 120


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _initial():
    import oracle
    orc = oracle.load()
    phi = np.full((H, W), 0.054)
    phi[:, 20:23] = 0.0975
    u, v = orc.rest_field(phi)
    orc.seed_disk(u, 10.0, 14.0, 6.0, 0.8)
    orc.seed_disk(u, 30.0, 3.0, 4.0, 1.0)
    return orc, phi, u, v


def _strip_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    orc, phi, u, v = _initial()
    bounds = np.linspace(0, H, world + 1).astype(int)
    r0, r1 = bounds[rank], bounds[rank + 1]
    up = rank > 0            # a neighbour above
    dn = rank < world - 1    # a neighbour below
    us, vs, ph = u[r0:r1].copy(), v[r0:r1].copy(), phi[r0:r1]
    for _ in range(STEPS):
        halo_top = torch.empty(W, dtype=torch.float64)
        halo_bot = torch.empty(W, dtype=torch.float64)
        reqs = []
        if up:
            reqs.append(dist.isend(torch.from_numpy(us[0].copy()), rank - 1))
            reqs.append(dist.irecv(halo_top, rank - 1))
        if dn:
            reqs.append(dist.isend(torch.from_numpy(us[-1].copy()), rank + 1))
            reqs.append(dist.irecv(halo_bot, rank + 1))
        for q in reqs:
            q.wait()
        rows_u = ([halo_top.numpy()] if up else []) + list(us) + ([halo_bot.numpy()] if dn else [])
        ext_u = np.ascontiguousarray(np.stack(rows_u))
        # v and phi of the halo rows only feed the halo rows' own (discarded) update
        pad = lambda a: np.ascontiguousarray(np.concatenate(  # noqa: E731
            ([a[:1]] if up else []) + [a] + ([a[-1:]] if dn else [])))
        u1, v1, rc, _ = orc.step(pad(ph), ext_u, pad(vs))
        a = 1 if up else 0
        us = u1[a:a + (r1 - r0)].copy()
        vs = v1[a:a + (r1 - r0)].copy()
    if rank == 0:
        parts_u, parts_v = [us], [vs]
        for src in range(1, world):
            n = (bounds[src + 1] - bounds[src]) * W
            tu = torch.empty(n, dtype=torch.float64)
            tv = torch.empty(n, dtype=torch.float64)
            dist.recv(tu, src)
            dist.recv(tv, src)
            parts_u.append(tu.numpy().reshape(-1, W))
            parts_v.append(tv.numpy().reshape(-1, W))
        np.savez(out_path, u=np.concatenate(parts_u), v=np.concatenate(parts_v))
    else:
        dist.send(torch.from_numpy(us.ravel().copy()), 0)
        dist.send(torch.from_numpy(vs.ravel().copy()), 0)
    dist.barrier()
    dist.destroy_process_group()


def test_row_strips_with_halo_exchange_equal_unsplit(tmp_path):
    out = str(tmp_path / "strips.npz")
    mp.start_processes(_strip_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    orc, phi, u, v = _initial()
    ref = orc.run(phi, u, v, STEPS)
    got = np.load(out)
    assert np.array_equal(got["u"], ref["u"]) and np.array_equal(got["v"], ref["v"])


def _kblock_strip_worker(rank, world, port, out_path, K):
    """Temporally blocked strips: every K steps each rank exchanges K rows of
    u and v with each neighbour and steps its strip, extended by those halo
    rows, K times; the halo's cut edge corrupts one row per step, so after K
    steps exactly the owned rows are still exact (ghost-zone recompute)."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    orc, phi, u, v = _initial()
    bounds = np.linspace(0, H, world + 1).astype(int)
    r0, r1 = bounds[rank], bounds[rank + 1]
    up, dn = rank > 0, rank < world - 1
    us, vs = u[r0:r1].copy(), v[r0:r1].copy()
    e0, e1 = (r0 - K if up else r0), (r1 + K if dn else r1)
    ph = phi[e0:e1]
    assert STEPS % K == 0
    for _ in range(STEPS // K):
        got = {}
        reqs = []
        for name, nb, rows in (("top", rank - 1, slice(0, K)), ("bot", rank + 1, slice(-K, None))):
            if (name == "top" and not up) or (name == "bot" and not dn):
                continue
            for arr, key in ((us, "u"), (vs, "v")):
                reqs.append(dist.isend(torch.from_numpy(arr[rows].ravel().copy()), nb))
                buf = torch.empty(K * W, dtype=torch.float64)
                reqs.append(dist.irecv(buf, nb))
                got[(name, key)] = buf
        for q in reqs:
            q.wait()
        def ext(a, key):
            parts = ([got[("top", key)].numpy().reshape(K, W)] if up else []) + [a] + \
                    ([got[("bot", key)].numpy().reshape(K, W)] if dn else [])
            return np.ascontiguousarray(np.concatenate(parts))
        out = orc.run(np.ascontiguousarray(ph), ext(us, "u"), ext(vs, "v"), K)
        a = K if up else 0
        us = out["u"][a:a + (r1 - r0)].copy()
        vs = out["v"][a:a + (r1 - r0)].copy()
    if rank == 0:
        parts_u, parts_v = [us], [vs]
        for src in range(1, world):
            n = (bounds[src + 1] - bounds[src]) * W
            tu = torch.empty(n, dtype=torch.float64)
            tv = torch.empty(n, dtype=torch.float64)
            dist.recv(tu, src)
            dist.recv(tv, src)
            parts_u.append(tu.numpy().reshape(-1, W))
            parts_v.append(tv.numpy().reshape(-1, W))
        np.savez(out_path, u=np.concatenate(parts_u), v=np.concatenate(parts_v))
    else:
        dist.send(torch.from_numpy(us.ravel().copy()), 0)
        dist.send(torch.from_numpy(vs.ravel().copy()), 0)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("K", [4, 6])
def test_kblocked_strips_equal_unsplit(tmp_path, K):
    """K rows of u and v every K steps suffice (the temporally blocked form of
    the strip exchange); the result equals the unsplit oracle bit for bit."""
    out = str(tmp_path / f"kstrips{K}.npz")
    mp.start_processes(_kblock_strip_worker, args=(2, _free_port(), out, K), nprocs=2,
                       join=True, start_method="spawn")
    orc, phi, u, v = _initial()
    ref = orc.run(phi, u, v, STEPS)
    got = np.load(out)
    assert np.array_equal(got["u"], ref["u"]) and np.array_equal(got["v"], ref["v"])


def _plan_worker(rank, world, port, out_path, halo, steps):
    """One strip per rank, exchanged as strip_plan's copies say: a copy whose
    sender is this rank is a send, one whose receiver is this rank a receive."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1901_06535_gb300.strips import strip_plan
    orc, phi, u, v = _initial()
    strips, transfers = strip_plan(H, world, halo)
    me = strips[rank]
    us, vs = u[me.e0:me.e1].copy(), v[me.e0:me.e1].copy()
    ph = np.ascontiguousarray(phi[me.e0:me.e1])
    left = steps
    while left > 0:
        m = min(left, halo)
        reqs, recvd = [], []
        for t in transfers:
            if t.src == rank:
                for a in (us, vs):
                    reqs.append(dist.isend(torch.from_numpy(
                        a[t.src_row:t.src_row + t.nrows].ravel().copy()), t.dst))
            if t.dst == rank:
                bufs = [torch.empty(t.nrows * W, dtype=torch.float64) for _ in range(2)]
                for b in bufs:
                    reqs.append(dist.irecv(b, t.src))
                recvd.append((t, bufs))
        for q in reqs:
            q.wait()
        for t, (bu, bv) in recvd:
            us[t.dst_row:t.dst_row + t.nrows] = bu.numpy().reshape(t.nrows, W)
            vs[t.dst_row:t.dst_row + t.nrows] = bv.numpy().reshape(t.nrows, W)
        out = orc.run(ph, us, vs, m)
        us, vs = out["u"], out["v"]
        left -= m
    own_u = np.ascontiguousarray(us[me.r0 - me.e0:me.r1 - me.e0])
    own_v = np.ascontiguousarray(vs[me.r0 - me.e0:me.r1 - me.e0])
    if rank == 0:
        parts_u, parts_v = [own_u], [own_v]
        for src in range(1, world):
            n = (strips[src].r1 - strips[src].r0) * W
            tu = torch.empty(n, dtype=torch.float64)
            tv = torch.empty(n, dtype=torch.float64)
            dist.recv(tu, src)
            dist.recv(tv, src)
            parts_u.append(tu.numpy().reshape(-1, W))
            parts_v.append(tv.numpy().reshape(-1, W))
        np.savez(out_path, u=np.concatenate(parts_u), v=np.concatenate(parts_v))
    else:
        dist.send(torch.from_numpy(own_u.ravel().copy()), 0)
        dist.send(torch.from_numpy(own_v.ravel().copy()), 0)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("halo,steps", [(3, 47), (5, 60)])
def test_strip_plan_on_three_ranks_equals_unsplit(tmp_path, halo, steps):
    out = str(tmp_path / f"plan{halo}.npz")
    mp.start_processes(_plan_worker, args=(3, _free_port(), out, halo, steps), nprocs=3,
                       join=True, start_method="spawn")
    orc, phi, u, v = _initial()
    ref = orc.run(phi, u, v, steps)
    got = np.load(out)
    assert np.array_equal(got["u"], ref["u"]) and np.array_equal(got["v"], ref["v"])


def _agg_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = [2.0, 3.0][rank]
    t_max = bench.max_over_ranks(t, world)
    val = bench.weak_scaling_value(1e9, world, t_max)
    if rank == 0:
        np.save(out_path, np.array([t_max, val]))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_rank_aggregation(tmp_path):
    out = str(tmp_path / "agg.npy")
    mp.start_processes(_agg_worker, args=(2, _free_port(), out), nprocs=2, join=True,
                       start_method="spawn")
    t_max, val = np.load(out)
    assert t_max == 3.0
    assert val == pytest.approx(2 * 1e9 / 3.0 / 1e9)
