"""The sharded filter's host side (the exchange plan, the collectives and
the order of the data) on CPU ranks: two gloo processes run
``shard.step`` over a stand-in for the device steps built from the oracle's
functions (per-rank inputs made here), and the whole particle system and
the records equal those of the single-process oracle filter.  The device
steps themselves are checked against a single context on the GPU
(tests/test_gpu_shard.py)."""
import math
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import cv as ocv
from oracle import philox, resample as ores, weights as ow
from paper_1306_5583_b300 import shard, workloads

SEED = 7


class OracleShard:
    """The device steps of one rank's shard, written with the oracle's
    functions in float64 (CPU tensors for the gloo collectives)."""

    def __init__(self, n_global, rank, world, y, threshold):
        self.n_global, self.rank, self.world = n_global, rank, world
        self.gmm, self.width = False, 4  # a particle filter: four state values per copy
        self.offs, self.sizes = shard.partition(n_global, world)
        self.n = self.sizes[rank]
        self.idx = np.arange(self.offs[rank], self.offs[rank] + self.n)
        self.y, self.thr = y, threshold
        self.p = ocv.CVParams(**workloads.CV_DEFAULT)
        self.t = -1
        self.x = None
        self.base = np.full(self.n, -math.log(n_global))
        self.logz = 0.0

    def move(self):
        self.t += 1
        t = self.t
        if t == 0:
            self.x = ocv.init_state(self.n, SEED, self.p, index=self.idx)
        else:
            self.x = ocv.move(self.x, t, SEED, self.p, index=self.idx)
        self.lw = self.base + ocv.loglik(self.x, self.y[t], self.p)
        m = float(np.max(self.lw))
        e = np.exp(self.lw - m)
        v = np.array([m, e.sum(), (e * e).sum(), (e * self.x[0]).sum(), (e * self.x[1]).sum(), 0, 0, 0])
        return torch.from_numpy(v.view(np.uint8).copy())

    def finalize(self, parts):
        P = parts.numpy().view(np.float64).reshape(-1, 8)
        M = float(P[:, 0].max())
        sc = np.exp(P[:, 0] - M)
        S1, S2 = float(np.sum(P[:, 1] * sc)), float(np.sum(P[:, 2] * sc * sc))
        L = M + math.log(S1)
        ess = S1 * S1 / S2
        self.M, self.L = M, L
        self.logz += L
        due = ow.resample_decision(ess, self.n_global, self.thr)
        self.base = self.lw - L
        return dict(t=self.t, L=L, logZ=self.logz, ess=ess, resampled=due,
                    mean_x=float(np.sum(P[:, 3] * sc)) / S1, mean_y=float(np.sum(P[:, 4] * sc)) / S1)

    def fixed_total(self):
        F = ores.frac_bits(self.n_global)
        self.q = [int(math.floor(v * 2.0 ** F)) for v in np.exp(self.lw - self.M)]
        return torch.tensor([sum(self.q)], dtype=torch.int64)

    def select(self, totals):
        tot = [int(v) for v in totals.numpy()]
        qb, qn = sum(tot[:self.rank]), sum(tot)
        P, D = ores.systematic_targets(self.n_global, philox.systematic_u24(SEED, self.t))
        Q = [qb + int(v) for v in ores.cdf(self.q)]
        self.src = np.full(self.n_global, -1, dtype=np.int64)
        import bisect
        k_lo, k_hi = None, None
        for k, pk in enumerate(P):
            tau = (qn * pk) // D
            if qb <= tau < Q[-1]:
                self.src[k] = bisect.bisect_right(Q, tau)
                k_lo = k if k_lo is None else k_lo
                k_hi = k + 1
        if k_lo is None:  # no output of this rank: an empty range at its place in the order
            k_lo = k_hi = sum(1 for pk in P if (qn * pk) // D < qb)
        if self.rank == self.world - 1:
            k_hi = self.n_global
        return torch.tensor([k_lo, k_hi], dtype=torch.int64)

    def pack(self, k_lo, count):
        s = self.src[k_lo:k_lo + count]
        return torch.from_numpy(np.ascontiguousarray(self.x[:, s].T).reshape(-1))

    def unpack(self, recv):
        self.x = recv.numpy().reshape(self.n, 4).T.copy()
        self.base = np.full(self.n, -math.log(self.n_global))


def _worker(rank, world, port, n_global, T, threshold, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _, y = workloads.cv_data(T, seed=0, **workloads.CV_DEFAULT)
        sh = OracleShard(n_global, rank, world, y, threshold)
        comm = shard.Collectives()
        recs = [shard.step(sh, comm) for _ in range(T - 1)]
        # the last iteration up to its weighting (the oracle run's final state)
        recs.append(sh.finalize(comm.all_gather(sh.move())))
        m = max(sh.sizes)  # all_gather wants equal sizes: pad, then trim
        x = torch.zeros(4, m, dtype=torch.float64)
        x[:, :sh.n] = torch.from_numpy(sh.x)
        xs = [torch.empty(4, m, dtype=torch.float64) for _ in sh.sizes]
        dist.all_gather(xs, x)
        if rank == 0:
            out.put((recs, torch.cat([v[:, :sz] for v, sz in zip(xs, sh.sizes)], dim=1).numpy()))
    except Exception as e:  # reported to the test instead of a silent hang
        out.put(repr(e))
        raise
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_plan_exchange_counts_and_refusals():
    offs, sizes = shard.partition(10, 3)
    assert offs == [0, 4, 7] and sizes == [4, 3, 3]
    ranges = [(0, 2), (2, 9), (9, 10)]
    plans = [shard.plan_exchange(ranges, offs, sizes, me) for me in range(3)]
    assert plans[0] == ([2, 0, 0], [2, 2, 0])
    assert plans[1] == ([2, 3, 2], [0, 3, 0])
    assert plans[2] == ([0, 0, 1], [0, 2, 1])
    # sends and receives agree pairwise
    for a in range(3):
        for b in range(3):
            assert plans[a][0][b] == plans[b][1][a]
    with pytest.raises(ValueError):
        shard.plan_exchange([(0, 2), (3, 9), (9, 10)], offs, sizes, 0)


@pytest.mark.parametrize("n_global,threshold", [(37, 1.0), (64, 0.6)])
def test_two_gloo_ranks_equal_the_single_process_filter(n_global, threshold):
    T = 9
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, n_global, T, threshold, q)) for r in range(2)]
    for p in procs:
        p.start()
    import queue
    res = None
    for _ in range(240):
        try:
            res = q.get(timeout=1)
            break
        except queue.Empty:
            if any(p.exitcode not in (None, 0) for p in procs):
                break
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert isinstance(res, tuple), res
    assert all(p.exitcode == 0 for p in procs)
    recs, x = res
    _, y = workloads.cv_data(T, seed=0, **workloads.CV_DEFAULT)
    ref, last = ocv.run(y, n_global, SEED, ocv.CVParams(**workloads.CV_DEFAULT), scheme="systematic",
                        threshold=threshold)
    assert any(r["resampled"] for r in ref)
    for r, o in zip(recs, ref):
        assert r["resampled"] == o["resampled"]
        assert abs(r["L"] - o["L"]) < 1e-12 and abs(r["logZ"] - o["logZ"]) < 1e-11
        assert abs(r["mean_x"] - o["mean_x"]) < 1e-12
    if threshold >= 1.0:
        assert np.array_equal(x, last.x)  # bit for bit: every step resampled, ancestors exact
    else:
        assert np.max(np.abs(x - last.x)) < 1e-10


# ---- independent filters of a batch spread over ranks ------------------------

def test_assign_filters_packs_by_cost():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        cost = [int(v) for v in rng.integers(1, 10_000, size=37)]
        parts = shard.assign_filters(cost, world)
        assert sorted(b for p in parts for b in p) == list(range(37))  # every filter once
        assert all(p == sorted(p) for p in parts)
        loads = [sum(cost[b] for b in p) for p in parts]
        bound = max(max(cost), sum(cost) / world)  # no packing does better than this
        assert max(loads) <= 4 / 3 * bound + 1e-9
    assert shard.assign_filters([1, 1, 1], 4) == [[0], [1], [2], []]
    assert shard.assign_filters([5, 3, 3, 2, 2, 1], 2) == [[0, 3, 5], [1, 2, 4]]
    with pytest.raises(ValueError):
        shard.assign_filters([1, -1], 2)


def _oracle_batch_runner(config, n, T, obs, streams):
    """Stand-in for one rank's batch: each filter as the oracle's run on its
    own Philox stream (the GPU batch is checked against plain runs and the
    oracle in tests/test_gpu_batch.py)."""
    p = ocv.CVParams(**workloads.CV_DEFAULT)
    return [ocv.run(y, nb, int(config.seed), p, scheme="systematic", threshold=0.5, stream=s)[0][-1]["logZ"]
            for nb, y, s in zip(n, obs, streams)]


BATCH_N = [40, 7, 64, 3, 25, 16, 1]
BATCH_T = [6, 9, 4, 8, 5, 7, 3]


def _batch_data():
    return [workloads.cv_data(t, seed=1 + b, **workloads.CV_DEFAULT)[1] for b, t in enumerate(BATCH_T)]


def _batch_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_1306_5583_b300 import smc
        cfg = smc.make_config(model="cv", n=1, precision=64, seed=SEED, stream_id=11)
        lz = shard.run_batch_over_ranks(cfg, BATCH_N, BATCH_T, _batch_data(), shard.Collectives(),
                                        runner=_oracle_batch_runner)
        out.put((rank, lz.tolist()))
    except Exception as e:
        out.put(repr(e))
        raise
    finally:
        dist.destroy_process_group()


def test_batch_over_two_gloo_ranks_equals_one_rank():
    """Two ranks, each running its share of the filters on their own Philox
    streams, gather the same log-evidence as one rank running them all."""
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_batch_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    import queue
    got = []
    for _ in range(240):
        try:
            got.append(q.get(timeout=1))
            if len(got) == 2:
                break
        except queue.Empty:
            if any(p.exitcode not in (None, 0) for p in procs):
                break
    for p in procs:
        p.join(timeout=60)
        if p.is_alive():
            p.kill()
    assert len(got) == 2 and all(isinstance(g, tuple) for g in got), got
    assert all(p.exitcode == 0 for p in procs)
    from paper_1306_5583_b300 import smc
    cfg = smc.make_config(model="cv", n=1, precision=64, seed=SEED, stream_id=11)
    ref = _oracle_batch_runner(cfg, BATCH_N, BATCH_T, _batch_data(), [11 + b for b in range(len(BATCH_N))])
    for _, lz in got:
        assert lz == ref  # bit for bit: the same arithmetic on the same streams
