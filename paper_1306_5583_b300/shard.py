"""A particle filter or the mixture sampler partitioned over ranks: one
shard per GPU, the weight set normalised across ranks and resampling global
(the paper's MPI module, Sec. 3.1, and its distributed weights; Sec. 5.2.5
runs the GMM sampler that way).  The mixture sampler's iteration adds its
moves after the exchange and one more gather of partials for the
path-sampling integrand and the acceptance rates.

A filter of N particles is split in blocks: rank r holds the particles
[off_r, off_r + n_r) under their global Philox indices, so each particle
evolves exactly as in a single context of N particles.  One iteration:

1. every shard moves and weighs its particles and reduces them to one
   partial (``smc_shard_move``);
2. an all-gather of the partials in rank order, which every rank combines
   and finalises identically (``smc_shard_finalize``): global normaliser,
   ESS, evidence increment, means and resampling decision;
3. when the ESS test asks: an all-gather of the shards' exact fixed-point
   totals; each rank selects the global outputs of its own particles on the
   global CDF (``smc_shard_select``), whose range [k_lo, k_hi) is gathered;
4. the copies travel to the ranks that own their output slots: each rank
   sends the part of its output range that falls in rank d's slot block to
   rank d (``plan_exchange``), packed in output order (``smc_shard_pack``);
   an all-to-all; the received copies, in output order, are the rank's new
   particles (``smc_shard_unpack``).

The fixed-point CDF makes the global selection exact and order-independent,
so the sharded filter's ancestors are those of one context of N particles.

Independent filters (the batched form) need no exchange: ``assign_filters``
packs them over ranks by cost N_b T_b, each rank runs its share as one
batch on the filters' own Philox streams, and ``run_batch_over_ranks``
gathers the log-evidence estimates at the end.

Every data-parallel step runs in the library's kernels; this module only
plans the exchange and calls the collectives.  ``Collectives`` wraps
torch.distributed (NCCL between GPUs, gloo on CPU); ``run_local`` drives
several shards of one process in lockstep with copies in place of the
collectives.
"""
import ctypes

import numpy as np

from . import smc

PARTIAL_BYTES = 64


def partition(n_global, world):
    """Block partition of n_global particles: (offsets, sizes), rank order."""
    base, extra = divmod(int(n_global), int(world))
    sizes = [base + (1 if r < extra else 0) for r in range(world)]
    offs = [0] * world
    for r in range(1, world):
        offs[r] = offs[r - 1] + sizes[r - 1]
    return offs, sizes


def plan_exchange(ranges, offs, sizes, me):
    """Send and receive counts of rank `me` (copies, not bytes).

    ranges[r] = [k_lo, k_hi): the global outputs whose parents rank r holds;
    they are consecutive and cover [0, N) in rank order.  Rank `me` sends to
    rank d the outputs of its range inside d's slot block [off_d, off_d +
    n_d), and receives from rank s the outputs of s's range inside its own
    block; in both directions the outputs stay in increasing order, so the
    received copies, concatenated in rank order, fill the rank's slots in
    order."""
    world = len(offs)
    n = offs[-1] + sizes[-1]
    lo = [int(r[0]) for r in ranges]
    hi = [int(r[1]) for r in ranges]
    if lo[0] != 0 or hi[-1] != n or any(hi[r] != lo[r + 1] for r in range(world - 1)):
        raise ValueError(f"output ranges {list(zip(lo, hi))} do not partition [0, {n}) in rank order")

    def overlap(a0, a1, b0, b1):
        return max(0, min(a1, b1) - max(a0, b0))

    send = [overlap(lo[me], hi[me], offs[d], offs[d] + sizes[d]) for d in range(world)]
    recv = [overlap(lo[s], hi[s], offs[me], offs[me] + sizes[me]) for s in range(world)]
    assert sum(send) == hi[me] - lo[me] and sum(recv) == sizes[me]
    return send, recv


class Collectives:
    """The collectives of the exchange over a torch.distributed process
    group (NCCL for device tensors, gloo for host tensors)."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)

    def all_gather(self, t):
        """Every rank's t, concatenated in rank order."""
        import torch
        parts = [torch.empty_like(t) for _ in range(self.world)]
        self.dist.all_gather(parts, t, group=self.group)
        return torch.cat(parts)

    def all_gather_object(self, obj):
        """Every rank's picklable obj, in rank order."""
        out = [None] * self.world
        self.dist.all_gather_object(out, obj, group=self.group)
        return out

    def all_to_all(self, send, send_counts, recv_counts, width):
        """Rank-order all-to-all of rows of `width` values."""
        import torch
        recv = torch.empty(sum(recv_counts) * width, dtype=send.dtype, device=send.device)
        self.dist.all_to_all_single(recv, send, [c * width for c in recv_counts], [c * width for c in send_counts],
                                    group=self.group)
        return recv


class Shard:
    """One rank's shard of a filter of `n_global` particles (the device
    steps of one iteration, in the order ``step`` calls them)."""

    def __init__(self, config, n_global, rank, world, stream=None, device=None):
        import copy
        import torch
        self.torch = torch
        self.rank, self.world = int(rank), int(world)
        self.n_global = int(n_global)
        offs, sizes = partition(self.n_global, self.world)
        self.offs, self.sizes = offs, sizes
        cfg = copy.copy(config)
        cfg.n_particles = sizes[self.rank]
        self.sampler = smc.Sampler(cfg, stream=stream, device=device)
        self.ctx = self.sampler.ctx
        smc.check(smc.lib().smc_shard_configure(self.ctx, self.n_global, offs[self.rank]), "smc_shard_configure")
        dev = self.sampler.device
        self.gmm = config.model == smc.MODEL_GMM
        self.width = self.sampler.dim  # state values per copy in the exchange
        self.rdtype = torch.float32 if config.precision == 32 else torch.float64
        self.partial = torch.zeros(PARTIAL_BYTES, dtype=torch.uint8, device=dev)
        self.total = torch.zeros(1, dtype=torch.int64, device=dev)
        self.range = torch.zeros(2, dtype=torch.int64, device=dev)
        self.src = torch.zeros(self.n_global, dtype=torch.int32, device=dev)

    @staticmethod
    def _p(t):
        return ctypes.c_void_p(t.data_ptr())

    def set_data(self, obs):
        self.sampler.set_data(obs)

    def initialize(self):
        self.sampler.initialize()

    def move(self):
        smc.check(smc.lib().smc_shard_move(self.ctx, self._p(self.partial)), "smc_shard_move")
        return self.partial

    def finalize(self, partials):
        smc.check(smc.lib().smc_shard_finalize(self.ctx, self._p(partials), self.world), "smc_shard_finalize")
        return self.sampler.history(1)[0]

    def fixed_total(self):
        smc.check(smc.lib().smc_shard_total(self.ctx, self._p(self.total)), "smc_shard_total")
        return self.total

    def select(self, totals):
        smc.check(smc.lib().smc_shard_select(self.ctx, self._p(totals), self.rank, self.world, self._p(self.src),
                                             self._p(self.range)), "smc_shard_select")
        return self.range

    def pack(self, k_lo, count):
        send = self.torch.empty(max(count, 1) * self.width, dtype=self.rdtype, device=self.partial.device)
        smc.check(smc.lib().smc_shard_pack(self.ctx, self._p(self.src), int(k_lo), int(count), self._p(send)),
                  "smc_shard_pack")
        return send[:count * self.width]

    def unpack(self, recv):
        smc.check(smc.lib().smc_shard_unpack(self.ctx, self._p(recv)), "smc_shard_unpack")

    def mcmc(self):
        """The mixture sampler's moves of the shard's particles; its partial."""
        smc.check(smc.lib().smc_shard_mcmc(self.ctx, self._p(self.partial)), "smc_shard_mcmc")
        return self.partial

    def mcmc_finalize(self, partials):
        smc.check(smc.lib().smc_shard_mcmc_finalize(self.ctx, self._p(partials), self.world),
                  "smc_shard_mcmc_finalize")
        return self.sampler.history(1)[0]

    def state(self):
        return self.sampler.state()

    def close(self):
        self.sampler.close()


def step(shard, comm):
    """One iteration of a shard in a process group (every rank calls it).
    Returns the iteration's record (the same on every rank)."""
    parts = comm.all_gather(shard.move())
    rec = shard.finalize(parts)
    if rec["resampled"]:
        totals = comm.all_gather(shard.fixed_total())
        ranges = comm.all_gather(shard.select(totals)).view(-1, 2).cpu().numpy()
        send_counts, recv_counts = plan_exchange(ranges, shard.offs, shard.sizes, shard.rank)
        k_lo = int(ranges[shard.rank][0])
        send = shard.pack(k_lo, int(ranges[shard.rank][1]) - k_lo)
        shard.unpack(comm.all_to_all(send, send_counts, recv_counts, shard.width))
    if shard.gmm and rec["t"] >= 1:  # the mixture sampler's moves, then its path-sampling record
        rec = shard.mcmc_finalize(comm.all_gather(shard.mcmc()))
    return rec


def run_local(shards, steps):
    """Several shards of one filter in one process, advanced in lockstep
    with copies in place of the collectives (the same plan and the same
    order of data as ``step``).  Returns the records of rank 0."""
    import torch
    world = len(shards)
    recs = []
    for _ in range(steps):
        parts = torch.cat([s.move().clone() for s in shards])
        rr = [s.finalize(parts) for s in shards]
        if rr[0]["resampled"]:
            totals = torch.cat([s.fixed_total().clone() for s in shards])
            ranges = torch.cat([s.select(totals).clone() for s in shards]).view(-1, 2).cpu().numpy()
            sends = []
            for s in shards:
                k_lo = int(ranges[s.rank][0])
                sends.append((s.pack(k_lo, int(ranges[s.rank][1]) - k_lo), plan_exchange(ranges, s.offs, s.sizes,
                                                                                        s.rank)[0]))
            for me, s in enumerate(shards):
                _, recv_counts = plan_exchange(ranges, s.offs, s.sizes, me)
                pieces = []
                w = s.width
                for src in range(world):
                    send, counts = sends[src]
                    start = sum(counts[:me]) * w
                    pieces.append(send[start:start + counts[me] * w])
                s.unpack(torch.cat(pieces))
        if shards[0].gmm and rr[0]["t"] >= 1:
            parts = torch.cat([s.mcmc().clone() for s in shards])
            rr = [s.mcmc_finalize(parts) for s in shards]
        recs.append(rr[0])
    return recs


# ---- independent filters of a batch spread over ranks ------------------------

def assign_filters(cost, world):
    """The filters of a batch split over `world` ranks by cost (N_b T_b
    particle-updates): in decreasing cost (ties by index) each filter goes
    to the rank with the smallest load so far (ties to the lower rank), the
    greedy longest-processing-time packing, whose largest load is within
    4/3 of the best possible.  Returns, per rank, its filters in increasing
    index order."""
    cost = [int(c) for c in cost]
    if world < 1 or any(c < 0 for c in cost):
        raise ValueError("assign_filters: world >= 1 and costs >= 0")
    load = [0] * world
    mine = [[] for _ in range(world)]
    for b in sorted(range(len(cost)), key=lambda i: (-cost[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += cost[b]
        mine[r].append(b)
    return [sorted(m) for m in mine]


def gpu_batch_runner(config, n, T, obs, streams, stream=None, device=None):
    """One rank's filters as one batch on its GPU (smc.Batch), each with its
    own Philox stream; returns their log-evidence estimates."""
    b = smc.Batch(config, n, T, stream=stream, device=device)
    try:
        b.set_streams(streams)
        for f, y in enumerate(obs):
            b.set_data(f, y)
        b.run()
        return [float(v) for v in b.log_evidence()]
    finally:
        b.close()


def run_batch_over_ranks(config, n, T, obs, comm, runner=gpu_batch_runner, **runner_kw):
    """Independent filters spread over ranks (no collective on the data
    path): rank `comm.rank` runs the filters `assign_filters` gives it, each
    on the Philox stream config.stream_id + its index in the whole batch, so
    every filter computes what it computes in one batch of all of them; one
    gather of (index, log-evidence) pairs at the end.  Returns every
    filter's log-evidence in filter order on every rank."""
    mine = assign_filters([int(a) * int(b) for a, b in zip(n, T)], comm.world)[comm.rank]
    res = {}
    if mine:
        vals = runner(config, [int(n[b]) for b in mine], [int(T[b]) for b in mine], [obs[b] for b in mine],
                      [(int(config.stream_id) + b) & 0xFFFFFFFF for b in mine], **runner_kw)
        res = dict(zip(mine, vals))
    out = np.full(len(n), np.nan)
    for part in comm.all_gather_object(res):
        for b, v in part.items():
            out[b] = v
    return out
