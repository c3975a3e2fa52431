"""GPU: the batched form (many filters of uneven N and T in one launch per
kernel) gives every filter the plain path's results on the same Philox
stream: bit for bit in FP32; in FP64 the same decisions and particles and
records equal to 1e-13 relative (the two kernels inline the same float64
arithmetic, whose multiply-add fusion the compiler chooses per kernel); the
plain path is itself parity-tested against the oracle, and the FP64 batch
below as well."""
import numpy as np
import pytest

from gpu_common import need_gpu, torch
from paper_1306_5583_b300 import smc, workloads

pytestmark = pytest.mark.gpu

NS = [1000, 3000, 70000, 2049, 1, 64, 4096, 1 << 14]
TS = [12, 5, 9, 12, 3, 7, 1, 10]


def _data(T, seed):
    return workloads.cv_data(T, seed=seed, **workloads.CV_DEFAULT)[1]


@pytest.mark.parametrize("precision,scheme", [(32, "systematic"), (32, "stratified"), (64, "systematic")])
def test_batch_equals_plain_runs_bit_for_bit(precision, scheme):
    need_gpu()
    cfg = smc.make_config(model="cv", n=1, precision=precision, scheme=scheme, threshold=0.7, seed=4,
                          max_data=max(TS), keep_cdf=False)
    bt = smc.Batch(cfg, NS, TS)
    for b, T in enumerate(TS):
        bt.set_data(b, _data(T, 1 + b))
    bt.run()
    lz = bt.log_evidence()
    for b, (n, T) in enumerate(zip(NS, TS)):
        pc = smc.make_config(model="cv", n=n, precision=precision, scheme=scheme, threshold=0.7, seed=4,
                             stream_id=b, max_data=T, keep_cdf=False)
        s = smc.Sampler(pc)
        s.set_data(_data(T, 1 + b))
        s.initialize()
        s.iterate(T - 1)
        hp = s.history(T)
        hb = bt.history(b, T)
        assert len(hb) == T
        for rp, rb in zip(hp, hb):
            for k in ("t", "resampled"):
                assert rp[k] == rb[k], (b, rp["t"], k, rp[k], rb[k])
            for k in ("L", "logZ", "ess", "mean_x", "mean_y"):
                if precision == 32:
                    assert rp[k] == rb[k], (b, rp["t"], k, rp[k], rb[k])
                else:
                    assert abs(rp[k] - rb[k]) <= 1e-13 * max(1.0, abs(rp[k])), (b, rp["t"], k, rp[k], rb[k])
        assert np.array_equal(s.state(), bt.state(b))
        if precision == 32:
            assert lz[b] == s.log_evidence()
        else:
            assert abs(lz[b] - s.log_evidence()) <= 1e-13 * max(1.0, abs(lz[b]))
        s.close()


def test_batch_tune_and_iterate_in_pieces():
    need_gpu()
    cfg = smc.make_config(model="cv", n=1, precision=32, scheme="systematic", threshold=0.5, seed=7,
                          max_data=max(TS), keep_cdf=False)
    bt = smc.Batch(cfg, NS, TS)
    for b, T in enumerate(TS):
        bt.set_data(b, _data(T, 1 + b))
    g, c = bt.tune()
    assert g in (1, 2, 3, 4, 6, 8) and c in (1, 2, 4)
    bt.iterate(4)
    bt.iterate(max(TS) - 1 - 4)
    a = bt.log_evidence()
    bt.run()
    assert np.array_equal(a, bt.log_evidence())
    with pytest.raises(smc.SMCError):
        bt.iterate(1)   # past the longest filter


def test_batch_fp64_filters_match_the_oracle():
    """FP64 batch: a one-particle filter, a ragged one (N = 2049, one
    particle past a tile), one at the paper's N = 1000 and one of 2^14
    particles, each against the free-running oracle filter on the same
    Philox stream (stream id = filter index): records at the FP64
    tolerances of the plain path, identical resampling decisions, final
    particle system within 1e-10."""
    need_gpu()
    from gpu_common import assert_close, oracle_params
    from oracle import cv as ocv
    ns = [1, 2049, 1000, 1 << 14]
    ts = [6, 14, 20, 10]
    seed, thr = 21, 0.7
    p = dict(workloads.CV_DEFAULT)
    cfg = smc.make_config(model="cv", n=1, precision=64, scheme="systematic", threshold=thr, seed=seed,
                          max_data=max(ts), keep_cdf=False)
    bt = smc.Batch(cfg, ns, ts)
    data = [_data(T, 1 + b) for b, T in enumerate(ts)]
    for b in range(len(ns)):
        bt.set_data(b, data[b])
    bt.run()
    lz = bt.log_evidence()
    op = oracle_params(p)
    any_resampled = False
    for b, (n, T) in enumerate(zip(ns, ts)):
        ref, last = ocv.run(data[b], n, seed, op, scheme="systematic", threshold=thr, stream=b)
        hb = bt.history(b, T)
        assert len(hb) == T
        for r, o in zip(hb, ref):
            assert r["t"] == o["t"]
            assert r["resampled"] == o["resampled"], (b, r["t"])
            assert abs(r["L"] - o["L"]) < 1e-9, (b, r["t"])
            assert abs(r["logZ"] - o["logZ"]) < 1e-9, (b, r["t"])
            assert abs(r["ess"] - o["ess"]) < 1e-7 * n
            assert abs(r["mean_x"] - o["mean_x"]) < 1e-9 and abs(r["mean_y"] - o["mean_y"]) < 1e-9
            any_resampled |= bool(o["resampled"])
        assert_close(bt.state(b), last.x, 1e-10, f"final state of filter {b}")
        assert abs(lz[b] - ref[-1]["logZ"]) < 1e-9
    assert any_resampled


def test_batch_launch_shapes_give_identical_results():
    """Whatever launch shape the autotuner picks (blocks per SM, tiles per
    work item), every filter's results are the same bit for bit: two
    batches of the same filters, one tuned, one on the default shape."""
    need_gpu()
    cfg = smc.make_config(model="cv", n=1, precision=32, scheme="systematic", threshold=0.6, seed=9,
                          max_data=max(TS), keep_cdf=False)
    out = []
    for tune in (False, True):
        bt = smc.Batch(cfg, NS, TS)
        for b, T in enumerate(TS):
            bt.set_data(b, _data(T, 1 + b))
        if tune:
            bt.tune()
        bt.run()
        out.append((bt.log_evidence(), [bt.state(b) for b in range(len(NS))]))
        bt.close()
    assert np.array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        assert np.array_equal(a, b)


def test_batch_split_over_ranks_equals_one_batch():
    """The filters of a batch split as two ranks would run them
    (shard.assign_filters by cost N_b T_b, each subset one batch with the
    filters' own Philox streams via smc_batch_set_streams): every filter's
    log-evidence is bit-identical to the one-batch run."""
    need_gpu()
    from paper_1306_5583_b300 import shard
    cfg = smc.make_config(model="cv", n=1, precision=32, scheme="systematic", threshold=0.6, seed=5, stream_id=3,
                          max_data=max(TS), keep_cdf=False)
    data = [_data(T, 1 + b) for b, T in enumerate(TS)]
    whole = smc.Batch(cfg, NS, TS)
    for b, y in enumerate(data):
        whole.set_data(b, y)
    whole.run()
    ref = whole.log_evidence()
    whole.close()
    parts = shard.assign_filters([n * T for n, T in zip(NS, TS)], 2)
    assert all(parts)
    got = np.full(len(NS), np.nan)
    for mine in parts:
        vals = shard.gpu_batch_runner(cfg, [NS[b] for b in mine], [TS[b] for b in mine], [data[b] for b in mine],
                                      [3 + b for b in mine])
        got[mine] = vals
    assert np.array_equal(got, np.asarray(ref, dtype=np.float64))


def test_benchmarked_batch_equals_plain_runs():
    """The benchmarked batch: 256 filters, N log-uniform in [2^10, 2^18],
    T uniform in [50, 2000], FP32, systematic at ESS < N/2, launch shape
    from the autotuner.  Every filter's log-evidence equals its plain run's
    bit for bit; the records and final particles of the four smallest and
    four largest filters too."""
    need_gpu()
    ns, ts = workloads.batch_shapes(256, seed=0)
    p = dict(workloads.CV_DEFAULT)
    data = [workloads.cv_data(int(T), seed=1 + b, **p)[1] for b, T in enumerate(ts)]
    cfg = smc.make_config(model="cv", n=1, precision=32, scheme="systematic", threshold=0.5, seed=3,
                          max_data=int(ts.max()), keep_cdf=False, cv=p)
    bt = smc.Batch(cfg, ns, ts)
    for b in range(len(ns)):
        bt.set_data(b, data[b])
    bt.tune()
    bt.initialize()
    bt.run()
    lz = bt.log_evidence()
    order = np.argsort(ns)
    full = set(order[:4].tolist()) | set(order[-4:].tolist())
    for b in range(len(ns)):
        n, T = int(ns[b]), int(ts[b])
        pc = smc.make_config(model="cv", n=n, precision=32, scheme="systematic", threshold=0.5, seed=3,
                             stream_id=b, max_data=T, keep_cdf=False, cv=p)
        s = smc.Sampler(pc)
        s.set_data(data[b])
        s.initialize()
        if T > 1:
            s.iterate(T - 1)
        assert lz[b] == s.log_evidence(), (b, n, T)
        if b in full:
            hp, hb = s.history(T), bt.history(b, T)
            assert [(r["t"], r["resampled"], r["L"], r["ess"]) for r in hp] == \
                   [(r["t"], r["resampled"], r["L"], r["ess"]) for r in hb], b
            assert np.array_equal(s.state(), bt.state(b)), b
        s.close()
    bt.close()
