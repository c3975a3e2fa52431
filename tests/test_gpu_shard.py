"""GPU: the device steps of the sharded filter (smc_shard_*).  Two or three
shards of one filter in one process, advanced in lockstep with copies in
place of the collectives (shard.run_local), against one context of the
whole filter: when every step resamples the particle systems are
identical bit for bit (the same Philox streams by global index, the same
exact fixed-point selection), and the records agree to the rounding of the
normaliser's summation order; with the ESS threshold they also match the
FP64 oracle."""
import numpy as np
import pytest

from gpu_common import need_gpu, oracle_params, torch
from oracle import cv as ocv
from paper_1306_5583_b300 import shard, smc, workloads

pytestmark = pytest.mark.gpu


def _single(n, T, precision, scheme, threshold, seed, y):
    cfg = smc.make_config(model="cv", n=n, precision=precision, scheme=scheme, threshold=threshold, seed=seed,
                          max_data=T, keep_cdf=False)
    s = smc.Sampler(cfg)
    s.set_data(y)
    s.initialize()
    return s


def _shards(n, world, T, precision, scheme, threshold, seed, y):
    cfg = smc.make_config(model="cv", n=n, precision=precision, scheme=scheme, threshold=threshold, seed=seed,
                          max_data=T, keep_cdf=False)
    out = []
    for r in range(world):
        sh = shard.Shard(cfg, n, r, world)
        sh.set_data(y)
        sh.initialize()
        out.append(sh)
    return out


@pytest.mark.parametrize("precision,scheme,n,world",
                         [(p, sc, n, w) for p in (32, 64) for sc in ("systematic", "stratified")
                          for n, w in ((5000, 2), (70001, 3))] + [(32, "systematic", (1 << 20) + 5, 2)])
def test_shards_equal_one_context_when_every_step_resamples(precision, scheme, n, world):
    """Shards in one process against one context; the last case is the
    benchmarked size (two shards of about 2^19 particles, ragged)."""
    need_gpu()
    T, seed = 8, 5
    _, y = workloads.cv_data(T, seed=1, **workloads.CV_DEFAULT)
    one = _single(n, T, precision, scheme, 1.0, seed, y)
    shs = _shards(n, world, T, precision, scheme, 1.0, seed, y)
    # after each step the shards hold the resampled copies (the exchange
    # materialises them); the single context holds the weighted particles
    # and the ancestors its next move gathers by
    def resampled(s):
        return s.state()[:, s.ancestors().astype(np.int64)]

    recs = shard.run_local(shs, 1)  # t = 0
    assert np.array_equal(np.concatenate([s.state() for s in shs], axis=1), resampled(one))
    for t in range(1, T):
        one.iterate(1)
        recs += shard.run_local(shs, 1)
        x = np.concatenate([s.state() for s in shs], axis=1)
        assert np.array_equal(x, resampled(one)), t
    ref = one.history(T)
    tol = 1e-5 if precision == 32 else 1e-11
    for r, o in zip(recs, ref):
        assert r["t"] == o["t"] and r["resampled"] and o["resampled"]
        assert r["max_lw"] == o["max_lw"]
        assert abs(r["L"] - o["L"]) < tol and abs(r["logZ"] - o["logZ"]) < tol * T
    for s in shs:
        s.close()
    one.close()


def test_fp64_shards_with_the_ess_test_match_the_oracle():
    need_gpu()
    n, T, seed, thr = 3001, 30, 2, 0.5
    _, y = workloads.cv_data(T, seed=0, **workloads.CV_DEFAULT)
    shs = _shards(n, 2, T, 64, "systematic", thr, seed, y)
    recs = shard.run_local(shs, T)
    ref, last = ocv.run(y, n, seed, oracle_params(dict(workloads.CV_DEFAULT)), scheme="systematic", threshold=thr)
    assert any(o["resampled"] for o in ref) and not all(o["resampled"] for o in ref)
    for r, o in zip(recs, ref):
        assert r["resampled"] == o["resampled"], r["t"]
        assert abs(r["L"] - o["L"]) < 1e-9 and abs(r["logZ"] - o["logZ"]) < 1e-9
        assert abs(r["mean_x"] - o["mean_x"]) < 1e-9
    for s in shs:
        s.close()


def test_shard_refusals():
    need_gpu()
    cfg = smc.make_config(model="cv", n=100, precision=32, scheme="multinomial", max_data=4)
    s = smc.Sampler(cfg)
    assert smc.lib().smc_shard_configure(s.ctx, 200, 0) == smc.E_ARG   # scheme
    cfg = smc.make_config(model="cv", n=100, precision=32, scheme="systematic", max_data=4)
    s = smc.Sampler(cfg)
    assert smc.lib().smc_shard_configure(s.ctx, 150, 60) == smc.E_ARG  # past the filter
    assert smc.lib().smc_shard_configure(s.ctx, 200, 100) == smc.OK
    s.set_data(np.zeros((4, 2)))
    s.initialize()
    with pytest.raises(smc.SMCError):
        s.iterate(1)  # a shard moves only through the exchange


def _gmm_cfg(n, T, precision, move, threshold, nd):
    mv = {"rw": smc.GMM_RW, "mala": smc.GMM_MALA}[move]
    return smc.make_config(model="gmm", n=n, precision=precision, scheme="systematic", threshold=threshold, seed=3,
                           max_data=nd, max_records=T + 1, keep_cdf=False,
                           gmm=dict(n_comp=2, n_iter=T, move=mv, mala_step=0.05, schedule=smc.ALPHA_PRIOR))


@pytest.mark.parametrize("precision", [32, 64])
@pytest.mark.parametrize("move", ["rw", "mala"])
@pytest.mark.parametrize("n,world", [(3001, 2), (4096, 3)])
def test_gmm_shards_equal_one_context(precision, move, n, world):
    """The mixture sampler partitioned over shards (reweight, global
    resampling and exchange, the moves, the path-sampling gather) against
    one sampler: identical particles after every iteration when every step
    resamples; the records (normaliser, evidence, path sampling, acceptance)
    to the rounding of the sums' order."""
    need_gpu()
    T, nd = 7, 200
    y = workloads.gmm_data(nd, seed=0)
    one = smc.Sampler(_gmm_cfg(n, T, precision, move, 1.0, nd))
    one.set_data(y)
    one.initialize()
    shs = []
    for r in range(world):
        sh = shard.Shard(_gmm_cfg(n, T, precision, move, 1.0, nd), n, r, world)
        sh.set_data(y)
        sh.initialize()
        shs.append(sh)
    recs = shard.run_local(shs, 1)  # t = 0: the prior draws
    assert np.array_equal(np.concatenate([s.state() for s in shs], axis=1), one.state())
    for t in range(1, T):
        one.iterate(1)
        recs += shard.run_local(shs, 1)
        assert np.array_equal(np.concatenate([s.state() for s in shs], axis=1), one.state()), t
    ref = one.history(T)
    tol = 1e-5 if precision == 32 else 1e-10
    for r, o in zip(recs, ref):
        assert r["t"] == o["t"] and r["resampled"] == o["resampled"]
        for k in ("L", "logZ", "path_u", "path_log_z"):
            assert abs(r[k] - o[k]) <= tol * max(1.0, abs(o[k])), (r["t"], k, r[k], o[k])
        assert r["accept"] == o["accept"] and r["accept_mala"] == o["accept_mala"]
    for s in shs:
        s.close()
    one.close()


def test_gmm_shard_refuses_an_adaptive_schedule():
    need_gpu()
    cfg = _gmm_cfg(1000, 5, 32, "rw", 0.5, 50)
    cfg.gmm.schedule = smc.ALPHA_ADAPTIVE
    with pytest.raises(smc.SMCError) as e:
        shard.Shard(cfg, 2000, 0, 2)
    assert e.value.code == smc.E_ARG


def test_gmm_fp64_shards_with_the_ess_test_equal_one_context():
    """With the ESS test (some steps resample, some not): the same decisions,
    particles and records as one sampler."""
    need_gpu()
    n, T, nd = 5000, 12, 200
    y = workloads.gmm_data(nd, seed=0)
    one = smc.Sampler(_gmm_cfg(n, T, 64, "rw", 0.5, nd))
    one.set_data(y)
    one.initialize()
    one.iterate(T - 1)
    shs = []
    for r in range(2):
        sh = shard.Shard(_gmm_cfg(n, T, 64, "rw", 0.5, nd), n, r, 2)
        sh.set_data(y)
        sh.initialize()
        shs.append(sh)
    recs = shard.run_local(shs, T)
    ref = one.history(T)
    assert any(o["resampled"] for o in ref[1:]) and not all(o["resampled"] for o in ref[1:])
    for r, o in zip(recs, ref):
        assert r["resampled"] == o["resampled"]
        for k in ("L", "logZ", "ess", "path_log_z"):
            assert abs(r[k] - o[k]) <= 1e-9 * max(1.0, abs(o[k])), (r["t"], k, r[k], o[k])
    assert np.array_equal(np.concatenate([s.state() for s in shs], axis=1), one.state())
    for s in shs:
        s.close()
    one.close()
