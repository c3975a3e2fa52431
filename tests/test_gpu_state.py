"""GPU tests of the state-changing calls of the boundary: WeightSet::
add_log_weight (Sec. 4.1.6), replacing the log-weights, and checkpoint /
resume (a restored sampler continues bit-identically)."""
import math

import numpy as np
import pytest

from gpu_common import assert_close, cv_params, make_pf, need_gpu, torch
from oracle import weights as ow
from paper_1306_5583_b300 import smc, workloads

pytestmark = pytest.mark.gpu


def _moved(precision, n=6000, T=12, threshold=0.3, seed=4, steps=4):
    """A filter after `steps` full iterations and one more move (no
    resampling pending)."""
    s, y, op = make_pf(n, T, precision, threshold=threshold, seed=seed)
    s.initialize()
    for _ in range(steps):
        s.move()
        s.resample()
    s.move()
    return s


@pytest.mark.parametrize("precision", [64, 32])
def test_add_log_weight_matches_oracle(precision):
    need_gpu()
    s = _moved(precision)
    rel = 1e-12 if precision == 64 else 1e-5
    lw = s.log_weight()
    x = s.state().astype(np.float64)
    before = s.history(2)
    rec0, prev = before[-1], before[-2]
    inc = (np.random.default_rng(1).standard_normal(s.n) * 0.7).astype(lw.dtype)
    s.add_log_weight(inc)
    lw2 = s.log_weight()
    assert np.array_equal(lw2, (lw + inc).astype(lw.dtype))
    rec = s.history(1)[0]
    assert rec["t"] == rec0["t"] and rec["status"] == 0
    m, L = ow.log_sum_exp(lw2.astype(np.float64))
    W = np.exp(lw2.astype(np.float64) - L)
    assert_close(rec["L"], L, rel, "L")
    assert_close(rec["ess"], 1.0 / np.sum(W * W), 10 * rel, "ESS")
    assert_close([rec["mean_x"], rec["mean_y"]], [np.sum(W * x[0]), np.sum(W * x[1])], 10 * rel, "means")
    # the evidence increment of iteration t is replaced, not added
    assert abs(rec["logZ"] - (prev["logZ"] + rec["L"])) < 1e-9
    assert rec["resampled"] == (rec["ess"] < 0.3 * s.n)
    s.resample()
    s.move()  # the filter carries on
    assert s.history(1)[0]["status"] == 0


def test_add_log_weight_after_queued_resampling_is_rejected():
    need_gpu()
    s, y, op = make_pf(2000, 8, 32, threshold=1.0, seed=1)
    s.initialize()  # t = 0 resampled (threshold 1): the gather is pending
    with pytest.raises(smc.SMCError) as e:
        s.add_log_weight(np.zeros(s.n, np.float32))
    assert e.value.code == smc.E_STATE


def test_write_log_weight_recomputes_the_normaliser():
    need_gpu()
    s = _moved(64)
    prev = s.history(2)[-2]
    lw = np.random.default_rng(2).standard_normal(s.n) * 2.0 - 5.0
    s.write_log_weight(lw)
    assert np.array_equal(s.log_weight(), lw)
    rec = s.history(1)[0]
    m, L = ow.log_sum_exp(lw)
    assert_close(rec["L"], L, 1e-12, "L")
    assert abs(rec["logZ"] - (prev["logZ"] + L)) < 1e-9


def _bits(v):
    """A record value in a form whose equality is bit equality (NaN too)."""
    if isinstance(v, float):
        return np.float64(v).tobytes()
    if isinstance(v, tuple):
        return tuple(_bits(u) for u in v)
    return v


def _snapshot(s, T):
    return (s.state(), s.log_weight(), s.ancestors(), s.log_evidence(),
            [tuple(sorted((k, _bits(v)) for k, v in r.items())) for r in s.history(T)])


@pytest.mark.parametrize("scheme,precision", [("systematic", 32), ("multinomial", 32), ("residual", 64)])
def test_checkpoint_resume_is_bit_identical_pf(scheme, precision):
    need_gpu()
    n, T, k1 = 20000, 30, 11
    p = cv_params()
    _, y = workloads.cv_data(T, seed=3, **p)
    mk = lambda: smc.Sampler(smc.make_config(model="cv", n=n, precision=precision, scheme=scheme, threshold=0.5,
                                             seed=7, max_data=T, max_records=T, cv=p))
    a = mk()
    a.set_data(y)
    a.initialize()
    a.iterate(k1)
    blob = a.checkpoint()
    a.iterate(T - 1 - k1)
    ref = _snapshot(a, T)
    b = mk()
    b.set_data(y)
    b.restore(blob)
    assert b.iteration() == k1
    b.iterate(T - 1 - k1)
    got = _snapshot(b, T)
    for u, v in zip(ref, got):
        if isinstance(u, np.ndarray):
            assert np.array_equal(u, v)
        else:
            assert u == v


def test_checkpoint_resume_is_bit_identical_gmm():
    need_gpu()
    from test_gpu_gmm import make_gmm
    T, k1 = 40, 17
    a, y, _ = make_gmm(4096, nd=300, T=T, seed=5)
    a.initialize()
    a.iterate(k1)
    blob = a.checkpoint()
    a.iterate(T - k1)
    ref = (a.state(), a.log_weight(), a.log_evidence(), a.path_sampling())
    b, _, _ = make_gmm(4096, nd=300, T=T, seed=5)
    b.restore(blob)
    b.iterate(T - k1)
    got = (b.state(), b.log_weight(), b.log_evidence(), b.path_sampling())
    for u, v in zip(ref, got):
        assert np.array_equal(np.asarray(u), np.asarray(v))


def test_restore_rejects_another_configuration():
    need_gpu()
    s, y, op = make_pf(3000, 10, 32, seed=1)
    s.initialize()
    blob = s.checkpoint()
    other, _, _ = make_pf(3000, 10, 32, seed=2)
    with pytest.raises(smc.SMCError) as e:
        other.restore(blob)
    assert e.value.code == smc.E_ARG
    with pytest.raises(smc.SMCError):
        s.restore(blob[:100])


@pytest.mark.parametrize("on_stream", [False, True])
@pytest.mark.parametrize("precision", [32, 64])
def test_iterate_host_matches_stored_observations(precision, on_stream):
    """smc_iterate_host with each observation sent from host memory gives
    the same records and final particle system, bit for bit, as iterating
    over the same observations stored up front: on the legacy stream (stream
    copies) and on a stream of its own (one graph launch, the observation
    and the record through the mapped staging)."""
    _host_vs_stored(precision, on_stream, 5000)


def test_iterate_host_at_the_benchmarked_size():
    """The same at N = 2^20 in FP32 on a stream of its own: the end-to-end
    call as the benchmark makes it."""
    _host_vs_stored(32, True, 1 << 20)


def _host_vs_stored(precision, on_stream, n):
    need_gpu()
    T = 10
    p = cv_params()
    _, y = workloads.cv_data(T, seed=0, **p)

    def sampler():
        cfg = smc.make_config(model="cv", n=n, precision=precision, scheme="systematic", threshold=0.6, seed=2,
                              max_data=T, cv=p)
        return smc.Sampler(cfg, stream=torch.cuda.Stream() if on_stream else None)

    a = sampler()
    a.set_data(y)
    a.initialize()
    a.iterate(T - 1)
    ha = a.history(T)
    b = sampler()
    b.set_data(y[:1])
    b.initialize()
    hb = [b.iterate_host(y[t]).as_dict() for t in range(1, T)]
    assert any(r["resampled"] for r in ha[1:])
    for ra, rb in zip(ha[1:], hb):
        for k in ("t", "L", "logZ", "ess", "mean_x", "mean_y", "resampled"):
            assert ra[k] == rb[k], (ra["t"], k, ra[k], rb[k])
    assert np.array_equal(a.state(), b.state())
    a.close()
    b.close()


def test_iterate_host_graph_stored_data_limits_and_errors():
    """The graph path of smc_iterate_host: with the observations stored up
    front a NULL observation replays them (records equal to smc_iterate);
    a step past the last observation is refused; a NaN observation comes
    back as the step's device error word."""
    need_gpu()
    n, T = 4096, 6
    p = cv_params()
    _, y = workloads.cv_data(T, seed=0, **p)

    def sampler():
        cfg = smc.make_config(model="cv", n=n, precision=32, scheme="stratified", threshold=0.7, seed=3,
                              max_data=T, cv=p)
        s = smc.Sampler(cfg, stream=torch.cuda.Stream())
        s.set_data(y)
        s.initialize()
        return s

    a, b = sampler(), sampler()
    a.iterate(T - 1)
    ha = a.history(T)
    hb = [b.iterate_host(None).as_dict() for _ in range(1, T)]
    for ra, rb in zip(ha[1:], hb):
        assert {k: _bits(v) for k, v in ra.items()} == {k: _bits(v) for k, v in rb.items()}
    with pytest.raises(smc.SMCError) as e:
        b.iterate_host(None)
    assert e.value.code == smc.E_ARG
    c = sampler()
    c.iterate_host(y[1])
    bad = y[2].copy()
    bad[0] = np.nan
    with pytest.raises(smc.SMCError) as e:
        c.iterate_host(bad)
    assert e.value.code == smc.E_NONFINITE
    for s in (a, b, c):
        s.close()


def test_iterate_host_graph_gmm():
    """GMM sampler stepped through smc_iterate_host on a stream (no
    observation): the same records as smc_iterate."""
    need_gpu()
    y = workloads.gmm_data(300, seed=1)
    T = 12

    def sampler():
        cfg = smc.make_config(model="gmm", n=2048, precision=32, scheme="systematic", threshold=0.5, seed=4,
                              max_data=300, max_records=T + 1,
                              gmm=dict(n_comp=3, n_iter=T, power=4.0, move=smc.GMM_RW))
        s = smc.Sampler(cfg, stream=torch.cuda.Stream())
        s.set_data(y)
        s.initialize()
        return s

    a, b = sampler(), sampler()
    a.iterate(T)
    ha = a.history(T + 1)
    hb = [b.iterate_host().as_dict() for _ in range(T)]
    for ra, rb in zip(ha[1:], hb):
        assert {k: _bits(v) for k, v in ra.items()} == {k: _bits(v) for k, v in rb.items()}
    with pytest.raises(smc.SMCError):
        b.iterate_host()
    a.close()
    b.close()


def test_bounded_wait_gives_up_and_the_context_recovers():
    """Failure detection on the device: with a short wait limit, one block
    waiting at the grid barrier for an arrival that never comes gives up,
    the next synchronising call returns SMC_E_TIMEOUT, the particle system
    is untouched, and restoring a checkpoint continues exactly like a run
    that never failed."""
    need_gpu()
    import ctypes
    from paper_1306_5583_b300 import smc as S
    n, T, seed = 5000, 10, 4
    s, y, op = make_pf(n, T, 32, scheme="systematic", seed=seed)
    ref, _, _ = make_pf(n, T, 32, scheme="systematic", seed=seed)
    s.initialize()
    ref.initialize()
    s.iterate(3)
    ref.iterate(3)
    blob = s.checkpoint()
    x0, lw0 = s.state(), s.log_weight()
    try:
        S.set_wait_limit(2000)
        s.wait_selftest()
        assert S.lib().smc_sync(s.ctx) == S.E_TIMEOUT
        # the reads still copy, and report the error
        x1 = np.empty_like(x0)
        assert S.lib().smc_read_state(s.ctx, x1.ctypes.data_as(ctypes.c_void_p), 0) == S.E_TIMEOUT
        assert np.array_equal(x1, x0)
        with pytest.raises(S.SMCError):
            s.iterate(1)
            s.sync()
    finally:
        S.set_wait_limit(0)
    s.restore(blob)
    assert np.array_equal(s.log_weight(), lw0)
    s.iterate(T - 1 - 3)
    ref.iterate(T - 1 - 3)
    assert np.array_equal(s.state(), ref.state())
    assert s.log_evidence() == ref.log_evidence()


@pytest.mark.parametrize("move", ["rw", "mala"])
def test_iterate_host_mixture_sampler(move):
    """smc_iterate_host on the mixture sampler (its graph ends with the
    record kernel and the completion word): every record equals the one
    smc_iterate writes, bit for bit, and so does the final particle
    system."""
    need_gpu()
    n, T, nd = 4096, 12, 200
    y = workloads.gmm_data(nd, seed=0)
    mv = {"rw": smc.GMM_RW, "mala": smc.GMM_MALA}[move]

    def sampler():
        cfg = smc.make_config(model="gmm", n=n, precision=32, scheme="systematic", threshold=0.5, seed=4,
                              max_data=nd, max_records=T + 1,
                              gmm=dict(n_comp=3, n_iter=T, power=5.0, move=mv, mala_step=0.05))
        s = smc.Sampler(cfg, stream=torch.cuda.Stream())
        s.set_data(y)
        s.initialize()
        return s

    a, b = sampler(), sampler()
    a.iterate(T)
    ha = a.history(T + 1)
    hb = [b.iterate_host(None).as_dict() for _ in range(T)]
    for ra, rb in zip(ha[1:], hb):
        assert {k: _bits(v) for k, v in ra.items()} == {k: _bits(v) for k, v in rb.items()}
    assert np.array_equal(a.state(), b.state())
    with pytest.raises(smc.SMCError) as e:
        b.iterate_host(None)  # past the schedule
    assert e.value.code == smc.E_ARG
    a.close()
    b.close()
