"""GPU: the batched form (many filters of uneven N and T in one launch per
kernel) gives every filter exactly the plain path's results on the same
Philox stream; the plain path is itself parity-tested against the oracle."""
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
            for k in ("t", "L", "logZ", "ess", "mean_x", "mean_y", "resampled"):
                assert rp[k] == rb[k], (b, rp["t"], k, rp[k], rb[k])
        assert np.array_equal(s.state(), bt.state(b))
        assert lz[b] == s.log_evidence()
        s.close()


def test_batch_tune_and_iterate_in_pieces():
    need_gpu()
    cfg = smc.make_config(model="cv", n=1, precision=32, scheme="systematic", threshold=0.5, seed=7,
                          max_data=max(TS), keep_cdf=False)
    bt = smc.Batch(cfg, NS, TS)
    for b, T in enumerate(TS):
        bt.set_data(b, _data(T, 1 + b))
    g = bt.tune()
    assert g in (1, 2, 4, 8)
    bt.iterate(4)
    bt.iterate(max(TS) - 1 - 4)
    a = bt.log_evidence()
    bt.run()
    assert np.array_equal(a, bt.log_evidence())
    with pytest.raises(smc.SMCError):
        bt.iterate(1)   # past the longest filter
