"""GPU tests of how Sampler::iterate (smc_iterate) runs its iterations:
whole chunks of iterations per graph launch, and the iterations recorded
into a caller's own CUDA graph capture (the caller then owns the replays;
an iteration replayed past the observation buffer raises SMC_E_RANGE on the
device instead of reading past it)."""
import numpy as np
import pytest

from gpu_common import cv_params, need_gpu, torch
from oracle import cv as ocv
from paper_1306_5583_b300 import smc, workloads

pytestmark = pytest.mark.gpu


def _sampler(n, T, precision, scheme, threshold, stream, seed=3):
    p = cv_params()
    _, y = workloads.cv_data(T, seed=0, **p)
    cfg = smc.make_config(model="cv", n=n, precision=precision, scheme=scheme, threshold=threshold, seed=seed,
                          max_data=T, max_records=T, cv=p)
    s = smc.Sampler(cfg, stream=stream)
    s.set_data(y)
    return s, y, p


def _records(s, count):
    return [(r["t"], r["resampled"], r["logZ"], r["ess"], r["mean_x"]) for r in s.history(count)]


@pytest.mark.parametrize("scheme", ["systematic", "stratified", "residual"])
def test_chunked_iterate_equals_single_launches(scheme):
    """smc_iterate(n) with n >= 8 replays an 8-iteration graph: the same
    particles and records as n one-iteration calls."""
    need_gpu()
    n, T = 20011, 30
    stream = torch.cuda.Stream()
    a, _, _ = _sampler(n, T, 32, scheme, 0.5, stream)
    b, _, _ = _sampler(n, T, 32, scheme, 0.5, stream)
    with torch.cuda.stream(stream):
        a.initialize()
        a.iterate(T - 1)  # three chunks of 8 and five single launches
        b.initialize()
        for _ in range(T - 1):
            b.iterate(1)
        stream.synchronize()
    assert np.array_equal(a.state(), b.state())
    assert np.array_equal(a.log_weight(), b.log_weight())
    assert _records(a, T) == _records(b, T)
    a.close()
    b.close()


def test_chunked_iterate_fp64_matches_oracle():
    """The chunked path of a double-precision filter against the oracle."""
    need_gpu()
    n, T = 3000, 20
    stream = torch.cuda.Stream()
    s, y, p = _sampler(n, T, 64, "systematic", 0.5, stream, seed=5)
    with torch.cuda.stream(stream):
        s.initialize()
        s.iterate(T - 1)
        stream.synchronize()
    ref, last = ocv.run(y, n, 5, ocv.CVParams(**p), scheme="systematic", threshold=0.5)
    for r, o in zip(s.history(T), ref):
        assert r["resampled"] == o["resampled"]
        assert abs(r["logZ"] - o["logZ"]) < 1e-9
    assert np.max(np.abs(s.state() - last.x)) < 1e-9
    s.close()


@pytest.mark.parametrize("precision,scheme,threshold", [(32, "systematic", 0.5), (32, "systematic", 1.0),
                                                        (64, "stratified", 0.5), (32, "multinomial", 0.5)])
def test_iterations_in_a_callers_graph(precision, scheme, threshold):
    """Iterations recorded into the caller's capture and replayed by the
    caller give the same particles and records as smc_iterate."""
    need_gpu()
    n, T, W, K = 50000, 40, 3, 12
    stream = torch.cuda.Stream()
    s, _, _ = _sampler(n, T, precision, scheme, threshold, stream)
    ref, _, _ = _sampler(n, T, precision, scheme, threshold, stream)
    with torch.cuda.stream(stream):
        s.initialize()
        s.iterate(1)  # the context's own iteration graph (the launch form the capture takes)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(K):
                s.iterate(1)
        s.initialize()
        s.iterate(W)
        g.replay()
        stream.synchronize()
        ref.initialize()
        ref.iterate(W + K)
        stream.synchronize()
    assert np.array_equal(s.state(), ref.state())
    assert _records(s, W + K + 1) == _records(ref, W + K + 1)
    s.close()
    ref.close()


def test_callers_graph_replayed_past_the_data_raises_range():
    """A caller's graph replayed until its iterations pass the observation
    buffer: the device raises SMC_E_RANGE and runs nothing further."""
    need_gpu()
    n, T, K = 4096, 12, 5
    stream = torch.cuda.Stream()
    s, _, _ = _sampler(n, T, 32, "systematic", 0.5, stream)
    with torch.cuda.stream(stream):
        s.initialize()
        s.iterate(1)
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            s.iterate(K)
        s.initialize()
        s.iterate(1)
        stream.synchronize()
        g.replay()  # iterations 2 .. 6
        g.replay()  # 7 .. 11: the last observation row
        stream.synchronize()
        s.sync()
        last = s.history(1)[0]
        assert last["t"] == T - 1 and last["status"] == smc.OK
        g.replay()  # 12: past the data
        stream.synchronize()
        with pytest.raises(smc.SMCError) as e:
            s.sync()
        assert e.value.code == smc.E_RANGE
    s.close()


@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty")
def test_capture_refused_without_own_graph():
    """A capture on a context that has no iteration graph yet is refused
    (SMC_E_STATE) and leaves the caller's capture intact (and empty, which
    PyTorch warns about)."""
    need_gpu()
    stream = torch.cuda.Stream()
    s, _, _ = _sampler(2048, 10, 32, "systematic", 0.5, stream)
    with torch.cuda.stream(stream):
        s.initialize()
        stream.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=stream):
            with pytest.raises(smc.SMCError) as e:
                s.iterate(1)
        assert e.value.code == smc.E_STATE
    s.close()
