"""GPU: the allocation-free systematic resampling entry point gives the same
ancestors as the context API's resampling step on the same log-weights,
seed, stream and iteration, on two calls in a row (its scratch array is
shared and reused between calls).  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

from gpu_common import make_pf, need_gpu, torch
from paper_1306_5583_b300 import smc

pytestmark = pytest.mark.gpu


def _noalloc(lw_dev, n, seed, t, out):
    return smc.lib().smc_resample_systematic_noalloc(
        ctypes.c_void_p(lw_dev.data_ptr()), n, seed, 0, t, ctypes.c_void_p(out.data_ptr()),
        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_noalloc_matches_context_resampling_twice():
    need_gpu()
    n, seed = 300000 + 7, 13
    s, y, op = make_pf(n, 6, 32, scheme="systematic", threshold=1.0, seed=seed)
    s.initialize()
    for t in (1, 2):
        s.move()
        lw = torch.from_numpy(s.log_weight()).cuda()
        s.resample()
        ref = s.ancestors()
        out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
        assert _noalloc(lw, n, seed, t, out) == smc.OK
        torch.cuda.synchronize()
        assert np.array_equal(out.cpu().numpy(), ref), t


def test_noalloc_rejects_sizes_beyond_its_scratch():
    need_gpu()
    n = (1 << 22) + 1
    lw = torch.zeros(16, dtype=torch.float32, device="cuda")
    out = torch.zeros(16, dtype=torch.int32, device="cuda")
    assert _noalloc(lw, n, 1, 0, out) == smc.E_ARG


def _status():
    v = ctypes.c_int32(-1)
    assert smc.lib().smc_resample_noalloc_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                                  ctypes.byref(v)) == smc.OK
    return v.value


@pytest.mark.parametrize("bad", ["nan", "all_neg_inf"])
def test_noalloc_reports_nonfinite_weights_and_writes_nothing(bad):
    """A NaN log-weight (which a maximum alone would skip) or all weights
    zero: the call writes no ancestor and its status word says
    SMC_E_NONFINITE, as the context API's weighting step does; a good call
    afterwards clears the status."""
    need_gpu()
    n = 5000
    lw = torch.randn(n, dtype=torch.float32, device="cuda")
    if bad == "nan":
        lw[1234] = float("nan")
    else:
        lw.fill_(float("-inf"))
    out = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    assert _noalloc(lw, n, 3, 1, out) == smc.OK
    assert _status() == smc.E_NONFINITE
    assert bool((out == -1).all())
    good = torch.randn(n, dtype=torch.float32, device="cuda")
    assert _noalloc(good, n, 3, 1, out) == smc.OK
    assert _status() == smc.OK
    o = out.cpu().numpy()
    assert o.min() >= 0 and np.all(np.diff(o) >= 0)
