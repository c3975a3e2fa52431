"""Host checks of the CUDA path's header-only arithmetic (compiled with g++).

* the exact 64-bit resampling thresholds tau_k = floor(Q_N (2^25 k + c) / (N 2^25))
  of systematic / stratified selection against Python integers;
* the double-float helpers of the FP32 finalisation (logarithm, division,
  exact integer and double conversions) against 40-digit decimal arithmetic.
"""
import ctypes
import decimal
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SHIM = os.path.join(HERE, "host_support", "df_shim.cpp")


@pytest.fixture(scope="module")
def shim(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("shim") / "df_shim.so")
    subprocess.run([gxx, "-O2", "-std=c++17", "-shared", "-fPIC", "-o", out, SHIM], check=True)
    lib = ctypes.CDLL(out)
    lib.shim_df_log.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_void_p]
    lib.shim_df_div.argtypes = [ctypes.c_float] * 4 + [ctypes.c_void_p]
    lib.shim_df_to_double.argtypes = [ctypes.c_float, ctypes.c_float]
    lib.shim_df_to_double.restype = ctypes.c_double
    lib.shim_df_from_int.argtypes = [ctypes.c_longlong, ctypes.c_void_p]
    lib.shim_df_from_u64.argtypes = [ctypes.c_ulonglong, ctypes.c_void_p]
    lib.shim_grid_tau.argtypes = [ctypes.c_ulonglong] * 4 + [ctypes.c_int, ctypes.c_int, ctypes.c_void_p]
    return lib


def _df(x):
    hi = np.float32(x)
    lo = np.float32(x - float(hi))
    return float(hi), float(lo)


def test_grid_thresholds_are_exact(shim):
    rng = np.random.default_rng(0)
    out = (ctypes.c_ulonglong * 8)()
    for n in (1, 2, 3, 7, 1000, 1024, 65535, 1 << 20, (1 << 20) + 1, 12345678, (1 << 31) - 1):
        f = 61 - int(np.ceil(np.log2(n))) if n > 1 else 61
        qmax = min(n << f, (1 << 62) - 1)
        for rep in range(300):
            qn = int(qmax - rng.integers(0, 1000)) if rep % 3 == 0 else int(rng.integers(1, qmax))
            c = 2 * int(rng.integers(0, 1 << 24)) + 1
            k0 = int(rng.integers(0, n + 1))
            for incremental in (0, 1):
                shim.shim_grid_tau(qn, n, k0, c, 8, incremental, out)
                for j in range(8):
                    k = k0 + j
                    if k > n:  # thresholds past the last output are never used
                        break
                    assert out[j] == (qn * ((k << 25) + c)) // (n << 25), (n, qn, k, c, incremental)


def test_df_log_accuracy(shim):
    decimal.getcontext().prec = 40
    rng = np.random.default_rng(1)
    out = (ctypes.c_float * 2)()
    worst = 0.0
    for _ in range(20000):
        x = 2.0 ** rng.uniform(-20, 31)
        hi, lo = _df(x * (1 + rng.uniform(-1e-8, 1e-8)))
        shim.shim_df_log(hi, lo, out)
        got = decimal.Decimal(float(out[0])) + decimal.Decimal(float(out[1]))
        ref = (decimal.Decimal(hi) + decimal.Decimal(lo)).ln()
        worst = max(worst, float(abs(got - ref)))
    assert worst < 5e-13, worst
    for v in (1.0, 2.0, 0.5, float(2 ** 20)):
        shim.shim_df_log(v, 0.0, out)
        assert abs(float(out[0]) + float(out[1]) - np.log(v)) < 1e-14


def test_df_div_accuracy(shim):
    decimal.getcontext().prec = 40
    rng = np.random.default_rng(2)
    out = (ctypes.c_float * 2)()
    for _ in range(20000):
        a, b = rng.uniform(1e-3, 1e6, size=2)
        ah, al = _df(a)
        bh, bl = _df(b)
        shim.shim_df_div(ah, al, bh, bl, out)
        got = decimal.Decimal(float(out[0])) + decimal.Decimal(float(out[1]))
        ref = (decimal.Decimal(ah) + decimal.Decimal(al)) / (decimal.Decimal(bh) + decimal.Decimal(bl))
        assert float(abs(got - ref) / ref) < 1e-13


def test_df_conversions(shim):
    out = (ctypes.c_float * 2)()
    for x in (0, 1, 255, 256, 257, (1 << 24) + 1, (1 << 31) - 1, 123456789):
        shim.shim_df_from_int(x, out)
        assert int(out[0]) + int(out[1]) == x
    rng = np.random.default_rng(3)
    for _ in range(1000):
        hi, lo = _df(rng.normal() * 10 ** rng.uniform(-5, 5))
        assert shim.shim_df_to_double(hi, lo) == hi + lo
    for x in [0, 1, 3, (1 << 24) - 1, (1 << 24) + 1, (1 << 40) + 12345, (1 << 62) - 1, (1 << 64) - 1] + \
            [int(v) for v in rng.integers(0, 1 << 63, size=2000, dtype=np.uint64)]:
        shim.shim_df_from_u64(x, out)
        got = decimal.Decimal(float(out[0])) + decimal.Decimal(float(out[1]))
        assert abs(got - x) <= max(x, 1) * decimal.Decimal(2) ** -47, x
    assert shim.shim_df_to_double(float("inf"), 0.0) == float("inf")
    assert np.isnan(shim.shim_df_to_double(float("nan"), 0.0))
    assert shim.shim_df_to_double(-0.0, 0.0) == 0.0
