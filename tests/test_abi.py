"""The C-ABI library loads, exports every symbol include/smc.h declares,
and its structs have the layout the Python binding assumes (no GPU needed)."""
import ctypes
import os
import re
import subprocess
import tempfile

import pytest

from paper_1306_5583_b300 import build, smc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "smc.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(smc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return smc.lib()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert "smc_create" in names and "smc_resample" in names
    for name in names:
        assert hasattr(L, name), name


def test_binding_covers_the_header():
    assert set(_declared()) == set(smc._SIGS)


def test_struct_layout_matches_c():
    src = r"""
#include <stdio.h>
#include <stddef.h>
#include "smc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(smc_config), sizeof(smc_record), sizeof(smc_cv_params),
         sizeof(smc_gmm_params), offsetof(smc_config, max_data), offsetof(smc_config, gmm),
         offsetof(smc_record, t));
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "l.c")
        exe = os.path.join(d, "l")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", exe, c], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()]
    assert vals == [ctypes.sizeof(smc.Config), ctypes.sizeof(smc.Record), ctypes.sizeof(smc.CVParams),
                    ctypes.sizeof(smc.GMMParams), smc.Config.max_data.offset, smc.Config.gmm.offset,
                    smc.Record.t.offset]


def test_workspace_sizing_is_host_only_and_validates(L):
    cfg = smc.make_config(n=1 << 20, precision=32, scheme="systematic", max_data=1000)
    b = L.smc_workspace_bytes(ctypes.byref(cfg))
    # state (2 x 4 x N floats) + log-weights (2 x N) + ancestors + CDF at least
    assert b >= (1 << 20) * (32 + 8 + 4 + 8)
    for bad in (dict(n=0), dict(precision=16), dict(scheme=9), dict(max_data=0)):
        kw = dict(n=1024, precision=32, scheme="systematic", max_data=10)
        kw.update(bad)
        c = smc.make_config(**kw)
        assert L.smc_workspace_bytes(ctypes.byref(c)) == 0
    # residual needs its extra arrays
    cr = smc.make_config(n=1 << 20, scheme="residual", max_data=1000)
    assert L.smc_workspace_bytes(ctypes.byref(cr)) > b


def test_create_rejects_bad_workspace_without_touching_the_device(L):
    cfg = smc.make_config(n=1000, precision=64, max_data=10)
    ctx = ctypes.c_void_p()
    assert L.smc_create(ctypes.byref(ctx), ctypes.byref(cfg), None, 0, None) == smc.E_WORKSPACE
    assert not ctx.value
    assert L.smc_create(ctypes.byref(ctx), ctypes.byref(cfg), ctypes.c_void_p(4096 + 8), 1 << 30, None) \
        == smc.E_WORKSPACE


def test_error_strings(L):
    for code in range(8):
        assert L.smc_error_string(code)
    assert L.smc_error_string(99) == b"unknown error"
