"""Build step: compile the CUDA sources into in-tree shared libraries.

* ``paper_1306_5583_b300/libsmc.so``: the SMC hot path behind include/smc.h
  (csrc/smc.cu) and the special-function pipe rate measurement
  (csrc/mufu_peak.cu).
* ``tests/gpu_support/libcurand_philox.so``: a test-only kernel that calls
  the CUDA toolkit's own Philox4x32-10 (curand device API) so the GPU tests
  can cross-check the library's generator against an independent
  implementation.

All code is compiled for sm_103a only.
"""
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIB = os.path.join(PKG, "libsmc.so")
TEST_SUPPORT = os.path.join(ROOT, "tests", "gpu_support")
CURAND_SRC = os.path.join(TEST_SUPPORT, "curand_philox.cu")
CURAND_LIB = os.path.join(TEST_SUPPORT, "libcurand_philox.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsmc.so")


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))
            if f.endswith((".cu", ".cuh", ".h"))] + [os.path.join(ROOT, "include", "smc.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force=False, verbose=False):
    nvcc = _nvcc()
    out = []
    if force or _stale(LIB, _sources()):
        cmd = [nvcc, *ARCH, *FLAGS, "-o", LIB + ".tmp", os.path.join(CSRC, "smc.cu"), os.path.join(CSRC, "mufu_peak.cu")]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        out.append(_run(cmd))
        os.replace(LIB + ".tmp", LIB)
    if os.path.exists(CURAND_SRC) and (force or _stale(CURAND_LIB, [CURAND_SRC])):
        cmd = [nvcc, *ARCH, *FLAGS, "-o", CURAND_LIB + ".tmp", CURAND_SRC]
        out.append(_run(cmd))
        os.replace(CURAND_LIB + ".tmp", CURAND_LIB)
    return "".join(out)


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
