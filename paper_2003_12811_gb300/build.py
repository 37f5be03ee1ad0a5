"""Build libsbp.so in-tree with nvcc for sm_103a (GB300)."""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsbp.so")
SOURCES = ["sbp_api.cu"]
DEPS = ["sbp_api.cu", "sbp_kernels.cuh", "sbp_adjoint.cuh", "sbp_device.cuh", "sbp_interior_march.cuh",
        "sbp_batch.cuh", "sbp_wide.cuh", "sbp_tables.inc"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr", "-shared",
              "--split-compile", "0"]   # device code compiled in parallel on all host cores


def nvcc_path():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    return cand if os.path.exists(cand) else None


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(HERE, "..", "include", "sbp.h"), __file__]
    return all(os.path.getmtime(s) <= t for s in srcs)


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    nvcc = nvcc_path()
    if nvcc is None:
        raise RuntimeError("nvcc not found: cannot build libsbp")
    tmp = LIB + ".tmp"
    cmd = [nvcc] + NVCC_FLAGS + ["-o", tmp] + [os.path.join(CSRC, s) for s in SOURCES]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose:
        print(res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
