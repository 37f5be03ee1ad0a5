"""Build libsbp.so in-tree with nvcc for sm_103a (GB300)."""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsbp.so")
SOURCES = ["sbp_api.cu", "sbp3d_api.cu"]
DEPS = ["sbp_api.cu", "sbp_kernels.cuh", "sbp_adjoint.cuh", "sbp_device.cuh", "sbp_interior_march.cuh",
        "sbp_batch.cuh", "sbp_wide.cuh", "sbp_tables.inc", "sbp3d_api.cu", "sbp3d.cuh"]
HEADERS = ["sbp.h", "sbp3.h"]
NVCC_FLAGS = ["-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
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
    srcs = [os.path.join(CSRC, d) for d in DEPS] + [os.path.join(HERE, "..", "include", x) for x in HEADERS] + [__file__]
    return all(os.path.getmtime(s) <= t for s in srcs)


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    nvcc = nvcc_path()
    if nvcc is None:
        raise RuntimeError("nvcc not found: cannot build libsbp")
    tmp = LIB + ".tmp"
    # one object per translation unit, compiled side by side, then one shared library
    objs = [os.path.join(HERE, "_" + os.path.splitext(s)[0] + ".tmp.o") for s in SOURCES]
    procs = [subprocess.Popen([nvcc] + NVCC_FLAGS + ["-c", "-o", o, os.path.join(CSRC, s)],
                              stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for s, o in zip(SOURCES, objs)]
    outs = [p.communicate() for p in procs]
    log = "".join(a + b for a, b in outs)
    try:
        if any(p.returncode != 0 for p in procs):
            raise RuntimeError("nvcc failed:\n" + log)
        res = subprocess.run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", tmp] + objs,
                             capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc link failed:\n" + res.stdout + res.stderr)
    finally:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
    if verbose:
        print(log)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
