"""Builds libfsmc.so in-tree with nvcc for sm_103a (B300)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libfsmc.so")
SOURCES = ["engine.cu", "ess.cu", "ess_block.cu", "ess_tc.cu", "dr.cu", "nuts.cu", "slice.cu", "serving.cu",
           "noalloc.cu", "autotune.cu", "probe.cu", "stats.cu"]
HEADERS = ["fsmc_device.cuh", "fsmc_kernels.h", "engine_internal.h", "target_logp.cuh", "ess_common.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread"]


def _stale():
    if not os.path.exists(LIB):
        return True
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(HERE, "..", "include", "fsmc.h"))
    deps.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in deps) > os.path.getmtime(LIB)


def build(force=False, verbose=False, jobs=None):
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    procs = []
    objs = []
    hdr_time = max(os.path.getmtime(p) for p in
                   [os.path.join(CSRC, f) for f in HEADERS] +
                   [os.path.join(HERE, "..", "include", "fsmc.h"), os.path.abspath(__file__)])
    for src in SOURCES:
        obj = os.path.join(objdir, src.replace(".cu", ".o"))
        objs.append(obj)
        # an object newer than its source and every header is up to date
        if (not force and not verbose and os.path.exists(obj) and
                os.path.getmtime(obj) > max(hdr_time, os.path.getmtime(os.path.join(CSRC, src)))):
            continue
        cmd = [nvcc] + FLAGS + ARCH + ["-I", os.path.join(HERE, "..", "include"), "-c",
                                       os.path.join(CSRC, src), "-o", obj]
        if verbose:
            cmd.append("-Xptxas=-v")
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode())
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = LIB + ".tmp"
    subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
