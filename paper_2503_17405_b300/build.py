"""Builds libfsmc.so (and the benchmark's probe library) in-tree with nvcc for sm_103a (B300)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libfsmc.so")
SOURCES = ["engine.cu", "ess.cu", "ess_block.cu", "ess_tc.cu", "dr.cu", "nuts.cu", "slice.cu", "serving.cu",
           "noalloc.cu", "autotune.cu", "stats.cu"]
# sources compiled as several objects, each with its own -D (disjoint explicit instantiations)
PARTS = {"ess.cu": [("ess_p%d" % p, ["-DFSMC_ESS_PART=%d" % p]) for p in (1, 2, 3, 4)]}
# the benchmark's throughput probe: a separate library, not part of libfsmc.so or its C ABI
PROBE_LIB = os.path.join(HERE, "libfsmc_probe.so")
PROBE_SOURCES = ["bench_probe.cu"]
HEADERS = ["fsmc_device.cuh", "fsmc_kernels.h", "engine_internal.h", "target_logp.cuh", "ess_common.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread"]


def _header_time():
    return max(os.path.getmtime(p) for p in
               [os.path.join(CSRC, f) for f in HEADERS] +
               [os.path.join(HERE, "..", "include", "fsmc.h"), os.path.abspath(__file__)])


def _stale(lib, sources):
    if not os.path.exists(lib):
        return True
    newest = max([_header_time()] + [os.path.getmtime(os.path.join(CSRC, f)) for f in sources])
    return newest > os.path.getmtime(lib)


def _build_lib(lib, sources, force, verbose):
    if not force and not _stale(lib, sources):
        return lib
    nvcc = os.environ.get("NVCC", "nvcc")
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    procs, objs = [], []
    hdr_time = _header_time()
    for src in sources:
        for name, defs in PARTS.get(src, [(src.replace(".cu", ""), [])]):
            obj = os.path.join(objdir, name + ".o")
            objs.append(obj)
            # an object newer than its source and every header is up to date
            if (not force and not verbose and os.path.exists(obj) and
                    os.path.getmtime(obj) > max(hdr_time, os.path.getmtime(os.path.join(CSRC, src)))):
                continue
            cmd = [nvcc] + FLAGS + ARCH + defs + ["-I", os.path.join(HERE, "..", "include"), "-c",
                                                  os.path.join(CSRC, src), "-o", obj]
            if verbose:
                cmd.append("-Xptxas=-v")
            procs.append((name, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0 or verbose:
            sys.stderr.write(out.decode())
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = lib + ".tmp"
    subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"], check=True)
    os.replace(tmp, lib)
    return lib


def build(force=False, verbose=False, jobs=None):
    """Builds libfsmc.so and libfsmc_probe.so where stale; returns the path of libfsmc.so."""
    _build_lib(PROBE_LIB, PROBE_SOURCES, force, verbose)
    return _build_lib(LIB, SOURCES, force, verbose)


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
