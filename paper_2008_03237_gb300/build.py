"""Builds libpairf12.so (sm_103a) in-tree with nvcc.

    python -m paper_2008_03237_gb300.build            # from the repository root

Each translation unit is compiled in parallel to an object file under _build/,
then linked into paper_2008_03237_gb300/libpairf12.so against the shared CUDA
runtime.  Nothing is installed outside the repository.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libpairf12.so")
# host-side translation units, then one per kernel variant (csrc/inst/): the
# variants are large fused kernels, and compiling them apart lets them build
# in parallel
SOURCES = ["pf12_api.cu", "pf12_forward.cu", "pf12_backward.cu", "pf12_full.cu"] + sorted(
    os.path.join("inst", f) for f in os.listdir(os.path.join(CSRC, "inst")) if f.endswith(".cu"))
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpairf12")
    return exe


def cuda_lib_dir():
    base = os.path.dirname(os.path.dirname(os.path.realpath(nvcc())))
    for sub in ("lib64", "lib", os.path.join("targets", "sbsa-linux", "lib"),
                os.path.join("targets", "x86_64-linux", "lib")):
        d = os.path.join(base, sub)
        if os.path.exists(os.path.join(d, "libcudart.so")):
            return d
    return os.path.join(base, "lib64")


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.splitext(src)[0].replace(os.sep, "_") + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def needs_build():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [
        os.path.join(CSRC, "inst", f) for f in os.listdir(os.path.join(CSRC, "inst"))] + [
        os.path.join(ROOT, "include", "pairf12.h"), os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, ptxas_info=False, force=False):
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    extra = ["-Xptxas", "-v"] if ptxas_info else []
    with cf.ThreadPoolExecutor(min(len(SOURCES), max(2, os.cpu_count() or 2))) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    objs = [o for o, _ in results]
    if verbose or ptxas_info:
        for (_, log), s in zip(results, SOURCES):
            if log.strip():
                print(f"--- {s}\n{log}")
    tmp = LIB + ".tmp"
    libdir = cuda_lib_dir()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "shared",
           "-Xlinker", "-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


PROBE_SRC = os.path.join(CSRC, "probe", "fp64_peak.cu")
PROBE_LIB = os.path.join(PKG, "libpf12probe.so")


def build_probe(force=False):
    """libpf12probe.so: the FP64 FMA-pipe throughput probe the benchmark uses
    as its roofline denominator (not part of the pair-F12 library)."""
    if not force and os.path.exists(PROBE_LIB) and os.path.getmtime(PROBE_LIB) >= max(
            os.path.getmtime(PROBE_SRC), os.path.getmtime(os.path.abspath(__file__))):
        return PROBE_LIB
    tmp = PROBE_LIB + ".tmp"
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           PROBE_SRC, "-o", tmp, "-cudart", "shared", "-Xlinker", "-rpath," + cuda_lib_dir()]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for the FP64 probe:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, PROBE_LIB)
    return PROBE_LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv, force="-f" in sys.argv))
