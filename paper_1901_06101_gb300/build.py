"""Build libhbaca.so in-tree for sm_103a (GB300).

Each translation unit is compiled by its own nvcc process (in parallel),
then the objects are linked into ``paper_1901_06101_gb300/libhbaca.so``; the
FP64 unit-rate probe the benchmark reports goes to ``libhbaca_probe.so``.
Usage: ``python -m paper_1901_06101_gb300.build`` (or ``build()``).
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhbaca.so")
LIB_PROBE = os.path.join(HERE, "libhbaca_probe.so")
SOURCES = ["hbaca_f64.cu", "hbaca_c128.cu", "plan.cpp", "api.cpp", "noalloc.cu", "adjoint.cu", "errnorm.cu", "hmatrix.cpp"]
PROBE_SOURCES = ["probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src, verbose_ptxas=False):
    obj = os.path.join(OBJ, os.path.splitext(src)[0] + ".o")
    cmd = [_nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, "-O3", "-std=c++17",
           "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"), "-I", CSRC] + ARCH
    if src.endswith(".cu"):
        cmd += ["-lineinfo"]
        if verbose_ptxas:
            cmd += ["-Xptxas", "-v"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(verbose_ptxas=False, quiet=False):
    os.makedirs(OBJ, exist_ok=True)
    allsrc = SOURCES + PROBE_SOURCES
    with ThreadPoolExecutor(max_workers=len(allsrc)) as ex:
        results = dict(zip(allsrc, ex.map(lambda s: _compile(s, verbose_ptxas), allsrc)))
    if verbose_ptxas and not quiet:
        for _, log in results.values():
            sys.stderr.write(log)
    for lib_path, srcs in ((LIB, SOURCES), (LIB_PROBE, PROBE_SOURCES)):
        cmd = [_nvcc(), "-shared", "-o", lib_path] + [results[s][0] for s in srcs] + ARCH
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    return LIB


if __name__ == "__main__":
    build(verbose_ptxas="-v" in sys.argv)
    print(LIB)
