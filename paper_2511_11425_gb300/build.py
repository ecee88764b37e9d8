"""Build libsph (paper_2511_11425_gb300/_libsph.so) for GB300 (sm_103a).

Each translation unit in csrc/ is compiled in parallel with nvcc, then linked
into one shared library with a plain C ABI (include/sph.h).  The FP32 FMA
throughput probe the benchmark uses for its roofline (probe/fma_probe.cu) is
compiled at the same time into its own library, _fma_probe.so, which is not
part of libsph.  A library is rebuilt only when a source or header is newer
than it.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "_libsph.so")
PROBE_SRC = os.path.join(HERE, "probe", "fma_probe.cu")
PROBE_LIB = os.path.join(HERE, "_fma_probe.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", os.path.join(ROOT, "include")]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsph")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib, deps) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    return any(os.path.getmtime(d) > t for d in list(deps) + [os.path.abspath(__file__)])


def _lib_deps():
    headers = glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h"))
    return sources() + headers + [
        os.path.join(ROOT, "include", "sph.h")]


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    lib_stale = force or _stale(LIB, _lib_deps())
    probe_stale = force or _stale(PROBE_LIB, [PROBE_SRC])
    if not (lib_stale or probe_stale):
        return LIB
    nvcc = _nvcc()
    os.makedirs(OBJ, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(OBJ, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, file=sys.stderr)
        return obj

    def probe():
        tmp = PROBE_LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc, *ARCH, "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared", PROBE_SRC,
               "-o", tmp]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (PROBE_SRC, r.stdout, r.stderr))
        os.replace(tmp, PROBE_LIB)

    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        fprobe = ex.submit(probe) if probe_stale else None
        if lib_stale:
            objs = list(ex.map(compile_one, sources()))
            tmp = LIB + ".tmp%d" % os.getpid()
            r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True,
                               text=True)
            if r.returncode != 0:
                raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
            os.replace(tmp, LIB)
        if fprobe is not None:
            fprobe.result()
    return LIB


if __name__ == "__main__":
    v = "-v" in sys.argv
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=v or bool(extra), extra=extra))
