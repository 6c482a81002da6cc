"""Build the sm_103a shared library libqhd.so in-tree (nvcc, no CMake).

The translation units compile in parallel; the result is
paper_2303_01471_gb300/_lib/libqhd.so, a plain C ABI (include/qhd.h) with
the CUDA runtime linked statically and no other library.  The arithmetic throughput probe
that the benchmark uses to state roofline peaks is built beside it as its own
library, _lib/libqhd_probe.so (include/qhd_probe.h), outside the simulator's
ABI.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libqhd.so")
SOURCES = ["qhd_kernels.cu", "qhd_plane.cu", "qhd_host.cu", "qhd_static.cu", "qhd_tcdft.cu", "qhd_fno.cu", "qhd_spectrum.cu",
           "qhd_lattice.cu", "qhd_group.cu", "qhd_umma_gemm.cu"]
PROBE_SOURCE = "qhd_probe.cu"
PROBE_LIB = os.path.join(LIBDIR, "libqhd_probe.so")
HEADERS = ["qhd_device.cuh", "qhd_kernels.h", "qhd_plane.cuh", "qhd_tcdft.h", "qhd_spectrum.h", "qhd_sched.cuh",
           "qhd_prep.cuh", "qhd_group.h", "qhd_umma.cuh", "qhd_trace.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _cuda_home() -> str:
    return os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc() -> str:
    cand = os.path.join(_cuda_home(), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB) or not os.path.exists(PROBE_LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, s) for s in SOURCES + HEADERS + [PROBE_SOURCE]]
    deps.append(os.path.join(ROOT, "include", "qhd.h"))
    deps.append(os.path.join(ROOT, "include", "qhd_probe.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags=None, out: str = None,
          csrc: str = None) -> str:
    """Compile libqhd.so.  extra_flags / out / csrc build a variant elsewhere (for
    experiments); the default library is LIB from CSRC."""
    target = out or LIB
    src_dir = csrc or CSRC
    if not force and out is None and not extra_flags and not _stale():
        return LIB
    libdir = os.path.dirname(target)
    os.makedirs(libdir, exist_ok=True)
    nvcc = _nvcc()
    flags = ["-std=c++17", "-O3", "-lineinfo", *ARCH, "-Xcompiler", "-fPIC",
             "-I" + os.path.join(ROOT, "include"), "-I" + src_dir, "-diag-suppress", "550"]
    if verbose:
        flags += ["-Xptxas", "-v"]
    flags += list(extra_flags or [])

    def compile_one(src):
        obj = os.path.join(libdir, os.path.splitext(src)[0] + ".o")
        cmd = [nvcc, *flags, "-c", os.path.join(src_dir, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES) + 1) as ex:
        objs = list(ex.map(compile_one, SOURCES + [PROBE_SOURCE]))
    cudalib = os.path.join(_cuda_home(), "lib64")

    def link(out_path, objects, extra):
        tmp = out_path + ".tmp"
        cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objects, "-cudart", "static", *extra]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out_path)

    link(target, objs[:-1], [])
    link(os.path.join(libdir, "libqhd_probe.so"), objs[-1:], [])
    return target


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
