"""Builds the in-tree shared library libspeedup_gb300.so with nvcc (sm_103a).

The translation units are compiled in parallel and linked with the static
CUDA runtime; the result lands in ``paper_1105_0542_gb300/_lib/`` (ignored by
git), objects in ``paper_1105_0542_gb300/_build/``.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libspeedup_gb300.so")
CLI = os.path.join(LIBDIR, "speedup")
SOURCES = ["sampler.cu", "api.cu", "generator.cpp", "peaks.cu", "proposal.cu", "train.cu", "evolution.cu", "nd.cu", "spectrum.cu"]
# the sampler kernel, once per (precision, ring): compiled in parallel
INSTANCES = [(prec, ring, 0) for prec in (64, 32) for ring in (0, 1, 2)] + [(64, 3, 0)]
# double-precision samplers that read tables too large for shared memory from global memory
INSTANCES += [(64, ring, 1) for ring in (0, 1, 2)]
# single-precision even-ring samplers and batched kernels with the table
# shapes of fixed_shapes.h compiled in, spread over eight units (kFixedGroups)
FIXED_GROUPS = 8
HEADERS = ["sampler.h", "generator.h", "sampler_impl.cuh", "sampler_inst.cu", "boxmuller.cuh", "mlp.cuh",
           "proposal.h", "train.h", "philox.cuh", "spectrum.h", "erf_poly.h", "fixed_shapes.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return path


def _inputs():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    files.append(os.path.join(ROOT, "include", "speedup.h"))
    files.append(os.path.join(CSRC, "speedup_cli.c"))
    files.append(os.path.abspath(__file__))
    return files


def up_to_date():
    if not os.path.exists(LIB) or not os.path.exists(CLI):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(f) <= t for f in _inputs())


def _compile(job, verbose):
    src, defs = job
    tag = "".join(f"_{v}" for v in defs.values())
    obj = os.path.join(BUILD, os.path.basename(src) + tag + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-c", src, "-o", obj,
           "-Xcompiler", "-fPIC,-ffp-contract=off", "-I", os.path.join(ROOT, "include")]
    cmd += [f"-D{k}={v}" for k, v in defs.items()]
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-v"] if verbose else []
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, r.stderr


def build(force=False, verbose=False):
    """Compile and link; returns the library path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    jobs = [(os.path.join(CSRC, "sampler_inst.cu"), {"SU_PREC": p, "SU_RING": r, "SU_GTAB": g})
            for p, r, g in INSTANCES]
    jobs += [(os.path.join(CSRC, "sampler_inst.cu"), {"SU_FIXED": g}) for g in range(FIXED_GROUPS)]
    jobs += [(os.path.join(CSRC, f), {}) for f in SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        results = list(ex.map(lambda j: _compile(j, verbose), jobs))
    if verbose:
        for _, log in results:
            if log:
                print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp] + [o for o, _ in results]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    # the command-line front end, plain C over the C ABI, beside the library
    cli = [os.environ.get("CC", "gcc"), "-O2", "-std=c11", "-Wall", "-I", os.path.join(ROOT, "include"),
           os.path.join(CSRC, "speedup_cli.c"), "-o", CLI + f".tmp{os.getpid()}", "-L", LIBDIR, "-lspeedup_gb300",
           "-Wl,-rpath,$ORIGIN"]
    r = subprocess.run(cli, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"cli build failed:\n{r.stdout}\n{r.stderr}")
    os.replace(CLI + f".tmp{os.getpid()}", CLI)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
