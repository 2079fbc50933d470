"""Build step of the CUDA library: compiles ``csrc/*.cu`` for sm_103a with nvcc
(one translation unit per process, in parallel) and links
``_build/libebvisc.so`` in-tree."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libebvisc.so")
# Measurement variant: the same sources with the FP32 V-cycle reading FP32
# face coefficients instead of BF16 ones (only solvers.cu differs).
VARIANT_LIB = os.path.join(OUT, "libebvisc_fp32faces.so")
VARIANT_SRC = "solvers.cu"
VARIANT_DEFINE = "-DEBV_VCYCLE_FP32_FACES"
INCLUDE = os.path.join(ROOT, "include")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE]


def _nvcc():
    for cand in (os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"), "nvcc"):
        if os.path.sep not in cand or os.path.exists(cand):
            return cand
    return "nvcc"


def sources():
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cu"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "ebvisc.h"))
    nvcc = _nvcc()
    jobs = []
    objs = []
    for s in sources():
        o = os.path.join(OUT, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            jobs.append([nvcc] + ARCH + FLAGS + ["-c", s, "-o", o])
    vobj = os.path.join(OUT, "solvers_fp32faces.o")
    if force or _stale(vobj, [os.path.join(SRC, VARIANT_SRC)] + headers):
        jobs.append([nvcc] + ARCH + FLAGS + [VARIANT_DEFINE, "-c", os.path.join(SRC, VARIANT_SRC), "-o", vobj])
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        res = list(ex.map(lambda cmd: subprocess.run(cmd, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, res):
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: " + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
    vobjs = [vobj if os.path.basename(o) == "solvers.o" else o for o in objs]
    for lib, ob in ((LIB, objs), (VARIANT_LIB, vobjs)):
        if force or jobs or _stale(lib, ob):
            tmp = lib + f".{os.getpid()}.tmp"
            r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + ob, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("link failed\n" + r.stdout + r.stderr)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
