"""In-tree build of the package's native parts.

* ``libbcm.so``     -- the CUDA library behind the C-ABI in ``include/bcm.h``
                       (sm_103a only, built with nvcc).
* ``libbcmgen.so``  -- the seeded graph generators (plain C, host only).

Both land in ``paper_1507_01490_gb300/_lib/``.  A library is rebuilt when any
of its sources is newer than the built file.  Compilation happens on the
machine that runs the code (the GPU host is AArch64, this one may be x86-64),
so nothing built here is assumed to run elsewhere.
"""
from __future__ import annotations

import os
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

PKG_DIR = os.path.dirname(os.path.abspath(__file__))
REPO_DIR = os.path.dirname(PKG_DIR)
LIB_DIR = os.path.join(PKG_DIR, "_lib")
CSRC_DIR = os.path.join(PKG_DIR, "csrc")
GEN_DIR = os.path.join(PKG_DIR, "gen")
INCLUDE_DIR = os.path.join(REPO_DIR, "include")

NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a"]

_lock = threading.Lock()


def _newer(target: str, sources: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _run(cmd: list[str]) -> None:
    res = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if res.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(cmd) + "\n" + res.stdout)


def cuda_sources() -> list[str]:
    return sorted(os.path.join(CSRC_DIR, f) for f in os.listdir(CSRC_DIR) if f.endswith(".cu"))


def cuda_headers() -> list[str]:
    hs = [os.path.join(CSRC_DIR, f) for f in os.listdir(CSRC_DIR) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE_DIR, f) for f in os.listdir(INCLUDE_DIR) if f.endswith(".h")]
    return sorted(hs)


def build_gen(force: bool = False) -> str:
    src = os.path.join(GEN_DIR, "graphgen.c")
    out = os.path.join(LIB_DIR, "libbcmgen.so")
    with _lock:
        os.makedirs(LIB_DIR, exist_ok=True)
        if force or _newer(out, [src]):
            tmp = out + ".tmp%d" % os.getpid()
            _run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                  "-Wall", "-o", tmp, src, "-lm"])
            os.replace(tmp, out)
    return out


def build_cuda(force: bool = False, verbose_ptxas: bool = False) -> str:
    """Compile every .cu under csrc/ for sm_103a (in parallel) and link libbcm.so."""
    out = os.path.join(LIB_DIR, "libbcm.so")
    srcs = cuda_sources()
    deps = srcs + cuda_headers()
    with _lock:
        os.makedirs(LIB_DIR, exist_ok=True)
        if not (force or _newer(out, deps)):
            return out
        objs = []
        cmds = []
        for s in srcs:
            o = os.path.join(LIB_DIR, os.path.basename(s)[:-3] + ".o")
            objs.append(o)
            cmd = [NVCC, *ARCH_FLAGS, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I", INCLUDE_DIR, "-I", CSRC_DIR, "-c", s, "-o", o]
            if verbose_ptxas:
                cmd += ["-Xptxas", "-v"]
            cmds.append(cmd)
        with ThreadPoolExecutor(max_workers=min(8, len(cmds))) as ex:
            for f in [ex.submit(_run, c) for c in cmds]:
                f.result()
        tmp = out + ".tmp%d" % os.getpid()
        _run([NVCC, *ARCH_FLAGS, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, out)
    return out


def build_all(force: bool = False) -> dict:
    return {"gen": build_gen(force), "cuda": build_cuda(force)}


if __name__ == "__main__":
    print(build_all(force="--force" in sys.argv))
