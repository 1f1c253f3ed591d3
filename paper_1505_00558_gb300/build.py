"""Builds libtsqs.so in-tree with nvcc for sm_103a (a few translation units compiled
in parallel, then linked against the shared CUDA runtime)."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libtsqs.so")

SOURCES = ["tsqs_common.cu", "tsqs_k4.cu", "tsqs_k8.cu", "tsqs_k16.cu", "tsqs_host.cu",
           "tsqs_autotune.cu", "tsqs_server.cu", "tsqs_noalloc.cu", "tsqs_wide.cu"]
EXTRA: list[str] = []


def _cuda_home() -> str:
    for c in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if c and os.path.exists(os.path.join(c, "bin", "nvcc")):
            return c
    return "/usr/local/cuda"


def nvcc_flags() -> list[str]:
    return ["-std=c++17", "-O3", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
            "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _sources() -> list[str]:
    return SOURCES + [s for s in EXTRA if os.path.exists(os.path.join(CSRC, s))]


def _deps() -> list[str]:
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "tsqs.h")]


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = os.path.join(_cuda_home(), "bin", "nvcc")
    headers = [d for d in _deps() if d.endswith((".h", ".cuh"))]
    jobs = []
    objs = []
    for src in _sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src + ".o")
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [nvcc] + nvcc_flags() + (extra_flags or []) + ["-c", s, "-o", o]
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed:\n{' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with ThreadPoolExecutor(max_workers=min(8, max(1, len(jobs)))) as ex:
        for err in ex.map(run, jobs):
            if verbose and err:
                print(err, file=sys.stderr)
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + f".tmp{os.getpid()}"
        cudalib = os.path.join(_cuda_home(), "lib64")
        run([nvcc, "-shared", "-o", tmp] + objs +
            ["-cudart", "shared", "-Xlinker", f"-rpath,{cudalib}", "-lpthread"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
