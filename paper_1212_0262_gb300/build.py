"""Build libmd.so (and libmdpeaks.so) in-tree for sm_103a with nvcc.

Translation units compile in parallel (one nvcc per .cu), then link into a
shared library next to this file.  No cmake, one -gencode.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INC = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INC, "-I", CSRC,
                "--expt-relaxed-constexpr"]

LIBS = {
    "libmd.so": ["api.cu", "hmf.cu", "pairs.cu", "sym.cu", "energy.cu", "ic.cu", "grad.cu", "tangent.cu", "batch.cu", "noalloc.cu", "shard.cu"],
    "libmdpeaks.so": ["peaks.cu"],
}


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _stale(target: str, deps: list[str]) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INC, f) for f in os.listdir(INC) if f.endswith(".h")]
    return hs


def build(verbose: bool = False, force: bool = False) -> dict[str, str]:
    """Compile every library; returns {name: path}."""
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = _headers()
    jobs = []
    for lib, srcs in LIBS.items():
        for s in srcs:
            src = os.path.join(CSRC, s)
            obj = os.path.join(BUILD, s.replace(".cu", ".o"))
            if force or _stale(obj, [src] + headers):
                jobs.append((src, obj))

    def compile_one(job):
        src, obj = job
        cmd = [nvcc] + FLAGS + ["-c", src, "-o", obj]
        if verbose:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stderr}")
        return src, r.stderr

    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for src, err in ex.map(compile_one, jobs):
            if verbose and err:
                sys.stderr.write(f"== {os.path.basename(src)}\n{err}")
    out = {}
    for lib, srcs in LIBS.items():
        objs = [os.path.join(BUILD, s.replace(".cu", ".o")) for s in srcs]
        target = os.path.join(PKG, lib)
        if force or _stale(target, objs):
            tmp = target + f".tmp{os.getpid()}"
            cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"link failed for {lib}:\n{r.stderr}")
            os.replace(tmp, target)
        out[lib] = target
    return out


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
