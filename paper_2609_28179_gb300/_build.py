"""Build libglass.so (sm_103a) in-tree: one nvcc process per translation
unit, in parallel, then one link.  Re-runs only what changed."""
from __future__ import annotations

import concurrent.futures as cf
import glob
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libglass.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libglass.so")


def _headers_digest() -> str:
    h = hashlib.sha1()
    for p in sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) +
                    [os.path.join(ROOT, "include", "glass.h")]):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _obj(src: str, digest: str, extra: list[str]) -> str:
    with open(src, "rb") as f:
        h = hashlib.sha1(f.read() + digest.encode() + " ".join(extra).encode()).hexdigest()[:16]
    return os.path.join(BUILD, os.path.basename(src)[:-3] + "." + h + ".o")


def _compile(src: str, obj: str, extra: list[str], verbose: bool) -> str:
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", obj + ".tmp"]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    os.replace(obj + ".tmp", obj)
    return r.stderr


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, jobs: int | None = None) -> str:
    """Compile every csrc/*.cu for sm_103a and link libglass.so; returns its path."""
    extra = list(extra or [])
    os.makedirs(BUILD, exist_ok=True)
    digest = _headers_digest()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")))
    objs = [_obj(s, digest, extra) for s in srcs]
    todo = [(s, o) for s, o in zip(srcs, objs) if force or not os.path.exists(o)]
    logs = {}
    if todo:
        jobs = jobs or min(len(todo), max(1, os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = {ex.submit(_compile, s, o, extra, verbose): s for s, o in todo}
            for f in cf.as_completed(futs):
                logs[futs[f]] = f.result()
    stamp = LIB + ".inputs"
    want = "\n".join(objs)
    have = open(stamp).read() if os.path.exists(stamp) else ""
    if todo or force or have != want or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        with open(stamp, "w") as f:
            f.write(want)
    # drop objects of earlier source versions
    keep = set(objs)
    for stale in glob.glob(os.path.join(BUILD, "*.o")):
        if stale not in keep:
            try:
                os.remove(stale)
            except OSError:
                pass
    if verbose:
        for s, log in sorted(logs.items()):
            sys.stderr.write(f"== {os.path.basename(s)}\n{log}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
