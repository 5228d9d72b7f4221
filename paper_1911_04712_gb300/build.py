"""Build libdpd.so in-tree for sm_103a (nvcc, one -gencode, parallel objects)."""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdpd.so")
PHILOX_ROUNDS = 10  # the noise generator's round count (Philox-4x32-10)


def lib_path(philox_rounds: int = PHILOX_ROUNDS, checked: bool = False) -> str:
    """The library file.  Other round counts (for a round-count study) and the
    checked build (kernels test their derived indices, see DPD_IN_BOUNDS)
    build beside it."""
    name = "libdpd"
    if philox_rounds != PHILOX_ROUNDS:
        name += f"_r{philox_rounds}"
    if checked:
        name += "_checked"
    return os.path.join(HERE, name + ".so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _headers() -> list[str]:
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "dpd.h"))
    return hs


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None,
          philox_rounds: int = PHILOX_ROUNDS, checked: bool = False) -> str:
    nvcc = _nvcc()
    if not 1 <= philox_rounds <= 16:
        raise ValueError("Philox round count must be 1..16")
    lib = lib_path(philox_rounds, checked)
    bdir = BUILD if philox_rounds == PHILOX_ROUNDS else BUILD + f"_r{philox_rounds}"
    if checked:
        bdir += "_checked"
    os.makedirs(bdir, exist_ok=True)
    flags = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2,-fvisibility=hidden",
                    "-I", os.path.join(ROOT, "include"), "-I", CSRC]
    if philox_rounds != PHILOX_ROUNDS:
        flags += [f"-DDPD_PHILOX_ROUNDS={philox_rounds}"]
    if checked:
        flags += ["-DDPD_CHECKED=1"]
    if extra:
        flags += extra
    if verbose:
        flags += ["-Xptxas", "-v"]
    hdrs = _headers()
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            jobs.append([nvcc] + flags + ["-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed: {' '.join(cmd)}")
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static", "-lrt", "-ldl",
                                                              "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    rounds = PHILOX_ROUNDS
    if "--philox-rounds" in sys.argv:
        rounds = int(sys.argv[sys.argv.index("--philox-rounds") + 1])
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, philox_rounds=rounds,
                checked="--checked" in sys.argv))
