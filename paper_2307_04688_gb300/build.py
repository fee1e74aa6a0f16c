"""Build libcheb.so in-tree with nvcc for sm_103a (no cmake, parallel compile).

The same sources also build libcheb_check.so, the checked build (-DCHEB_CHECK:
device bounds checks that report CHEB_EBOUNDS instead of trapping); both
variants compile in one parallel batch."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libcheb.so")
BUILD_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libcheb_check.so")
INCLUDE = os.path.join(ROOT, "include")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-lineinfo",
              "-Xcompiler", "-fPIC,-fvisibility=hidden", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(target: str, deps) -> bool:
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, check: bool = True) -> str:
    """Compile every .cu under csrc/ (in parallel) and link libcheb.so, and with
    `check` also libcheb_check.so from the same sources with -DCHEB_CHECK."""
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "cheb.h"))
    nvcc = _nvcc()
    variants = [(BUILD, LIB, [])]
    if check:
        variants.append((BUILD_CHECK, LIB_CHECK, ["-DCHEB_CHECK"]))
    procs, links = [], []
    for bdir, lib, extra in variants:
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for src in sources():
            obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            if force or _stale(obj, [src] + headers):
                cmd = [nvcc] + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
                if verbose:
                    print(" ".join(cmd), file=sys.stderr)
                procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        links.append((lib, objs))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out.decode(errors="replace")))
        elif verbose and out:
            print(out.decode(errors="replace"), file=sys.stderr)
    if failed:
        msg = "\n".join(f"--- {s}\n{o}" for s, o in failed)
        raise RuntimeError("nvcc failed:\n" + msg)
    for lib, objs in links:
        if force or _stale(lib, objs):
            cmd = [nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a", "-o", lib] + objs + ["-ldl"]
            subprocess.check_call(cmd)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
