"""Build the CUDA library ``libfdtd_llg.so`` in-tree for sm_103a with nvcc."""
from __future__ import annotations

import glob
import hashlib
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libfdtd_llg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
    return sorted(deps + glob.glob(os.path.join(ROOT, "include", "*.h")))


def sources_hash() -> str:
    """sha1 over the library's sources and headers (names and contents)."""
    h = hashlib.sha1()
    for d in _deps():
        h.update(os.path.relpath(d, ROOT).encode())
        with open(d, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def stale() -> bool:
    """True when the library is missing or was built from other sources than
    the present ones (recorded beside it at build time; file times are not
    trusted, they do not survive copies of the tree)."""
    try:
        with open(LIB + ".sha1") as f:
            return f.read().strip() != sources_hash() or not os.path.exists(LIB)
    except OSError:
        return True


_stale = stale


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-shared",
           "-o", LIB + ".tmp", *sources(), "-I", os.path.join(ROOT, "include")]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    with open(LIB + ".sha1", "w") as f:
        f.write(sources_hash() + "\n")
    return LIB


if __name__ == "__main__":
    import sys

    print(build(force="-f" in sys.argv, verbose="-v" in sys.argv))
