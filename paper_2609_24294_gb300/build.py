"""Build libzfpx.so in-tree with nvcc for sm_103a.

Each translation unit is compiled in parallel to an object file, then linked
into ``paper_2609_24294_gb300/libzfpx.so``.  The library is rebuilt unless a
stamp beside it records the same hash of every source and header, the compiler
flags, the nvcc version and the host machine (a library compiled on another
machine, or from other sources, is never reused).  One line on stderr says
whether it compiled.  ``python -m paper_2609_24294_gb300.build`` does the same
from the command line.
"""
import glob
import hashlib
import os
import platform
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
ROOT = os.path.dirname(PKG)
LIB = os.path.join(PKG, "libzfpx.so")
BUILD = os.path.join(PKG, "_build")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fvisibility=hidden",
         "-I", os.path.join(ROOT, "include")]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "zfpx.h"), os.path.abspath(__file__)]


STAMP = LIB + ".sha256"


def _nvcc_version(nvcc):
    try:
        return subprocess.run([nvcc, "--version"], capture_output=True, text=True).stdout
    except OSError:
        return "nvcc not found"


def source_hash(nvcc=None):
    """Hash of everything the library is built from, and of where it is built."""
    nvcc = nvcc or _nvcc()
    h = hashlib.sha256()
    for d in sorted(_deps()):
        h.update(os.path.relpath(d, ROOT).encode() + b"\0")
        h.update(open(d, "rb").read())
    h.update(" ".join(ARCH + FLAGS[:-1]).encode())
    h.update(_nvcc_version(nvcc).encode())
    h.update(platform.machine().encode())
    return h.hexdigest()


def up_to_date(digest=None):
    if not (os.path.exists(LIB) and os.path.exists(STAMP)):
        return False
    try:
        return open(STAMP).read().strip() == (digest or source_hash())
    except OSError:
        return False


def build(force=False, verbose=False):
    nvcc = _nvcc()
    digest = source_hash(nvcc)
    if not force and up_to_date(digest):
        sys.stderr.write("libzfpx: up to date (sources sha256 %s, %s)\n" % (digest[:12], platform.machine()))
        return LIB
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + FLAGS + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and r.stderr:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(digest + "\n")
    sys.stderr.write("libzfpx: compiled %d translation units for sm_103a (sources sha256 %s, %s)\n"
                     % (len(objs), digest[:12], platform.machine()))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
