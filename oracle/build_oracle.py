"""Build the oracle's C library (test infrastructure only).

`python oracle/build_oracle.py` compiles zfp_oracle.c with the host C compiler
into oracle/libzfporacle.so.  Plain C99, no architecture-specific flags, so
the same source builds on x86_64 and aarch64 hosts.  The library is rebuilt
unless a stamp beside it records the same hash of the source, the command and
the host machine.
"""
import hashlib
import os
import platform
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "zfp_oracle.c")
LIB = os.path.join(HERE, "libzfporacle.so")


STAMP = LIB + ".sha256"


def build(force: bool = False) -> str:
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [cc, "-std=c99", "-O2", "-fPIC", "-shared", "-fno-fast-math",
           "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    h = hashlib.sha256(open(SRC, "rb").read())
    h.update(" ".join(cmd[:1] + cmd[2:-4]).encode() + platform.machine().encode())
    digest = h.hexdigest()
    if (not force and os.path.exists(LIB) and os.path.exists(STAMP)
            and open(STAMP).read().strip() == digest):
        return LIB
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    with open(STAMP, "w") as f:
        f.write(digest + "\n")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
