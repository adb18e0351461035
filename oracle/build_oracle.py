"""Build the oracle's C library (test infrastructure only).

`python oracle/build_oracle.py` compiles zfp_oracle.c with the host C compiler
into oracle/libzfporacle.so.  Plain C99, no architecture-specific flags, so
the same source builds on x86_64 and aarch64 hosts.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "zfp_oracle.c")
LIB = os.path.join(HERE, "libzfporacle.so")


def build(force: bool = False) -> str:
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [cc, "-std=c99", "-O2", "-fPIC", "-shared", "-fno-fast-math",
           "-Wall", "-Wextra", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
