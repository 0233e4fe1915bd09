"""Compile the oracle's C part (binary128 Legendre recurrence) with gcc.

TEST INFRASTRUCTURE: builds the checker, not the product.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "pnm_binary128.c")
LIB = os.path.join(HERE, "_pnm_binary128.so")


def build(force: bool = False) -> str:
    """Compile ``pnm_binary128.c`` to ``_pnm_binary128.so`` if it is stale."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-Wall", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
