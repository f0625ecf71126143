"""Compile the oracle's C numerics into a shared library next to this file.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain gcc, -O2, no
architecture-specific flags, so the same source builds on x86_64 and aarch64.
"""
import os
import subprocess
import sys
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc", "oracle_linalg.c")
LIB = os.path.join(HERE, "liboracle_linalg.so")
_LOCK = threading.Lock()  # threads of one process that load the oracle at once build it once


def build(force: bool = False) -> str:
    with _LOCK:
        if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
            return LIB
        tmp = LIB + f".{os.getpid()}.{threading.get_ident()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
