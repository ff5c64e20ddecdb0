"""Compile the C oracle into oracle/liboracle.so (gcc, no GPU needed).

Test infrastructure: builds the checker, never the product.
"""
import fcntl
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["darts_oracle.c"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["darts_oracle.h"]
    return any(os.path.getmtime(os.path.join(HERE, s)) > t for s in deps)


def build(force: bool = False) -> str:
    if not (force or _stale()):
        return LIB
    # one builder at a time (ranks of a multi-process launch build together)
    with open(os.path.join(HERE, ".build.lock"), "w") as lock:
        fcntl.flock(lock, fcntl.LOCK_EX)
        if force or _stale():
            cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-pthread",
                   "-Wall", "-o", LIB + ".tmp"] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
            subprocess.run(cmd, check=True)
            os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
