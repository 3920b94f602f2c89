"""Compile the oracle's C solver (``csolve.c``) into ``oracle/libsgo.so`` with gcc and OpenMP.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

    python -m oracle.cbuild
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csolve.c")
LIB = os.path.join(HERE, "libsgo.so")


def build(force=False):
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    cc = os.environ.get("CC", "gcc")
    cmd = [cc, "-O2", "-fopenmp", "-std=c99", "-shared", "-fPIC", SRC, "-o", LIB, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle C build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
