"""Build step for the oracle's C part (TEST INFRASTRUCTURE ONLY).

Compiles ``fd_oracle.c`` with gcc into ``oracle/_build/liboracle_fd.so``.
Only tests/, ``__graft_entry__`` and bench.py's cpu_baseline leg use it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle_fd.so")
SRC = os.path.join(HERE, "fd_oracle.c")


def build(force=False):
    """Compile the oracle library if it is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fno-fast-math", "-fopenmp", "-shared", "-fPIC",
           "-o", tmp, SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
