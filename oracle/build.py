"""Compile the C oracle into ``oracle/liboracle.so`` with gcc.

The oracle is test infrastructure: this builds the checker, it does not put
the oracle on any product path. Floating-point contraction is switched off so
that the x86 and Arm builds round identically.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["oracle_core.c", "oracle_split.c", "oracle_sai.c", "oracle_krylov.c", "oracle_smw.c", "oracle_backward.c",
           "oracle_perm.c", "oracle_block.c"]
LIB = os.path.join(HERE, "liboracle.so")


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = SOURCES + ["oracle.h", "oracle_internal.h"]
    return any(os.path.getmtime(os.path.join(HERE, f)) > t for f in deps)


def build_oracle(force=False, verbose=False):
    """Build liboracle.so if missing or older than its sources; return its path."""
    if not force and not _stale():
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-Wall", "-Wno-unused-function", "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    if verbose:
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv, verbose=True))
