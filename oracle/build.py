"""Builds the oracle's shared library (real FP64 + complex-step FP64 forms).

Plain gcc, no FMA contraction (so the x86 and Arm builds round alike), OpenMP
over cells for the CPU baseline.  Test infrastructure only.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "nlc_oracle.c")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "liboracle.so")

CFLAGS = ["-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math",
          "-fopenmp", "-fPIC", "-Wall"]


def build(force=False):
    """Compile liboracle.so if it is missing or older than its source."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    objs = []
    procs = []
    for tag, extra in (("real", []), ("cs", ["-DORC_COMPLEX"])):
        obj = os.path.join(LIBDIR, f"oracle_{tag}.o")
        objs.append(obj)
        procs.append(subprocess.Popen(["gcc", *CFLAGS, *extra, "-c", SRC,
                                       "-o", obj]))
    for p in procs:
        if p.wait() != 0:
            raise RuntimeError("oracle compile failed")
    tmp = LIB + ".tmp"
    subprocess.check_call(["gcc", "-shared", "-fopenmp", *objs, "-o", tmp,
                           "-lm"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
