"""Build the FP64 CPU oracle (test infrastructure) into oracle/liborc.so.

Plain C11, compiled with -ffp-contract=off so that no multiply-add is fused
behind the source's back (the FP32 decision paths and the FP64 depth must
follow the written operation order exactly), and OpenMP for the loops over
chunks, views and rows (which does not change any arithmetic).
"""
import fcntl
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_geometry.c", "orc_gaussians.c", "orc_voxels.c", "orc_composite.c", "orc_filter.c"]
LIB = os.path.join(HERE, "liborc.so")


def _current() -> bool:
    srcs = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "lf_oracle.h")]
    return os.path.exists(LIB) and os.path.getmtime(LIB) >= max(os.path.getmtime(s) for s in srcs)


def build(force: bool = False) -> str:
    if not force and _current():
        return LIB
    # one build at a time when several processes start together
    with open(LIB + ".lock", "w") as lk:
        fcntl.flock(lk, fcntl.LOCK_EX)
        try:
            if not force and _current():
                return LIB
            return _build()
        finally:
            fcntl.flock(lk, fcntl.LOCK_UN)


def _build() -> str:
    cc = os.environ.get("CC", "gcc")
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = [cc, "-std=gnu11", "-O2", "-ffp-contract=off", "-fno-math-errno", "-fopenmp",
           "-shared", "-fPIC", "-Wall", "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
