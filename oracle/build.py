"""Build the oracle shared library (plain C, FP64) with gcc.

Test infrastructure only.  OpenMP is used when the compiler supports it; the
ion-ion loop keeps a fixed per-target order, so results do not depend on it.
"""
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")


def _openmp_ok(cc):
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "t.c")
        with open(src, "w") as f:
            f.write("#include <omp.h>\nint main(void){return omp_get_max_threads()>0?0:1;}\n")
        r = subprocess.run([cc, "-fopenmp", src, "-o", os.path.join(td, "t")], capture_output=True)
        return r.returncode == 0


def build(force=False, openmp=True):
    src = os.path.join(HERE, "oracle.c")
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(src), os.path.getmtime(os.path.join(HERE, "oracle.h"))
    ):
        return LIB
    cc = os.environ.get("CC", "gcc")
    # -ffp-contract=off: no fused multiply-add, so every operation rounds once as written
    flags = ["-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    if openmp and _openmp_ok(cc):
        flags.append("-fopenmp")
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [cc] + flags + [src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
