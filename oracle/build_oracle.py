"""Compile the C oracle into ``oracle/liboracle.so`` (test infrastructure).

Plain gcc, FP64, ``-O2 -ffp-contract=off`` so that no multiply-add is fused
and the oracle's rounding follows its source line by line.  Builds on x86-64
and aarch64 alike (no target-specific flags).
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, "cp_oracle.c"), os.path.join(HERE, "or_mlp.c")]
HDR = os.path.join(HERE, "cp_oracle.h")
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    newest = max(os.path.getmtime(f) for f in SRCS + [HDR])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11", "-fPIC",
           "-shared", "-Wall", "-o", tmp, *SRCS, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
