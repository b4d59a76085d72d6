"""Build the FP64 CPU oracle (test infrastructure) into oracle/_build/liboracle.so.

Plain gcc, no fused multiply-add (-ffp-contract=off), so every operation of the
canonical distance is an IEEE round-to-nearest double operation on x86-64 and
aarch64 alike.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "liboracle.so")
SRCS = [os.path.join(HERE, "grng_oracle.c"), os.path.join(HERE, "mlp_oracle.c"), os.path.join(HERE, "guided_oracle.c")]


def build(force: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    srcs = [s for s in SRCS if os.path.exists(s)]
    newest = max(os.path.getmtime(s) for s in srcs)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-o", LIB + ".tmp"] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
