"""Build the oracle's plain-C helper (oracle/c/*.c -> oracle/liboracle.so) with gcc.

TEST INFRASTRUCTURE ONLY (see the package header)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "liboracle.so")


def build(force=False):
    srcs = [os.path.join(HERE, "c", f) for f in sorted(os.listdir(os.path.join(HERE, "c"))) if f.endswith(".c")]
    if not force and os.path.exists(LIB) and all(os.path.getmtime(s) <= os.path.getmtime(LIB) for s in srcs):
        return LIB
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", LIB + ".tmp", *srcs, "-lm"], check=True)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
