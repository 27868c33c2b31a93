"""Build the CPU FP64 oracle shared library (test infrastructure only).

The oracle is plain C99 compiled with gcc; floating-point contraction is off so
that x86_64 and aarch64 hosts round every operation the same way.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "librecon_oracle.so")
SRC = os.path.join(HERE, "recon_oracle.c")


def build(force: bool = False) -> str:
    """Compile recon_oracle.c into librecon_oracle.so next to it; return the path."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "recon_oracle.h"))
    ):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-ffp-contract=off",
           "-fPIC", "-shared", "-o", tmp, SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
