"""Build the CPU FP64 oracle shared library (test infrastructure only).

The oracle is plain C99 compiled with gcc; floating-point contraction is off so
that x86_64 and aarch64 hosts round every operation the same way.  It is built
with OpenMP where gcc supports it (the threaded loops give the same bits as the
serial ones), else single-threaded.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "librecon_oracle.so")
SRC = os.path.join(HERE, "recon_oracle.c")
BASE = ["gcc", "-O2", "-std=c99", "-Wall", "-Wextra", "-ffp-contract=off", "-fPIC", "-shared"]


def build(force: bool = False, openmp: bool = True, out: str = LIB) -> str:
    """Compile recon_oracle.c into a shared library (librecon_oracle.so next to
    it by default); return the path."""
    if not force and out == LIB and os.path.exists(LIB) and os.path.getmtime(LIB) >= max(
        os.path.getmtime(SRC), os.path.getmtime(os.path.join(HERE, "recon_oracle.h")),
        os.path.getmtime(os.path.abspath(__file__))
    ):
        return out
    tmp = out + f".tmp{os.getpid()}"
    flags = [["-fopenmp"], []] if openmp else [[]]
    for extra in flags:
        r = subprocess.run([*BASE, *extra, "-o", tmp, SRC, "-lm"], capture_output=True, text=True)
        if r.returncode == 0:
            break
    else:
        raise RuntimeError("gcc failed to build the oracle:\n" + r.stderr)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force=True))
