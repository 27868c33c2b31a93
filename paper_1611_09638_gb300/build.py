"""Build librecon.so (the CUDA solver behind include/recon.h) in-tree for
sm_103a with nvcc: one object per translation unit, compiled in parallel,
then linked into a shared library next to this file.

build(checked=True) builds librecon_checked.so instead: the same library
compiled with -DRECON_CHECKED, whose kernels check their computed shared- and
global-memory offsets and report a failed check as a status (never a trap).
The package loads it in place of librecon.so when RECON_BUILD=checked is set
in the environment."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librecon.so")
LIB_CHECKED = os.path.join(HERE, "librecon_checked.so")
SOURCES = ["recon_api.cu", "mg_kernels.cu", "step_kernels.cu", "smoother.cu", "transfer.cu", "control.cu", "adjoint.cu", "noalloc.cu", "coarse_cluster.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(os.path.dirname(HERE), "include", "recon.h"))
    return max(os.path.getmtime(f) for f in files)


def lib_path(checked: bool = False) -> str:
    return LIB_CHECKED if checked else LIB


def build(force: bool = False, verbose: bool = False, extra=(), checked: bool = False) -> str:
    """Compile and link librecon.so (librecon_checked.so with checked) if any
    source is newer; return its path."""
    lib = lib_path(checked)
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps():
        return lib
    build_dir = os.path.join(BUILD, "checked") if checked else BUILD
    os.makedirs(build_dir, exist_ok=True)
    if checked:
        extra = tuple(extra) + ("-DRECON_CHECKED",)
    nvcc = _nvcc()
    procs, objs = [], []
    for src in SOURCES:
        obj = os.path.join(build_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    errs = []
    for src, pr in procs:
        out, _ = pr.communicate()
        if pr.returncode != 0:
            errs.append(f"{src}:\n{out.decode(errors='replace')}")
        elif verbose and out:
            print(out.decode(errors="replace"))
    if errs:
        raise RuntimeError("nvcc failed:\n" + "\n".join(errs))
    tmp = lib + f".tmp{os.getpid()}"
    subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose="-v" in sys.argv,
                extra=("-Xptxas", "-v") if "--ptxas" in sys.argv else ()))
