"""Build step of the CUDA library: compiles csrc/*.cu for sm_103a into
lib/libreactflow.so (in-tree, so the shared object travels with the sources)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "lib", "libreactflow.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def deps():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC)) + [os.path.join(ROOT, "include", "reactflow.h")]


def up_to_date() -> bool:
    if not os.path.exists(OUT):
        return False
    t = os.path.getmtime(OUT)
    return all(os.path.getmtime(d) <= t for d in deps())


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and up_to_date():
        return OUT
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    # -fmad=true: multiply-add pairs contract into FMAs (the flux sweeps are issue-bound,
    # the FP64 path FP64-bound).  Kernels that inline the same device code (single-grid
    # and ensemble launches, chunked and whole cell-state launches) still round alike:
    # the tests compare them bit for bit.  ptxas compiles the kernels on all host cores.
    cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-fmad=true", "-std=c++17", "-shared", "-Xcompiler", "-fPIC",
           "-I", os.path.join(ROOT, "include"), "-I", CSRC, "--expt-relaxed-constexpr",
           "-cudart", "static", "-Xptxas", "--split-compile=0", *extra, *sources(), "-o", OUT + ".tmp"]
    if verbose:
        print(" ".join(cmd), flush=True)
    subprocess.run(cmd, check=True)
    os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    ex = [a for a in sys.argv[1:] if a not in ("-f", "-v")]
    print(build(force="-f" in sys.argv, verbose="-v" in sys.argv, extra=ex))
