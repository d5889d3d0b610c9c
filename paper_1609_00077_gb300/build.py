"""Build the CUDA library in-tree: generate the site-algebra tables, then
compile csrc/ppq_capi.cu for sm_103a into libppq.so next to this file."""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libppq.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libppq.so")
    return exe


def generate_tables():
    sys.path.insert(0, os.path.dirname(HERE))
    from paper_1609_00077_gb300 import tables
    return tables.emit_header(os.path.join(CSRC, "ppq_tables.h"))


def build(verbose=False, extra=()):
    generate_tables()
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-Xptxas", "-v" if verbose else "-O3", *extra,
           "-o", LIB, os.path.join(CSRC, "ppq_capi.cu")]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stderr[-6000:])
    if verbose:
        print(res.stderr)
    return LIB


if __name__ == "__main__":
    build(verbose="-v" in sys.argv)
    print(LIB)
