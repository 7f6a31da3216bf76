"""Build the CUDA library libspgemm_predict.so in-tree for GB300 (sm_103a).

One translation unit (csrc/api.cu includes the kernel headers), compiled by
nvcc with the CUDA runtime linked statically, so the library depends only on
the driver at run time.  The output goes to ``lib/`` next to this file.
"""
import os
import pathlib
import shutil
import subprocess
import tempfile

HERE = pathlib.Path(__file__).resolve().parent
ROOT = HERE.parent
CSRC = HERE / "csrc"
HEADER = ROOT / "include" / "spgemm_predict.h"
LIBDIR = HERE / "lib"
LIB = LIBDIR / "libspgemm_predict.so"
ARCH = "arch=compute_103a,code=sm_103a"


def nvcc_path():
    p = shutil.which("nvcc")
    if p:
        return p
    for cand in ("/usr/local/cuda/bin/nvcc",):
        if os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def sources():
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cuh")) + [HEADER]


def up_to_date():
    if not LIB.exists():
        return False
    t = LIB.stat().st_mtime
    return all(s.stat().st_mtime <= t for s in sources())


def build(force=False, verbose=False, extra_flags=()):
    """Compile the library unless it is newer than every source; returns its path."""
    if not force and up_to_date():
        return LIB
    LIBDIR.mkdir(exist_ok=True)
    fd, tmp = tempfile.mkstemp(prefix=".libspgemm.", suffix=".so", dir=str(LIBDIR))
    os.close(fd)
    cmd = [nvcc_path(), "-shared", "-Xcompiler", "-fPIC", "-gencode", ARCH, "-O3", "-lineinfo",
           "-std=c++17", *extra_flags, str(CSRC / "api.cu"), "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        os.unlink(tmp)
        raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    if verbose:
        print(r.stdout + r.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
