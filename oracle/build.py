"""Compile the CPU oracle (oracle.c) into liboracle.so next to this file.

Test infrastructure: builds the checker, not the product.  Plain gcc, no
architecture-specific flags, so the same source builds on x86-64 and aarch64.
OpenMP is used when the compiler supports it.
"""
import os
import pathlib
import subprocess
import tempfile

HERE = pathlib.Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
LIB = HERE / "liboracle.so"


def _compile(extra):
    # Compile to a temporary name and rename, so a concurrent reader never sees
    # a half-written library.
    fd, tmp = tempfile.mkstemp(prefix=".liboracle.", suffix=".so", dir=str(HERE))
    os.close(fd)
    cmd = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *extra, str(SRC), "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        os.unlink(tmp)
        return False, r.stderr
    os.replace(tmp, LIB)
    return True, ""


def build(force=False):
    """Build liboracle.so if it is missing or older than oracle.c."""
    if not force and LIB.exists() and LIB.stat().st_mtime >= SRC.stat().st_mtime:
        return LIB
    ok, err = _compile(["-fopenmp"])
    if not ok:
        ok, err2 = _compile([])
        if not ok:
            raise RuntimeError("oracle build failed:\n" + err + "\n" + err2)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
