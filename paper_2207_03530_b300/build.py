"""Build the CUDA library libvmas.so in-tree for sm_103a with nvcc.

The host code is three translation units (the world and its step, the
packed ragged worlds, the surrogate); each compiles to an object in its own
nvcc process, in parallel, and one nvcc call links them.

With VMAS_CHECKED=1 in the environment the same sources build
libvmas_checked.so instead, with -DVMAS_CHECKED: every shared- and
global-memory index of the step kernels is checked on the device; an index
out of range is not used, sets bit 2 of the device error word (reported by
vmas_check as VMAS_EDEVICE) and records where it happened.  The binding
loads that library when the same variable is set, so
``VMAS_CHECKED=1 python -m pytest tests -m gpu`` runs the GPU suite on it.
"""
from __future__ import annotations

import glob
import os
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CHECKED = os.environ.get("VMAS_CHECKED") == "1"
LIB = os.path.join(PKG, "libvmas_checked.so" if CHECKED else "libvmas.so")
SOURCES = [os.path.join(PKG, "csrc", f) for f in ("vmas.cu", "ragged.cu", "surrogate_host.cu")]
NVCC_FLAGS = ["-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
              "-Xcompiler", "-fPIC"] + (["-DVMAS_CHECKED"] if CHECKED else [])


def _inputs():
    return SOURCES + glob.glob(os.path.join(PKG, "csrc", "*.cuh")) + \
        [os.path.join(PKG, "csrc", "host.h"), os.path.join(ROOT, "include", "vmas.h"), __file__]


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(p) > t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library (libvmas.so, or libvmas_checked.so with
    VMAS_CHECKED=1) unless it is up to date; returns its path."""
    if not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    tag = ".tmp%d" % os.getpid()
    objs = [LIB[:-3] + "_" + os.path.basename(src)[:-3] + tag + ".o" for src in SOURCES]
    procs = []
    try:
        for src, obj in zip(SOURCES, objs):
            cmd = [nvcc, *NVCC_FLAGS, "-I", os.path.join(ROOT, "include"), "-c", "-o", obj, src]
            if verbose:
                cmd.insert(1, "-Xptxas=-v")
            procs.append((cmd, subprocess.Popen(cmd)))
        for cmd, pr in procs:
            if pr.wait() != 0:
                raise subprocess.CalledProcessError(pr.returncode, cmd)
        tmp = LIB + tag
        subprocess.run([nvcc, "-shared", "-gencode", "arch=compute_103a,code=sm_103a",
                        "-o", tmp, *objs], check=True)
        os.replace(tmp, LIB)
    finally:
        for pr in procs:
            if pr[1].poll() is None:
                pr[1].kill()
                pr[1].wait()
        for obj in objs:
            if os.path.exists(obj):
                os.remove(obj)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
