"""Build libdecolor.so (the C ABI of include/decolor.h) for sm_103a with nvcc.

Translation units compile in parallel (one per input sample type plus the host
ABI); objects go to ``_build/`` next to this file and the shared library to
``libdecolor.so``.  Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OBJDIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdecolor.so")
SOURCES = ["dc_engine_u8.cu", "dc_engine_f16.cu", "dc_engine_f32.cu", "dc_abi.cu", "dc_noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
_lock = threading.Lock()


def nvcc_path() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdecolor.so")


def _deps() -> list[str]:
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(CSRC, "*.h")) + [os.path.join(ROOT, "include", "decolor.h"), __file__])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          lib_path: str | None = None, obj_dir: str | None = None) -> str:
    """Compile and link libdecolor.so (or `lib_path`); returns its path.  Raises on
    compiler errors.  `extra_flags` go to every nvcc compile (e.g. -D options)."""
    lib = lib_path or LIB
    objdir = obj_dir or OBJDIR
    with _lock:
        if not force and lib_path is None and up_to_date():
            return LIB
        nvcc = nvcc_path()
        os.makedirs(objdir, exist_ok=True)
        flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                        "-I", os.path.join(ROOT, "include")] + list(extra_flags or [])
        procs = []
        for src in SOURCES:
            obj = os.path.join(objdir, src.replace(".cu", ".o"))
            cmd = [nvcc] + flags + ["-c", os.path.join(CSRC, src), "-o", obj]
            procs.append((cmd, obj, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs, errors = [], []
        for cmd, obj, pr in procs:
            out, _ = pr.communicate()
            if verbose and out:
                print(out.decode(errors="replace"))
            if pr.returncode != 0:
                errors.append(" ".join(cmd) + "\n" + out.decode(errors="replace"))
            objs.append(obj)
        if errors:
            raise RuntimeError("nvcc failed:\n" + "\n".join(errors))
        tmp = lib + ".tmp%d" % os.getpid()
        link = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
            "-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        res = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n" + " ".join(link) + "\n" + res.stdout.decode(errors="replace"))
        os.replace(tmp, lib)
        return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
