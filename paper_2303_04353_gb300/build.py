"""Build libddgemm (the CUDA kernels and the C ABI of include/ddgemm.h) in
tree, for sm_103a only.  Translation units compile in parallel; the result
is paper_2303_04353_gb300/_build/libddgemm_<machine>.so."""
from __future__ import annotations

import glob
import os
import platform
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
SOURCES = ["api.cu", "split.cu", "cascade_fp64.cu", "probe.cu", "noalloc.cu", "split_int8.cu",
           "cascade_int8.cu", "cascade_int8_tc.cu", "cascade_int8_tc8.cu", "batched.cu",
           "batched_int8_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
                     "-I" + INCLUDE, "-I" + CSRC]


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA 13 toolkit is required to build libddgemm")
    return path


def lib_path() -> str:
    return os.path.join(OUT_DIR, f"libddgemm_{platform.machine()}.so")


def _inputs():
    return ([os.path.join(CSRC, s) for s in SOURCES] + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def up_to_date() -> bool:
    out = lib_path()
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(p) <= t for p in _inputs())


def build(force: bool = False, verbose: bool = False) -> str:
    out = lib_path()
    if not force and up_to_date():
        return out
    os.makedirs(OUT_DIR, exist_ok=True)
    tag = f"{platform.machine()}.{os.getpid()}"
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, f"{os.path.splitext(src)[0]}.{tag}.o")
        cmd = [nvcc()] + NVCC_FLAGS + ["-c", os.path.join(CSRC, src), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for src, p in procs:
        log = p.communicate()[0].decode(errors="replace")
        if p.returncode != 0:
            failed.append(f"{src}:\n{log}")
        elif verbose and log.strip():
            print(log)
    if failed:
        raise RuntimeError("nvcc failed\n" + "\n".join(failed))
    tmp = out + f".{tag}.tmp"
    subprocess.run([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs, check=True)
    os.replace(tmp, out)
    for o in objs:
        os.remove(o)
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
