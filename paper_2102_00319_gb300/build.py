"""Builds libhecnn.so in-tree with nvcc for sm_103a (no torch types involved).

Each translation unit compiles in parallel; the host file is compiled with
-ffp-contract=off so its double arithmetic is the plain IEEE one on every
host architecture.
"""
import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhecnn.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"
SOURCES = ["hc_ntt.cu", "hc_kernels.cu", "hc_api.cu", "hc_noalloc.cu", "hc_probe.cu", "hc_host.cpp"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhecnn")
    return cand


def _compile(src, obj):
    common = ["-O3", "-std=c++17", "-I" + os.path.join(ROOT, "include"), "-I" + CSRC,
              "-Xcompiler", "-fPIC,-ffp-contract=off"]
    cmd = [_nvcc(), ARCH, "-lineinfo", "-c", src, "-o", obj] + common
    if src.endswith(".cu"):
        cmd += ["-Xptxas", "-O3"]
    else:
        cmd += ["-x", "c++"]
    subprocess.check_call(cmd)


def build(force=False, verbose=False):
    os.makedirs(OUT, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    headers = [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith((".h", ".cuh"))]
    headers.append(os.path.join(ROOT, "include", "hecnn.h"))
    newest = max(os.path.getmtime(f) for f in srcs + headers + [__file__])
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= newest:
        return LIB
    objs = [os.path.join(OUT, os.path.basename(s) + ".o") for s in srcs]
    with concurrent.futures.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        list(ex.map(lambda a: _compile(*a), zip(srcs, objs)))
    tmp = LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call([_nvcc(), ARCH, "-shared", "-o", tmp] + objs)
    os.replace(tmp, LIB)
    if verbose:
        print("built", LIB)
    return LIB


if __name__ == "__main__":
    build(force=True, verbose=True)
