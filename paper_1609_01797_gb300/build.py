"""Builds libtaser.so (all CUDA kernels + the C ABI) in-tree for sm_103a with nvcc.

Usage: python -m paper_1609_01797_gb300.build   (or build() from Python)
"""
import concurrent.futures
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIBDIR = os.path.join(PKG, "lib")
LIB = os.path.join(LIBDIR, "libtaser.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["taser_api.cu", "build_T.cu", "spectral.cu", "detect_fp32.cu", "detect_tc.cu", "detect_tc64.cu", "detect_fx14.cu", "static_scratch.cu", "unfolded.cu", "unfolded_tc.cu", "uneven.cu"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtaser")
    return cand


def _flags(verbose_ptxas=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(INCLUDE, "taser.h"), __file__] + [
        os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(verbose_ptxas=False, force=False, jobs=None):
    """Compile every kernel source (in parallel) and link libtaser.so. Returns its path."""
    nvcc = _nvcc()
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    flags = _flags(verbose_ptxas)

    def compile_one(name):
        src = os.path.join(CSRC, name)
        obj = os.path.join(objdir, name.replace(".cu", ".o"))
        if force or verbose_ptxas or _stale(obj, src):
            cmd = [nvcc] + flags + ["-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, r.stdout, r.stderr))
            return obj, r.stderr
        return obj, ""

    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs or len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    logs = "".join(r[1] for r in results)
    objs = [r[0] for r in results]
    if force or verbose_ptxas or not os.path.exists(LIB) or any(
            os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        tmp = LIB + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
    if verbose_ptxas:
        print(logs)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose_ptxas="-v" in sys.argv, force="-f" in sys.argv))
