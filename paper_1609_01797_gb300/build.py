"""Builds libtaser.so (all CUDA kernels + the C ABI) in-tree for sm_103a with nvcc, and its
bounds-checked variant libtaser_debug.so (-DTASER_DEBUG: every run-time index is checked
and counted, see taser_debug_report in include/taser.h).

Usage: python -m paper_1609_01797_gb300.build [-f] [-v] [--debug]   (or build() from Python)
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
LIB_DEBUG = os.path.join(LIBDIR, "libtaser_debug.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["taser_api.cu", "build_T.cu", "spectral.cu", "detect_fp32.cu", "detect_tc.cu", "detect_fx14.cu", "static_scratch.cu", "unfolded.cu", "unfolded_tc.cu", "uneven.cu"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libtaser")
    return cand


def _flags(verbose_ptxas=False, debug=False):
    f = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    if debug:
        f += ["-DTASER_DEBUG"]
    if verbose_ptxas:
        f += ["-Xptxas", "-v"]
    return f


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    deps = [src, os.path.join(INCLUDE, "taser.h"), __file__] + [
        os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".cuh")]
    return any(os.path.getmtime(d) > os.path.getmtime(obj) for d in deps)


def build(verbose_ptxas=False, force=False, jobs=None, debug=False):
    """Compile every kernel source (in parallel) and link libtaser.so (debug: the
    bounds-checked libtaser_debug.so). Returns its path."""
    nvcc = _nvcc()
    objdir = os.path.join(LIBDIR, "obj_debug" if debug else "obj")
    lib_path = LIB_DEBUG if debug else LIB
    os.makedirs(objdir, exist_ok=True)
    flags = _flags(verbose_ptxas, debug)

    def compile_one(name):
        src = os.path.join(CSRC, name)
        obj = os.path.join(objdir, name.replace(".cu", ".o"))
        if force or verbose_ptxas or _stale(obj, src):
            # TASER_TU numbers the source in the debug build's failure records.
            cmd = [nvcc] + flags + ["-DTASER_TU=%d" % (SOURCES.index(name) + 1), "-c", src, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, r.stdout, r.stderr))
            return obj, r.stderr
        return obj, ""

    with concurrent.futures.ThreadPoolExecutor(max_workers=jobs or len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    logs = "".join(r[1] for r in results)
    objs = [r[0] for r in results]
    if force or verbose_ptxas or not os.path.exists(lib_path) or any(
            os.path.getmtime(o) > os.path.getmtime(lib_path) for o in objs):
        tmp = lib_path + ".tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, lib_path)
    if verbose_ptxas:
        print(logs)
    return lib_path


def source_of(tu):
    """The kernel source that a debug failure record's file number names."""
    return SOURCES[tu - 1] if 1 <= tu <= len(SOURCES) else None


if __name__ == "__main__":
    import sys
    print(build(verbose_ptxas="-v" in sys.argv, force="-f" in sys.argv, debug="--debug" in sys.argv))
