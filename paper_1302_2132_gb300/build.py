"""In-tree build of libgks.so for sm_103a (nvcc, one translation unit per kernel family, compiled
in parallel)."""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libgks.so")
UNITS = ["gks_serve.cu", "gks_step_2d.cu", "gks_step_2d_tiles.cu", "gks_step_2d_tiles2.cu", "gks_step_acc64.cu", "gks_step_pair.cu", "gks_step_rar.cu", "gks_step_3d.cu", "gks_step_3d_tiles.cu", "gks_step_1d.cu", "gks_face.cu", "gks_capi.cu", "gks_count.cpp", "gks_probe.cu", "gks_noalloc.cu", "gks_komega.cu", "gks_step_muscl3.cu", "gks_step_weno5.cu", "gks_curv.cu", "gks_curv_recon.cu", "gks_curv_kw.cu", "gks_curv_rar.cu", "gks_steady.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found")


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, jobs=None):
    os.makedirs(BUILD, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(INCLUDE, "gks.h"))
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]

    def compile_unit(u):
        src = os.path.join(CSRC, u)
        obj = os.path.join(BUILD, os.path.splitext(u)[0] + ".o")
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc()] + flags + ["-c", src, "-o", obj + ".tmp"]
            if verbose:
                print(" ".join(cmd), file=sys.stderr)
            subprocess.check_call(cmd)
            os.replace(obj + ".tmp", obj)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs or min(len(UNITS), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_unit, UNITS))
    if force or _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call([nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
