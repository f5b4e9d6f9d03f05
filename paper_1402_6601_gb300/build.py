"""Build the CUDA library in-tree: paper_1402_6601_gb300/_build/libchol_gb300.so.

Every translation unit is compiled for sm_103a only, in parallel, then linked into one
shared library with the CUDA runtime linked statically (the library needs only the driver
at run time). No cmake: plain nvcc.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libchol_gb300.so")
SOURCES = ["csrc/adjoint.cu", "csrc/api.cu", "csrc/batched.cu", "csrc/factor.cu", "csrc/lu.cu", "csrc/solve.cu",
           "csrc/refine.cu", "csrc/probe.cu"]
HEADERS = ["csrc/blockacc.cuh", "csrc/common.cuh", "csrc/dag.cuh", "csrc/dag_lu.cuh", "csrc/internal.cuh", "csrc/sched.cuh",
           "csrc/tiles_f32.cuh", "csrc/tiles_f64.cuh", "csrc/tiles_lu.cuh", "csrc/tiles_tc.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _deps():
    return [os.path.join(HERE, p) for p in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "chol.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force=False, verbose=False, extra_flags=()):
    if not force and up_to_date():
        return LIB
    os.makedirs(os.path.join(OUT, "obj"), exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(HERE, "csrc")]

    def compile_one(src):
        obj = os.path.join(OUT, "obj", os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + FLAGS + list(extra_flags) + inc + ["-c", os.path.join(HERE, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    flags = [a for a in sys.argv[1:] if a.startswith("-X") or a.startswith("--")]
    print(build(force=True, verbose="-v" in sys.argv, extra_flags=[f for f in flags if f != "--force"]))
