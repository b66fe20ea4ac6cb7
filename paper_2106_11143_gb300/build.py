"""Build libnb.so in-tree for sm_103a with nvcc.

Each translation unit under csrc/ is compiled in parallel to an object file
in _build/, then linked into paper_2106_11143_gb300/libnb.so.  The CUDA
runtime is linked statically; the library shares the device's primary
context (and therefore streams) with PyTorch.
"""
import os
import shutil
import subprocess
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libnb.so")
SOURCES = ["nb_pair.cu", "nb_sym.cu", "nb_integrate.cu", "nb_batched.cu", "nb_adjoint.cu",
           "nb_api.cu", "nb_noalloc.cu", "nb_probe.cu",
           "nb_vjp.cu", "nb_small.cu"]
HEADERS = ["nb_common.cuh", "nb_pairterm.cuh", "nb_vjpterm.cuh", "nb_symsched.cuh", "nb_verlet.cuh",
           os.path.join("..", "..", "include", "nb.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(out, deps):
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    hdrs = [os.path.normpath(os.path.join(CSRC, h)) for h in HEADERS]
    objs, procs = [], []
    t0 = time.time()
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xptxas", "-v" if verbose else "-O3", *extra, "-c", s, "-o", o]
            procs.append((src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE,
                                                     stderr=subprocess.STDOUT, text=True)))
    failed = []
    for src, cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append((src, out))
        elif verbose and out:
            print(out)
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join("%s:\n%s" % f for f in failed))
    if force or procs or _stale(LIB, objs):
        tmp = LIB + ".tmp"
        subprocess.check_call([nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-ldl"])  # dlopen for NVTX
        os.replace(tmp, LIB)
    if verbose:
        print("built %s in %.1fs" % (LIB, time.time() - t0))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
