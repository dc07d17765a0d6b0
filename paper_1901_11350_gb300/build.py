"""Build ``libspirit_gb.so`` (the C-ABI library) for sm_103a, in-tree.

Each translation unit under ``csrc/`` is compiled by nvcc in parallel, then
linked into a shared library next to this file.  Only rebuilds what changed.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libspirit_gb.so")
SOURCES = ["api.cu", "field_llg.cu", "minimise.cu", "dipole.cu", "cubic.cu", "cubic_lean.cu", "topo.cu", "static_step.cu", "dipole_fast.cu", "unet.cu", "mc.cu", "hessian.cu", "htst.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
                "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"]
# extra nvcc flags for experiments (e.g. -DSPGB_CUBIC_MINB=4); a change of
# flags rebuilds everything
EXTRA = os.environ.get("SPGB_NVCC_EXTRA", "").split()


def _deps():
    out = [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    out += [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    return out


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.splitext(os.path.basename(src))[0] + ".o")
    if _stale(obj, [src] + _deps()):
        cmd = [NVCC, "-c", src, "-o", obj + ".tmp"] + FLAGS + extra
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
        os.replace(obj + ".tmp", obj)
    return obj


def build(verbose=False, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    extra = list(extra) + EXTRA
    stamp = os.path.join(BUILD, "flags.txt")
    flags = " ".join(FLAGS + extra)
    if not os.path.exists(stamp) or open(stamp).read() != flags:
        for f in os.listdir(BUILD):
            if f.endswith(".o"):
                os.remove(os.path.join(BUILD, f))
        with open(stamp, "w") as fh:
            fh.write(flags)
    srcs = [os.path.join(CSRC, s) for s in SOURCES if os.path.exists(os.path.join(CSRC, s))]
    with cf.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        objs = list(ex.map(lambda s: _compile(s, list(extra)), srcs))
    if _stale(LIB, objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [NVCC, "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "shared"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        os.replace(tmp, LIB)
    if verbose:
        print(LIB)
    return LIB


if __name__ == "__main__":
    build(verbose=True)
