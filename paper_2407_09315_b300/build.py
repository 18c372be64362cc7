"""Build the CUDA library librbmd.so in-tree for sm_103a (B300).

nvcc cross-compiles without a GPU.  The library is plain C ABI (include/rbmd.h)
with the CUDA runtime linked statically, so the Python binding loads it with
ctypes and nothing else.
"""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "librbmd.so")
# the same sources with every list and cell index bounds-checked on the device
# (-DRBMD_CHECKED: a bad index latches RBMD_ERR_BOUNDS instead of being used)
OUT_CHECKED = os.path.join(HERE, "librbmd_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    for p in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if p and (os.path.isabs(p) and os.path.exists(p) or not os.path.isabs(p)):
            return p
    return "nvcc"


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [os.path.join(ROOT, "include", "rbmd.h")]


def up_to_date(out=OUT) -> bool:
    if not os.path.exists(out):
        return False
    t = os.path.getmtime(out)
    return all(os.path.getmtime(f) <= t for f in sources() + headers())


def build(force: bool = False, verbose: bool = False, extra=None, checked: bool = False) -> str:
    """Compile every csrc/*.cu to an object file (in parallel), then link them
    into librbmd.so (librbmd_checked.so with checked=True) with the CUDA runtime
    linked statically."""
    out = OUT_CHECKED if checked else OUT
    if not force and up_to_date(out):
        return out
    if checked:
        extra = list(extra or []) + ["-DRBMD_CHECKED"]
    from concurrent.futures import ThreadPoolExecutor

    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    flags = ["-O3", "-lineinfo", "-std=c++17", *ARCH, "-Xcompiler", "-fPIC",
             "-Xcompiler", "-ffp-contract=off", "-I", os.path.join(ROOT, "include")]
    if verbose:
        flags.insert(0, "-Xptxas=-v")
    if extra:
        flags[0:0] = list(extra)
    objs = []
    cmds = []
    for src in sources():
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".%s%d.o" % ("c" if checked else "",
                                                                           os.getpid()))
        objs.append(obj)
        cmds.append([nvcc(), *flags, "-c", "-o", obj, src])
    with ThreadPoolExecutor(max_workers=min(len(cmds), os.cpu_count() or 1)) as ex:
        for f in [ex.submit(subprocess.check_call, c) for c in cmds]:
            f.result()
    tmp = out + ".tmp%d" % os.getpid()
    subprocess.check_call([nvcc(), *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs])
    for o in objs:
        os.remove(o)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
