"""In-tree build of the CUDA libraries (sm_103a) with plain nvcc, no cmake.

libtopomag.so        -- the product: FFT passes, tensor setup, C ABI (include/topomag.h)
libtopomag_cufft.so  -- the comparison pipeline built on cuFFT (bench only)

Translation units compile in parallel; a unit is rebuilt when it or a header
is newer than its object file.
"""

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
INCLUDE = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE]

PRODUCT_UNITS = ["api.cu", "k_xfwd.cu", "k_xinv.cu", "k_yz.cu", "k_zdir.cu", "tensor.cu", "misc.cu", "unet.cu", "lbfgsb.cu", "k_yzfused.cu", "k_xobj.cu"]
CUFFT_UNITS = ["cufft_pipeline.cu"]

LIB = os.path.join(HERE, "libtopomag.so")
LIB_CUFFT = os.path.join(HERE, "libtopomag_cufft.so")


def nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return max((os.path.getmtime(h) for h in hs), default=0.0)


def _compile(src, force, extra):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    if not force and os.path.exists(obj):
        t = os.path.getmtime(obj)
        if t >= os.path.getmtime(src) and t >= _headers():
            return obj
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj


def _link(objs, out, libs=()):
    cmd = [nvcc(), *ARCH, "-shared", "-o", out, *objs, *libs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed for {out}:\n{r.stdout}\n{r.stderr}")


def build(force=False, verbose=False, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    units = [(os.path.join(CSRC, u), "p") for u in PRODUCT_UNITS]
    units += [(os.path.join(CSRC, u), "c") for u in CUFFT_UNITS if os.path.exists(os.path.join(CSRC, u))]
    workers = min(len(units), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(workers) as ex:
        futs = {ex.submit(_compile, src, force, list(extra)): (src, kind) for src, kind in units}
        objs = {"p": [], "c": []}
        for f in cf.as_completed(futs):
            src, kind = futs[f]
            objs[kind].append(f.result())
            if verbose:
                print("compiled", os.path.basename(src), flush=True)
    _link(sorted(objs["p"]), LIB)
    if objs["c"]:
        _link(sorted(objs["c"]), LIB_CUFFT, ["-lcufft"])
    return LIB


if __name__ == "__main__":
    import sys

    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
