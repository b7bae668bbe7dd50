"""Build libdgmg.so (the C-ABI library of include/dgmg.h) for sm_103a.

Each translation unit is compiled by its own nvcc / g++ process, in
parallel; the per-order kernel file is compiled once per n = p+1 with
-DDGMG_N=n.  The output goes to paper_1805_11930_gb300/_build/ and is rebuilt
only when a source or header is newer than the library.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "libdgmg.so")
ORDERS = range(2, 10)            # n = p + 1, p = 1..8
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdgmg.so")


def _jobs():
    nv = _nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
    jobs = []
    for n in ORDERS:
        obj = os.path.join(BUILD, f"cell_kernels_n{n}.o")
        jobs.append((obj, [nv] + common + [f"-DDGMG_N={n}", "-c", os.path.join(CSRC, "cell_kernels.cu"), "-o", obj]))
    for name in ("vec_kernels", "capi", "noalloc"):
        obj = os.path.join(BUILD, name + ".o")
        jobs.append((obj, [nv] + common + ["-c", os.path.join(CSRC, name + ".cu"), "-o", obj]))
    gxx = shutil.which("g++") or "g++"
    obj = os.path.join(BUILD, "setup_host.o")
    jobs.append((obj, [gxx, "-O3", "-fPIC", "-std=c++17", "-I", INCLUDE, "-I", CSRC, "-c",
                       os.path.join(CSRC, "setup_host.cpp"), "-o", obj]))
    return nv, jobs


def _sources():
    out = [os.path.join(INCLUDE, "dgmg.h")]
    for f in os.listdir(CSRC):
        out.append(os.path.join(CSRC, f))
    return out


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False):
    """Compile and link libdgmg.so; returns its path."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nv, jobs = _jobs()

    def run(job):
        obj, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=max(2, min(len(jobs), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(run, jobs))
    tmp = LIB + ".tmp"
    cmd = [nv] + ARCH + ["-shared", "-Xcompiler", "-fPIC", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
