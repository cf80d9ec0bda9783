"""Build libgf2x_gb300.so (sm_103a) in-tree with nvcc, translation units in parallel."""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
OUT_DIR = os.path.join(PKG, "_lib")
LIB = os.path.join(OUT_DIR, "libgf2x_gb300.so")
INCLUDE = os.path.join(ROOT, "include")
EXPERIMENTS = os.path.join(PKG, "experiments")
# the two experiments (tensor-core Toeplitz multiplier, bitsliced leaves) as
# small libraries with test entry points, so that GPU tests can check them
EXPERIMENT_LIBS = {"libgf2x_exp_tc.so": "tc_toeplitz.cu", "libgf2x_exp_bitsliced.so": "bitsliced_leaf.cu"}

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH


def sources():
    out = []
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cpp")):
            out.append(os.path.join(CSRC, f))
    return out


def _deps_mtime():
    files = sources() + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    files.append(os.path.join(INCLUDE, "gf2x_gb300.h"))
    files += [os.path.join(EXPERIMENTS, f) for f in EXPERIMENT_LIBS.values()]
    return max(os.path.getmtime(f) for f in files)


def experiment_lib(name: str) -> str:
    return os.path.join(OUT_DIR, name)


def _up_to_date() -> bool:
    outs = [LIB] + [experiment_lib(k) for k in EXPERIMENT_LIBS]
    return all(os.path.exists(o) for o in outs) and min(os.path.getmtime(o) for o in outs) >= _deps_mtime()


def build(force: bool = False, verbose: bool = False, jobs: int = 0) -> str:
    """Compile every translation unit and link the shared library (and the
    experiments' test libraries); returns the library's path."""
    if not force and _up_to_date():
        return LIB
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")

    def build_experiment(item):
        name, src = item
        out = experiment_lib(name)
        tmp = out + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", "-DGF2X_EXPERIMENT_LIB", os.path.join(EXPERIMENTS, src), "-o", tmp] + NVCC_FLAGS
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, out)
        return out

    def compile_one(src):
        obj = os.path.join(obj_dir, os.path.basename(src) + ".o")
        cmd = [nvcc, "-c", src, "-o", obj] + NVCC_FLAGS
        if src.endswith(".cpp"):
            cmd = [nvcc, "-x", "cu", "-c", src, "-o", obj] + NVCC_FLAGS
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout, r.stderr, file=sys.stderr)
        return obj

    jobs = jobs or min(8, os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        exps = [ex.submit(build_experiment, it) for it in EXPERIMENT_LIBS.items()]
        objs = list(ex.map(compile_one, sources()))
        for f in exps:
            f.result()
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
