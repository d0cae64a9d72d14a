"""Builds liblbm.so in-tree with nvcc for sm_103a (translation units compiled in
parallel, then linked into one shared library with the C ABI of include/lbm.h)."""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.environ.get("LBM_CSRC") or os.path.join(HERE, "csrc")
# LBM_BUILD_DIR / LBM_NVCC_EXTRA redirect the build and add nvcc flags (tuning runs)
BUILD = os.environ.get("LBM_BUILD_DIR") or os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liblbm.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xptxas", "-v",
         "-I", CSRC, "-I", os.path.join(ROOT, "include")]

EXTRA = os.environ.get("LBM_NVCC_EXTRA", "").split()
UNITS = [("setup", "setup.cu", []), ("api", "api.cu", []), ("wss", "wss.cu", ["--use_fast_math"]),
         ("porosity", "porosity.cu", []), ("aniso", "aniso.cu", [])]
# Resident blocks of the time step per SM (its launch bound): 6 (80 registers)
# for FP32; 8 (64 registers) for the 2-byte storage types, measured 2.5 %
# faster there and slower for FP32.
STEP_MIN_BLOCKS = {"f32": 6, "f16": 8, "bf16": 8}
for q in (19, 27):
    for s, name in ((0, "f32"), (1, "f16"), (2, "bf16")):
        UNITS.append((f"step_{q}_{name}", "step.cu", [f"-DLBM_Q={q}", f"-DLBM_STORE={s}", "--use_fast_math",
                                                      f"-DLBM_MIN_BLOCKS={STEP_MIN_BLOCKS[name]}"]))
        UNITS.append((f"adjoint_{q}_{name}", "adjoint.cu",
                      [f"-DLBM_Q={q}", f"-DLBM_STORE={s}", "--use_fast_math"]))


def _sources():
    return [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(ROOT, "include", "lbm.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    stamp = os.path.join(BUILD, "flags.txt")
    if not os.path.exists(stamp) or open(stamp).read() != " ".join(EXTRA):
        return False
    return all(os.path.getmtime(s) <= t for s in _sources())


def _compile(unit):
    name, src, defs = unit
    obj = os.path.join(BUILD, name + ".o")
    cmd = [NVCC, *ARCH, *FLAGS, *defs, *EXTRA, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    with open(os.path.join(BUILD, name + ".log"), "w") as fh:
        fh.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr[-4000:]}")
    return obj


def build(force=False, jobs=None):
    """Compiles every translation unit and links _build/liblbm.so."""
    os.makedirs(BUILD, exist_ok=True)
    if not force and up_to_date():
        return LIB
    jobs = jobs or min(len(UNITS), os.cpu_count() or 4)
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        objs = list(ex.map(_compile, UNITS))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lcudart_static", "-lrt", "-ldl",
           "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr[-4000:]}")
    os.replace(tmp, LIB)
    with open(os.path.join(BUILD, "flags.txt"), "w") as fh:
        fh.write(" ".join(EXTRA))
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
