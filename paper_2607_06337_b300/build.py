"""Build liborchard.so (the CUDA path, sm_103a) in-tree with nvcc."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC_DIR = os.path.join(HERE, "csrc")
LIB_DIR = os.path.join(HERE, "_lib")
LIB_PATH = os.path.join(LIB_DIR, "liborchard.so")
# the profiling build: the same library with the step's phase clocks compiled in
PHASE_LIB_PATH = os.path.join(LIB_DIR, "liborchard_phase.so")
VARIANTS = {"": (LIB_PATH, []), "phase": (PHASE_LIB_PATH, ["-DORCHARD_PHASE_CLOCKS"])}
SOURCES = ["step_kernel.cu", "adjoint_kernel.cu", "orchard_abi.cu", "static_scratch.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def sources():
    return [os.path.join(SRC_DIR, s) for s in SOURCES]


def _stale(path: str = LIB_PATH) -> bool:
    if not os.path.exists(path):
        return True
    t = os.path.getmtime(path)
    deps = sources() + [os.path.join(SRC_DIR, f) for f in os.listdir(SRC_DIR)] + \
        [os.path.join(ROOT, "include", "orchard.h")]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, variant: str = "") -> str:
    """Compile the library (variant "") or its phase-clock profiling build (variant "phase")."""
    path, defs = VARIANTS[variant]
    os.makedirs(LIB_DIR, exist_ok=True)
    if not force and not _stale(path):
        return path
    nvcc = os.environ.get("NVCC", "nvcc")
    cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-shared", "-Xcompiler", "-fPIC", *defs,
           "-I", os.path.join(ROOT, "include"), "-o", path + ".tmp", *sources()]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.run(cmd, check=True)
    os.replace(path + ".tmp", path)
    return path


if __name__ == "__main__":
    var = "phase" if "--phase" in sys.argv else ""
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv, variant=var))
