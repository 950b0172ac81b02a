"""Build libei.so in-tree: nvcc for sm_103a, one object per translation unit
compiled in parallel, then one shared link (static CUDA runtime)."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libei.so")
# the debug build: device-side bounds checks in the projector and the adjoint
CHECK_LIB = os.path.join(HERE, "libei_check.so")
CHECK_OBJ = os.path.join(HERE, "_build_check")
SOURCES = ["ei_api.cu", "k_project.cu", "k_ic.cu", "k_backproject.cu", "solver.cu",
           "ei_noalloc.cu", "k_fbp.cu", "nn_kernels.cu", "nn_unet.cu", "k_peaks.cu", "nn_conv_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps_mtime() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(HERE, "..", "include", "ei.h"))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False, extra=(), lib: str = LIB,
          obj_dir: str = OBJ) -> str:
    """Compile and link; `extra` nvcc flags (e.g. -D tunables) and another output
    path may be given to build variants side by side."""
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= _deps_mtime():
        return lib
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(obj_dir, src.replace(".cu", ".o"))
        cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


def build_checked(force: bool = False) -> str:
    """The library with device-side bounds checks (-DEI_DEVICE_CHECKS) as
    libei_check.so beside the regular one (load it with EI_LIBRARY)."""
    return build(force=force, extra=("-DEI_DEVICE_CHECKS",), lib=CHECK_LIB, obj_dir=CHECK_OBJ)


if __name__ == "__main__":
    extra = [a for a in sys.argv[1:] if a.startswith("-X") or a.startswith("--")]
    print(build(force=True, verbose="-v" in sys.argv, extra=[e for e in extra if e != "--force"]))
