"""Build libpwa (the CUDA library behind the C ABI in include/pwa.h) in-tree.

nvcc compiles the .cu sources for sm_103a only (B300) into
paper_2403_09225_b300/_lib/libpwa.so.  Each translation unit compiles in its
own nvcc process (they run in parallel), then the objects are linked.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libpwa.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++20", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
SOURCES = ["pwa_api.cu", "fit.cu", "hessian.cu", "multi.cu", "noalloc.cu", "coupling.cu", "mlp.cu", "generate.cu", "variant.cu"]
HEADERS = ["pass_kernel.cuh", "pwa_internal.h", "tcgen05.cuh"]

#: compiled shapes of the fused pass: S (projections) x W (warps per block) x
#: KPW (resonances per warp in the second sweep)
SHAPES_S = (1, 2, 3, 4)
SHAPES_W = (1, 2, 4, 8)
SHAPES_KPW = (1, 2, 3, 4, 5, 6, 7, 8)
MODES = {"nll": "MODE_NLL", "grad": "MODE_GRAD", "hvp": "MODE_HVP", "hvpr": "MODE_HVP_REUSE"}


def _instance_units() -> dict:
    """Translation units that instantiate the fused pass, one per (mode, S):
    each defines pick_pass_<mode>_s<S>(W, KPW) returning the kernel."""
    units = {}
    for mode, enum in MODES.items():
        for S in SHAPES_S:
            lines = ['// generated by build.py: instances of pass_kernel for %s, S = %d' % (enum, S),
                     '#include "pass_kernel.cuh"', '#include "pwa_internal.h"', 'namespace pwa {',
                     'KernelFn pick_pass_%s_s%d(int W, int kpw)' % (mode, S), '{']
            if mode == "nll":
                lines.append('    (void)kpw;  // no second sweep')
                for W in SHAPES_W:
                    lines.append('    if (W == %d) return pass_kernel<%s, %d, %d, 1>;' % (W, enum, S, W))
            else:
                for W in SHAPES_W:
                    for kpw in SHAPES_KPW:
                        lines.append('    if (W == %d && kpw == %d) return pass_kernel<%s, %d, %d, %d>;'
                                     % (W, kpw, enum, S, W, kpw))
            lines += ['    return nullptr;', '}', '}  // namespace pwa', '']
            units['pass_%s_s%d.cu' % (mode, S)] = '\n'.join(lines)
    return units


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: libpwa needs the CUDA toolkit to build")


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(ROOT, "include", "pwa.h"),
                                                                   os.path.abspath(__file__)]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libpwa.so if it is missing or older than its sources."""
    if not force and not _stale():
        return LIB
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)

    def compile_one(src):
        obj = os.path.join(objdir, os.path.splitext(os.path.basename(src))[0] + ".o")
        cmd = [nvcc, *ARCH, *FLAGS, "-I", os.path.join(ROOT, "include"), "-I", CSRC, "-c", src, "-o", obj]
        if verbose:
            cmd.append("-Xptxas=-v")
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, res.stderr))
        if verbose:
            sys.stderr.write(res.stderr)
        return obj

    gendir = os.path.join(LIBDIR, "gen")
    os.makedirs(gendir, exist_ok=True)
    gen = []
    for name, text in _instance_units().items():
        path = os.path.join(gendir, name)
        if not os.path.exists(path) or open(path).read() != text:
            with open(path, "w") as f:
                f.write(text)
        gen.append(path)
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 8) as ex:
        objs = list(ex.map(compile_one, [os.path.join(CSRC, f) for f in SOURCES] + gen))
    tmp = LIB + ".tmp%d" % os.getpid()
    res = subprocess.run([nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs],
                         capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("link failed:\n%s" % res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
