"""In-tree build of the CUDA library ``_build/libxamg_gpu.so`` for sm_103a.

Host setup code is compiled with g++ without floating-point contraction (its
results are a deterministic function of the input); the kernels and the C ABI
with nvcc for ``arch=compute_103a,code=sm_103a``.  Translation units compile in
parallel.  Usage: ``python -m paper_2103_07329_gb300.build``.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libxamg_gpu.so")
ROOT = os.path.dirname(HERE)

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _nvcc() -> str:
    p = shutil.which("nvcc") or os.path.join(CUDA_HOME, "bin", "nvcc")
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found: the CUDA library cannot be built")
    return p


def sources():
    return [os.path.join(CSRC, f) for f in ("setup.cpp", "hier_io.cpp", "kernels.cu", "capi.cu", "noalloc.cu",
                                            "rows_nv1.cu", "rows_nv2.cu", "rows_nv4.cu",
                                            "rows_nv8.cu", "rows_nv16.cu", "rows_nv32.cu",
                                            "rowsf_nv1.cu", "rowsf_nv2.cu", "rowsf_nv4.cu",
                                            "rowsf_nv8.cu", "rowsf_nv16.cu", "rowsf_nv32.cu",
                                            "net.cu", "batch.cu", "batch_stage1.cu",
                                            "batch_stage2.cu", "batch_stage3.cu",
                                            "bicg_variants.cu", "vtail_f64.cu", "vtail_f32.cu")]


def _deps():
    return sources() + [os.path.join(CSRC, f) for f in ("hier_host.h", "launch.h", "kernels.cuh",
                                                              "rows_inst.cuh", "elem.cuh", "batch.h",
                                                              "vtail.cuh", "vtail_kern.cuh",
                                                              "batch_stage.cuh")] + [
        os.path.join(ROOT, "include", "xamg_gpu.h")]


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", os.path.join(ROOT, "include")]
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        objs.append(obj)
        if src.endswith(".cpp"):
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-pthread", "-ffp-contract=off", *inc,
                   "-c", src, "-o", obj]
        else:
            cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-Xcompiler", "-ffp-contract=off", *inc, "-c", src, "-o", obj]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
        if verbose:
            print(" ".join(cmd), flush=True)
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in jobs:
        out, _ = p.communicate()
        if p.returncode != 0 or (verbose or ptxas_info) and out:
            sys.stdout.write(out.decode(errors="replace"))
        if p.returncode != 0:
            failed.append(" ".join(cmd))
    if failed:
        raise RuntimeError("CUDA library build failed:\n" + "\n".join(failed))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs, "-lpthread",
            "-Xlinker", "-rpath", "-Xlinker", os.path.join(CUDA_HOME, "lib64")]
    if verbose:
        print(" ".join(link), flush=True)
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
