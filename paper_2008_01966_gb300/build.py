"""Build the CUDA library libcavity.so in-tree for sm_103a.

Each translation unit is compiled in parallel with nvcc and the objects are
linked into a shared library next to this file.  No CMake, no torch extension
machinery: the library exposes the plain C ABI of include/cavity.h.
"""

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libcavity.so")
BUILD = os.path.join(HERE, "_build")
SOURCES = ["api.cu", "tbc.cu", "tbc_f32.cu", "tbc_df.cu", "tbc_df_k2.cu", "tbc_df_k5.cu",
           "tbc_df_k7.cu", "tbc_df_k9.cu", "tbc_df_k10.cu", "zsweep.cu", "khat.cu", "rhs.cu",
           "precond.cu", "gmres.cu", "bgmres.cu", "dense.cu", "field.cu", "field_fused.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fcx-limited-range",
         "-Xptxas", "-O3"]
# The pair-of-FP32 pass kernels are instantiated in tbc_df_k*.cu (one unit per
# size group, compiled in parallel) and launched from tbc_df.cu, which only
# declares them: their host stubs need external linkage.  Each of these
# kernels is instantiated in exactly one unit, so the linker's choice of stub
# is unique.
SPLIT = {"tbc_df.cu", "tbc_df_k2.cu", "tbc_df_k5.cu", "tbc_df_k7.cu", "tbc_df_k9.cu", "tbc_df_k10.cu"}
SPLIT_FLAGS = ["-static-global-template-stub=false"]


def _nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(home, "bin", "nvcc")
    return p if os.path.exists(p) else "nvcc"


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    deps.append(os.path.join(HERE, "..", "include", "cavity.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(verbose=False, ptxas_info=False):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        if _stale(obj, src) or ptxas_info:
            cmd = [nvcc] + ARCH + FLAGS + (SPLIT_FLAGS if s in SPLIT else []) + ["-c", src, "-o", obj]
            if ptxas_info:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or ptxas_info:
                    sys.stderr.write(r.stderr)
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
    if jobs or not os.path.exists(OUT):
        cmd = [nvcc] + ARCH + ["-shared", "-o", OUT] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    return OUT


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
    print(OUT)
