"""Build librlbm.so in-tree with nvcc for sm_103a (no torch extension
machinery: plain nvcc/g++ objects compiled in parallel, then one link)."""
import concurrent.futures as cf
import os
import platform
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "librlbm.so")

CUDA_SOURCES = ["rlbm_kernels_f64.cu", "rlbm_kernels_f32.cu", "rlbm_kernels_io.cu",
                "rlbm_fused_m1.cu", "rlbm_fused_g16.cu", "rlbm_fused_e5.cu", "rlbm_fused_s2.cu", "rlbm_noalloc.cu",
                "rlbm_kernels3d.cu", "rlbm_fused3d.cu", "rlbm_kernels_o3.cu", "rlbm_fused_o3.cu", "rlbm_peak.cu"]
CXX_SOURCES = ["rlbm_stencil.cpp", "rlbm_host.cpp", "rlbm_host3d.cpp"]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librlbm.so")
    return cand


def _cuda_home():
    return os.path.dirname(os.path.dirname(os.path.realpath(_nvcc())))


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "rlbm.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(force=False, verbose=False):
    """Compile (if stale) and return the path of librlbm.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    inc = ["-I", CSRC, "-I", os.path.join(ROOT, "include"), "-I", os.path.join(_cuda_home(), "include")]
    jobs = []
    for src in CUDA_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append([nvcc, *GENCODE, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xptxas", "-v", *inc, "-c", os.path.join(CSRC, src), "-o", obj])
    for src in CXX_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-pthread", *inc, "-c",
                     os.path.join(CSRC, src), "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(_run, jobs))
    objs = [os.path.join(BUILD, s + ".o") for s in CUDA_SOURCES + CXX_SOURCES]
    libs = (["-lquadmath"] if platform.machine() in ("x86_64", "i686") else []) + ["-lpthread"]
    tmp = LIB + ".tmp"
    _run([nvcc, *GENCODE, "-shared", "-o", tmp, *objs, *libs])
    os.replace(tmp, LIB)
    with open(os.path.join(BUILD, "ptxas.log"), "w") as fh:
        fh.write("\n".join(logs))
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=False))
