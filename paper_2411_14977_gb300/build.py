"""In-tree build of the native library ``libpmg.so`` (CUDA kernels for sm_103a + C ABI).

Every translation unit is compiled in parallel with nvcc (one -gencode, sm_103a only) and
linked into ``paper_2411_14977_gb300/_lib/libpmg.so`` against the shared CUDA runtime.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libpmg.so")
SOURCES = ["k_apply_aniso.cu", "k_apply.cu", "k_apply_bathy.cu", "k_apply_tc.cu", "k_levels_aniso.cu", "k_dense.cu", "k_levels.cu", "k_fdm32.cu", "k_fdm32z.cu", "k_fdm32_batch.cu", "k_vtail.cu", "k_stepper.cu", "k_nn.cu", "k_coarse_vec.cu", "solver.cu",
           "warmstart.cu", "noalloc.cu", "host_basis.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libpmg.so")
    return cand


def _common_flags():
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3",
            "-I", os.path.join(ROOT, "include"), "-I", CSRC, "--expt-relaxed-constexpr"]


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    deps.append(os.path.join(ROOT, "include", "pmg.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, force=False):
    """Compile and link libpmg.so if any source changed; returns the library path."""
    nvcc = _nvcc()
    os.makedirs(OUT_DIR, exist_ok=True)
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(OUT_DIR, src + ".o")
        if force or _stale(o, s):
            cmd = [nvcc] + ARCH + _common_flags() + ["-c", s, "-o", o]
            if src.endswith(".cpp"):
                cmd = [nvcc] + _common_flags() + ["-x", "c++", "-c", s, "-o", o]
            jobs.append((src, cmd))

    def run(job):
        src, cmd = job
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    if jobs:
        with ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for msg in ex.map(run, jobs):
                if verbose and msg:
                    print(msg)
    objs = [os.path.join(OUT_DIR, s + ".o") for s in SOURCES]
    if jobs or not os.path.exists(LIB):
        cmd = [nvcc] + ARCH + ["-shared", "-cudart", "shared", "-o", LIB] + objs + \
              ["-Xlinker", "-rpath,/usr/local/cuda/lib64"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
