"""Compile the CUDA library for sm_103a into paper_2006_15698_gb300/lib/.

nvcc only (no cmake): the translation units compile in parallel, then link
into one shared library exporting the C ABI of include/dg.h.  Works the same
on the x86_64 build host and on the aarch64 GPU hosts.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIBDIR = os.path.join(HERE, "lib")
LIB = os.path.join(LIBDIR, "libdg_gb300.so")
SOURCES = ["dg_api.cu", "dg_kernels_f64.cu", "dg_kernels_f32.cu", "dg_batch_f32.cu",
           "dg_f32_deg01.cu", "dg_f32_deg2.cu", "dg_f32_deg3.cu", "dg_f32_deg4.cu",
           "dg_f32_deg5.cu", "dg_f32_deg6.cu", "dg_probe.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _flags():
    return [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
            "-Xptxas", "-v" if os.environ.get("DG_PTXAS_VERBOSE") else "-O3",
            f"-I{os.path.join(HERE, '..', 'include')}"]


def _compile(src):
    out = os.path.join(OBJ, src.replace(".cu", ".o"))
    cmd = [NVCC, *_flags(), "-c", os.path.join(CSRC, src), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return out, r.stderr


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "dg.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False):
    """Build (if stale) and return the path of libdg_gb300.so."""
    if not force and not _stale():
        return LIB
    os.makedirs(OBJ, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    with cf.ThreadPoolExecutor(len(SOURCES)) as ex:
        results = list(ex.map(_compile, SOURCES))
    if verbose:
        for _, log in results:
            if log:
                print(log)
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
