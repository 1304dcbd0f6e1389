"""Build the C-ABI shared library libsaq.so in-tree with nvcc for sm_103a.

Each translation unit compiles in parallel; the objects are linked into
paper_2509_12086_gb300/libsaq.so together with cuSOLVER and cuBLAS (used by
the fit only).
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libsaq.so")
BUILD = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["saq_host.cpp", "saq_encode.cu", "k_simt.cu", "k_caq1.cu", "k_estimate.cu",
           "k_fit.cu", "k_tc.cu", "saq_noalloc.cu", "saq_ingest.cu"]


def _nvcc():
    home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    p = os.path.join(home, "bin", "nvcc")
    return p if os.path.exists(p) else (shutil.which("nvcc") or "nvcc")


def _flags():
    return ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "-I" + os.path.join(ROOT, "include"), "-I" + CSRC,
                   "--expt-relaxed-constexpr", "-Xptxas", "-v" if os.environ.get("SAQ_PTXAS_V") else "-O3"]


def _compile(src):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    srcp = os.path.join(CSRC, src)
    deps = [srcp, os.path.join(CSRC, "saq_internal.h"), os.path.join(ROOT, "include", "saq.h")]
    if os.path.exists(obj) and all(os.path.getmtime(obj) >= os.path.getmtime(d) for d in deps):
        return obj, ""
    cmd = [_nvcc()] + _flags() + ["-x", "cu", "-c", srcp, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build(verbose=False):
    import platform
    marker = os.path.join(BUILD, "arch")
    if not (os.path.exists(marker) and open(marker).read() == platform.machine()):
        shutil.rmtree(BUILD, ignore_errors=True)
        if os.path.exists(OUT):
            os.remove(OUT)
    os.makedirs(BUILD, exist_ok=True)
    with open(marker, "w") as f:
        f.write(platform.machine())
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 2)) as ex:
        results = list(ex.map(_compile, SOURCES))
    if verbose:
        for _, log in results:
            if log:
                print(log)
    objs = [o for o, _ in results]
    if (not os.path.exists(OUT)
            or any(os.path.getmtime(o) > os.path.getmtime(OUT) for o in objs)):
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", OUT + ".tmp"] + objs + [
            "-lcusolver", "-lcublas", "-lcudart", "-lpthread",
            "-Xlinker", "-rpath=" + os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64")]
        subprocess.check_call(cmd)
        os.replace(OUT + ".tmp", OUT)
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
