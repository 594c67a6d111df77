"""Build the CUDA library ``libmktfhe.so`` in-tree for sm_103a.

Two translation units compiled in parallel: the kernels with nvcc
(``-gencode arch=compute_103a,code=sm_103a``) and the host runtime with g++;
nvcc links them into one shared library with the CUDA runtime linked
statically.  Output: ``paper_2205_05825_gb300/_build/libmktfhe.so``.
Set MK_PTXAS_VERBOSE=1 to print ptxas register / shared-memory usage.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libmktfhe.so")
CUDA_HOME = os.environ.get("CUDA_HOME", "/usr/local/cuda")
NVCC = os.path.join(CUDA_HOME, "bin", "nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

CU_SOURCES = ["mk_kernels.cu", "mk_noalloc.cu", "mk_tensor.cu", "mk_tensor_tc05.cu"]
# mk_br.cu is compiled once per (log2 N, blind-rotation variant).
BR_SOURCE = "mk_br.cu"
BR_INSTANCES = [(logn, f, v) for logn in (8, 10) for f in (0, 1) for v in range(9)] + \
    [(logn, 2, 0) for logn in (8, 10)]
# mk_brc.cu (the cluster kernel) is compiled once per (log2 N, field).
BRC_SOURCE = "mk_brc.cu"
BRC_INSTANCES = [(logn, f) for logn in (8, 10) for f in (0, 1)]
CPP_SOURCES = ["mk_host.cpp", "mk_circuits.cpp", "mk_server.cpp"]
HEADERS = ["mk_internal.h", "mk_ctx.h", "mk_bootstrap.cuh", "mk_bulk.cuh", "mk_bootstrap_fft.cuh", "mk_bootstrap_cluster.cuh",
           "mk_bootstrap_staged.cuh", "mk_bootstrap_split.cuh", "mk_netlist.cuh",
           BR_SOURCE, BRC_SOURCE]


def _newest_input():
    files = [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES + HEADERS]
    files.append(os.path.join(INCLUDE, "mk_tfhe.h"))
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT_DIR, exist_ok=True)
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _newest_input():
        return LIB
    objs, procs = [], []
    ptxas_v = ["-Xptxas", "-v"] if os.environ.get("MK_PTXAS_VERBOSE") else []
    for src in CU_SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
               "-I", INCLUDE, *ptxas_v, "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for logn, f, v in BR_INSTANCES:
        obj = os.path.join(OUT_DIR, "mk_br_%d_f%d_v%d.o" % (logn, f, v))
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
               "-DMK_LOGN=%d" % logn, "-DMK_FIELD=%d" % f, "-DMK_VARIANT=%d" % v, *ptxas_v, "-c",
               os.path.join(CSRC, BR_SOURCE), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for logn, f in BRC_INSTANCES:
        obj = os.path.join(OUT_DIR, "mk_brc_%d_f%d.o" % (logn, f))
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
               "-DMK_LOGN=%d" % logn, "-DMK_FIELD=%d" % f, *ptxas_v, "-c", os.path.join(CSRC, BRC_SOURCE), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    for src in CPP_SOURCES:
        obj = os.path.join(OUT_DIR, src + ".o")
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-Wall",
               "-I", os.path.join(CUDA_HOME, "include"), "-I", INCLUDE,
               "-c", os.path.join(CSRC, src), "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = []
    for cmd, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append(" ".join(cmd) + "\n" + text)
        elif verbose or ptxas_v:
            sys.stdout.write(text)
    if failed:
        raise RuntimeError("build failed:\n" + "\n".join(failed))
    tmp = LIB + ".tmp.%d" % os.getpid()
    subprocess.check_call([NVCC, *ARCH, "-shared", "-Xlinker", "-z,defs", "-o", tmp, *objs, "-lpthread"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
