"""Build libfsm.so (the C-ABI library) in-tree for sm_103a.

Translation units are compiled in parallel with nvcc, then linked into
paper_2603_28160_gb300/libfsm.so against the shared CUDA runtime.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libfsm.so")
OBJ = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I" + os.path.join(ROOT, "include")]
SOURCES = ["fsm_kernels.cu", "fsm_filter.cu", "fsm_api.cpp", "fsm_batch.cpp", "fsm_serve.cpp"]
# the micro-benchmarks of the units the kernels are bound by: a library of their own
PROBE_SOURCES = ["fsm_probe.cu"]
PROBE_LIB = os.path.join(HERE, "libfsm_probe.so")


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every translation unit (in parallel) and link libfsm.so and
    libfsm_probe.so; returns the path of libfsm.so."""
    os.makedirs(OBJ, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers += [os.path.join(ROOT, "include", f) for f in ("fsm.h", "fsm_probe.h")]
    jobs = []
    for src in SOURCES + PROBE_SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(OBJ, src + ".o")
        if force or _stale(obj, [path] + headers):
            jobs.append([nvcc()] + ARCH + FLAGS + ["-c", path, "-o", obj])
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES) + len(PROBE_SOURCES)) as ex:
        for cmd, rc in zip(jobs, ex.map(lambda c: subprocess.run(c, capture_output=not verbose), jobs)):
            if rc.returncode != 0:
                sys.stderr.write((rc.stderr or b"").decode())
                raise RuntimeError("nvcc failed: " + " ".join(cmd))
    for lib, srcs in ((LIB, SOURCES), (PROBE_LIB, PROBE_SOURCES)):
        objs = [os.path.join(OBJ, s + ".o") for s in srcs]
        if force or jobs or _stale(lib, objs):
            tmp = lib + ".tmp%d" % os.getpid()
            cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "shared", "-o", tmp] + objs + [
                "-Xlinker", "-rpath,/usr/local/cuda/lib64", "-Xlinker", "-z,defs", "-lpthread"]
            subprocess.check_call(cmd)
            os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
