"""Build the in-tree shared library ``lib/libterra_wedge.so`` for sm_103a.

Each translation unit is compiled by its own nvcc process (in parallel) and then
linked; host code is compiled with -ffp-contract=off so that x86 and Arm hosts
build bitwise-identical mesh tables.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "lib")
LIBNAME = "libterra_wedge.so"
# (source, extra flags): kernels.cu is compiled in five parts (the FP64 and the FP32 A-apply
# launchers of each quadrature rule apart)
SOURCES = [("kernels.cu", ["-DTN_PART=1"]), ("kernels.cu", ["-DTN_PART=2"]), ("kernels.cu", ["-DTN_PART=3"]),
           ("kernels.cu", ["-DTN_PART=4"]), ("kernels.cu", ["-DTN_PART=5"]),
           ("solver.cu", []), ("server.cu", []), ("api.cu", []), ("noalloc.cu", []), ("probe.cu", []), ("energy.cu", []), ("mesh.cpp", [])]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def library_path():
    return os.path.join(LIBDIR, LIBNAME)


def build(verbose=False, extra_flags=()):
    """Compile every source and link the shared library; returns its path."""
    os.makedirs(os.path.join(LIBDIR, "obj"), exist_ok=True)
    common = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-ffp-contract=off", *ARCH, *extra_flags]
    procs, objs = [], []
    for i, (src, flags) in enumerate(SOURCES):
        obj = os.path.join(LIBDIR, "obj", "%d_%s.o" % (i, src))
        lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
        cmd = [nvcc(), *common, *flags, *lang, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        procs.append((src, cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)))
        objs.append(obj)
    failed = []
    for src, cmd, p in procs:
        out, _ = p.communicate()
        if verbose or p.returncode != 0:
            sys.stdout.write(out)
        if p.returncode != 0:
            failed.append(src)
    if failed:
        raise RuntimeError("nvcc failed for " + ", ".join(failed))
    tmp = library_path() + ".tmp"
    link = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        sys.stdout.write(r.stdout)
        raise RuntimeError("link failed")
    os.replace(tmp, library_path())
    return library_path()


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
