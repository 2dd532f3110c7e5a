"""Build libdiffsim.so (CUDA, sm_103a) in-tree: one nvcc process per translation unit, in parallel.

    python -m paper_2409_07107_gb300.build          # or: import __graft_entry__; __graft_entry__.build()
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdiffsim.so")
OBJ_CHECK = os.path.join(HERE, "_build_check")
LIB_CHECK = os.path.join(HERE, "libdiffsim_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for c in (os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc"), "nvcc"):
        if os.path.sep not in c or os.path.exists(c):
            return c
    return "nvcc"


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


def _stale(src, obj):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".inc"))]
    deps.append(os.path.join(INCLUDE, "diffsim.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose=False, jobs=None, check=False):
    """Compile every .cu under csrc/ and link libdiffsim.so (with check=True: the checked build,
    -DDS_CHECK, as libdiffsim_check.so, objects apart).  Returns the library path."""
    obj_dir = OBJ_CHECK if check else OBJ
    lib = LIB_CHECK if check else LIB
    flags = FLAGS + (["-DDS_CHECK"] if check else [])
    os.makedirs(obj_dir, exist_ok=True)
    nvcc = _nvcc()
    srcs = sources()
    objs = [os.path.join(obj_dir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    todo = [(s, o) for s, o in zip(srcs, objs) if _stale(s, o)]

    def compile_one(so):
        s, o = so
        cmd = [nvcc] + ARCH + flags + ["-c", s, "-o", o]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (s, r.stdout, r.stderr))
        return s

    if todo:
        n = jobs or max(1, min(len(todo), os.cpu_count() or 1))
        with cf.ThreadPoolExecutor(max_workers=n) as ex:
            for s in ex.map(compile_one, todo):
                if verbose:
                    print("compiled", os.path.basename(s), flush=True)
    if todo or not os.path.exists(lib):
        cmd = [nvcc] + ARCH + ["-shared", "-o", lib + ".tmp"] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
    sys.exit(0)
