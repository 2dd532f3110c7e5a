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


def _unit_flags(src):
    """Relocatable device code for the persistent kernel's units (its per-shape steps are device
    functions of other units, resolved by a device link); the steps' units at the kernel's register
    budget (128 per thread: __launch_bounds__(128, 4))."""
    name = os.path.basename(src)
    if name.startswith("ds_persist_part_"):
        return ["-rdc=true", "-maxrregcount=128"]
    if name.startswith("ds_persist"):
        return ["-rdc=true"]
    return []


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
    # the large units (the humanoid shapes and the persistent kernel) first, so that they do not
    # start last and set the build's length
    todo = sorted(((s, o) for s, o in zip(srcs, objs) if _stale(s, o)),
                  key=lambda so: (not any(t in os.path.basename(so[0]) for t in ("_31_36_", "persist_part")), so[0]))

    def compile_one(so):
        s, o = so
        cmd = [nvcc] + ARCH + flags + _unit_flags(s) + ["-c", s, "-o", o]
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
        # device link of the relocatable units (the persistent kernel and its per-shape steps)
        rdc = [o for s, o in zip(srcs, objs) if _unit_flags(s)]
        link_objs = list(objs)
        if rdc:
            dlink = os.path.join(obj_dir, "ds_dlink.o")
            r = subprocess.run([nvcc] + ARCH + ["-dlink", "-Xcompiler", "-fPIC"] + rdc + ["-o", dlink],
                               capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("device link failed:\n%s\n%s" % (r.stdout, r.stderr))
            link_objs.append(dlink)
        cmd = [nvcc] + ARCH + ["-shared", "-o", lib + ".tmp"] + link_objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
    sys.exit(0)
