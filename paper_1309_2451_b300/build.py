"""Build libctap.so (the CUDA library behind include/ctap.h) in place, for
sm_103a only.  nvcc cross-compiles without a GPU."""
import glob
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libctap.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-Wall",
         "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _compile(src, obj, extra, verbose):
    cmd = ["nvcc", *ARCH, *FLAGS, *extra, "-c", "-o", obj, src]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return obj


DEBUG_LIB = os.path.join(HERE, "libctap_debug.so")


def build(force=False, verbose=False, extra=(), debug=False):
    """Compile the csrc/*.cu files whose objects are out of date in parallel
    (one nvcc per file; the largest file bounds the wall time), then link
    libctap.so.  debug=True also links libctap_debug.so, the bounds-checked
    build: the sources that include bounds.cuh recompiled with
    -DCTAP_DEBUG_BOUNDS (objects under _build/debug), the others shared."""
    from concurrent.futures import ThreadPoolExecutor
    objdir = os.path.join(HERE, "_build")
    os.makedirs(objdir, exist_ok=True)
    srcs = sources()
    objs = [os.path.join(objdir, os.path.basename(s)[:-3] + ".o") for s in srcs]
    def deps(path, seen):
        """path and every file it includes with #include "..." (recursively)."""
        if path in seen or not os.path.exists(path):
            return seen
        seen.add(path)
        with open(path, errors="replace") as f:
            for line in f:
                line = line.strip()
                if line.startswith("#include") and '"' in line:
                    inc = line.split('"')[1]
                    deps(os.path.normpath(os.path.join(os.path.dirname(path), inc)), seen)
        return seen

    def stale(src, obj):
        if force or extra or not os.path.exists(obj):
            return True
        t = os.path.getmtime(obj)
        return any(os.path.getmtime(d) > t for d in deps(src, set()))

    todo = [(s, o) for s, o in zip(srcs, objs) if stale(s, o)]
    if todo:
        with ThreadPoolExecutor(max_workers=len(todo)) as ex:
            list(ex.map(lambda so: _compile(so[0], so[1], extra, verbose), todo))
    if todo or not os.path.exists(LIB) or \
            any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        _link(LIB, objs, verbose)
    if debug:
        bounds = os.path.join(CSRC, "bounds.cuh")
        ddir = os.path.join(objdir, "debug")
        os.makedirs(ddir, exist_ok=True)
        dobjs = []
        for src, obj in zip(srcs, objs):
            if bounds in deps(src, set()):
                dobj = os.path.join(ddir, os.path.basename(obj))
                if stale(src, dobj):
                    _compile(src, dobj, ["-DCTAP_DEBUG_BOUNDS", *extra], verbose)
                dobjs.append(dobj)
            else:
                dobjs.append(obj)
        if not os.path.exists(DEBUG_LIB) or \
                any(os.path.getmtime(o) > os.path.getmtime(DEBUG_LIB) for o in dobjs):
            _link(DEBUG_LIB, dobjs, verbose)
    return LIB


def _link(lib, objs, verbose):
    cmd = ["nvcc", *ARCH, "-shared", "-o", lib + ".tmp", *objs]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    os.replace(lib + ".tmp", lib)


if __name__ == "__main__":
    extra = ["-Xptxas", "-v"] if "--ptxas" in sys.argv else []
    print(build(force=True, verbose=True, extra=extra))
