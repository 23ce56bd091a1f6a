"""Build the CUDA library libchol.so in-tree for sm_103a (nvcc + g++, no cmake).

The translation units are compiled in parallel and linked into
``paper_2409_14009_gb300/_build/libchol.so``.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libchol.so")
# the bounds-checked variant (-DCHOL_BOUNDS_CHECK), built on request
OUT_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(OUT_CHECKED, "libchol.so")
INC = os.path.join(ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")


def _sources():
    return sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs += [os.path.join(INC, f) for f in os.listdir(INC) if f.endswith(".h")]
    return hs


def _compile(src, out=OUT, defs=()):
    obj = os.path.join(out, src + ".o")
    path = os.path.join(CSRC, src)
    if src.endswith(".cu"):
        cmd = [NVCC, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", *defs,
               "-I", INC, "-I", CSRC, "-c", path, "-o", obj]
    else:
        cmd = [NVCC, "-O2", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-pthread", "-x", "c++", *defs,
               "-I", INC, "-I", CSRC, "-c", path, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("compile failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return obj


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    """Build libchol.so (or, with checked=True, the bounds-checked variant in _build_checked/)."""
    out, lib = (OUT_CHECKED, LIB_CHECKED) if checked else (OUT, LIB)
    defs = ("-DCHOL_BOUNDS_CHECK",) if checked else ()
    os.makedirs(out, exist_ok=True)
    srcs = _sources()
    deps = [os.path.join(CSRC, s) for s in srcs] + _headers() + [os.path.abspath(__file__)]
    if not force and os.path.exists(lib):
        t = os.path.getmtime(lib)
        if all(os.path.getmtime(d) <= t for d in deps):
            return lib
    with ThreadPoolExecutor(max_workers=max(2, len(srcs))) as ex:
        objs = list(ex.map(lambda f: _compile(f, out, defs), srcs))
    tmp = lib + ".%d.tmp" % os.getpid()
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static", "-lpthread", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    os.replace(tmp, lib)
    if verbose:
        print(lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv))
