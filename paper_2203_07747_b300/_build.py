"""Build librtn.so in-tree with nvcc for sm_103a (B300): every .cu file is
compiled to an object in parallel, then the objects are linked."""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "librtn.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-Xptxas", "-v"]
LIBS = []


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + [
        os.path.join(HERE, "..", "include", "rtn.h")]


def stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in sources() + headers())


def _obj(src):
    return os.path.join(OBJ, os.path.basename(src)[:-3] + ".o")


def _compile(nvcc, src, force):
    o = _obj(src)
    newest = max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in headers()])
    if not force and os.path.exists(o) and os.path.getmtime(o) >= newest:
        return src, 0, ""
    tmp = o + ".tmp%d" % os.getpid()
    r = subprocess.run([nvcc] + ARCH + FLAGS + ["-c", "-o", tmp, src], capture_output=True, text=True)
    if r.returncode == 0:
        os.replace(tmp, o)
    return src, r.returncode, r.stdout + r.stderr


def build(force=False, verbose=False):
    if not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    srcs = sources()
    with ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        results = list(ex.map(lambda s: _compile(nvcc, s, force), srcs))
    failed = [r for r in results if r[1] != 0]
    for src, rc, log in results:
        if verbose or rc != 0:
            sys.stderr.write(log)
    if failed:
        raise RuntimeError("nvcc failed building librtn.so: " + ", ".join(os.path.basename(f[0]) for f in failed))
    tmp = LIB + ".tmp%d" % os.getpid()
    r = subprocess.run([nvcc] + ARCH + ["-shared", "-o", tmp] + [_obj(s) for s in srcs] + LIBS,
                       capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
        raise RuntimeError("nvcc failed linking librtn.so")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
