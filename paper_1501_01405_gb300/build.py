"""Build the engine's shared library (libmrip.so) for sm_103a, in-tree.

Every translation unit under csrc/ is compiled by nvcc in parallel with
`-gencode arch=compute_103a,code=sm_103a -lineinfo -O3`, then linked into
paper_1501_01405_gb300/_build/libmrip.so with the CUDA runtime linked
statically.  A unit is recompiled only when it or a header is newer than its
object file.

build(variant="debug") compiles the same sources with -DMRIP_DEBUG (the
kernels' bounds checks, read by mrip_debug_checks) into
_build_debug/libmrip_debug.so, linked -Bsymbolic so that it can be loaded
beside the release library.
"""
import glob
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libmrip.so")
VARIANTS = {
    "release": (OUT, LIB, [], []),
    "debug": (os.path.join(HERE, "_build_debug"), os.path.join(HERE, "_build_debug", "libmrip_debug.so"),
              ["-DMRIP_DEBUG"], ["-Xlinker", "-Bsymbolic"]),
}
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _headers():
    return sorted(glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h")))


def _compile(src, extra, out=OUT):
    obj = os.path.join(out, os.path.basename(src) + ".o")
    newest = max([os.path.getmtime(src)] + [os.path.getmtime(h) for h in _headers()])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest:
        return obj
    tmp = obj + ".tmp.%d.o" % os.getpid()
    cmd = [nvcc()] + ARCH + NVCC_FLAGS + extra + ["-c", src, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    os.replace(tmp, obj)
    return obj


def build(force=False, extra_flags=None, jobs=None, variant="release"):
    """Compile csrc/*.cu and link the variant's library (release:
    _build/libmrip.so); returns the library path."""
    out, lib, vflags, lflags = VARIANTS[variant]
    os.makedirs(out, exist_ok=True)
    extra = vflags + list(extra_flags or [])
    if force:
        for o in glob.glob(os.path.join(out, "*.o")):
            os.remove(o)
    srcs = _sources()
    with ThreadPoolExecutor(max_workers=jobs or min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra, out), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if os.path.exists(lib) and os.path.getmtime(lib) >= newest and not force:
        return lib
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [nvcc()] + ARCH + ["-shared", "-cudart", "static"] + lflags + ["-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


def ptxas_report():
    """Register / spill / shared-memory report of every kernel (-Xptxas -v)."""
    lines = []
    for src in _sources():
        cmd = [nvcc()] + ARCH + NVCC_FLAGS + ["-Xptxas", "-v", "-c", src, "-o", os.devnull]
        r = subprocess.run(cmd, capture_output=True, text=True)
        lines.append("== " + os.path.basename(src))
        lines.extend(l for l in r.stderr.splitlines() if "ptxas" in l)
    return "\n".join(lines)


if __name__ == "__main__":
    print(build(force=True))
