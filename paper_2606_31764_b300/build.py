"""Builds the CUDA library in-tree: csrc/*.cu -> libnurbs_splat.so (sm_103a).

Each translation unit is compiled on its own (in parallel) into _build/, then
the objects are linked into the shared library."""
import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIB = os.path.join(HERE, "libnurbs_splat.so")
OBJ = os.path.join(ROOT, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def sources():
    return sorted(glob.glob(os.path.join(HERE, "csrc", "*.cu")))


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r.returncode, r.stdout + r.stderr


def build(verbose=False, extra=()):
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ, exist_ok=True)
    inc = ["-I", os.path.join(ROOT, "include")]
    jobs = []
    for src in sources():
        obj = os.path.join(OBJ, os.path.splitext(os.path.basename(src))[0] + ".o")
        jobs.append((obj, [nvcc, *ARCH, *FLAGS, *inc, *extra, "-c", src, "-o", obj]))
    with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
        results = list(ex.map(lambda j: _run(j[1]), jobs))
    for (obj, cmd), (rc, out) in zip(jobs, results):
        if verbose:
            print(" ".join(cmd))
        if rc != 0:
            sys.stderr.write(out)
            raise RuntimeError("nvcc failed on " + cmd[-3])
        if verbose and out:
            print(out)
    rc, out = _run([nvcc, *ARCH, "-shared", "-o", LIB, *[j[0] for j in jobs]])
    if rc != 0:
        sys.stderr.write(out)
        raise RuntimeError("link failed")
    return LIB


if __name__ == "__main__":
    build(verbose=True, extra=sys.argv[1:])
