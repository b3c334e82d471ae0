"""Build libdg.so in-tree: hand-written CUDA for sm_103a plus the C++ host side.

Each translation unit is compiled by its own nvcc process (in parallel), then
linked into ``paper_1506_06140_gb300/libdg.so`` with the CUDA runtime linked
statically.  Objects go to ``paper_1506_06140_gb300/_build/``.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["dg_inst_3d_f64.cu", "dg_inst_3d_f32.cu", "dg_inst_2d_f64.cu", "dg_inst_2d_f32.cu", "dg_inst_2d_tensor.cu",
           "dg_mixed_3d.cu", "dg_mixed_2d.cu", "dg_common.cu", "dg_noalloc.cu", "dg_regrid.cu",
           "dg_host.cpp"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include"),
         "-I", CSRC]


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "dg.h"))
    return files


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(f) > t for f in _deps() + [src])


def build(force=False, verbose=False, extra_flags=()):
    """Compile stale objects and link libdg.so; returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        if not os.path.exists(path):
            continue
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        if force or _stale(obj, path):
            cmd = [NVCC] + ARCH + FLAGS + list(extra_flags) + ["-c", path, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [NVCC] + FLAGS + list(extra_flags) + ["-x", "c++", "-c", path, "-o", obj]
            jobs.append(cmd)

    def run(cmd):
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    relink = bool(jobs) or not os.path.exists(LIB)
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, r in ex.map(run, jobs):
            if r.returncode != 0:
                raise RuntimeError("nvcc failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
            if verbose and (r.stdout or r.stderr):
                print(r.stdout + r.stderr)
    if relink:
        cmd = [NVCC] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcuda"] * 0
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s" % (r.stdout, r.stderr))
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    extra = [a for a in sys.argv[1:] if a.startswith("-X") or a.startswith("--")]
    extra = [a for a in extra if a != "--force"]
    build(force="--force" in sys.argv, verbose=True, extra_flags=extra)
