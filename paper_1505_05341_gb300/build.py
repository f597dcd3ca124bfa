"""Build libystat.so in-tree for sm_103a with nvcc (no cmake).

    python -m paper_1505_05341_gb300.build          # or build_library() from Python

Every .cu file under csrc/ is compiled in parallel to csrc/../_build/*.o, then linked
into paper_1505_05341_gb300/libystat.so (static CUDA runtime).  The generated
k-polynomial table csrc/group_table.inc is refreshed from gen_group_table.py first.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libystat.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# Host code must not contract a + b*c into an FMA: the node offsets and shell edges
# it builds in FP64 have to round exactly as their plain definitions do (gcc on
# aarch64 contracts by default).
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
         "--expt-relaxed-constexpr"]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libystat")
    return cand


def _gen_table():
    out = os.path.join(CSRC, "group_table.inc")
    txt = subprocess.run([sys.executable, os.path.join(CSRC, "gen_group_table.py")], check=True,
                         capture_output=True, text=True).stdout
    old = open(out).read() if os.path.exists(out) else None
    if txt != old:
        with open(out, "w") as fh:
            fh.write(txt)


def _compile(nvcc, src, obj, verbose):
    extra = os.environ.get("YS_NVCC_FLAGS", "").split()
    cmd = [nvcc, *FLAGS, *extra, *ARCH, "-I", os.path.join(HERE, "..", "include"), "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed on {os.path.basename(src)}:\n{r.stdout}\n{r.stderr}")
    return r.stderr


def build_library(force: bool = False, verbose: bool = False, jobs: int | None = None) -> str:
    """Compile and link libystat.so; returns its path.  Skips the work when the
    library is newer than every source unless ``force``."""
    _gen_table()
    srcs = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(HERE, "..", "include", "ystat.h")]
    if not force and os.path.exists(LIB):
        t = os.path.getmtime(LIB)
        if all(os.path.getmtime(d) <= t for d in deps):
            return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs = [os.path.join(BUILD, os.path.basename(s)[:-3] + ".o") for s in srcs]
    jobs = jobs or min(len(srcs), os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        logs = list(ex.map(lambda so: _compile(nvcc, so[0], so[1], verbose), zip(srcs, objs)))
    if verbose:
        for s, log in zip(srcs, logs):
            print(f"== {os.path.basename(s)}\n{log}")
    tmp = LIB + ".tmp"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_library(force="--force" in sys.argv, verbose="-v" in sys.argv))
