"""Compile liblbmfreeze.so for sm_103a (nvcc, in-tree, no torch extension).

Each translation unit is compiled in parallel, then linked into
``paper_2403_16122_gb300/_build/liblbmfreeze.so``. The kernel source is
compiled once per part (``-DLBM_PART=k``: the storage dispatch with the tile,
initialisation and reduction kernels, then the strip kernels of each storage
type and kind), each compilation whole. nvcc's own partitioning of a file for
parallel compilation (``--split-compile``) is not deterministic: two builds
of the same source gave one kernel no spills and then 392 bytes of them.
Rebuilds only when a source or header is newer than the library.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import re
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(PKG, "_build")
LIB = os.path.join(OUT_DIR, "liblbmfreeze.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}"]
# sources compiled once per part, with the number of parts; a part leaves the
# helpers that only other parts use unreferenced (diagnostic 177)
PARTS = {"lbm_kernels.cu": 9}
PART_FLAGS = ["-diag-suppress=177"]


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build liblbmfreeze")
    return cand


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def jobs():
    """(source, part or None) of every compilation."""
    out = []
    for src in sources():
        n = PARTS.get(os.path.basename(src))
        out += [(src, k) for k in range(n)] if n else [(src, None)]
    return out


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) \
        + glob.glob(os.path.join(INCLUDE, "*.h")) + [os.path.abspath(__file__)]
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    cc = nvcc()
    objs = []

    def compile_one(job):
        src, part = job
        base = os.path.basename(src) + ("" if part is None else f".part{part}")
        obj = os.path.join(OUT_DIR, base + ".o")
        # the register and spill report of every kernel is kept beside the
        # object (ptxas_report reads it)
        cmd = [cc, *ARCH, *FLAGS, *([] if part is None else [f"-DLBM_PART={part}", *PART_FLAGS]),
               "-Xptxas=-v", "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        with open(obj + ".ptxas.txt", "w") as f:
            f.write(r.stderr)
        return obj, r.stderr

    todo = jobs()
    with cf.ThreadPoolExecutor(max_workers=max(1, len(todo))) as ex:
        for obj, log in ex.map(compile_one, todo):
            objs.append(obj)
            if verbose and log:
                print(log)
    tmp = LIB + f".tmp{os.getpid()}"
    r = subprocess.run([cc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


def ptxas_report() -> dict:
    """{mangled kernel name: (registers, spill store bytes)} from the report of
    the last build."""
    out = {}
    names = {os.path.basename(src) + ("" if k is None else f".part{k}") for src, k in jobs()}
    for path in glob.glob(os.path.join(OUT_DIR, "*.o.ptxas.txt")):
        if os.path.basename(path)[: -len(".o.ptxas.txt")] not in names:
            continue  # left by an earlier layout of the build
        cur, spill = None, 0
        for line in open(path):
            m = re.search(r"Compiling entry function '([^']+)'", line)
            if m:
                cur, spill = m.group(1), 0
                continue
            m = re.search(r"(\d+) bytes spill stores", line)
            if m and cur:
                spill = int(m.group(1))
            m = re.search(r"Used (\d+) registers", line)
            if m and cur:
                out[cur] = (int(m.group(1)), spill)
                cur = None
    return out


if __name__ == "__main__":
    print(build(force=True, verbose=True))
