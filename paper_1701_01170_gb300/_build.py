"""Build the CUDA library libgr.so for sm_103a (in-tree, under _build/).

Every translation unit in csrc/ is compiled by nvcc in parallel, then linked
into one shared library with the C ABI of include/gr.h.  No torch headers are
involved: the library only sees plain pointers and sizes.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libgr.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "--extended-lambda", "-lineinfo", "-Xcompiler", "-fPIC",
              "-I" + INCLUDE]


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libgr.so")


def sources() -> list[str]:
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))


# the sources each persistent kernel is compiled from (besides gr.h, whose
# declarations of other entry points do not enter the kernel's code)
KERNEL_SOURCES = {
    "bfs": ("gr_bfs.cu", "gr_bfs_body.cuh", "gr_internal.cuh"),
    "sssp": ("gr_sssp.cu", "gr_sssp_body.cuh", "gr_internal.cuh"),
}


def _code_only(text: str) -> bytes:
    """Source text without comments and blank lines (comments do not change a kernel)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln.strip()).encode()


def source_digest(kernel: str | None = None) -> str:
    """Content hash identifying a kernel version: of every CUDA source and the C ABI
    header, or, for kernel "bfs" / "sssp", of the code (comments stripped) of the
    sources that kernel is built from."""
    import hashlib
    h = hashlib.sha256()
    if kernel is None:
        files = sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cuh")))
    else:
        files = sorted(KERNEL_SOURCES[kernel])
    for f in files:
        h.update(f.encode())
        with open(os.path.join(CSRC, f), "rb") as fh:
            data = fh.read()
        h.update(_code_only(data.decode()) if kernel else data)
    if kernel is None:
        with open(os.path.join(INCLUDE, "gr.h"), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _stale(out: str, deps: list[str]) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, defines: tuple = (),
          out_dir: str | None = None) -> str:
    """Compile csrc/*.cu and link libgr.so; returns the library path.

    `defines` (e.g. ("GR_STREAM_COLUMNS=1",)) and `out_dir` build a variant of
    the library elsewhere, for A/B measurements of the build-time switches.
    """
    bdir = out_dir or BUILD
    lib = os.path.join(bdir, "libgr.so")
    os.makedirs(bdir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cuh")]
    headers.append(os.path.join(INCLUDE, "gr.h"))
    cc = nvcc()
    jobs = []
    objs = []
    for src in sources():
        obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            jobs.append([cc, *ARCH, *NVCC_FLAGS, *["-D" + d for d in defines], "-c", src, "-o", obj])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode:
                print(" ".join(cmd))
                print(r.stdout + r.stderr)
            if r.returncode:
                raise RuntimeError(f"nvcc failed for {cmd[-3]}")
    if force or jobs or _stale(lib, objs):
        tmp = lib + f".{os.getpid()}.tmp"
        subprocess.check_call([cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs])
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
