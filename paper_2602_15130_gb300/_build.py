"""In-tree build of the CUDA library ``libpic_gb300.so`` for sm_103a.

Each translation unit is compiled in parallel with nvcc, then linked with
nvcc -shared. Outputs live next to the sources and are git-ignored.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build_objs"
LIB = PKG / "libpic_gb300.so"
SOURCES = ["pic_api.cu", "k_particles.cu", "k_sort.cu", "k_field.cu", "k_mixed.cu", "k_batch.cu", "k_angles.cu",
           "k_adjoint.cu", "k_peaks.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = [
    "-O3", "-std=c++17", "-lineinfo", *ARCH,
    "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
    "--expt-relaxed-constexpr",
]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def _stale(target: Path, deps) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(d).stat().st_mtime > t for d in deps)


def build_library(force: bool = False, verbose: bool = False) -> Path:
    BUILD.mkdir(exist_ok=True)
    headers = [CSRC / "pic_internal.cuh", CSRC / "mixed_common.cuh", CSRC / "ntc_fp64.cuh", PKG.parent / "include" / "pic.h"]
    cc = nvcc()
    jobs = []
    for src in SOURCES:
        s = CSRC / src
        o = BUILD / (src + ".o")
        if force or _stale(o, [s, *headers]):
            jobs.append([cc, *NVCC_FLAGS, "-c", str(s), "-o", str(o)])
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for r in ex.map(lambda cmd: subprocess.run(cmd, capture_output=True, text=True), jobs):
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed:\n" + " ".join(r.args) + "\n" + r.stdout + r.stderr)
                if verbose and (r.stdout or r.stderr):
                    print(r.stdout + r.stderr)
    objs = [BUILD / (s + ".o") for s in SOURCES]
    if force or jobs or _stale(LIB, objs):
        tmp = LIB.with_suffix(f".so.{os.getpid()}.tmp")
        r = subprocess.run([cc, *ARCH, "-shared", *map(str, objs), "-o", str(tmp), "-lcudart"],
                           capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
        os.replace(tmp, LIB)
    return LIB
