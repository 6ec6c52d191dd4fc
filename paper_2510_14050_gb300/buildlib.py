"""Compile the in-tree shared libraries.

* ``libans.so``       -- the CUDA library behind ``include/ans.h`` (sm_103a only).
* ``libans_synth.so`` -- the seeded synthetic packet generator (host C).

Both land next to this file.  Compilation of the CUDA translation units runs
in parallel; a unit is rebuilt only when its source, a header it includes, or
the flags changed.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
ROOT = PKG.parent
INCLUDE = ROOT / "include"
OBJ = PKG / "_build"

LIBANS = PKG / "libans.so"
LIBSYNTH = PKG / "libans_synth.so"

CUDA_UNITS = ["ans_abi.cu", "ans_sort.cu", "ans_stats.cu", "ans_cluster.cu", "ans_merge.cu", "ans_hash.cu", "ans_noalloc.cu", "ans_plan.cu", "ans_winhash.cu", "ans_split.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libans.so")


def _digest(paths, flags) -> str:
    h = hashlib.sha256()
    for p in paths:
        h.update(Path(p).read_bytes())
    h.update(" ".join(flags).encode())
    return h.hexdigest()


def _run(cmd):
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"command failed ({res.returncode}): {' '.join(map(str, cmd))}\n"
                           f"{res.stdout}\n{res.stderr}")
    return res.stdout + res.stderr


def build_synth(force: bool = False) -> Path:
    src = CSRC / "synth.c"
    flags = ["-O2", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-std=c11"]
    stamp = OBJ / "libans_synth.sha"
    dig = _digest([src], flags)
    if not force and LIBSYNTH.exists() and stamp.exists() and stamp.read_text() == dig:
        return LIBSYNTH
    OBJ.mkdir(exist_ok=True)
    tmp = LIBSYNTH.with_suffix(".so.tmp")
    _run(["gcc", *flags, str(src), "-o", str(tmp), "-lm"])
    os.replace(tmp, LIBSYNTH)
    stamp.write_text(dig)
    return LIBSYNTH


def build_ans(force: bool = False, verbose: bool = False) -> Path:
    nvcc = _nvcc()
    headers = sorted(CSRC.glob("*.cuh")) + [INCLUDE / "ans.h"]
    flags = [*NVCC_FLAGS, *ARCH, f"-I{INCLUDE}", f"-I{CSRC}"]
    OBJ.mkdir(exist_ok=True)
    all_dig = _digest([CSRC / u for u in CUDA_UNITS] + headers, flags)
    stamp = OBJ / "libans.sha"
    if not force and LIBANS.exists() and stamp.exists() and stamp.read_text() == all_dig:
        return LIBANS

    def compile_unit(unit):
        obj = OBJ / (unit + ".o")
        dig = _digest([CSRC / unit] + headers, flags)
        ustamp = OBJ / (unit + ".sha")
        if not force and obj.exists() and ustamp.exists() and ustamp.read_text() == dig:
            return ""
        out = _run([nvcc, *flags, "-c", str(CSRC / unit), "-o", str(obj)])
        ustamp.write_text(dig)
        return out

    with cf.ThreadPoolExecutor(max_workers=len(CUDA_UNITS)) as ex:
        logs = list(ex.map(compile_unit, CUDA_UNITS))
    if verbose:
        for unit, log in zip(CUDA_UNITS, logs):
            if log.strip():
                print(f"--- {unit}\n{log}")
    tmp = LIBANS.with_suffix(".so.tmp")
    _run([nvcc, *ARCH, "-shared", "-o", str(tmp), *[str(OBJ / (u + ".o")) for u in CUDA_UNITS],
          "-lcudart"])
    os.replace(tmp, LIBANS)
    stamp.write_text(all_dig)
    return LIBANS


def build_all(force: bool = False, verbose: bool = False) -> None:
    with cf.ThreadPoolExecutor(max_workers=2) as ex:
        f1 = ex.submit(build_synth, force)
        f2 = ex.submit(build_ans, force, verbose)
        f1.result()
        f2.result()


if __name__ == "__main__":
    import sys
    build_all(force="--force" in sys.argv, verbose=True)
    print(LIBANS, LIBSYNTH)
