"""Builds libdoe.so (the C-ABI library in include/doe.h) in-tree with nvcc for sm_103a, and its
bounds-checked twin libdoe_debug.so (every kernel compiled with -DDOE_DEBUG: each global,
shared and distributed-shared-memory index is checked against its buffer before the access; a
violation sets DOE_FAULT_BOUNDS, see doe_fault_status, and skips the access).

    python -m paper_2505_22313_b300.build [--force] [-v]

Object files go to paper_2505_22313_b300/_build/ (release) and _build/debug/, the libraries to
paper_2505_22313_b300/libdoe.so and libdoe_debug.so.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
BUILD = PKG / "_build"
LIB = PKG / "libdoe.so"
DEBUG_LIB = PKG / "libdoe_debug.so"  # bounds-checked build, loaded by its own tests only
COMPARE_LIB = PKG / "libdoe_cufft.so"  # cuFFT comparison chain, loaded only by the benchmark
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC,-O2", f"-I{ROOT / 'include'}", f"-I{CSRC}"]
SOURCES = ["doe_pass_mr.cu", "doe_pass_pow2_large.cu", "doe_pass_big.cu", "doe_pass_pow2_small.cu",
           "doe_pass_render.cu", "doe_launch.cu", "doe_api.cu", "doe_render.cu", "doe_noalloc.cu", "doe_design.cu"]


def _deps() -> list[Path]:
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + [ROOT / "include" / "doe.h"]


def _stale(target: Path, deps: list[Path]) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(d.stat().st_mtime > t for d in deps)


def _library(lib: Path, objdir: Path, extra: list[str], link_extra: list[str], deps: list[Path], force: bool,
             verbose: bool) -> Path:
    """Compiles SOURCES into objdir (an object is rebuilt when its own source or any header is
    newer than it) and links them into lib."""
    objdir.mkdir(parents=True, exist_ok=True)
    headers = [d for d in deps if d.suffix != ".cu"]

    def compile_one(src: str) -> Path:
        obj = objdir / (Path(src).stem + ".o")
        if not force and not verbose and not _stale(obj, [CSRC / src, *headers]):
            return obj
        cmd = [NVCC, *FLAGS, *extra, *ARCH, "-c", str(CSRC / src), "-o", str(obj)]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    if force or _stale(lib, objs):
        tmp = lib.with_suffix(f".so.tmp{os.getpid()}")
        cmd = [NVCC, "-shared", *ARCH, "-o", str(tmp), *map(str, objs), "-lcudart", *link_extra]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed for {lib.name}:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    else:
        os.utime(lib)
    return lib


def build(force: bool = False, verbose: bool = False, debug: bool = True) -> Path:
    """Builds libdoe.so and the cuFFT comparison library; with debug also libdoe_debug.so."""
    deps = _deps()
    targets = [LIB, COMPARE_LIB] + ([DEBUG_LIB] if debug else [])
    if not force and not any(_stale(t, deps) for t in targets):
        return LIB
    if force or _stale(LIB, deps) or _stale(COMPARE_LIB, deps):
        _library(LIB, BUILD, [], [], deps, force, verbose)
        _build_compare(verbose)
    if debug and (force or _stale(DEBUG_LIB, deps)):
        # -Bsymbolic: the debug library's internal references bind to itself even when the
        # release library is loaded in the same process
        _library(DEBUG_LIB, BUILD / "debug", ["-DDOE_DEBUG"], ["-Xlinker", "-Bsymbolic"], deps, force, verbose)
    return LIB


def _build_compare(verbose: bool = False) -> Path:
    """The cuFFT-based comparison chain (benchmark only; libdoe never loads it)."""
    obj = BUILD / "compare_cufft.o"
    cmd = [NVCC, *FLAGS, *ARCH, "-c", str(CSRC / "compare_cufft.cu"), "-o", str(obj)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for compare_cufft.cu:\n{r.stdout}\n{r.stderr}")
    tmp = COMPARE_LIB.with_suffix(f".so.tmp{os.getpid()}")
    cmd = [NVCC, "-shared", *ARCH, "-o", str(tmp), str(obj), f"-L{PKG}", "-ldoe", "-lcufft", "-lcudart",
           "-Xlinker", "-rpath,$ORIGIN"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed for libdoe_cufft.so:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, COMPARE_LIB)
    return COMPARE_LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
