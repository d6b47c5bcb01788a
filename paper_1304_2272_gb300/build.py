"""In-tree build of the engine's C-ABI shared library for sm_103a (GB300).

Every ``csrc/*.cu`` file is compiled in parallel with nvcc into ``_build/`` and
linked into ``libgwas_gb300.so`` next to this file (CUDA runtime linked statically);
``cli/gwas_stream.cpp`` is then built against it into ``gwas_stream`` (a native
out-of-core driver of the C ABI). A source newer than its product triggers a rebuild;
``force=True`` always rebuilds.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

PKG = Path(__file__).resolve().parent
CSRC = PKG / "csrc"
INCLUDE = PKG.parent / "include"
BUILD = PKG / "_build"
LIB = PKG / "libgwas_gb300.so"
CLI_SRC = PKG / "cli" / "gwas_stream.cpp"
CLI = PKG / "gwas_stream"
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-I", str(INCLUDE)]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and Path(cand).exists():
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the engine")


def sources() -> list[Path]:
    return sorted(CSRC.glob("*.cu"))


def _deps() -> list[Path]:
    return sources() + sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + \
        sorted(INCLUDE.glob("*.h"))


def up_to_date() -> bool:
    if not LIB.exists():
        return False
    t = LIB.stat().st_mtime
    return all(p.stat().st_mtime <= t for p in _deps())


def build_cli(force: bool = False) -> Path:
    """Compile the streaming command-line driver against the library."""
    if not force and CLI.exists() and CLI.stat().st_mtime >= max(
            LIB.stat().st_mtime, CLI_SRC.stat().st_mtime, (INCLUDE / "gwas.h").stat().st_mtime):
        return CLI
    cxx = os.environ.get("CXX") or shutil.which("g++") or "g++"
    tmp = CLI.with_suffix(".tmp")
    cmd = [cxx, "-O2", "-std=c++17", "-I", str(INCLUDE), "-o", str(tmp), str(CLI_SRC),
           "-L", str(PKG), "-lgwas_gb300", "-Wl,-rpath,$ORIGIN", "-pthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"building gwas_stream failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, CLI)
    return CLI


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None) -> Path:
    """Compile the library (and the streaming driver) if needed; return the library path."""
    if not force and up_to_date():
        build_cli()
        return LIB
    BUILD.mkdir(exist_ok=True)
    cc = nvcc()
    extra = list(extra or [])

    def compile_one(src: Path) -> Path:
        obj = BUILD / (src.stem + ".o")
        cmd = [cc, *ARCH, *FLAGS, *extra, "-c", str(src), "-o", str(obj)]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src.name}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(len(sources()), os.cpu_count() or 4))) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = LIB.with_suffix(".so.tmp")
    cmd = [cc, *ARCH, "-shared", "-o", str(tmp), *map(str, objs), "-cudart", "static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    build_cli(force=True)
    return LIB


if __name__ == "__main__":
    force = "--force" in sys.argv
    print(build(force=force, verbose="-v" in sys.argv))
