"""In-tree build of the package's native libraries.

- ``scene/libscene.so``: the seeded scene generator (host C, OpenMP).
- ``lib/libsvgf.so``: the C-ABI denoiser library (CUDA for sm_103a + host C++).

Each library is rebuilt only when a source is newer than the built file. Sources compile in
parallel; the CUDA build uses one ``-gencode`` (compute_103a/sm_103a).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys
from pathlib import Path

PKG = Path(__file__).resolve().parent
SCENE_SRC = [PKG / "scene" / "scene.c"]
SCENE_LIB = PKG / "scene" / "libscene.so"
CSRC = PKG / "csrc"
SVGF_LIB = PKG / "lib" / "libsvgf.so"
INCLUDE = PKG.parent / "include"

NVCC_ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale(target: Path, sources) -> bool:
    if not target.exists():
        return True
    t = target.stat().st_mtime
    return any(Path(s).stat().st_mtime > t for s in sources)


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: " + " ".join(map(str, cmd)) + "\n" + r.stdout)
    return r.stdout


def build_scene(force: bool = False) -> Path:
    if force or _stale(SCENE_LIB, SCENE_SRC):
        tmp = SCENE_LIB.with_suffix(f".tmp{os.getpid()}.so")
        _run(["gcc", "-std=gnu11", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", str(tmp)]
             + [str(s) for s in SCENE_SRC] + ["-lm"])
        os.replace(tmp, SCENE_LIB)
    return SCENE_LIB


def _cuda_sources():
    return sorted(CSRC.glob("*.cu")) + sorted(CSRC.glob("*.cpp"))


def _headers():
    return sorted(CSRC.glob("*.cuh")) + sorted(CSRC.glob("*.h")) + sorted(INCLUDE.glob("*.h"))


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA library cannot be built")


def build_svgf(force: bool = False, extra_flags=()) -> Path:
    srcs = _cuda_sources()
    deps = srcs + _headers()
    if not (force or _stale(SVGF_LIB, deps)):
        return SVGF_LIB
    nvcc = nvcc_path()
    objdir = PKG / "lib" / "_obj"
    objdir.mkdir(parents=True, exist_ok=True)
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", f"-I{INCLUDE}", f"-I{CSRC}"]
    jobs = []
    for s in srcs:
        o = objdir / (s.stem + ".o")
        if s.suffix == ".cu":
            cmd = [nvcc, *NVCC_ARCH, "-lineinfo", *common, *extra_flags, "-c", str(s), "-o", str(o)]
        else:
            cmd = [nvcc, *common, *extra_flags, "-c", str(s), "-o", str(o)]
        jobs.append((cmd, o))
    with cf.ThreadPoolExecutor(max_workers=min(8, len(jobs))) as ex:
        list(ex.map(lambda j: _run(j[0]), jobs))
    tmp = SVGF_LIB.with_suffix(f".tmp{os.getpid()}.so")
    _run([nvcc, *NVCC_ARCH, "-shared", "-cudart", "shared", "-Xlinker", "-rpath", "-Xlinker",
          os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64"), "-o", str(tmp)] + [str(o) for _, o in jobs])
    os.replace(tmp, SVGF_LIB)
    return SVGF_LIB


if __name__ == "__main__":
    build_scene(force="--force" in sys.argv)
    build_svgf(force="--force" in sys.argv)
    print("built", SCENE_LIB, SVGF_LIB)
