"""In-tree build of the native libraries (sm_103a only).

  _build/libmg.so             the Mixture Graph library (C-ABI, include/mg.h)
  _build/libmgsynth_dev.so    GPU generator of the synthetic test volumes
  _build/libmgsynth_host.so   host generator of the synthetic test volumes

Translation units compile in parallel with nvcc / gcc; no cmake.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_CSRC = os.path.join(_HERE, "csrc")
_BUILD = os.path.join(_HERE, "_build")
_ROOT = os.path.dirname(_HERE)
_INCLUDE = os.path.join(_ROOT, "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "-Xptxas", "-warn-spills"]


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def _stale(out: str, deps) -> bool:
    if not os.path.exists(out):
        return True
    t = os.path.getmtime(out)
    return any(os.path.getmtime(d) > t for d in deps)


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed: %s\n%s\n%s" % (" ".join(cmd), r.stdout, r.stderr))
    return r.stdout + r.stderr


def _headers():
    return (glob.glob(os.path.join(_CSRC, "*.cuh")) + glob.glob(os.path.join(_CSRC, "*.h"))
            + glob.glob(os.path.join(_INCLUDE, "*.h")))


def build_synth_host(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_CSRC, "synth_host.c")
    out = os.path.join(_BUILD, "libmgsynth_host.so")
    if force or _stale(out, [src]):
        tmp = out + ".%d.tmp" % os.getpid()
        _run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", src, "-o", tmp, "-lm"])
        os.replace(tmp, out)
    return out


def build_synth_dev(force: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    src = os.path.join(_CSRC, "synth_dev.cu")
    out = os.path.join(_BUILD, "libmgsynth_dev.so")
    if force or _stale(out, [src]):
        tmp = out + ".%d.tmp" % os.getpid()
        _run([_nvcc()] + ARCH + NVCC_FLAGS + ["-shared", src, "-o", tmp])
        os.replace(tmp, out)
    return out


def mg_sources():
    return sorted(glob.glob(os.path.join(_CSRC, "mg_*.cu")))


def build_mg(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(_BUILD, exist_ok=True)
    out = os.path.join(_BUILD, "libmg.so")
    srcs = mg_sources()
    hdrs = _headers()
    objs = []
    jobs = []
    for s in srcs:
        o = os.path.join(_BUILD, os.path.basename(s)[:-3] + ".o")
        objs.append(o)
        if force or _stale(o, [s] + hdrs):
            cmd = [_nvcc()] + ARCH + NVCC_FLAGS + ["-I", _INCLUDE, "-I", _CSRC, "-c", s, "-o", o]
            if verbose:
                cmd += ["-Xptxas", "-v"]
            jobs.append(cmd)
    logs = []
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            logs = list(ex.map(_run, jobs))
    if force or jobs or _stale(out, objs):
        tmp = out + ".%d.tmp" % os.getpid()
        _run([_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"])
        os.replace(tmp, out)
    if verbose:
        for l in logs:
            print(l)
    return out


def build_all(force: bool = False, verbose: bool = False):
    with cf.ThreadPoolExecutor(max_workers=3) as ex:
        fs = [ex.submit(build_mg, force, verbose), ex.submit(build_synth_dev, force),
              ex.submit(build_synth_host, force)]
        return [f.result() for f in fs]


if __name__ == "__main__":
    import sys
    print(build_all(force="--force" in sys.argv, verbose="-v" in sys.argv))
