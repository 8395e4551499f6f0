"""Build libsinv.so in place (nvcc for sm_103a; host code with the same driver).

``python -m paper_2609_11363_b300.build`` or ``build_lib()``.  Objects go to
``_build/`` beside this file; the shared library to ``libsinv.so``.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
OUT = os.path.join(HERE, "libsinv.so")
BUILD = os.path.join(HERE, "_build")
# the checked build: every gather and scatter whose index comes from the plan or the
# maps checks it, records an out-of-range index in the status word and skips the access
OUT_CHECKED = os.path.join(HERE, "libsinv_checked.so")
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
SOURCES = ["api.cu", "selinv.cu", "selinv_tc.cu", "ninv.cu", "ninv_map.cu", "ninv_own.cu", "elementwise.cu", "mlp.cu", "spai.cu", "einv.cu", "symbolic.cpp"]
HEADERS = ["plan.h", "kernels.h", "device.cuh", "hash.cuh", "tc.cuh"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O3", "-I" + INCLUDE]


def _newest_dep():
    files = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(INCLUDE, "sinv.h"), __file__]
    return max(os.path.getmtime(f) for f in files)


def _compile(src, verbose=False, checked=False):
    obj = os.path.join(BUILD_CHECKED if checked else BUILD, src + ".o")
    cmd = [NVCC] + ARCH + FLAGS + (["-DSINV_CHECKED"] if checked else []) + ["-c", os.path.join(CSRC, src), "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    return obj, r.stderr


def build_lib(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    out = OUT_CHECKED if checked else OUT
    if not force and os.path.exists(out) and os.path.getmtime(out) >= _newest_dep():
        return out
    os.makedirs(BUILD_CHECKED if checked else BUILD, exist_ok=True)
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, checked), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_lib(force="--force" in sys.argv, verbose="-v" in sys.argv, checked="--checked" in sys.argv))
