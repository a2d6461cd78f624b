"""Build ``libnnm.so`` (the sm_103a CUDA library behind include/nnm.h) in-tree.

Every ``csrc/*.cu`` translation unit is compiled by nvcc in parallel for
``compute_103a``/``sm_103a`` only, then linked into
``paper_1402_3789_gb300/_build/libnnm.so``.  Cross-compiling needs no GPU.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# translation units: (output name, source, extra defines)
# (the FP32 sweep once per feature width, and the long units first)
UNITS = [(f"sweep_fp32_d{D}", "sweep_fp32.cu", [f"-DNNM_SWEEP_FP32_D={D}"]) for D in (25, 32, 28, 24, 20, 16, 12, 8, 4)] + [
    ("sweep_tc", "sweep_tc.cu", []),
    ("nnm_api", "nnm_api.cu", []),
    ("prep", "prep.cu", []),
    ("rerank", "rerank.cu", []),
    ("rounds", "rounds.cu", []),
    ("sort", "sort.cu", []),
    ("restrict", "restrict.cu", []),
    ("dendro", "dendro.cu", []),
    ("restrict_static", "restrict_static.cu", []),
    ("literal", "literal.cu", []),
]
# the arithmetic-peak microbenchmarks (roofline denominators): a library of their own
PEAK_UNITS = [("peaks", "peaks.cu", [])]


def nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def library_path() -> str:
    return os.path.join(BUILD, "libnnm.so")


def peaks_library_path() -> str:
    return os.path.join(BUILD, "libnnm_peaks.so")


def _sources_mtime() -> float:
    paths = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    paths.append(os.path.join(ROOT, "include", "nnm.h"))
    paths.append(os.path.abspath(__file__))
    return max(os.path.getmtime(p) for p in paths)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    out = library_path()
    peaks = peaks_library_path()
    if (not force and os.path.exists(out) and os.path.exists(peaks)
            and min(os.path.getmtime(out), os.path.getmtime(peaks)) >= _sources_mtime()):
        return out
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    common = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
                     "-I", CSRC]
    if ptxas_info:
        common += ["-Xptxas", "-v"]

    # a unit is recompiled when its object is older than its source, any header, this
    # script, or when the build is forced
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(ROOT, "include", "nnm.h"), os.path.abspath(__file__)]
    newest_header = max(os.path.getmtime(h) for h in headers)

    def compile_unit(unit):
        name, src, defs = unit
        obj = os.path.join(BUILD, name + ".o")
        if (not force and os.path.exists(obj)
                and os.path.getmtime(obj) >= max(newest_header, os.path.getmtime(os.path.join(CSRC, src)))):
            return obj, ""
        cmd = [cc] + common + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=min(len(UNITS), os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_unit, UNITS + PEAK_UNITS))
    if verbose or ptxas_info:
        for _, err in results:
            if err:
                sys.stderr.write(err)

    def link(target, objs):
        tmp = target + f".tmp{os.getpid()}"
        cmd = [cc] + ARCH + ["-shared", "-cudart", "shared", "-Xlinker", "-rpath=/usr/local/cuda/lib64",
                             "-o", tmp] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, target)

    link(peaks, [o for o, _ in results[len(UNITS):]])
    link(out, [o for o, _ in results[: len(UNITS)]])
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
