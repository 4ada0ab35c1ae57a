"""Build the CUDA libraries in-tree for sm_103a with nvcc (no cmake, no torch extension machinery).

  libdg.so       the RHS library declared in include/dg.h
  libdgpeaks.so  ALU-throughput microbenchmarks used for the roofline denominators

Translation units compile in parallel; a library is rebuilt only when a source or header is newer.
Usage: python -m paper_2112_10517_gb300.build [--force] [--ptxas-info]
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
NVFLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I", os.path.join(ROOT, "include")]

# volume_inst.cu is compiled once per (dimension, flux precision, node-count range): the volume kernels are the
# bulk of the compile time, and separate objects compile in parallel.
VOLUME_OBJS = [("volume_inst.cu", "vol%dd_%s_n%d%d" % (nd, t, lo, hi),
                ["-DVOL_ND=%d" % nd, "-DVOL_T=%s" % ("double" if t == "f64" else "float"),
                 "-DVOL_NLO=%d" % lo, "-DVOL_NHI=%d" % hi])
               for nd in (2, 3) for t in ("f64", "f32") for lo, hi in ((2, 5), (6, 7), (8, 8))]

LIBS = {
    "libdg.so": ["host.cu", "volume.cu", "interface.cu", "misc.cu", "noalloc.cu", "batch.cu", "vjp.cu", "gauss.cu"]
                + VOLUME_OBJS,
    "libdgpeaks.so": ["peaks.cu"],
}
HEADERS = ["dg_internal.h", "kernels.cuh", "dgmath.cuh", "volume_impl.cuh", "volume_pipe.cuh", "tile_plan.h"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libdg.so")


def _newest(paths):
    return max(os.path.getmtime(p) for p in paths)


def lib_path(name: str = "libdg.so") -> str:
    return os.path.join(HERE, name)


def build(force: bool = False, ptxas_info: bool = False, verbose: bool = False) -> dict:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "dg.h")]
    out = {}
    jobs = []
    for lib, srcs in LIBS.items():
        target = lib_path(lib)
        units = [(s, s, []) if isinstance(s, str) else s for s in srcs]  # (source, object name, defines)
        src_paths = sorted({os.path.join(CSRC, u[0]) for u in units})
        deps = src_paths + headers + [os.path.join(ROOT, "include", "dg_peaks.h")]
        if not force and os.path.exists(target) and os.path.getmtime(target) >= _newest(deps):
            out[lib] = target
            continue
        objs = []
        for src, name, defs in units:
            obj = os.path.join(BUILD, name + ".o")
            objs.append(obj)
            cmd = ([nvcc] + NVFLAGS + defs + (["-Xptxas", "-v"] if ptxas_info else []) +
                   ["-c", os.path.join(CSRC, src), "-o", obj])
            jobs.append((lib, cmd))
        out[lib] = (target, objs)

    def run(job):
        lib, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        return r.stderr

    jobs.sort(key=lambda j: 0 if any("volume_inst" in a for a in j[1]) else 1)  # longest units first
    logs = []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 8))) as ex:
        for log in ex.map(run, jobs):
            logs.append(log)
    for lib, val in list(out.items()):
        if isinstance(val, str):
            continue
        target, objs = val
        tmp = target + ".tmp%d" % os.getpid()
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
        os.replace(tmp, target)
        out[lib] = target
    if verbose or ptxas_info:
        sys.stderr.write("".join(logs))
    return out


if __name__ == "__main__":
    res = build(force="--force" in sys.argv, ptxas_info="--ptxas-info" in sys.argv, verbose=True)
    for k, v in res.items():
        print(k, v)
