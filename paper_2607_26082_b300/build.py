"""Build libdtt.so in-tree for sm_103a (B300) with nvcc.

    python -m paper_2607_26082_b300.build        (or build() from Python)

The shared library is written next to this file; object files go to _build/.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdtt.so")
SOURCES = ["dtt_api.cu", "k_residual.cu", "k_residual_f32.cu", "k_transform.cu", "k_fft.cu", "k_solver.cu", "k_util.cu",
           "dtt_net.cu", "k_net.cu", "k_tensor_z.cu", "k_wfft.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def build(verbose=False, force=False, jobs=None):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    objs, cmds = [], []
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    newest_dep = max(os.path.getmtime(d) for d in deps)
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(o)
        if not force and os.path.exists(o) and os.path.getmtime(o) >= newest_dep:
            continue
        cmds.append([nvcc] + ARCH + FLAGS + ["-c", s, "-o", o])
    # translation units compile independently: one nvcc process per file, in parallel
    jobs = jobs or max(1, min(len(cmds), os.cpu_count() or 1))
    if verbose:
        for cmd in cmds:
            print(" ".join(cmd))
    with ThreadPoolExecutor(max_workers=jobs) as ex:
        for cmd, rc in zip(cmds, ex.map(lambda c: subprocess.run(c).returncode, cmds)):
            if rc != 0:
                raise subprocess.CalledProcessError(rc, cmd)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        cmd = [nvcc] + ARCH + ["-shared", "-o", LIB] + objs + ["-lcudart"]
        if verbose:
            print(" ".join(cmd))
        subprocess.run(cmd, check=True)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
