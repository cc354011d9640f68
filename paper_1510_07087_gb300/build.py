"""Build the C-ABI shared library `libdh2.so` in-tree for sm_103a.

    python -m paper_1510_07087_gb300.build

Host sources are compiled with g++ (-ffp-contract=off: the tree builder's
floating-point decisions must not depend on FMA contraction), CUDA sources
with nvcc for sm_103a only, all in parallel, then linked with nvcc.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libdh2.so")

HOST_SOURCES = ["dh2_tree.cpp"]
CUDA_SOURCES = ["dh2_pair.cu", "dh2_gram.cu", "dh2_rq_tc.cu", "dh2_ops.cu", "dh2_api.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
# build-time tuning macros, read from the environment (integers; the defaults,
# the measured best, sit beside each #ifndef in csrc/)
TUNING_MACROS = ("DH2_PAIR_MINB", "DH2_PAIR_MINB192", "DH2_PAIR_MINB160", "DH2_PAIR_MINB128", "DH2_LQT",
                 "DH2_HOST_PANELS", "DH2_GRAM_MINB128", "DH2_GRAM_MINB160", "DH2_GRAM_MINB192", "DH2_RQ_MINB",
                 "DH2_PROJ_MINB")


def _nvcc() -> str:
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else (shutil.which("nvcc") or "nvcc")


def build(verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for src in HOST_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-pthread", "-ffp-contract=off", "-Wall", "-Wno-unused-function",
                     f"-I{os.path.join(HERE, '..', 'include')}", "-c", os.path.join(CSRC, src), "-o", obj])
    extra = ["-DDH2_CHECK"] if os.environ.get("DH2_CHECK") == "1" else []
    if os.environ.get("DH2_PROFILE") == "1":
        extra.append("-DDH2_PROFILE")
    for name in TUNING_MACROS:
        if os.environ.get(name):
            extra.append(f"-D{name}={int(os.environ[name])}")
    for src in CUDA_SOURCES:
        obj = os.path.join(BUILD, src + ".o")
        objs.append(obj)
        jobs.append([nvcc, "-std=c++17", "-O3", "-lineinfo", *ARCH, "--extended-lambda", *extra,
                     "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                     "-c", os.path.join(CSRC, src), "-o", obj])
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True) for j in jobs]
    failed = []
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        if verbose and out:
            print(out)
        if p.returncode != 0:
            failed.append((j, out))
    if failed:
        msg = "\n".join(" ".join(j) + "\n" + out for j, out in failed)
        raise RuntimeError("libdh2 build failed:\n" + msg)
    link = [nvcc, "-shared", *ARCH, "-o", LIB + ".tmp", *objs, "-lpthread"]
    r = subprocess.run(link, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("libdh2 link failed:\n" + r.stdout)
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
