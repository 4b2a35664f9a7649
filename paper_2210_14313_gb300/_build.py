"""Builds libsg.so in-tree for sm_103a (nvcc + g++, translation units in
parallel, CUDA runtime linked statically)."""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libsg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

SOURCES = ["sg_rules.cpp", "sg_plan.cpp", "sg_kernels.cu", "sg_api.cu", "sg_noalloc.cu", "sg_user.cu"]
# sources compiled at run time for user integrands, embedded into the library as strings
EMBEDDED = [("sg_src_internal", "sg_internal.h"), ("sg_src_fold_logic", "sg_fold_logic.h"),
            ("sg_src_xsum", "sg_xsum.h"), ("sg_src_reduce", "sg_reduce.cuh"),
            ("sg_src_user_kernel", "sg_user_kernel.cuh")]
HEADERS = ["sg_internal.h", "sg_kernels.h", "sg_rules.h", "sg_plan.h", "sg_fold_logic.h", "sg_reduce.cuh",
           "sg_ff.cuh", "sg_user.h", "sg_user_kernel.cuh", "sg_fixed.h", "sg_xsum.h"]
CUDA_INC = "/usr/local/cuda/include"


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS]
    deps.append(os.path.join(HERE, "..", "include", "sg.h"))
    deps.append(os.path.abspath(__file__))
    return any(os.path.getmtime(p) > t for p in deps if os.path.exists(p))


def _write_embedded() -> None:
    """_lib/sg_user_sources.h: the run-time compiled sources as raw string literals."""
    lines = ["// Generated by _build.py: sources that NVRTC compiles for user integrands."]
    for var, name in EMBEDDED:
        with open(os.path.join(CSRC, name)) as f:
            text = f.read()
        if ")SG_RAW\"" in text:
            raise RuntimeError("delimiter inside %s" % name)
        lines.append('static const char %s[] = R"SG_RAW(%s)SG_RAW";' % (var, text))
    path = os.path.join(OUT_DIR, "sg_user_sources.h")
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        f.write("\n".join(lines) + "\n")
    os.replace(tmp, path)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    _write_embedded()
    nvcc = _nvcc()
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, os.path.splitext(src)[0] + ".o")
        objs.append(obj)
        path = os.path.join(CSRC, src)
        if src.endswith(".cu"):
            cmd = [nvcc, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC,-fvisibility=hidden",
                   "-I" + OUT_DIR, "-c", path, "-o", obj]
        else:
            cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-fvisibility=hidden", "-ffp-contract=off",
                   "-I" + CUDA_INC, "-c", path, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    for cmd, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            raise RuntimeError("build failed: %s\n%s" % (" ".join(cmd), out.decode(errors="replace")))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc, *ARCH, "-shared", "-cudart=static", "-o", tmp, *objs, "-ldl"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed: %s\n%s" % (" ".join(cmd), r.stdout.decode(errors="replace")))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
