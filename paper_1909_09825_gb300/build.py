"""In-tree build of libfgt1d.so for sm_103a (nvcc, no cmake).

Each translation unit under csrc/ is compiled in parallel into _build/, then
linked into paper_1909_09825_gb300/libfgt1d.so.  sweep_inst.cu is compiled once
per (precision, term count) so that the heavy kernel instantiations spread over
all cores.  Rebuilds only what changed.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libfgt1d.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC] + ARCH
CXX_FLAGS = ["-O2", "-std=c++17", "-fPIC", "-I", INCLUDE, "-I", CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(INCLUDE, "fgt1d.h"))
    return max(os.path.getmtime(h) for h in hs)


# sweep_inst.cu: precision 0 FP64, 1 FP32, 2 double-float; tile shape 0 (128 x 32),
# 1 (256 x 16); term counts 1..8
VARIANTS = {"sweep_inst.cu": [("p%d_s%d_ne%d" % (p, sh, ne),
                               ["-DFGT_SW_PREC=%d" % p, "-DFGT_SW_SHAPE=%d" % sh, "-DFGT_SW_NE=%d" % ne])
                              for p in (0, 1, 2) for sh in (0, 1) for ne in range(1, 9)]}


def _sources():
    """(source, object name, extra flags) for every unit to compile."""
    out = []
    for f in sorted(f for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp"))):
        if f in VARIANTS:
            out += [(f, "%s.%s.o" % (f, tag), flags) for tag, flags in VARIANTS[f]]
        else:
            out.append((f, f + ".o", []))
    return out


def build(verbose=False, extra_flags=()):
    """Compile every CUDA/C++ source for sm_103a and link libfgt1d.so; returns its path."""
    os.makedirs(BUILD, exist_ok=True)
    hdr_time = _headers()
    nvcc = _nvcc()
    jobs = []
    objs = []
    for src, oname, vflags in _sources():
        s = os.path.join(CSRC, src)
        o = os.path.join(BUILD, oname)
        objs.append(o)
        if os.path.exists(o) and os.path.getmtime(o) >= max(os.path.getmtime(s), hdr_time) and not extra_flags:
            continue
        if src.endswith(".cu"):
            cmd = [nvcc, "-c", s, "-o", o] + NVCC_FLAGS + vflags + list(extra_flags)
        else:
            # no floating-point contraction on the host: the double-double SOE construction
            # relies on exact two-sums, and x86 and Arm hosts then give the same nodes
            cmd = [nvcc, "-c", s, "-o", o, "-x", "c++", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
                   "-O2", "-std=c++17", "-I", INCLUDE, "-I", CSRC]
        jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    # the kernel instantiation units (the longest) first
    jobs.sort(key=lambda cmd: os.path.basename(cmd[2]) not in VARIANTS)
    failed = []
    with ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                failed.append(cmd[2])
    if failed:
        raise RuntimeError("compilation failed: " + ", ".join(failed))
    if jobs or not os.path.exists(LIB):
        cmd = [nvcc, "-shared", "-o", LIB] + objs + ARCH + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n" + r.stdout + r.stderr)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
