"""Build librosen.so (the CUDA kernels and the C ABI) in-tree for sm_103a.

Every ``csrc/*.cu`` translation unit is compiled in parallel with
``nvcc -gencode arch=compute_103a,code=sm_103a`` and linked into
``paper_1704_04381_gb300/_build/librosen.so``.  Rebuilds only what changed.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT = os.path.join(PKG, "_build")
LIB = os.path.join(OUT, "librosen.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC]


def nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build librosen")


def _headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(INCLUDE, "*.h"))


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def _ff(x):
    """A double as a float-float pair (hi = nearest float, lo = nearest float
    to the remainder), as C hex-float literals."""
    import struct
    f32 = lambda v: struct.unpack("<f", struct.pack("<f", v))[0]
    hi = f32(x)
    lo = f32(x - hi)
    return float(hi).hex() + "f", float(lo).hex() + "f"


def write_turn_table():
    """Generate csrc/turn_table.cuh: cos and sin of 2 pi m / 256 (m = 0..255)
    and the constant 2 pi / 2^24 as float-float pairs, from the host's
    double-precision cos and sin.  Written only when its text changes."""
    import math
    lines = ["// turn_table.cuh -- generated by build.py (write_turn_table); do not edit.",
             "// Float-float values from double-precision cos and sin on the host:",
             "// kTurn[m] = {cos hi, sin hi, cos lo, sin lo} of 2 pi m / 256, and",
             "// 2 pi / 2^24 (the angle of one unit of a 24-bit turn fraction).",
             "#pragma once", "",
             "namespace rosen {", ""]
    kh, kl = _ff(2.0 * math.pi / 2.0 ** 24)
    lines.append("constexpr float kTurnUnitHi = %s, kTurnUnitLo = %s;" % (kh, kl))
    lines.append("")
    lines.append("__constant__ float4 kTurn[256] = {")
    for m in range(256):
        ch, cl = _ff(math.cos(2.0 * math.pi * m / 256.0))
        sh, sl = _ff(math.sin(2.0 * math.pi * m / 256.0))
        lines.append("    {%s, %s, %s, %s}," % (ch, sh, cl, sl))
    lines += ["};", "", "}  // namespace rosen", ""]
    text = "\n".join(lines)
    path = os.path.join(CSRC, "turn_table.cuh")
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)
    return path


def build(force=False, verbose=False, extra_flags=()):
    """Compile and link librosen.so if any source changed; return its path."""
    os.makedirs(OUT, exist_ok=True)
    write_turn_table()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    hdrs = _headers()
    exe = nvcc()
    objs, jobs = [], []
    for src in srcs:
        obj = os.path.join(OUT, os.path.basename(src) + ".o")
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            cmd = [exe] + ARCH + NVCC_FLAGS + list(extra_flags) + ["-c", src, "-o", obj]
            if src.endswith(".cpp"):
                cmd = [exe] + NVCC_FLAGS + list(extra_flags) + ["-x", "cu"] + ARCH + ["-c", src, "-o", obj]
            jobs.append(cmd)
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
        for cmd, r in zip(jobs, results):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed for " + cmd[-3])
    if force or jobs or _stale(LIB, objs):
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = [exe] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread", "-ldl", "-lrt"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            raise RuntimeError("link of librosen.so failed")
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
