"""Build libhbpc.so in-tree with nvcc for sm_103a.

Every translation unit is compiled in parallel into ``_build/`` next to this
file; the element-operator instantiations are split into the units listed in
``csrc/ops_units.h``.  ``build()`` is idempotent: a unit is recompiled only when
a source or header is newer than its object.
"""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libhbpc.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
           "--expt-relaxed-constexpr", "-I", CSRC, "-I", INCLUDE] + ARCH


def nvcc():
    exe = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(exe):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libhbpc")
    return exe


def _units():
    text = open(os.path.join(CSRC, "ops_units.h")).read()
    out = []
    for m in re.finditer(r"X\((\w+),\s*(\d),\s*(\d),\s*(0x[0-9A-Fa-f]+),\s*(0x[0-9A-Fa-f]+)\)", text):
        name, law, dim, lm, gm = m.groups()
        out.append((name, ["-DHBPC_LAW=" + law, "-DHBPC_DIM=" + dim, "-DHBPC_UNIT=" + name,
                           "-DHBPC_LOBATTO_MASK=" + lm, "-DHBPC_GAUSS_MASK=" + gm]))
    if not out:
        raise RuntimeError("no units parsed from ops_units.h")
    return out


def _jobs():
    jobs = []
    for name, defs in _units():
        jobs.append((os.path.join(CSRC, "ops_inst.cu"), os.path.join(BUILD, "ops_%s.o" % name), defs))
    for src in ("hbpc_api.cu", "hbpc_basis.cpp", "ops_table.cpp", "hbpc_probe.cu"):
        obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
        jobs.append((os.path.join(CSRC, src), obj, []))
    return jobs


def _newest_dep():
    t = 0.0
    for d in (CSRC, INCLUDE):
        for f in os.listdir(d):
            t = max(t, os.path.getmtime(os.path.join(d, f)))
    return t


def build(verbose=False, jobs=None):
    os.makedirs(BUILD, exist_ok=True)
    exe = nvcc()
    dep = max(_newest_dep(), os.path.getmtime(__file__))
    todo = [j for j in _jobs() if not os.path.exists(j[1]) or os.path.getmtime(j[1]) < dep]

    def run(job):
        src, obj, defs = job
        cmd = [exe] + NVFLAGS + defs + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (obj, " ".join(cmd), r.stderr[-4000:]))
        if verbose:
            print("built", os.path.basename(obj), flush=True)
        return obj

    workers = jobs or max(2, os.cpu_count() or 2)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        list(ex.map(run, todo))
    objs = [j[1] for j in _jobs()]
    if todo or not os.path.exists(LIB):
        cmd = [exe] + ARCH + ["-shared", "--cudart", "shared", "-o", LIB] + objs
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr[-4000:]))
    return LIB


if __name__ == "__main__":
    print(build(verbose=True))
