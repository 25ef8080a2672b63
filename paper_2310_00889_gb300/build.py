"""Build libsbq.so (the CUDA C-ABI library) in-tree for sm_103a.

Each translation unit under csrc/ is compiled by nvcc in parallel, then linked into
paper_2310_00889_gb300/_lib/libsbq.so.  No cmake, no torch extension machinery.
"""
from __future__ import annotations

import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIBDIR = os.path.join(HERE, "_lib")
LIB = os.path.join(LIBDIR, "libsbq.so")
ROOT = os.path.dirname(HERE)

GEN = os.path.join(LIBDIR, "gen")
RULES = os.path.join(HERE, "rules")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr",
              "-Xcompiler", "-fPIC,-fvisibility=hidden,-O2", "-I", os.path.join(ROOT, "include"),
              "-I", GEN]


def nvcc_path() -> str:
    p = shutil.which("nvcc")
    if p:
        return p
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsbq")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _rule_tables():
    return sorted(glob.glob(os.path.join(RULES, "angular_l*.txt")),
                  key=lambda f: int(os.path.basename(f)[len("angular_l"):-len(".txt")]))


def _deps():
    return _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) \
        + [os.path.join(ROOT, "include", "sbq.h"), os.path.abspath(__file__),
           os.path.join(os.path.dirname(os.path.abspath(__file__)), "angular_rules.py")] + _rule_tables() + _singular_tables()


def _rule_levels():
    """LEVELS + 1 of angular_rules.py, read from its source (the build imports no package code)."""
    import re
    src = open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "angular_rules.py")).read()
    return int(re.search(r"^LEVELS = (\d+)", src, re.M).group(1)) + 1


def write_rule_tables():
    """The compressed angular rules (rules/angular_l<l0>.txt, written by angular_rules.py)
    as a C include for the quadrature builder: per table its l0, the node count of each of
    the LEVELS + 1 distance levels, and the (offset, weight) pairs level by level, as hexadecimal
    floating-point literals (exact)."""
    os.makedirs(GEN, exist_ok=True)
    nlev = _rule_levels()
    l0s, cnts, data = [], [], []
    for path in _rule_tables():
        l0 = int(os.path.basename(path)[len("angular_l"):-len(".txt")])
        cnt = [0] * nlev
        lines = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
        i = 0
        while i < len(lines):
            lev, n = int(lines[i][0]), int(lines[i][1])
            cnt[lev] = n
            for k in range(n):
                a, b = lines[i + 1 + k]
                data.append(float(a).hex())
                data.append(float(b).hex())
            i += n + 1
        l0s.append(l0)
        cnts.append(cnt)
    out = ["// generated by paper_2310_00889_gb300/build.py from rules/angular_l*.txt", ""]
    out.append("static const int kRuleTables = %d;" % len(l0s))
    out.append("static const int kRuleL0[%d] = {%s};" % (max(1, len(l0s)), ", ".join(map(str, l0s)) or "0"))
    out.append("static const int kRuleLevels = %d;" % nlev)
    out.append("static const int kRuleCnt[%d][%d] = {%s};" % (
        max(1, len(l0s)), nlev, ", ".join("{" + ", ".join(map(str, c)) + "}" for c in cnts) or "{0}"))
    out.append("static const double kRuleData[%d] = {" % max(1, len(data)))
    for k in range(0, len(data), 4):
        out.append("    " + ", ".join(data[k:k + 4]) + ",")
    if not data:
        out.append("    0.0,")
    out.append("};")
    text = "\n".join(out) + "\n"
    path = os.path.join(GEN, "angular_rules_tables.inc")
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)
    return path


def _singular_tables():
    return sorted(glob.glob(os.path.join(RULES, "singular_ns*_l*.txt")))


def write_singular_tables():
    """The whole-element singular rules (rules/singular_ns<ns>_l<l0>.txt, written by
    singular_rules.py) as a C include: the table's ns, l0 and aspect levels, per (level, i0)
    the node count and the offset of its first node, and the (offset, weight) pairs, as
    hexadecimal floating-point literals (exact).  At most one table; none: kSingTables = 0."""
    os.makedirs(GEN, exist_ok=True)
    out = ["// generated by paper_2310_00889_gb300/build.py from rules/singular_ns*_l*.txt", ""]
    paths = _singular_tables()
    if paths:
        path = paths[0]
        base = os.path.basename(path)[len("singular_ns"):-len(".txt")]
        ns, l0 = int(base.split("_l")[0]), int(base.split("_l")[1])
        lines = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
        rules, i = {}, 0
        while i < len(lines):
            lev, i0, n = (int(v) for v in lines[i])
            rules[(lev, i0)] = lines[i + 1:i + 1 + n]
            i += n + 1
        lo = min(k[0] for k in rules)
        hi = max(k[0] for k in rules)
        cnt, off, data = [], [], []
        for lev in range(lo, hi + 1):
            for i0 in range(ns):
                r = rules.get((lev, i0), [])
                off.append(len(data) // 2)
                cnt.append(len(r))
                for a, b in r:
                    data.append(float(a).hex())
                    data.append(float(b).hex())
        out.append("static const int kSingTables = 1;")
        out.append("static const int kSingNs = %d, kSingL0 = %d, kSingLo = %d, kSingHi = %d;" % (ns, l0, lo, hi))
    else:
        cnt, off, data = [0], [0], []
        out.append("static const int kSingTables = 0;")
        out.append("static const int kSingNs = 0, kSingL0 = 0, kSingLo = 0, kSingHi = -1;")
    out.append("static const int kSingCnt[%d] = {%s};" % (len(cnt), ", ".join(map(str, cnt))))
    out.append("static const int kSingOff[%d] = {%s};" % (len(off), ", ".join(map(str, off))))
    out.append("static const double kSingData[%d] = {" % max(1, len(data)))
    for k in range(0, len(data), 4):
        out.append("    " + ", ".join(data[k:k + 4]) + ",")
    if not data:
        out.append("    0.0,")
    out.append("};")
    text = "\n".join(out) + "\n"
    path = os.path.join(GEN, "singular_rules_tables.inc")
    if not os.path.exists(path) or open(path).read() != text:
        with open(path, "w") as f:
            f.write(text)
    return path


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in _deps())


def build(force: bool = False, verbose: bool = False, extra_flags=None) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = nvcc_path()
    write_rule_tables()
    write_singular_tables()
    objdir = os.path.join(LIBDIR, "obj")
    os.makedirs(objdir, exist_ok=True)
    flags = NVCC_FLAGS + list(extra_flags or [])

    def compile_one(src):
        obj = os.path.join(objdir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *ARCH, *flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), flush=True)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr, flush=True)
        return obj

    srcs = _sources()
    with cf.ThreadPoolExecutor(max_workers=min(len(srcs), os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = LIB + ".tmp.%d" % os.getpid()
    cuda_lib = os.path.join(os.path.dirname(os.path.dirname(nvcc)), "lib64")
    cmd = [nvcc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs,
           "-Xlinker", "-rpath," + cuda_lib]
    if verbose:
        print(" ".join(cmd), flush=True)
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True,
          extra_flags=["-Xptxas", "-v"] if "--ptxas" in sys.argv else None)
    print(LIB)
