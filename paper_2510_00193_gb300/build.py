"""Builds libmtp_gb300.so in-tree for sm_103a.

Steps: generate the per-level basis code (basisgen), write one translation
unit per level plus the level registry, compile every unit with nvcc in
parallel, link one shared library with the CUDA runtime linked statically.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
GEN = os.path.join(BUILD, "gen")
LIB = os.path.join(HERE, "libmtp_gb300.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
LEVELS = (2, 4, 6, 8, 10, 12, 14, 16, 18, 20)


def nvcc_path():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmtp_gb300.so")
    return cand


def _common_flags(extra_ptxas=False):
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-I" + INCLUDE, "-I" + CSRC,
                    "-I" + GEN, "--expt-relaxed-constexpr"]
    if extra_ptxas:
        flags += ["-Xptxas", "-v"]
    return flags


def _write(path, text):
    if os.path.exists(path):
        with open(path) as fh:
            if fh.read() == text:
                return
    with open(path, "w") as fh:
        fh.write(text)


def generate_sources(levels=LEVELS):
    sys.path.insert(0, HERE)
    try:
        import basisgen
    finally:
        sys.path.pop(0)
    os.makedirs(GEN, exist_ok=True)
    basisgen.generate(GEN, levels)
    units = []
    for L in levels:
        path = os.path.join(GEN, "efv_level%d.cu" % L)
        _write(path, (
            "// Generated by paper_2510_00193_gb300/build.py.\n"
            "#include \"efv_kernel.cuh\"\n#include \"grade_kernel.cuh\"\n#include \"batch_kernel.cuh\"\n"
            "#include \"tangent_kernel.cuh\"\n#include \"efv_team.cuh\"\n"
            "#include \"mtp_level%d.cuh\"\n"
            "namespace mtp {\nint efv_level%d(const EfvArgs& a, int precision, bool want_dtheta, cudaStream_t s) {\n"
            "  return efv_launch<MtpLevel%d>(a, precision, want_dtheta, s);\n}\n"
            "int rows_level%d(const EfvArgs& a, const int32_t* list, int64_t n, double* rows, int64_t ld, double* bsum,"
            " cudaStream_t s) {\n  return basis_rows_launch<MtpLevel%d>(a, list, n, rows, ld, bsum, s);\n}\n"
            "int batch_level%d(const BatchArgs& b, int precision, bool want_dtheta, int threads, cudaStream_t s) {\n"
            "  return batch_launch<MtpLevel%d>(b, precision, want_dtheta, threads, s);\n}\n"
            "int tangent_level%d(const TangentArgs& t, int precision, cudaStream_t s) {\n"
            "  return tangent_launch<MtpLevel%d>(t, precision, s);\n}\n"
            "int split_level%d() { return MtpLevel%d::NGROUPS > 1 ? MtpLevel%d::NCOMP : 0; }\n"
            "int team_level%d(const EfvArgs& a, int precision, bool want_dtheta, cudaStream_t s) {\n"
            "  return efv_team_launch<MtpLevel%d>(a, precision, want_dtheta, s);\n}\n"
            "}  // namespace mtp\n") % (L, L, L, L, L, L, L, L, L, L, L, L, L, L))
        units.append(path)
    decl = "".join("int efv_level%d(const EfvArgs&, int, bool, cudaStream_t);\n"
                   "int rows_level%d(const EfvArgs&, const int32_t*, int64_t, double*, int64_t, double*, cudaStream_t);\n"
                   "int batch_level%d(const BatchArgs&, int, bool, int, cudaStream_t);\n"
                   "int tangent_level%d(const TangentArgs&, int, cudaStream_t);\n"
                   "int split_level%d();\n"
                   "int team_level%d(const EfvArgs&, int, bool, cudaStream_t);\n"
                   % (L, L, L, L, L, L) for L in levels)
    table = ",\n".join("  {%d, efv_level%d, rows_level%d, batch_level%d, tangent_level%d, split_level%d(), team_level%d}"
                        % (L, L, L, L, L, L, L) for L in levels)
    reg = os.path.join(GEN, "levels.cu")
    _write(reg, (
        "// Generated by paper_2510_00193_gb300/build.py.\n#include \"mtp_internal.cuh\"\nnamespace mtp {\n%s"
        "static const LevelEntry kEntries[] = {\n%s\n};\n"
        "const LevelEntry* find_level(int level) {\n"
        "  for (const auto& e : kEntries) if (e.level == level) return &e;\n  return nullptr;\n}\n}  // namespace mtp\n")
        % (decl, table))
    units.append(reg)
    return units


def _fingerprint(paths):
    h = hashlib.sha256()
    for p in sorted(paths):
        with open(p, "rb") as fh:
            h.update(p.encode())
            h.update(fh.read())
    return h.hexdigest()


def _compile(src, obj, verbose=False):
    cmd = [nvcc_path()] + _common_flags(verbose) + ["-c", src, "-o", obj]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), res.stderr[-6000:]))
    return res.stderr


def build(levels=LEVELS, jobs=None, verbose=False, force=False):
    """Compile and link; returns the path of the shared library."""
    os.makedirs(BUILD, exist_ok=True)
    units = generate_sources(levels)
    units += [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith(".cu")]
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    headers += [os.path.join(GEN, f) for f in os.listdir(GEN) if f.endswith((".cuh", ".h"))]
    objs = []
    todo = []
    hdr_fp = _fingerprint(headers + [__file__])
    for src in units:
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        stamp = obj + ".stamp"
        fp = _fingerprint([src]) + hdr_fp + " ".join(ARCH)
        objs.append(obj)
        if force or not (os.path.exists(obj) and os.path.exists(stamp) and open(stamp).read() == fp):
            todo.append((src, obj, stamp, fp))
    jobs = jobs or max(2, min(len(todo) or 1, os.cpu_count() or 4))
    logs = {}
    if todo:
        # biggest units first so the long poles start early
        todo.sort(key=lambda t: -os.path.getsize(t[0]) - 10 * sum(
            os.path.getsize(os.path.join(GEN, "mtp_level%d.cuh" % L)) for L in levels if ("level%d." % L) in t[0]))
        with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
            futs = {ex.submit(_compile, s, o, verbose): (s, o, st, fp) for s, o, st, fp in todo}
            for fu in cf.as_completed(futs):
                s, o, st, fp = futs[fu]
                logs[s] = fu.result()
                with open(st, "w") as fh:
                    fh.write(fp)
    need_link = bool(todo) or not os.path.exists(LIB)
    if need_link:
        tmp = LIB + ".tmp"
        cmd = [nvcc_path()] + ARCH + ["-shared", "-cudart", "static", "-o", tmp] + objs + ["-lrt", "-lpthread", "-ldl"]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), res.stderr[-4000:]))
        os.replace(tmp, LIB)
    if verbose:
        for s, log in logs.items():
            print("==", os.path.basename(s))
            print(log)
    return LIB


if __name__ == "__main__":
    args = sys.argv[1:]
    verbose = "-v" in args
    force = "-f" in args
    lv = tuple(int(a) for a in args if a.isdigit()) or LEVELS
    print(build(lv, verbose=verbose, force=force))
