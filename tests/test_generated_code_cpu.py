"""The generated per-level code compiled for the host (g++), against itself in
the plain form.

The generator writes the moment update, pair adjoint and contraction either
over every Cartesian moment component with a whole-DAG reverse pass (the
method as written), or in the form the kernels run: neighbour sweeps over the
components with a z-exponent of at most 1 (u^(a,b,c) = u^(a,b,c-2) -
u^(a+2,b,c-2) - u^(a,b+2,c-2) for a unit vector u) and, in FP32, a reverse
pass graph by graph.  Both must give the same site energy, basis values, pair
gradients and dE/dc chain factors on random neighbourhoods (double precision,
1e-12 relative); the FP32 forms must keep the FP32 rounding of the plain
form.  No GPU is used."""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2510_00193_gb300")
CSRC = os.path.join(PKG, "csrc")

HARNESS = r"""
#include <cstdio>
#include <cmath>
#include <random>
#include "mtp_level8.cuh"
#include "mtp_level16.cuh"
using namespace mtp;
template <class R, class LV> void run(unsigned seed, bool graph) {
  std::mt19937_64 g(seed);
  std::normal_distribution<double> nd(0, 1);
  const int NP = 26;
  double u[NP][3], f[NP][LV::NMU], df[NP][LV::NMU], r[NP];
  for (int p = 0; p < NP; ++p) {
    double x = nd(g), y = nd(g), z = nd(g), n = std::sqrt(x * x + y * y + z * z);
    u[p][0] = x / n; u[p][1] = y / n; u[p][2] = z / n; r[p] = 2.5 + std::fabs(nd(g));
    for (int m = 0; m < LV::NMU; ++m) { f[p][m] = 0.3 * nd(g); df[p][m] = 0.3 * nd(g); }
  }
  R xi[LV::NBASIS];
  for (int a = 0; a < LV::NBASIS; ++a) xi[a] = R(0.1 * nd(g));
  R M[LV::NCOMP] = {}, D[LV::NCOMP], B[LV::NBASIS];
  for (int p = 0; p < NP; ++p) {
    R fr[LV::NMU];
    for (int m = 0; m < LV::NMU; ++m) fr[m] = R(f[p][m]);
    LV::template moments<R>(M, fr, R(u[p][0]), R(u[p][1]), R(u[p][2]));
  }
  const R E = graph ? LV::template contract_graph<R, true>(M, xi, D, B) : LV::template contract<R, true>(M, xi, D, B);
  printf("%.17g\n", (double)E);
  for (int a = 0; a < LV::NBASIS; ++a) printf("%.17g\n", (double)B[a]);
  for (int p = 0; p < NP; ++p) {
    R fr[LV::NMU], dfr[LV::NMU], S[LV::NMU], gx, gy, gz;
    for (int m = 0; m < LV::NMU; ++m) { fr[m] = R(f[p][m]); dfr[m] = R(df[p][m]); }
    LV::template pair_adjoint<R>(D, fr, dfr, R(u[p][0]), R(u[p][1]), R(u[p][2]), R(1.0 / r[p]), gx, gy, gz, S);
    printf("%.17g\n%.17g\n%.17g\n", (double)gx, (double)gy, (double)gz);
    for (int m = 0; m < LV::NMU; ++m) printf("%.17g\n", (double)S[m]);
  }
}
int main() {
  for (unsigned seed = 1; seed <= 3; ++seed) {
    run<double, MtpLevel8>(seed, false);
    run<double, MtpLevel16>(seed, false);
    run<double, MtpLevel16>(seed, true);
    run<float, MtpLevel16>(seed, true);
  }
}
"""


def _build(tmp, sphere):
    sys.path.insert(0, PKG)
    try:
        import basisgen
    finally:
        sys.path.pop(0)
    saved = basisgen.SPHERE_MAX_LEVEL
    basisgen.SPHERE_MAX_LEVEL = saved if sphere else 0
    try:
        out = os.path.join(tmp, "sphere" if sphere else "plain")
        os.makedirs(out, exist_ok=True)
        for level in (8, 16):
            with open(os.path.join(out, "mtp_level%d.cuh" % level), "w") as fh:
                fh.write(basisgen.emit_header(basisgen.Level(level)))
    finally:
        basisgen.SPHERE_MAX_LEVEL = saved
    src = os.path.join(tmp, "harness.cpp")
    with open(src, "w") as fh:
        fh.write(HARNESS)
    exe = os.path.join(out, "harness")
    subprocess.run(["g++", "-O1", "-std=c++17", "-I" + out, "-I" + CSRC, src, "-o", exe], check=True,
                   capture_output=True, timeout=600)
    res = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120)
    return np.array([float(v) for v in res.stdout.split()])


@pytest.fixture(scope="module")
def outputs(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    tmp = str(tmp_path_factory.mktemp("gen"))
    return _build(tmp, False), _build(tmp, True)


def _blocks(v):
    """Split one seed's output into (double L8, double L16, double L16 per graph, float L16 per graph)."""
    sys.path.insert(0, PKG)
    try:
        import basisgen
    finally:
        sys.path.pop(0)
    sizes = []
    for level in (8, 16, 16, 16):
        lv = basisgen.Level(level)
        sizes.append(1 + lv.m + 26 * (3 + lv.nmu))
    per_seed = sum(sizes)
    assert len(v) == 3 * per_seed
    out = []
    for seed in range(3):
        base = seed * per_seed
        parts = []
        for n in sizes:
            parts.append(v[base:base + n])
            base += n
        out.append(parts)
    return out


def test_sphere_form_equals_plain_form_in_double(outputs):
    plain, sphere = (_blocks(v) for v in outputs)
    for p, s in zip(plain, sphere):
        for k in range(3):   # level 8, level 16, level 16 per-graph reverse pass
            ref = p[1] if k == 2 else p[k]
            scale = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
            assert np.max(np.abs(s[k] - ref) / scale) < 1e-12


def test_per_graph_form_equals_whole_dag_in_plain_code(outputs):
    plain, _ = (_blocks(v) for v in outputs)
    for p in plain:
        scale = np.maximum(np.abs(p[1]), 1e-3 * np.abs(p[1]).max())
        assert np.max(np.abs(p[2] - p[1]) / scale) < 1e-12


def test_fp32_rounding_unchanged_by_the_reduction(outputs):
    """The FP32 per-graph code of both forms against the double result: the
    reduced form must not lose more than a small factor of FP32 rounding."""
    plain, sphere = (_blocks(v) for v in outputs)
    ep = es = 0.0
    for p, s in zip(plain, sphere):
        ref = p[1]
        norm = np.linalg.norm(ref)
        ep = max(ep, np.linalg.norm(p[3] - ref) / norm)
        es = max(es, np.linalg.norm(s[3] - ref) / norm)
    assert ep < 1e-5 and es < 1e-5
    assert es < 3.0 * ep + 1e-7
