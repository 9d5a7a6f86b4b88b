// Per-thread interpreter of a contraction program (used for high levels,
// whose straight-line contraction code would be too large to compile).
// Program records: DOT = [0, dst, n, (a, b, w) * n] (V[dst] = sum w V[a] V[b]),
// PROD = [1, dst, n, g * n] (V[dst] = prod V[g]); V[0, NCOMP) holds the moment
// components, V[ONE] = 1, V[BOFF + alpha] the basis values.  The reverse pass
// walks the records backwards and accumulates adjoints A, starting from
// A[BOFF + alpha] = xi_alpha; D = A[0, NCOMP).
#pragma once
#include "mtp_math.cuh"

namespace mtp {

// Core: V[0, NCOMP) holds the moment components on entry; on return A[0,
// NCOMP) holds D = dE/dM.  V and A are caller arrays of NV values.
template <class R, bool WANT_B, int NCOMP, int NV, int ONE, int BOFF, int NB, int NREC>
__device__ __forceinline__ R interpret_values(const int32_t* __restrict__ prog, const int32_t* __restrict__ starts,
                                              R* V, R* A, const typename ScalarOf<R>::T* __restrict__ xi, R* B) {
  V[ONE] = R(1);
  for (int r = 0; r < NREC; ++r) {
    const int32_t* p = prog + starts[r];
    const int type = p[0], dst = p[1], cnt = p[2];
    if (type == 0) {
      R acc = R(0);
      for (int t = 0; t < cnt; ++t) {
        const int a = p[3 + 3 * t], b = p[4 + 3 * t], w = p[5 + 3 * t];
        acc = fmadd(V[a] * R((typename ScalarOf<R>::T)w), V[b], acc);
      }
      V[dst] = acc;
    } else {
      R acc = V[p[3]];
      for (int t = 1; t < cnt; ++t) acc = acc * V[p[3 + t]];
      V[dst] = acc;
    }
  }
  R E = R(0);
  for (int a = 0; a < NB; ++a) {
    E = fmadd(R(xi[a]), V[BOFF + a], E);
    if (WANT_B) B[a] = V[BOFF + a];
  }
  for (int v = 0; v < NV; ++v) A[v] = R(0);
  for (int a = 0; a < NB; ++a) A[BOFF + a] = R(xi[a]);
  for (int r = NREC - 1; r >= 0; --r) {
    const int32_t* p = prog + starts[r];
    const int type = p[0], dst = p[1], cnt = p[2];
    const R ad = A[dst];
    if (type == 0) {
      for (int t = 0; t < cnt; ++t) {
        const int a = p[3 + 3 * t], b = p[4 + 3 * t], w = p[5 + 3 * t];
        const R aw = ad * R((typename ScalarOf<R>::T)w);
        A[a] = fmadd(aw, V[b], A[a]);
        A[b] = fmadd(aw, V[a], A[b]);
      }
    } else {
      for (int k = 0; k < cnt; ++k) {
        R prod = ad;
        for (int t = 0; t < cnt; ++t)
          if (t != k) prod = prod * V[p[3 + t]];
        A[p[3 + k]] = A[p[3 + k]] + prod;
      }
    }
  }
  return E;
}

template <class R, bool WANT_B, int NCOMP, int NV, int ONE, int BOFF, int NB, int NREC>
__device__ __forceinline__ R interpret_contract(const int32_t* __restrict__ prog, const int32_t* __restrict__ starts,
                                                const R* __restrict__ M,
                                                const typename ScalarOf<R>::T* __restrict__ xi, R* __restrict__ D,
                                                R* __restrict__ B) {
  R V[NV];
  R A[NV];
  for (int c = 0; c < NCOMP; ++c) V[c] = M[c];
  const R E = interpret_values<R, WANT_B, NCOMP, NV, ONE, BOFF, NB, NREC>(prog, starts, V, A, xi, B);
  for (int c = 0; c < NCOMP; ++c) D[c] = A[c];
  return E;
}

}  // namespace mtp
