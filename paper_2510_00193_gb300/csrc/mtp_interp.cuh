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

// The same program run by one warp on shared arrays V and A of NV values:
// the records are grouped by dependency level (order[level_off[L] ..
// level_off[L + 1]) are the records of level L, whose inputs all come from
// lower levels), lane l takes every 32nd record of a level, and the warp
// meets between levels.  The reverse pass walks the levels downwards; a
// record's adjoint A[dst] is complete once the levels above it are done, and
// its contributions to lower values are added with shared-memory atomics
// (records of one level may share inputs).  The caller fills V[0, NCOMP)
// before and reads D = A[0, NCOMP) after; every lane returns E.  Basis value a
// goes to store_basis(B, a, V[BOFF + a]) on the lane that forms it.
template <class R, bool WANT_B, int NCOMP, int NV, int ONE, int BOFF, int NB, int NLEV, class BV>
__device__ R interpret_values_warp(const int32_t* __restrict__ prog, const int32_t* __restrict__ starts,
                                   const int32_t* __restrict__ order, const int32_t* __restrict__ level_off, R* V,
                                   R* A, const typename ScalarOf<R>::T* __restrict__ xi, BV B, int lane) {
  using S = typename ScalarOf<R>::T;
  if (lane == 0) V[ONE] = R(1);
  __syncwarp();
  for (int L = 0; L < NLEV; ++L) {
    for (int k = level_off[L] + lane; k < level_off[L + 1]; k += 32) {
      const int32_t* p = prog + starts[order[k]];
      const int type = p[0], dst = p[1], cnt = p[2];
      R acc;
      if (type == 0) {
        acc = R(0);
        for (int t = 0; t < cnt; ++t) acc = fmadd(V[p[3 + 3 * t]] * R((S)p[5 + 3 * t]), V[p[4 + 3 * t]], acc);
      } else {
        acc = V[p[3]];
        for (int t = 1; t < cnt; ++t) acc = acc * V[p[3 + t]];
      }
      V[dst] = acc;
    }
    __syncwarp();
  }
  R E = R(0);
  for (int a = lane; a < NB; a += 32) {
    E = fmadd(R(xi[a]), V[BOFF + a], E);
    if (WANT_B) store_basis(B, a, V[BOFF + a]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) E += __shfl_xor_sync(0xffffffffu, E, o);
  for (int v = lane; v < NV; v += 32) A[v] = R(0);
  __syncwarp();
  for (int a = lane; a < NB; a += 32) A[BOFF + a] = R(xi[a]);
  __syncwarp();
  for (int L = NLEV - 1; L >= 0; --L) {
    for (int k = level_off[L] + lane; k < level_off[L + 1]; k += 32) {
      const int32_t* p = prog + starts[order[k]];
      const int type = p[0], dst = p[1], cnt = p[2];
      const R ad = A[dst];
      if (type == 0) {
        for (int t = 0; t < cnt; ++t) {
          const int a = p[3 + 3 * t], b = p[4 + 3 * t];
          const R aw = ad * R((S)p[5 + 3 * t]);
          atomicAdd(A + a, aw * V[b]);
          atomicAdd(A + b, aw * V[a]);
        }
      } else {
        for (int j = 0; j < cnt; ++j) {
          R prod = ad;
          for (int t = 0; t < cnt; ++t)
            if (t != j) prod = prod * V[p[3 + t]];
          atomicAdd(A + p[3 + j], prod);
        }
      }
    }
    __syncwarp();
  }
  return E;
}

}  // namespace mtp
