// Directional second derivatives for force matching (the double backward of
// a loss on forces): along a direction v of the positions,
//   dtheta_tan = d/dt dE/dtheta (x + t v)   (mixed second derivative . v)
//   force_tan  = d/dt F (x + t v) = -H v     (Hessian-vector product)
// The energy/force code is run once with dual numbers (value, tangent): the
// pair vectors carry the tangent v_j - v_i, and every generated function
// (moments, contraction and its reverse pass, pair adjoint) propagates it.
// The tangent of dE/dxi_alpha is sum_i dB_alpha(i)/dt; the tangent of
// dE/dc[mu][k][zi][zj] is sum over pairs of d(Q_k S_mu)/dt; species energies
// have zero tangent.
#pragma once
#include <type_traits>

#include "efv_kernel.cuh"

namespace mtp {

template <class S>
__device__ __forceinline__ Dual<S> rsqrt_r(Dual<S> a) {
  const S r = rsqrt_r(a.v);
  return {r, S(-0.5) * r * r * r * a.t};
}

struct TangentArgs {
  EfvArgs base;
  const double* v;          // [N][3] direction
  double* dtheta_tan;       // [n_params]
  double* force_tan;        // [N][3] or null
};

// Dual pair vector: value from the precision's own geometry, tangent v_j - v_i.
template <class S>
struct TangentGeom {
  PairGeom<S> g;
  S vx, vy, vz;
  __device__ __forceinline__ void load_centre(const TangentArgs& t, int64_t i, const S* cell) {
    g.load_centre(t.base, i, cell);
    vx = S(t.v[3 * i]); vy = S(t.v[3 * i + 1]); vz = S(t.v[3 * i + 2]);
  }
  __device__ __forceinline__ void vec(const TangentArgs& t, int32_t j, const typename PairGeom<S>::Load& l,
                                      int32_t img, Dual<S>& dx, Dual<S>& dy, Dual<S>& dz) const {
    S x, y, z;
    g.vec(t.base, l, img, x, y, z);
    dx = Dual<S>(x, S(__ldg(t.v + 3 * (int64_t)j)) - vx);
    dy = Dual<S>(y, S(__ldg(t.v + 3 * (int64_t)j + 1)) - vy);
    dz = Dual<S>(z, S(__ldg(t.v + 3 * (int64_t)j + 2)) - vz);
  }
};

template <class LV, class S>
__global__ void __launch_bounds__(kEfvThreads) tangent_kernel(const TangentArgs t) {
  using R = Dual<S>;
  constexpr int NMU = LV::NMU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EfvArgs& a = t.base;
  EfvShared<S, NMU, true> sm;     // coefficients and (tangent) accumulators in S
  sm.setup(a, smem_raw);
  sm.zero_gradients();
  __syncthreads();
  const int64_t i = a.atom_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  S Bt[LV::NBASIS];
#pragma unroll
  for (int k = 0; k < LV::NBASIS; ++k) Bt[k] = S(0);
  if (i < a.atom_end) {
    TangentGeom<S> geom;
    geom.load_centre(t, i, cell_of<S>(a));
    const int zi = species_at(a.z, i, a.n_species);
    const int64_t beg = __ldg(a.offsets + i), end = __ldg(a.offsets + i + 1);
    R M[LV::NCOMP];
#pragma unroll
    for (int c = 0; c < LV::NCOMP; ++c) M[c] = R(0);
    const R rcut = R(sm.rcut), mid = R(sm.mid), scale = R(sm.scale);
    for (int64_t k = beg; k < end; ++k) {
      const int32_t j = __ldg(a.nbr_j + k);
      const int32_t img = __ldg(a.nbr_img + k);
      const auto l = geom.g.fetch(a, j);
      R dx, dy, dz;
      geom.vec(t, j, l, img, dx, dy, dz);
      const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
      const R rinv = rsqrt_r(r2);
      const R r = r2 * rinv;
      R f[NMU];
      radial<R, NMU, false, false>(sm.c + (zi * sm.S + l.species) * sm.cstride, sm.nq, r, mid, scale, rcut, f,
                                   (R*)nullptr, (R*)nullptr);
      LV::template moments<R>(M, f, dx * rinv, dy * rinv, dz * rinv);
    }
    R D[LV::NCOMP], B[LV::NBASIS];
    (void)LV::template contract<R, true>(M, sm.xi, D, B);
#pragma unroll
    for (int k = 0; k < LV::NBASIS; ++k) Bt[k] = B[k].t;
    S fx = S(0), fy = S(0), fz = S(0);
    constexpr int kAccS = 4;
    const bool own_acc = sm.S <= kAccS;
    S acc[kAccS * NMU * kMaxQ];
    if (own_acc) {
      for (int u = 0; u < sm.S * NMU * kMaxQ; ++u) acc[u] = S(0);
    }
    for (int64_t k = beg; k < end; ++k) {
      const int32_t j = __ldg(a.nbr_j + k);
      const int32_t img = __ldg(a.nbr_img + k);
      const auto l = geom.g.fetch(a, j);
      R dx, dy, dz;
      geom.vec(t, j, l, img, dx, dy, dz);
      const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
      const R rinv = rsqrt_r(r2);
      const R r = r2 * rinv;
      R f[NMU], df[NMU], q[kMaxQ];
      radial<R, NMU, true, true>(sm.c + (zi * sm.S + l.species) * sm.cstride, sm.nq, r, mid, scale, rcut, f, df, q);
      R gx, gy, gz, Smu[NMU];
      LV::template pair_adjoint<R>(D, f, df, dx * rinv, dy * rinv, dz * rinv, rinv, gx, gy, gz, Smu);
      fx += gx.t; fy += gy.t; fz += gz.t;
      if (t.force_tan) {
        atomicAdd(t.force_tan + 3 * (int64_t)j, -(double)gx.t);
        atomicAdd(t.force_tan + 3 * (int64_t)j + 1, -(double)gy.t);
        atomicAdd(t.force_tan + 3 * (int64_t)j + 2, -(double)gz.t);
      }
      if (own_acc) {
        S* dst = acc + l.species * NMU * kMaxQ;
#pragma unroll
        for (int mu = 0; mu < NMU; ++mu) {
#pragma unroll
          for (int kk = 0; kk < kMaxQ; ++kk)
            if (kk < sm.nq) dst[mu * kMaxQ + kk] += (q[kk] * Smu[mu]).t;
        }
      } else {
        S* dst = sm.dc + (zi * sm.S + l.species) * NMU * sm.nq;
#pragma unroll
        for (int mu = 0; mu < NMU; ++mu) {
#pragma unroll
          for (int kk = 0; kk < kMaxQ; ++kk)
            if (kk < sm.nq) atomicAdd(dst + mu * sm.nq + kk, (q[kk] * Smu[mu]).t);
        }
      }
    }
    if (own_acc) {
      for (int zj = 0; zj < sm.S; ++zj) {
        S* dst = sm.dc + (zi * sm.S + zj) * NMU * sm.nq;
        for (int mu = 0; mu < NMU; ++mu)
          for (int kk = 0; kk < sm.nq; ++kk) atomicAdd(dst + mu * sm.nq + kk, acc[(zj * NMU + mu) * kMaxQ + kk]);
      }
    }
    if (t.force_tan) {
      atomicAdd(t.force_tan + 3 * i, (double)fx);
      atomicAdd(t.force_tan + 3 * i + 1, (double)fy);
      atomicAdd(t.force_tan + 3 * i + 2, (double)fz);
    }
  }
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < LV::NBASIS; ++k) {
    const double v = warp_sum((double)Bt[k]);
    if (lane == 0) atomicAdd(sm.dxi + k, S(v));
  }
  __syncthreads();
  const int S_ = sm.S, SS = sm.SS, nq = sm.nq;
  for (int k = threadIdx.x; k < SS * NMU * nq; k += blockDim.x) {
    const int p = k / (NMU * nq);
    const int mk = k % (NMU * nq);
    atomicAdd(t.dtheta_tan + S_ + (int64_t)mk * SS + p, (double)sm.dc[k]);
  }
  for (int k = threadIdx.x; k < sm.m; k += blockDim.x)
    atomicAdd(t.dtheta_tan + S_ + (int64_t)NMU * nq * SS + k, (double)sm.dxi[k]);
}

// Levels with component groups and a scratch buffer (t.base.mbuf, [2][NCOMP]
// [atom] dual numbers) run the tangent as three kernels, as the energy does:
// dual moments per component group, the interpreted contraction at high
// occupancy, dual adjoint sweeps per group.
template <class LV, class S>
__global__ void __launch_bounds__(kEfvThreads) tangent_moments_kernel(const TangentArgs t) {
  using R = Dual<S>;
  constexpr int NMU = LV::NMU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EfvArgs& a = t.base;
  EfvShared<S, NMU, true> sm;
  sm.setup(a, smem_raw);
  __syncthreads();
  const int64_t n = a.atom_end - a.atom_begin;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  const int64_t i = a.atom_begin + u;
  TangentGeom<S> geom;
  geom.load_centre(t, i, cell_of<S>(a));
  const int zi = species_at(a.z, i, a.n_species);
  const int64_t beg = __ldg(a.offsets + i), end = __ldg(a.offsets + i + 1);
  const R rcut = R(sm.rcut), mid = R(sm.mid), scale = R(sm.scale);
  R* buf = static_cast<R*>(a.mbuf) + u;
  auto sweep = [&](auto group) {
    constexpr int G = decltype(group)::value;
    R Mg[LV::NCOMP];
#pragma unroll
    for (int c = 0; c < LV::NCOMP; ++c) Mg[c] = R(0);
    for (int64_t k = beg; k < end; ++k) {
      const int32_t j = __ldg(a.nbr_j + k);
      const int32_t img = __ldg(a.nbr_img + k);
      const auto l = geom.g.fetch(a, j);
      R dx, dy, dz;
      geom.vec(t, j, l, img, dx, dy, dz);
      const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
      const R rinv = rsqrt_r(r2);
      const R r = r2 * rinv;
      R f[NMU];
      radial<R, NMU, false, false>(sm.c + (zi * sm.S + l.species) * sm.cstride, sm.nq, r, mid, scale, rcut, f,
                                   (R*)nullptr, (R*)nullptr);
      LV::template moments_group<G, R>(Mg, f, dx * rinv, dy * rinv, dz * rinv);
    }
    LV::template store_group<G, R>(Mg, buf, n);
  };
  sweep(std::integral_constant<int, 0>());
  sweep(std::integral_constant<int, 1>());
}

template <class LV, class S>
__global__ void __launch_bounds__(kEfvThreads) tangent_contract_kernel(const TangentArgs t) {
  using R = Dual<S>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EfvArgs& a = t.base;
  EfvShared<S, LV::NMU, true> sm;
  sm.setup(a, smem_raw);
  sm.zero_gradients();
  __syncthreads();
  const int64_t n = a.atom_end - a.atom_begin;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = u < n;
  const int lane = threadIdx.x & 31;
  if (__any_sync(0xffffffffu, active)) {
    const R* __restrict__ mrow = static_cast<const R*>(a.mbuf) + (active ? u : 0);
    R* __restrict__ drow = static_cast<R*>(a.mbuf) + (size_t)LV::NCOMP * n + (active ? u : 0);
    R V[LV::NVALUES], A[LV::NVALUES], B[LV::NBASIS];
    for (int c = 0; c < LV::NCOMP; ++c) V[c] = active ? mrow[c * n] : R(0);
    (void)LV::template contract_values<R, true>(V, A, sm.xi, B);
    if (active)
      for (int c = 0; c < LV::NCOMP; ++c) drow[c * n] = A[c];
    for (int k = 0; k < LV::NBASIS; ++k) {
      const S v = warp_sum_r(active ? B[k].t : S(0));
      if (lane == 0) atomicAdd(sm.dxi + k, v);
    }
  }
  __syncthreads();
  const int S_ = sm.S, SS = sm.SS, nq = sm.nq;
  for (int k = threadIdx.x; k < sm.m; k += blockDim.x)
    atomicAdd(t.dtheta_tan + S_ + (int64_t)LV::NMU * nq * SS + k, (double)sm.dxi[k]);
}

template <class LV, class S>
__global__ void __launch_bounds__(kEfvThreads) tangent_adjoint_kernel(const TangentArgs t) {
  using R = Dual<S>;
  constexpr int NMU = LV::NMU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const EfvArgs& a = t.base;
  EfvShared<S, NMU, true> sm;
  sm.setup(a, smem_raw);
  sm.zero_gradients();
  __syncthreads();
  const int64_t n = a.atom_end - a.atom_begin;
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n) {
    const int64_t i = a.atom_begin + u;
    TangentGeom<S> geom;
    geom.load_centre(t, i, cell_of<S>(a));
    const int zi = species_at(a.z, i, a.n_species);
    const int64_t beg = __ldg(a.offsets + i), end = __ldg(a.offsets + i + 1);
    const R rcut = R(sm.rcut), mid = R(sm.mid), scale = R(sm.scale);
    const R* buf = static_cast<const R*>(a.mbuf) + (size_t)LV::NCOMP * n + u;
    S fx = S(0), fy = S(0), fz = S(0);
    constexpr int kAccS = 4;
    const bool own_acc = sm.S <= kAccS;
    S acc[kAccS * NMU * kMaxQ];
    if (own_acc) {
      for (int v = 0; v < sm.S * NMU * kMaxQ; ++v) acc[v] = S(0);
    }
    auto sweep = [&](auto group) {
      constexpr int G = decltype(group)::value;
      R Dg[LV::NCOMP];
      LV::template load_group<G, R>(buf, n, Dg);
      for (int64_t k = beg; k < end; ++k) {
        const int32_t j = __ldg(a.nbr_j + k);
        const int32_t img = __ldg(a.nbr_img + k);
        const auto l = geom.g.fetch(a, j);
        R dx, dy, dz;
        geom.vec(t, j, l, img, dx, dy, dz);
        const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
        const R rinv = rsqrt_r(r2);
        const R r = r2 * rinv;
        R f[NMU], df[NMU], q[kMaxQ];
        radial<R, NMU, true, true>(sm.c + (zi * sm.S + l.species) * sm.cstride, sm.nq, r, mid, scale, rcut, f, df,
                                   q);
        R gx, gy, gz, Smu[NMU];
        LV::template pair_adjoint_group<G, R>(Dg, f, df, dx * rinv, dy * rinv, dz * rinv, rinv, gx, gy, gz, Smu);
        fx += gx.t; fy += gy.t; fz += gz.t;
        if (t.force_tan) {
          atomicAdd(t.force_tan + 3 * (int64_t)j, -(double)gx.t);
          atomicAdd(t.force_tan + 3 * (int64_t)j + 1, -(double)gy.t);
          atomicAdd(t.force_tan + 3 * (int64_t)j + 2, -(double)gz.t);
        }
        constexpr int mu_lo = LV::GROUP_MU_LO[G], mu_hi = LV::GROUP_MU_HI[G];
        if (own_acc) {
          S* dst = acc + l.species * NMU * kMaxQ;
#pragma unroll
          for (int mu = mu_lo; mu < mu_hi; ++mu) {
#pragma unroll
            for (int kk = 0; kk < kMaxQ; ++kk)
              if (kk < sm.nq) dst[mu * kMaxQ + kk] += (q[kk] * Smu[mu]).t;
          }
        } else {
          S* dst = sm.dc + (zi * sm.S + l.species) * NMU * sm.nq;
#pragma unroll
          for (int mu = mu_lo; mu < mu_hi; ++mu) {
#pragma unroll
            for (int kk = 0; kk < kMaxQ; ++kk)
              if (kk < sm.nq) atomicAdd(dst + mu * sm.nq + kk, (q[kk] * Smu[mu]).t);
          }
        }
      }
    };
    sweep(std::integral_constant<int, 0>());
    sweep(std::integral_constant<int, 1>());
    if (own_acc) {
      for (int zj = 0; zj < sm.S; ++zj) {
        S* dst = sm.dc + (zi * sm.S + zj) * NMU * sm.nq;
        for (int mu = 0; mu < NMU; ++mu)
          for (int kk = 0; kk < sm.nq; ++kk) atomicAdd(dst + mu * sm.nq + kk, acc[(zj * NMU + mu) * kMaxQ + kk]);
      }
    }
    if (t.force_tan) {
      atomicAdd(t.force_tan + 3 * i, (double)fx);
      atomicAdd(t.force_tan + 3 * i + 1, (double)fy);
      atomicAdd(t.force_tan + 3 * i + 2, (double)fz);
    }
  }
  __syncthreads();
  const int S_ = sm.S, SS = sm.SS, nq = sm.nq;
  for (int k = threadIdx.x; k < SS * NMU * nq; k += blockDim.x) {
    const int p = k / (NMU * nq);
    const int mk = k % (NMU * nq);
    atomicAdd(t.dtheta_tan + S_ + (int64_t)mk * SS + p, (double)sm.dc[k]);
  }
}

template <class LV, class S>
int tangent_split_launch(const TangentArgs& t, cudaStream_t stream) {
  const EfvArgs& a = t.base;
  const int64_t n = a.atom_end - a.atom_begin;
  const int SS = a.n_species * a.n_species;
  const unsigned grid = (unsigned)((n + kEfvThreads - 1) / kEfvThreads);
  const size_t bytes = efv_smem_bytes<S, LV::NMU, true>(SS, a.n_q, a.m);
  int rc;
  if ((rc = set_smem(tangent_moments_kernel<LV, S>, bytes)) != MTP_OK) return rc;
  if ((rc = set_smem(tangent_contract_kernel<LV, S>, bytes)) != MTP_OK) return rc;
  if ((rc = set_smem(tangent_adjoint_kernel<LV, S>, bytes)) != MTP_OK) return rc;
  tangent_moments_kernel<LV, S><<<grid, kEfvThreads, bytes, stream>>>(t);
  tangent_contract_kernel<LV, S><<<grid, kEfvThreads, bytes, stream>>>(t);
  tangent_adjoint_kernel<LV, S><<<grid, kEfvThreads, bytes, stream>>>(t);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("tangent split kernels (level %d): %s", LV::LEVEL, cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  return MTP_OK;
}

template <class LV>
int tangent_launch(const TangentArgs& t, int precision, cudaStream_t stream) {
  const EfvArgs& a = t.base;
  const int64_t n = a.atom_end - a.atom_begin;
  if (n <= 0) return MTP_OK;
  if constexpr (LV::NGROUPS > 1) {
    if (a.mbuf)
      return precision == MTP_MIXED ? tangent_split_launch<LV, float>(t, stream)
                                    : tangent_split_launch<LV, double>(t, stream);
  }
  const int SS = a.n_species * a.n_species;
  const unsigned grid = (unsigned)((n + kEfvThreads - 1) / kEfvThreads);
  cudaError_t e;
  if (precision == MTP_MIXED) {
    const size_t bytes = efv_smem_bytes<float, LV::NMU, true>(SS, a.n_q, a.m);
    auto kern = tangent_kernel<LV, float>;
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    kern<<<grid, kEfvThreads, bytes, stream>>>(t);
  } else {
    const size_t bytes = efv_smem_bytes<double, LV::NMU, true>(SS, a.n_q, a.m);
    auto kern = tangent_kernel<LV, double>;
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    kern<<<grid, kEfvThreads, bytes, stream>>>(t);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("tangent kernel launch (level %d): %s", LV::LEVEL, cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  return MTP_OK;
}

}  // namespace mtp
