// Warp-per-atom energy/force kernel: the block-parallel variant for small
// systems and high levels (the paper keeps a separate GPU pair style that
// spreads one atom's work over a team of threads for this regime, Sec. 2.1,
// Table 1, and Sec. 4).  With few atoms the one-thread-per-atom kernel leaves
// most of the GPU idle and each thread walks all of its ~26-54 neighbours in
// sequence; here the 32 lanes of a warp share one atom:
//   sweep 1: lane l takes the pairs l, l + 32, ... and accumulates partial
//            moments in registers (the generated per-pair code);
//   reduce:  the partial moments go through a per-warp shared-memory
//            transpose [c][lane] and lane l sums the components c = l (mod 32);
//   contract: every lane loads the full moment vector (broadcast reads) and
//            runs the contraction and its reverse pass redundantly (one
//            instruction stream for the warp, so this costs the same issue
//            slots as one lane) and so holds D = dE_i/dM in registers;
//   sweep 2: lane l takes the same pairs as in sweep 1, scatters F_j -= g and
//            keeps its share of F_i, W and dE/dc; F_i is summed across the warp.
// Levels with component groups (18 and 20) have their own kernel below.
#pragma once
#include "efv_kernel.cuh"

namespace mtp {

constexpr int kTeamWarps = 4;   // atoms (warps) per block of 128 threads

template <class R>
__host__ __device__ __forceinline__ size_t team_buf_bytes(int ncomp) {
  return sizeof(R) * (size_t)kTeamWarps * (size_t)ncomp * 33;
}

template <class LV, class R, bool DTHETA, int NQ = 0>
__global__ void __launch_bounds__(kEfvThreads) efv_team_kernel(const EfvArgs a) {
  static_assert(LV::NGROUPS == 1, "warp-per-atom kernel: levels with one component group");
  constexpr int NMU = LV::NMU;
  const int nq = NQ > 0 ? NQ : a.n_q;
  constexpr int C = LV::NCOMP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EfvShared<R, NMU, DTHETA> sm;
  sm.setup(a, smem_raw);
  sm.zero_gradients();
  const int SS = a.n_species * a.n_species;
  R* tbuf = reinterpret_cast<R*>(smem_raw + ((efv_smem_bytes<R, NMU, DTHETA>(SS, a.n_q, a.m) + 15) & ~size_t(15)));
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  R* tb = tbuf + (size_t)warp * C * 33;   // [c][33]: 32 lane partials, then the total
  const int64_t i = a.atom_begin + (int64_t)blockIdx.x * kTeamWarps + warp;
  const bool active = i < a.atom_end;   // warp-uniform
  double e_i = 0.0;
  R w[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  if (active) {
    const R* cell = cell_of<R>(a);
    PairGeom<R> geom;
    geom.load_centre(a, i, cell);
    const int zi = species_at(a.z, i, a.n_species);
    const int64_t beg = __ldg(a.offsets + i), end = __ldg(a.offsets + i + 1);
    const R* cz = sm.c + zi * sm.S * sm.cstride;
    // sweep 1: partial moments of this lane's pairs
    R M[C];
#pragma unroll
    for (int c = 0; c < C; ++c) M[c] = R(0);
    for (int64_t k = beg + lane; k < end; k += 32) {
      const int32_t j = __ldg(a.nbr_j + k), img = __ldg(a.nbr_img + k);
      const typename PairGeom<R>::Load lj = geom.fetch(a, j);
      R dx, dy, dz;
      geom.vec(a, lj, img, dx, dy, dz);
      const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
      const R rinv = rsqrt_r(r2);
      const R r = r2 * rinv;
      R f[NMU];
      radial<R, NMU, false, false, NQ>(cz + lj.species * sm.cstride, sm.nq, r, sm.mid, sm.scale, sm.rcut, f,
                                       nullptr, nullptr);
      LV::template moments<R>(M, f, dx * rinv, dy * rinv, dz * rinv);
    }
    // reduce across the warp through the transpose buffer
#pragma unroll
    for (int c = 0; c < C; ++c) tb[c * 33 + lane] = M[c];
    __syncwarp();
    for (int c = lane; c < C; c += 32) {
      R s = R(0);
#pragma unroll 8
      for (int t = 0; t < 32; ++t) s += tb[c * 33 + t];
      tb[c * 33 + 32] = s;
    }
    __syncwarp();
#pragma unroll
    for (int c = 0; c < C; ++c) M[c] = tb[c * 33 + 32];
    // contraction (every lane, the same values)
    R D[C];
    R Bv[DTHETA ? LV::NBASIS : 1];
    R ei;
    if constexpr (DTHETA)
      ei = LV::template contract<R, true>(M, sm.xi, D, Bv);
    else
      ei = LV::template contract<R, true, const R*, DiscardBasisSink<R>>(
          M, sm.xi, D, DiscardBasisSink<R>{sm.discard + warp, lane == 0});
    if (lane == 0) {
      e_i = a.species_energy[zi] + (double)ei;
      a.e_atom[i] = e_i;
      if (DTHETA) {
        for (int t = 0; t < (DTHETA ? LV::NBASIS : 1); ++t) atomicAdd(sm.dxi + t, Bv[t]);
        atomicAdd(sm.cnt + zi, 1);
      }
    }
    // sweep 2: this lane's pairs
    R fx = R(0), fy = R(0), fz = R(0);
    constexpr int kAccS = 4;
    const bool own_acc = DTHETA && sm.S <= kAccS;
    R acc[DTHETA ? kAccS * NMU * kMaxQ : 1];
    if (own_acc) {
      for (int t = 0; t < sm.S * NMU * nq; ++t) acc[t] = R(0);
    }
    for (int64_t k = beg + lane; k < end; k += 32) {
      const int32_t j = __ldg(a.nbr_j + k), img = __ldg(a.nbr_img + k);
      const typename PairGeom<R>::Load lj = geom.fetch(a, j);
      const int zj = lj.species;
      R dx, dy, dz;
      geom.vec(a, lj, img, dx, dy, dz);
      const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
      const R rinv = rsqrt_r(r2);
      const R r = r2 * rinv;
      R f[NMU], df[NMU], q[DTHETA ? kMaxQ : 1];
      radial<R, NMU, true, DTHETA, NQ>(cz + zj * sm.cstride, sm.nq, r, sm.mid, sm.scale, sm.rcut, f, df, q);
      R gx, gy, gz, Smu[NMU];
      LV::template pair_adjoint<R>(D, f, df, dx * rinv, dy * rinv, dz * rinv, rinv, gx, gy, gz, Smu);
      fx += gx;
      fy += gy;
      fz += gz;
      scatter_force(a, j, -gx, -gy, -gz);
      w[0] = fmadd(-gx, dx, w[0]);
      w[1] = fmadd(-gy, dy, w[1]);
      w[2] = fmadd(-gz, dz, w[2]);
      w[3] = fmadd(R(-0.5), fmadd(gx, dy, gy * dx), w[3]);
      w[4] = fmadd(R(-0.5), fmadd(gx, dz, gz * dx), w[4]);
      w[5] = fmadd(R(-0.5), fmadd(gy, dz, gz * dy), w[5]);
      if (DTHETA) {
        if (own_acc) {
          R* dst = acc + zj * NMU * nq;
#pragma unroll
          for (int mu = 0; mu < NMU; ++mu)
#pragma unroll
            for (int kk = 0; kk < kMaxQ; ++kk)
              if (kk < nq) dst[mu * nq + kk] = fmadd(q[kk], Smu[mu], dst[mu * nq + kk]);
        } else {
          R* dst = sm.dc + (zi * sm.S + zj) * NMU * nq;
#pragma unroll
          for (int mu = 0; mu < NMU; ++mu)
#pragma unroll
            for (int kk = 0; kk < kMaxQ; ++kk)
              if (kk < nq) atomicAdd(dst + mu * nq + kk, q[kk] * Smu[mu]);
        }
      }
    }
    if (own_acc) {
      for (int zj = 0; zj < sm.S; ++zj) {
        R* dst = sm.dc + (zi * sm.S + zj) * NMU * sm.nq;
        for (int t = 0; t < NMU * sm.nq; ++t) atomicAdd(dst + t, acc[zj * NMU * sm.nq + t]);
      }
    }
    fx = warp_sum_r(fx);
    fy = warp_sum_r(fy);
    fz = warp_sum_r(fz);
    if (lane == 0) {
      scatter_force(a, i, fx, fy, fz);
      if (!isfinite(e_i) || !isfinite((double)fx) || !isfinite((double)fy) || !isfinite((double)fz))
        flag_status(a.status, MTP_ERR_NONFINITE);
    }
  }
  efv_block_flush<LV, R, DTHETA>(sm, e_i, w, a.e_total, a.virial, a.dtheta);
}

// Levels with component groups (18 and 20: interpreted contraction).  One
// warp per atom as above, with three differences: the neighbours are swept
// once per component group (a group's partial moments fit in registers), the
// transpose buffer holds one group at a time, and the contraction is the
// warp-parallel interpreter on per-warp shared arrays V and A (its records
// spread over the lanes level by level).  Pairs closer than R_min take the
// FP64 radial path, as in the three-kernel form of these levels.
template <class R> struct AtomicBasisSink {
  R* dxi;
  __device__ __forceinline__ void operator()(int a, R v) const { atomicAdd(dxi + a, v); }
};

template <class LV> constexpr int group_span() {
  int m = 0;
  for (int g = 0; g < LV::NGROUPS; ++g) m = (LV::GROUP_C_HI[g] - LV::GROUP_C_LO[g]) > m ? (LV::GROUP_C_HI[g] - LV::GROUP_C_LO[g]) : m;
  return m;
}

template <class R> constexpr int team_groups_warps() { return sizeof(R) == 4 ? 4 : 2; }

template <class LV, class R>
__host__ __device__ __forceinline__ size_t team_groups_warp_bytes() {
  return sizeof(R) * ((size_t)group_span<LV>() * 33 + 2 * (size_t)LV::NVALUES);
}

template <class LV, class R, bool DTHETA, int G>
__device__ __forceinline__ void team_group_moments(const EfvArgs& a, const EfvShared<R, LV::NMU, DTHETA>& sm,
                                                   const PairGeom<R>& geom, int zi, int64_t beg, int64_t end,
                                                   int lane, R* tb, R* V) {
  constexpr int NMU = LV::NMU;
  R Mg[LV::NCOMP];
#pragma unroll
  for (int c = 0; c < LV::NCOMP; ++c) Mg[c] = R(0);
  for (int64_t k = beg + lane; k < end; k += 32) {
    const int32_t j = __ldg(a.nbr_j + k);
    int32_t img = __ldg(a.nbr_img + k);
    const typename PairGeom<R>::Load lj = geom.fetch(a, j);
    R dx, dy, dz;
    geom.vec(a, lj, img, dx, dy, dz);
    const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
    R rinv = rsqrt_r(r2);
    const R r = r2 * rinv;
    R f[NMU];
    if constexpr (std::is_same<R, float>::value) {
      if (r < sm.rmin)
        close_pair_fp64<NMU, false, false>(a, a.cell, geom.ci, j, img, zi, lj.species, dx, dy, dz, rinv, f, nullptr,
                                           nullptr);
      else
        radial<R, NMU, false, false>(sm.c + (zi * sm.S + lj.species) * sm.cstride, sm.nq, r, sm.mid, sm.scale,
                                     sm.rcut, f, nullptr, nullptr);
    } else {
      radial<R, NMU, false, false>(sm.c + (zi * sm.S + lj.species) * sm.cstride, sm.nq, r, sm.mid, sm.scale, sm.rcut,
                                   f, nullptr, nullptr);
    }
    LV::template moments_group<G, R>(Mg, f, dx * rinv, dy * rinv, dz * rinv);
  }
  constexpr int lo = LV::GROUP_C_LO[G], hi = LV::GROUP_C_HI[G];
  LV::template store_group<G, R>(Mg, tb - lo * 33 + lane, 33);   // tb[(c - lo) * 33 + lane]
  __syncwarp();
  for (int c = lo + lane; c < hi; c += 32) {
    R t = R(0);
#pragma unroll 8
    for (int u = 0; u < 32; ++u) t += tb[(c - lo) * 33 + u];
    V[c] = t;
  }
  __syncwarp();
}

template <class LV, class R, bool DTHETA, int G>
__device__ __forceinline__ void team_group_adjoint(const EfvArgs& a, const EfvShared<R, LV::NMU, DTHETA>& sm,
                                                   const PairGeom<R>& geom, int zi, int64_t beg, int64_t end,
                                                   int lane, const R* A, R& fx, R& fy, R& fz, R* w, R* acc,
                                                   bool own_acc) {
  constexpr int NMU = LV::NMU;
  R Dg[LV::NCOMP];
  LV::template load_group<G, R>(A, 1, Dg);
  for (int64_t k = beg + lane; k < end; k += 32) {
    const int32_t j = __ldg(a.nbr_j + k);
    int32_t img = __ldg(a.nbr_img + k);
    const typename PairGeom<R>::Load lj = geom.fetch(a, j);
    const int zj = lj.species;
    R dx, dy, dz;
    geom.vec(a, lj, img, dx, dy, dz);
    const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
    R rinv = rsqrt_r(r2);
    const R r = r2 * rinv;
    R f[NMU], df[NMU], q[DTHETA ? kMaxQ : 1];
    if constexpr (std::is_same<R, float>::value) {
      if (r < sm.rmin)
        close_pair_fp64<NMU, true, DTHETA>(a, a.cell, geom.ci, j, img, zi, zj, dx, dy, dz, rinv, f, df, q);
      else
        radial<R, NMU, true, DTHETA>(sm.c + (zi * sm.S + zj) * sm.cstride, sm.nq, r, sm.mid, sm.scale, sm.rcut, f,
                                     df, q);
    } else {
      radial<R, NMU, true, DTHETA>(sm.c + (zi * sm.S + zj) * sm.cstride, sm.nq, r, sm.mid, sm.scale, sm.rcut, f, df,
                                   q);
    }
    R gx, gy, gz, Smu[NMU];
    LV::template pair_adjoint_group<G, R>(Dg, f, df, dx * rinv, dy * rinv, dz * rinv, rinv, gx, gy, gz, Smu);
    fx += gx;
    fy += gy;
    fz += gz;
    scatter_force(a, j, -gx, -gy, -gz);
    w[0] = fmadd(-gx, dx, w[0]);
    w[1] = fmadd(-gy, dy, w[1]);
    w[2] = fmadd(-gz, dz, w[2]);
    w[3] = fmadd(R(-0.5), fmadd(gx, dy, gy * dx), w[3]);
    w[4] = fmadd(R(-0.5), fmadd(gx, dz, gz * dx), w[4]);
    w[5] = fmadd(R(-0.5), fmadd(gy, dz, gz * dy), w[5]);
    if (DTHETA) {
      constexpr int mu_lo = LV::GROUP_MU_LO[G], mu_hi = LV::GROUP_MU_HI[G];
      if (own_acc) {
        R* dst = acc + zj * NMU * sm.nq;
#pragma unroll
        for (int mu = mu_lo; mu < mu_hi; ++mu)
#pragma unroll
          for (int kk = 0; kk < kMaxQ; ++kk)
            if (kk < sm.nq) dst[mu * sm.nq + kk] = fmadd(q[kk], Smu[mu], dst[mu * sm.nq + kk]);
      } else {
        R* dst = sm.dc + (zi * sm.S + zj) * NMU * sm.nq;
#pragma unroll
        for (int mu = mu_lo; mu < mu_hi; ++mu)
#pragma unroll
          for (int kk = 0; kk < kMaxQ; ++kk)
            if (kk < sm.nq) atomicAdd(dst + mu * sm.nq + kk, q[kk] * Smu[mu]);
      }
    }
  }
}

template <class LV, class R, bool DTHETA>
__global__ void __launch_bounds__(128) efv_team_groups_kernel(const EfvArgs a) {
  static_assert(LV::NGROUPS == 2, "two component groups");
  constexpr int NMU = LV::NMU;
  constexpr int W = team_groups_warps<R>();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EfvShared<R, NMU, DTHETA> sm;
  sm.setup(a, smem_raw);
  sm.zero_gradients();
  const int SS = a.n_species * a.n_species;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  R* wbase = reinterpret_cast<R*>(smem_raw + ((efv_smem_bytes<R, NMU, DTHETA>(SS, a.n_q, a.m) + 15) & ~size_t(15)) +
                                  (size_t)warp * team_groups_warp_bytes<LV, R>());
  R* tb = wbase;
  R* V = tb + group_span<LV>() * 33;
  R* A = V + LV::NVALUES;
  __syncthreads();
  const int64_t i = a.atom_begin + (int64_t)blockIdx.x * W + warp;
  const bool active = i < a.atom_end;   // warp-uniform
  double e_i = 0.0;
  R w[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  if (active) {
    PairGeom<R> geom;
    geom.load_centre(a, i, cell_of<R>(a));
    const int zi = species_at(a.z, i, a.n_species);
    const int64_t beg = __ldg(a.offsets + i), end = __ldg(a.offsets + i + 1);
    team_group_moments<LV, R, DTHETA, 0>(a, sm, geom, zi, beg, end, lane, tb, V);
    team_group_moments<LV, R, DTHETA, 1>(a, sm, geom, zi, beg, end, lane, tb, V);
    R ei;
    if constexpr (DTHETA) ei = LV::template contract_warp<R, true>(V, A, sm.xi, AtomicBasisSink<R>{sm.dxi}, lane);
    else ei = LV::template contract_warp<R, false>(V, A, sm.xi, (R*)nullptr, lane);
    if (lane == 0) {
      e_i = a.species_energy[zi] + (double)ei;
      a.e_atom[i] = e_i;
      if (DTHETA) atomicAdd(sm.cnt + zi, 1);
    }
    R fx = R(0), fy = R(0), fz = R(0);
    constexpr int kAccS = 4;
    const bool own_acc = DTHETA && sm.S <= kAccS;
    R acc[DTHETA ? kAccS * NMU * kMaxQ : 1];
    if (own_acc) {
      for (int t = 0; t < sm.S * NMU * sm.nq; ++t) acc[t] = R(0);
    }
    team_group_adjoint<LV, R, DTHETA, 0>(a, sm, geom, zi, beg, end, lane, A, fx, fy, fz, w, acc, own_acc);
    team_group_adjoint<LV, R, DTHETA, 1>(a, sm, geom, zi, beg, end, lane, A, fx, fy, fz, w, acc, own_acc);
    if (own_acc) {
      for (int zj = 0; zj < sm.S; ++zj) {
        R* dst = sm.dc + (zi * sm.S + zj) * NMU * sm.nq;
        for (int t = 0; t < NMU * sm.nq; ++t) atomicAdd(dst + t, acc[zj * NMU * sm.nq + t]);
      }
    }
    fx = warp_sum_r(fx);
    fy = warp_sum_r(fy);
    fz = warp_sum_r(fz);
    if (lane == 0) {
      scatter_force(a, i, fx, fy, fz);
      if (!isfinite(e_i) || !isfinite((double)fx) || !isfinite((double)fy) || !isfinite((double)fz))
        flag_status(a.status, MTP_ERR_NONFINITE);
    }
  }
  efv_block_flush<LV, R, DTHETA>(sm, e_i, w, a.e_total, a.virial, a.dtheta);
}

template <class LV, class R, bool DTHETA>
int efv_team_launch_typed(const EfvArgs& a, cudaStream_t stream) {
  if constexpr (LV::NGROUPS == 2) {
    constexpr int W = team_groups_warps<R>();
    const int SS = a.n_species * a.n_species;
    const size_t bytes = ((efv_smem_bytes<R, LV::NMU, DTHETA>(SS, a.n_q, a.m) + 15) & ~size_t(15)) +
                         W * team_groups_warp_bytes<LV, R>();
    auto kern = efv_team_groups_kernel<LV, R, DTHETA>;
    int rc = set_smem(kern, bytes);
    if (rc != MTP_OK) return rc;
    const int64_t n = a.atom_end - a.atom_begin;
    if (n <= 0) return MTP_OK;
    const unsigned grid = (unsigned)((n + W - 1) / W);
    kern<<<grid, 32 * W, bytes, stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error("warp-per-atom kernel launch (level %d): %s", LV::LEVEL, cudaGetErrorString(e));
      return MTP_ERR_CUDA;
    }
    return MTP_OK;
  } else if constexpr (LV::NGROUPS != 1) {
    set_error("warp-per-atom kernel: level %d runs only as one thread per atom", LV::LEVEL);
    return MTP_ERR_UNSUPPORTED;
  } else {
    const int SS = a.n_species * a.n_species;
    const size_t bytes = ((efv_smem_bytes<R, LV::NMU, DTHETA>(SS, a.n_q, a.m) + 15) & ~size_t(15)) +
                         team_buf_bytes<R>(LV::NCOMP);
    auto kern = efv_team_kernel<LV, R, DTHETA>;
    if constexpr (std::is_same<R, float>::value) {
      if (a.n_q == kFixedQ) kern = efv_team_kernel<LV, R, DTHETA, kFixedQ>;
    }
    int rc = set_smem(kern, bytes);
    if (rc != MTP_OK) return rc;
    const int64_t n = a.atom_end - a.atom_begin;
    if (n <= 0) return MTP_OK;
    const unsigned grid = (unsigned)((n + kTeamWarps - 1) / kTeamWarps);
    kern<<<grid, kEfvThreads, bytes, stream>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error("warp-per-atom kernel launch (level %d): %s", LV::LEVEL, cudaGetErrorString(e));
      return MTP_ERR_CUDA;
    }
    return MTP_OK;
  }
}

template <class LV>
int efv_team_launch(const EfvArgs& a, int precision, bool want_dtheta, cudaStream_t stream) {
  if (precision == MTP_MIXED)
    return want_dtheta ? efv_team_launch_typed<LV, float, true>(a, stream)
                       : efv_team_launch_typed<LV, float, false>(a, stream);
  return want_dtheta ? efv_team_launch_typed<LV, double, true>(a, stream)
                     : efv_team_launch_typed<LV, double, false>(a, stream);
}

}  // namespace mtp
