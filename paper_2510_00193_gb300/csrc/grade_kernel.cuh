// Basis rows for the extrapolation grade (paper Sec. 2.1 and Sec. 2.3:
// neighbourhood- and configuration-mode grades with selection and break
// thresholds; the grade of a neighbourhood b_i against an active set A is
// gamma_i = max_k |(b_i A^-1)_k|).
//
// basis_rows_kernel: one thread per listed atom; the forward neighbour sweep
// and the generated contraction (same code as the energy kernel) give the
// basis row b_i in FP64, written to rows[r][0..m); the configuration-mode
// sum sum_i b_i is accumulated in FP64 (warp shuffles, then one atomic per
// warp and basis function).
#pragma once
#include "efv_kernel.cuh"

namespace mtp {

constexpr int kRowsThreads = 128;

template <class LV>
__global__ void __launch_bounds__(kRowsThreads) basis_rows_kernel(const EfvArgs a, const int32_t* __restrict__ list,
                                                                  int64_t n_rows, double* __restrict__ rows,
                                                                  int64_t ld, double* __restrict__ bsum) {
  using R = double;
  constexpr int NMU = LV::NMU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int S = a.n_species;
  const int SS = S * S;
  const int nq = a.n_q;
  const int cstride = CoefLayout<R, NMU>::cstride(nq);
  R* s_c = reinterpret_cast<R*>(smem_raw);
  R* s_xi = s_c + SS * cstride;
  fill_coefs<R, NMU>(s_c, a.radial_d, SS, nq);
  for (int t = threadIdx.x; t < a.m; t += blockDim.x) s_xi[t] = a.xi_d[t];
  __syncthreads();

  const R rcut = R(a.r_cut);
  const R mid = R(0.5 * (a.r_min + a.r_cut));
  const R scale = R(2.0 / (a.r_cut - a.r_min));
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = r < n_rows;
  R B[LV::NBASIS];
#pragma unroll
  for (int t = 0; t < LV::NBASIS; ++t) B[t] = R(0);
  if (active) {
    const int64_t i = list ? (int64_t)list[r] : a.atom_begin + r;
    PairGeom<R> geom;
    geom.load_centre(a, i, a.cell);
    const int zi = species_at(a.z, i, a.n_species);
    R M[LV::NCOMP];
#pragma unroll
    for (int c = 0; c < LV::NCOMP; ++c) M[c] = R(0);
    PairStream<R> ps;
    int32_t j, img;
    typename PairGeom<R>::Load lj;
    ps.start(a, geom, __ldg(a.offsets + i), __ldg(a.offsets + i + 1));
    while (ps.next(a, geom, j, img, lj)) {
      R dx, dy, dz;
      geom.vec(a, lj, img, dx, dy, dz);
      const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
      const R rinv = rsqrt_r(r2);
      const R rr = r2 * rinv;
      R f[NMU];
      radial<R, NMU, false, false>(s_c + (zi * S + lj.species) * cstride, nq, rr, mid, scale, rcut, f, nullptr,
                                   nullptr);
      LV::template moments<R>(M, f, dx * rinv, dy * rinv, dz * rinv);
    }
    R D[LV::NCOMP];
    (void)LV::template contract<R, true>(M, s_xi, D, B);
    double* dst = rows + r * ld;
#pragma unroll
    for (int t = 0; t < LV::NBASIS; ++t) dst[t] = B[t];
  }
  if (bsum) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int t = 0; t < LV::NBASIS; ++t) {
      const double v = warp_sum(B[t]);
      if (lane == 0) atomicAdd(bsum + t, v);
    }
  }
}

template <class LV>
int basis_rows_launch(const EfvArgs& a, const int32_t* list, int64_t n_rows, double* rows, int64_t ld, double* bsum,
                      cudaStream_t stream) {
  if (n_rows <= 0) return MTP_OK;
  const int SS = a.n_species * a.n_species;
  const size_t bytes = sizeof(double) * ((size_t)SS * CoefLayout<double, LV::NMU>::cstride(a.n_q) + a.m);
  auto kern = basis_rows_kernel<LV>;
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
      set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
      return MTP_ERR_CUDA;
    }
  }
  kern<<<(unsigned)((n_rows + kRowsThreads - 1) / kRowsThreads), kRowsThreads, bytes, stream>>>(a, list, n_rows,
                                                                                                  rows, ld, bsum);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("basis_rows kernel launch (level %d): %s", LV::LEVEL, cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  return MTP_OK;
}

}  // namespace mtp
