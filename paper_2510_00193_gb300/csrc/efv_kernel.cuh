// Energy / force / virial / parameter-gradient kernel for one MTP level.
//
// One thread per centre atom i, two sweeps over its neighbours:
//   sweep 1: pair vector, radial functions f_mu (Chebyshev basis times
//            (R_cut - r)^2), moment components M[c] += f_mu rhat^K, all in
//            registers (straight-line code generated per level);
//   contraction: graph values, basis products, E_i = s + sum xi B and the
//            reverse pass D = dE_i/dM (generated straight-line code);
//   sweep 2: per pair g_ij = dE_i/dr_ij from D (generated), F_i += g,
//            F_j -= g (FP64 atomics), W -= sym(g (x) r_ij), and with DTHETA
//            dE/dc[mu][k][zi][zj] += Q_k(r) S_mu.
// Reductions of E, W and dE/dtheta are FP64 (warp shuffles, then one atomic
// per block).
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "mtp_internal.cuh"
#include "mtp_math.cuh"

namespace mtp {

constexpr int kEfvThreads = 128;       // split and warp-per-atom kernels
constexpr int kEfvFusedThreads = 128;  // the fused one-thread-per-atom kernel

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_sum_r(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_r(double v) { return warp_sum(v); }

__device__ __forceinline__ void flag_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Pair vector r_ij = x_j + n.H - x_i, in two steps so that the loads of the
// next pair can be issued before the current pair is processed:
// fetch(j) loads what the pair needs from atom j, vec() forms the vector.
template <class R> struct PairGeom;

template <> struct PairGeom<double> {
  // FP64: positions directly, shift s = (n1 a + n2 b) + n3 c.
  struct Load {
    double x, y, z;
    int species;
  };
  double xi, yi, zi;
  const double* c;   // cell rows of the configuration
  __device__ __forceinline__ void load_centre(const EfvArgs& a, int64_t i, const double* cell) {
    xi = a.x[3 * i]; yi = a.x[3 * i + 1]; zi = a.x[3 * i + 2];
    c = cell;
  }
  __device__ __forceinline__ Load fetch(const EfvArgs& a, int32_t j) const {
    Load l;
    l.x = __ldg(a.x + 3 * (int64_t)j);
    l.y = __ldg(a.x + 3 * (int64_t)j + 1);
    l.z = __ldg(a.x + 3 * (int64_t)j + 2);
    l.species = species_at(a.z, j, a.n_species);
    return l;
  }
  __device__ __forceinline__ void vec(const EfvArgs& a, const Load& l, int32_t img, double& dx, double& dy,
                                      double& dz) const {
    int n1, n2, n3;
    unpack_image(img, n1, n2, n3);
    const double sx = ((double)n1 * c[0] + (double)n2 * c[3]) + (double)n3 * c[6];
    const double sy = ((double)n1 * c[1] + (double)n2 * c[4]) + (double)n3 * c[7];
    const double sz = ((double)n1 * c[2] + (double)n2 * c[5]) + (double)n3 * c[8];
    dx = (l.x + sx) - xi;
    dy = (l.y + sy) - yi;
    dz = (l.z + sz) - zi;
  }
};

// Exact int -> float for |v| < 2^22 without a conversion instruction: the
// integer is added to the mantissa of 1.5 * 2^23.
__device__ __forceinline__ float small_int_to_float(int v) {
  return __int_as_float(0x4B400000 + v) - 12582912.0f;
}

// 32.32 fixed-point difference (int64) to a float in units of one cell:
// v = hi 2^16 + lo with hi = floor(v / 2^16) and 0 <= lo < 2^16.  Both parts
// are exact as floats (hi through the mantissa trick while |hi| < 2^22, that
// is up to 64 cells), so the single rounding is in the final sum, and no
// conversion runs on the FP64 pipe.
__device__ __forceinline__ float fixed_to_float(long long v) {
  const int hi = (int)(v >> 16);
  const float lo = small_int_to_float((int)(v & 0xFFFF));
  const float h = ((unsigned)(hi + (1 << 22)) < (1u << 23)) ? small_int_to_float(hi) : (float)hi;
  return fmaf(h, 65536.0f, lo) * 2.3283064365386963e-10f;
}

template <> struct PairGeom<float> {
  // Mixed: exact integer difference of 32.32 fixed-point fractional
  // coordinates plus the image, converted to FP32 and mapped by the cell.
  struct Load {
    longlong2 xy, zs;   // (qx, qy), (qz, species)
    int species;
  };
  long long qx, qy, qz;
  const float* c;    // cell rows of the configuration
  int32_t ci;        // centre atom (for the FP64 evaluation of close pairs)
  __device__ __forceinline__ void load_centre(const EfvArgs& a, int64_t i, const float* cell) {
    const longlong2 p = *reinterpret_cast<const longlong2*>(a.xq + 4 * i);
    const longlong2 q = *reinterpret_cast<const longlong2*>(a.xq + 4 * i + 2);
    qx = p.x; qy = p.y; qz = q.x;
    c = cell;
    ci = (int32_t)i;
  }
  __device__ __forceinline__ Load fetch(const EfvArgs& a, int32_t j) const {
    Load l;
    l.xy = __ldg(reinterpret_cast<const longlong2*>(a.xq + 4 * (int64_t)j));
    l.zs = __ldg(reinterpret_cast<const longlong2*>(a.xq + 4 * (int64_t)j + 2));
    l.species = (int)l.zs.y;
    return l;
  }
  __device__ __forceinline__ void vec(const EfvArgs& a, const Load& l, int32_t img, float& dx, float& dy,
                                      float& dz) const {
    int n1, n2, n3;
    unpack_image(img, n1, n2, n3);
    const float fx = fixed_to_float(l.xy.x - qx + ((long long)n1 << 32));
    const float fy = fixed_to_float(l.xy.y - qy + ((long long)n2 << 32));
    const float fz = fixed_to_float(l.zs.x - qz + ((long long)n3 << 32));
    dx = fmaf(fz, c[6], fmaf(fy, c[3], fx * c[0]));
    dy = fmaf(fz, c[7], fmaf(fy, c[4], fx * c[1]));
    dz = fmaf(fz, c[8], fmaf(fy, c[5], fx * c[2]));
  }
};

// Neighbour stream with software prefetch: the entry two pairs ahead and
// the atom data one pair ahead are in flight while a pair is processed.
template <class R>
struct PairStream {
  using Geom = PairGeom<R>;
  int64_t k, end;
  int32_t j1, im1, j2, im2;
  typename Geom::Load l1;
  __device__ __forceinline__ void start(const EfvArgs& a, const Geom& g, int64_t beg, int64_t end_) {
    k = beg;
    end = end_;
    j1 = im1 = j2 = im2 = 0;
    if (k < end) { j1 = __ldg(a.nbr_j + k); im1 = __ldg(a.nbr_img + k); }
    if (k + 1 < end) { j2 = __ldg(a.nbr_j + k + 1); im2 = __ldg(a.nbr_img + k + 1); }
    if (k < end) l1 = g.fetch(a, j1);
  }
  __device__ __forceinline__ bool next(const EfvArgs& a, const Geom& g, int32_t& j, int32_t& img,
                                       typename Geom::Load& l) {
    if (k >= end) return false;
    j = j1; img = im1; l = l1;
    j1 = j2; im1 = im2;
    if (k + 1 < end) l1 = g.fetch(a, j1);
    if (k + 2 < end) { j2 = __ldg(a.nbr_j + k + 2); im2 = __ldg(a.nbr_img + k + 2); }
    ++k;
    return true;
  }
  // Branch-free step for the software-pipelined sweeps (beg < end): past the
  // end it returns the last entry again, whose data are valid, and the caller
  // discards what it computes from it.
  __device__ __forceinline__ void step(const EfvArgs& a, const Geom& g, int32_t& j, int32_t& img,
                                       typename Geom::Load& l) {
    j = j1; img = im1; l = l1;
    const int64_t k2 = k + 2 < end ? k + 2 : end - 1;
    if (k + 1 < end) { j1 = j2; im1 = im2; }
    l1 = g.fetch(a, j1);
    j2 = __ldg(a.nbr_j + k2);
    im2 = __ldg(a.nbr_img + k2);
    ++k;
  }
};

// Force accumulation: FP64 atomics on the FP64 path; FP32 atomics into the
// FP32 accumulator on the mixed path (converted to FP64 once per atom at the end).
__device__ __forceinline__ void scatter_force(const EfvArgs& a, int64_t k, double gx, double gy, double gz) {
  atomicAdd(a.forces + 3 * k, gx);
  atomicAdd(a.forces + 3 * k + 1, gy);
  atomicAdd(a.forces + 3 * k + 2, gz);
}
__device__ __forceinline__ void scatter_force(const EfvArgs& a, int64_t k, float gx, float gy, float gz) {
  atomicAdd(a.forces_f + 3 * k, gx);
  atomicAdd(a.forces_f + 3 * k + 1, gy);
  atomicAdd(a.forces_f + 3 * k + 2, gz);
}

template <class R> __device__ __forceinline__ const R* cell_of(const EfvArgs& a);
template <> __device__ __forceinline__ const double* cell_of<double>(const EfvArgs& a) { return a.cell; }
template <> __device__ __forceinline__ const float* cell_of<float>(const EfvArgs& a) { return a.cellf; }

__device__ __forceinline__ float rsqrt_r(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsqrt_r(double v) { return rsqrt(v); }

// Radial functions of one pair.  c points at the (zi, zj) block, [mu][k].
// Radial coefficients in shared memory: per species pair (zi, zj) a block
// [k][mu] with mu padded to whole 16-byte vectors (KS entries per k), so that
// the NMU coefficients of one k arrive in one or two vector loads; successive
// pair blocks start one vector apart beyond that, which spreads the lanes of
// a warp (different neighbour species) over the banks.
template <class C, int NMU>
struct CoefLayout {
  static constexpr int V = 16 / (int)sizeof(C);   // entries per 16-byte vector
  static constexpr int KS = (NMU + V - 1) / V * V;
  __host__ __device__ static constexpr int cstride(int nq) { return nq * KS + V; }
  // shared index of c[mu][k] within a pair block
  __host__ __device__ static constexpr int at(int mu, int k) { return k * KS + mu; }
};

template <class C, int NMU>
__device__ __forceinline__ void load_coefs(const C* __restrict__ p, C (&v)[CoefLayout<C, NMU>::KS]) {
  constexpr int KS = CoefLayout<C, NMU>::KS;
  if constexpr (sizeof(C) == 4) {
#pragma unroll
    for (int g = 0; g < KS / 4; ++g) {
      const float4 t = reinterpret_cast<const float4*>(p)[g];
      v[4 * g] = t.x; v[4 * g + 1] = t.y; v[4 * g + 2] = t.z; v[4 * g + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int g = 0; g < KS / 2; ++g) {
      const double2 t = reinterpret_cast<const double2*>(p)[g];
      v[2 * g] = t.x; v[2 * g + 1] = t.y;
    }
  }
}

// f_mu = cut^2 sum_k c T_k, df_mu/dr = scale cut^2 sum_k c T'_k - 2 cut sum_k c T_k,
// with T_k(xi) the Chebyshev polynomials, xi = (r - mid) scale, cut = R_cut - r.
// c: the pair's coefficient block (CoefLayout).  NQ > 0 fixes n_q at compile
// time (nq is then ignored).
template <class R, int NMU, bool DERIV, bool WANT_Q, int NQ = 0, class C>
__device__ __forceinline__ void radial(const C* __restrict__ c, int nq_rt, R r, R mid, R scale, R rcut, R* f,
                                       R* df, R* q) {
  // c holds scalar coefficients (C); R may be C or a dual number over C
  using L = CoefLayout<C, NMU>;
  const int nq = NQ > 0 ? NQ : nq_rt;
  const R x = (r - mid) * scale;
  const R cut = rcut - r;
  const R cut2 = cut * cut;
  R t0 = R(1), t1 = x, d0 = R(0), d1 = R(1);
  R A[NMU], Bd[NMU];
  C cc[L::KS];
  load_coefs<C, NMU>(c, cc);
#pragma unroll
  for (int mu = 0; mu < NMU; ++mu) {
    A[mu] = R(cc[mu]);
    Bd[mu] = R(0);
  }
  if (WANT_Q) q[0] = cut2;
  if (nq > 1) {
    load_coefs<C, NMU>(c + L::KS, cc);
#pragma unroll
    for (int mu = 0; mu < NMU; ++mu) {
      A[mu] = fmadd(R(cc[mu]), x, A[mu]);
      if (DERIV) Bd[mu] = R(cc[mu]);
    }
    if (WANT_Q) q[1] = x * cut2;
  }
#pragma unroll
  for (int k = 2; k < kMaxQ; ++k) {
    if (k < nq) {
      const R t2 = fmadd(R(2) * x, t1, -t0);
      const R d2 = fmadd(R(2) * x, d1, fmadd(R(2), t1, -d0));
      load_coefs<C, NMU>(c + k * L::KS, cc);
#pragma unroll
      for (int mu = 0; mu < NMU; ++mu) {
        A[mu] = fmadd(R(cc[mu]), t2, A[mu]);
        if (DERIV) Bd[mu] = fmadd(R(cc[mu]), d2, Bd[mu]);
      }
      if (WANT_Q) q[k] = t2 * cut2;
      t0 = t1; t1 = t2; d0 = d1; d1 = d2;
    }
  }
#pragma unroll
  for (int mu = 0; mu < NMU; ++mu) {
    f[mu] = cut2 * A[mu];
    if (DERIV) df[mu] = fmadd(scale * cut2, Bd[mu], R(-2) * cut * A[mu]);
  }
}

// Fills the pair blocks of CoefLayout from the global layout [mu][k][zi][zj]
// (called by every thread of the block).
template <class C, int NMU, class SRC>
__device__ __forceinline__ void fill_coefs(C* dst, const SRC* __restrict__ src, int SS, int nq) {
  using L = CoefLayout<C, NMU>;
  for (int t = threadIdx.x; t < NMU * nq * SS; t += blockDim.x) {
    const int pair = t % SS, mk = t / SS;
    dst[pair * L::cstride(nq) + L::at(mk / nq, mk % nq)] = C(src[t]);
  }
}

// Pairs closer than R_min on the mixed path.  Below R_min the radial basis is
// extrapolated: the Chebyshev polynomials are evaluated at xi < -1, where
// they grow like cosh(k arccosh |xi|) and are steep, so the FP32 rounding of
// the distance (a few units in the last place) is amplified in f_mu and
// df_mu/dr, and at such close contacts the pair gradient is a sum of large
// basis-function terms that cancel (on the 256,000-atom level-20 workload this
// gave force errors of 0.15 eV/A against FP64 on the atoms of its closest
// pairs).  These pairs are rare (about 7e-4 per atom there), so for them the
// pair vector comes from the FP64 positions and the distance, the radial
// functions, their derivatives and (with WANT_Q) the basis values Q_k are
// evaluated in FP64 with the FP64 coefficients, then rounded to FP32 once.
// `cell` holds the FP64 rows of the configuration's cell.  Used by the
// level-18/20 split kernels; the fused kernels keep FP32 for every pair
// (an inlined FP64 branch cost them 20% at level 16, where no pair of the
// 1,024,000-atom workload comes closer than R_min, and 3x on the random
// gases, where a third of the warp iterations hold a pair between the 1.9 A
// minimum separation and R_min = 2 A and GB300's FP64 pipe serialises them).
template <int NMU, bool DERIV, bool WANT_Q>
__device__ __forceinline__ void close_pair_fp64(const EfvArgs& a, const double* cell, int32_t ci, int32_t j,
                                                int32_t img, int zi, int zj, float& dx, float& dy, float& dz,
                                                float& rinv, float* f, float* df, float* q) {
  int n1, n2, n3;
  unpack_image(img, n1, n2, n3);
  const double sx = ((double)n1 * cell[0] + (double)n2 * cell[3]) + (double)n3 * cell[6];
  const double sy = ((double)n1 * cell[1] + (double)n2 * cell[4]) + (double)n3 * cell[7];
  const double sz = ((double)n1 * cell[2] + (double)n2 * cell[5]) + (double)n3 * cell[8];
  const double ex = (a.x[3 * (int64_t)j] + sx) - a.x[3 * (int64_t)ci];
  const double ey = (a.x[3 * (int64_t)j + 1] + sy) - a.x[3 * (int64_t)ci + 1];
  const double ez = (a.x[3 * (int64_t)j + 2] + sz) - a.x[3 * (int64_t)ci + 2];
  const double r = sqrt(fma(ez, ez, fma(ey, ey, ex * ex)));
  const double ri = 1.0 / r;
  dx = (float)ex;
  dy = (float)ey;
  dz = (float)ez;
  rinv = (float)ri;
  const int S = a.n_species, nq = a.n_q;
  const double x = (r - 0.5 * (a.r_min + a.r_cut)) * (2.0 / (a.r_cut - a.r_min));
  const double scale = 2.0 / (a.r_cut - a.r_min);
  const double cut = a.r_cut - r;
  const double cut2 = cut * cut;
  double A[NMU], B[NMU];
  const double* cz = a.radial_d + (int64_t)zi * S + zj;   // c[mu][k][zi][zj] at cz[(mu nq + k) S^2]
  const int64_t ss = (int64_t)S * S;
  double t0 = 1.0, t1 = x, d0 = 0.0, d1 = 1.0;
#pragma unroll
  for (int mu = 0; mu < NMU; ++mu) {
    A[mu] = cz[(int64_t)mu * nq * ss];
    B[mu] = 0.0;
  }
  if (WANT_Q) q[0] = (float)cut2;
  for (int k = 1; k < nq; ++k) {
    double tk = t1, dk = d1;
    if (k >= 2) {
      tk = 2.0 * x * t1 - t0;
      dk = 2.0 * x * d1 + 2.0 * t1 - d0;
      t0 = t1; t1 = tk; d0 = d1; d1 = dk;
    }
#pragma unroll
    for (int mu = 0; mu < NMU; ++mu) {
      const double cc = cz[((int64_t)mu * nq + k) * ss];
      A[mu] = fma(cc, tk, A[mu]);
      if (DERIV) B[mu] = fma(cc, dk, B[mu]);
    }
    if (WANT_Q) q[k] = (float)(tk * cut2);
  }
#pragma unroll
  for (int mu = 0; mu < NMU; ++mu) {
    f[mu] = (float)(cut2 * A[mu]);
    if (DERIV) df[mu] = (float)(scale * cut2 * B[mu] - 2.0 * cut * A[mu]);
  }
}

// Byte offset of the FP64 reduction area in the kernel's dynamic shared memory.
template <class R, int NMU, bool DTHETA>
__host__ __device__ __forceinline__ size_t efv_red_offset(int SS, int nq, int m) {
  const size_t cstride = (size_t)CoefLayout<R, NMU>::cstride(nq);
  size_t bytes = sizeof(R) * ((size_t)SS * cstride + m);
  if (DTHETA) bytes += sizeof(R) * ((size_t)SS * NMU * nq + m);
  return (bytes + 15) & ~size_t(15);
}

constexpr int kMaxWarps = 8;   // blocks of up to 256 threads

template <class R, int NMU, bool DTHETA>
__host__ __device__ __forceinline__ size_t efv_smem_bytes(int SS, int nq, int m) {
  // ... then the per-species atom counts and one 8-byte discard slot per warp
  return efv_red_offset<R, NMU, DTHETA>(SS, nq, m) + sizeof(double) * 8 * kMaxWarps +
         ((sizeof(int) * kMaxSpecies + 7) & ~size_t(7)) + sizeof(double) * kMaxWarps;
}

// Mixed path with DTHETA: each thread's dE/dc accumulators [zj][mu][k] in
// shared memory, strided by the block size ([entry][thread], conflict-free),
// after the areas above.  (As a thread-private array indexed with the
// run-time n_q they lived in local memory, whose lines the batch kernel wrote
// back to DRAM.)  The FP64 path keeps the thread-private array.
template <class R, int NMU, bool DTHETA>
__host__ __device__ __forceinline__ size_t efv_acc_bytes(int S, int nq, int threads) {
  return (DTHETA && sizeof(R) == 4 && S <= 4) ? sizeof(R) * (size_t)S * NMU * nq * threads : 0;
}

__device__ __forceinline__ uint32_t dynamic_smem_size() {
  uint32_t r;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

// Accumulator array with a stride: thread-private (stride 1) or a thread's
// column of the shared [entry][thread] array.
// Basis-value sink of the contraction: the warp's sum of basis value a
// (lanes without an atom add zero) is added to the block's dE/dxi slot.
template <class R> struct WarpBasisSink {
  R* dxi;
  int lane;
  bool active;
  __device__ __forceinline__ void operator()(int a, R v) const {
    const R s = warp_sum_r(active ? v : R(0));
    if (lane == 0) atomicAdd(dxi + a, s);
  }
};

// Consumes each basis value as the contraction forms it: lane 0 of the warp
// writes it to the warp's own shared word, which nothing reads.  Used where the basis values
// are not wanted: with a use of this kind the level-16 energy/force kernel
// compiles without stack (the contraction alone fits in its registers);
// without one, ptxas keeps values of the contraction live into the adjoint
// sweep and spills about 1.1 KB per thread.
template <class R> struct DiscardBasisSink {
  R* slot;
  bool lane0;
  __device__ __forceinline__ void operator()(int, R v) const {
    if (lane0) *slot = v;
  }
};

template <class R> struct AccView {
  R* p;
  int stride;
  __device__ __forceinline__ R& operator[](int t) const { return p[t * stride]; }
};

// Shared-memory view: radial coefficients (pair blocks of CoefLayout), xi,
// and with DTHETA the per-block gradient accumulators.
template <class R, int NMU, bool DTHETA>
struct EfvShared {
  R* c;
  R* xi;
  R* dc;      // [SS][NMU][nq]
  R* dxi;     // [m]
  R* acc;     // mixed DTHETA: per-thread dE/dc accumulators [S NMU nq][blockDim], or null
  double* red;
  int* cnt;   // [S]
  R* discard; // [kMaxWarps] words that DiscardBasisSink writes and nothing reads
  int S, SS, nq, cstride, m;
  R rcut, mid, scale, rmin;

  __device__ __forceinline__ void setup(const EfvArgs& a, unsigned char* raw) {
    S = a.n_species;
    SS = S * S;
    nq = a.n_q;
    m = a.m;
    cstride = CoefLayout<R, NMU>::cstride(nq);
    c = reinterpret_cast<R*>(raw);
    xi = c + SS * cstride;
    dc = xi + m;
    dxi = dc + (DTHETA ? SS * NMU * nq : 0);
    red = reinterpret_cast<double*>(raw + efv_red_offset<R, NMU, DTHETA>(SS, nq, m));
    cnt = reinterpret_cast<int*>(red + 8 * kMaxWarps);
    discard = reinterpret_cast<R*>(red + 8 * kMaxWarps + (sizeof(int) * kMaxSpecies + 7) / 8);
    acc = nullptr;
    if (DTHETA && sizeof(R) == 4 && S <= 4) {
      const size_t off = (efv_smem_bytes<R, NMU, DTHETA>(SS, nq, m) + 15) & ~size_t(15);
      if ((size_t)dynamic_smem_size() >= off + efv_acc_bytes<R, NMU, DTHETA>(S, nq, blockDim.x))
        acc = reinterpret_cast<R*>(raw + off);
    }
    const R* radial_src;
    const R* xi_src;
    if constexpr (sizeof(R) == 8) {
      radial_src = reinterpret_cast<const R*>(a.radial_d);
      xi_src = reinterpret_cast<const R*>(a.xi_d);
    } else {
      radial_src = reinterpret_cast<const R*>(a.radial_f);
      xi_src = reinterpret_cast<const R*>(a.xi_f);
    }
    fill_coefs<R, NMU>(c, radial_src, SS, nq);
    for (int t = threadIdx.x; t < m; t += blockDim.x) xi[t] = xi_src[t];
    rcut = R(a.r_cut);
    rmin = R(a.r_min);
    mid = R(0.5 * (a.r_min + a.r_cut));
    scale = R(2.0 / (a.r_cut - a.r_min));
  }

  __device__ __forceinline__ void zero_gradients() {
    if (!DTHETA) return;
    for (int t = threadIdx.x; t < SS * NMU * nq; t += blockDim.x) dc[t] = R(0);
    for (int t = threadIdx.x; t < m; t += blockDim.x) dxi[t] = R(0);
    for (int t = threadIdx.x; t < S; t += blockDim.x) cnt[t] = 0;
  }
};

// First neighbour sweep: M[c] += f_mu(r_ij) rhat^K for the components of
// group G (G < 0: all components; G >= 0: the level's component group G).
// CLOSE64 (mixed path only): pairs closer than R_min take close_pair_fp64.
// Which sweeps are software-pipelined when DTHETA is set (without it both are).
constexpr bool kPipeMomentsDtheta = true;
constexpr bool kPipeAdjointDtheta = false;

// Geometry and radial functions of one pair for the first sweep: f_mu(r) and
// the unit vector u = r_ij / r.
template <class LV, class R, bool DTHETA, int NQ>
__device__ __forceinline__ void pair_radial(const EfvArgs& a, const EfvShared<R, LV::NMU, DTHETA>& sm,
                                            const PairGeom<R>& geom, int zi, const typename PairGeom<R>::Load& lj,
                                            int32_t img, R* f, R& ux, R& uy, R& uz) {
  R dx, dy, dz;
  geom.vec(a, lj, img, dx, dy, dz);
  const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
  const R rinv = rsqrt_r(r2);
  const R r = r2 * rinv;
  radial<R, LV::NMU, false, false, NQ>(sm.c + (zi * sm.S + lj.species) * sm.cstride, sm.nq, r, sm.mid, sm.scale,
                                       sm.rcut, f, nullptr, nullptr);
  ux = dx * rinv;
  uy = dy * rinv;
  uz = dz * rinv;
}

// The same for the second sweep: also df_mu/dr, the pair vector, 1/r and,
// with DTHETA, the basis values Q_k(r).
template <class LV, class R, bool DTHETA, int NQ>
struct PairTerms {
  R f[LV::NMU], df[LV::NMU], q[DTHETA ? kMaxQ : 1];
  R dx, dy, dz, rinv;
  int32_t j;
  int zj;
  __device__ __forceinline__ void eval(const EfvArgs& a, const EfvShared<R, LV::NMU, DTHETA>& sm,
                                       const PairGeom<R>& geom, int zi, int32_t j_, int32_t img,
                                       const typename PairGeom<R>::Load& lj) {
    j = j_;
    zj = lj.species;
    geom.vec(a, lj, img, dx, dy, dz);
    const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
    rinv = rsqrt_r(r2);
    const R r = r2 * rinv;
    radial<R, LV::NMU, true, DTHETA, NQ>(sm.c + (zi * sm.S + zj) * sm.cstride, sm.nq, r, sm.mid, sm.scale,
                                         sm.rcut, f, df, q);
  }
};

template <class LV, class R, bool DTHETA, int G, bool CLOSE64 = false, int NQ = 0>
__device__ __forceinline__ void moment_sweep(const EfvArgs& a, const EfvShared<R, LV::NMU, DTHETA>& sm,
                                             const PairGeom<R>& geom, const double* cell64, int zi, int64_t beg,
                                             int64_t end, R* M) {
  constexpr int NMU = LV::NMU;
  PairStream<R> ps;
  int32_t j, img;
  typename PairGeom<R>::Load lj;
  ps.start(a, geom, beg, end);
  if constexpr (!CLOSE64 && (kPipeMomentsDtheta || !DTHETA)) {
    // software-pipelined: the geometry and radial functions of the next pair
    // (one basic block with this pair's moment terms, so that the scheduler
    // overlaps the latency chain of the one with the independent FMAs of
    // the other)
    if (beg >= end) return;
    R f[NMU], ux, uy, uz;
    ps.step(a, geom, j, img, lj);
    pair_radial<LV, R, DTHETA, NQ>(a, sm, geom, zi, lj, img, f, ux, uy, uz);
    for (int64_t p = beg; p < end; ++p) {
      R fn[NMU], uxn, uyn, uzn;
      ps.step(a, geom, j, img, lj);
      pair_radial<LV, R, DTHETA, NQ>(a, sm, geom, zi, lj, img, fn, uxn, uyn, uzn);
      if constexpr (G < 0) LV::template moments<R>(M, f, ux, uy, uz);
      else LV::template moments_group<G, R>(M, f, ux, uy, uz);
#pragma unroll
      for (int mu = 0; mu < NMU; ++mu) f[mu] = fn[mu];
      ux = uxn; uy = uyn; uz = uzn;
    }
    return;
  }
  while (ps.next(a, geom, j, img, lj)) {
    R dx, dy, dz;
    geom.vec(a, lj, img, dx, dy, dz);
    const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
    R rinv = rsqrt_r(r2);
    const R r = r2 * rinv;
    R f[NMU];
    if constexpr (CLOSE64 && std::is_same<R, float>::value) {
      if (r < sm.rmin)
        close_pair_fp64<NMU, false, false>(a, cell64, geom.ci, j, img, zi, lj.species, dx, dy,
                                           dz, rinv, f, nullptr, nullptr);
      else
        radial<R, NMU, false, false, NQ>(sm.c + (zi * sm.S + lj.species) * sm.cstride, sm.nq, r, sm.mid,
                                         sm.scale, sm.rcut, f, nullptr, nullptr);
    } else {
      radial<R, NMU, false, false, NQ>(sm.c + (zi * sm.S + lj.species) * sm.cstride, sm.nq, r, sm.mid, sm.scale,
                                       sm.rcut, f, nullptr, nullptr);
    }
    if constexpr (G < 0) LV::template moments<R>(M, f, dx * rinv, dy * rinv, dz * rinv);
    else LV::template moments_group<G, R>(M, f, dx * rinv, dy * rinv, dz * rinv);
  }
}

// One pair of the second sweep: g = dE_i/dr_ij from D, the force and virial
// terms and, with DTHETA, the dE/dc terms Q_k(r) S_mu.
template <class LV, class R, bool DTHETA, int G, int NQ>
__device__ __forceinline__ void adjoint_pair(const EfvArgs& a, const EfvShared<R, LV::NMU, DTHETA>& sm, int zi,
                                             int32_t j, int zj, R dx, R dy, R dz, R rinv, const R* f, const R* df,
                                             const R* q, const R* D, R& fx, R& fy, R& fz, R* w, AccView<R> acc,
                                             bool own_acc) {
  constexpr int NMU = LV::NMU;
  R gx, gy, gz, Smu[NMU];
  if constexpr (G < 0)
    LV::template pair_adjoint<R>(D, f, df, dx * rinv, dy * rinv, dz * rinv, rinv, gx, gy, gz, Smu);
  else
    LV::template pair_adjoint_group<G, R>(D, f, df, dx * rinv, dy * rinv, dz * rinv, rinv, gx, gy, gz, Smu);
  fx += gx; fy += gy; fz += gz;
  scatter_force(a, j, -gx, -gy, -gz);
  w[0] = fmadd(-gx, dx, w[0]);
  w[1] = fmadd(-gy, dy, w[1]);
  w[2] = fmadd(-gz, dz, w[2]);
  w[3] = fmadd(R(-0.5), fmadd(gx, dy, gy * dx), w[3]);
  w[4] = fmadd(R(-0.5), fmadd(gx, dz, gz * dx), w[4]);
  w[5] = fmadd(R(-0.5), fmadd(gy, dz, gz * dy), w[5]);
  if (DTHETA) {
    int mu_lo = 0, mu_hi = NMU;
    if constexpr (G >= 0) {
      mu_lo = LV::GROUP_MU_LO[G];
      mu_hi = LV::GROUP_MU_HI[G];
    }
    const int nq = NQ > 0 ? NQ : sm.nq;
    if (own_acc) {
      const int base = zj * NMU * nq;
#pragma unroll
      for (int mu = 0; mu < NMU; ++mu) {
        if (mu < mu_lo || mu >= mu_hi) continue;
#pragma unroll
        for (int kk = 0; kk < kMaxQ; ++kk)
          if (kk < nq) {
            R& d = acc[base + mu * nq + kk];
            d = fmadd(q[kk], Smu[mu], d);
          }
      }
    } else {
      R* dst = sm.dc + (zi * sm.S + zj) * NMU * nq;
#pragma unroll
      for (int mu = 0; mu < NMU; ++mu) {
        if (mu < mu_lo || mu >= mu_hi) continue;
#pragma unroll
        for (int kk = 0; kk < kMaxQ; ++kk)
          if (kk < nq) atomicAdd(dst + mu * nq + kk, q[kk] * Smu[mu]);
      }
    }
  }

}

// Second neighbour sweep for the components of group G (G < 0: all): per pair
// g_ij = dE_i/dr_ij from D (the group's share), F_i += g, F_j -= g,
// W -= sym(g (x) r_ij) and, with DTHETA, the group's radial functions'
// dE/dc terms Q_k(r) S_mu into acc (own_acc) or the shared accumulators.
// CLOSE64 as in moment_sweep; without it and without DTHETA the sweep is
// software-pipelined like moment_sweep (with DTHETA the next pair's Q_k
// values would stay live as well, which measured slower).
template <class LV, class R, bool DTHETA, int G, bool CLOSE64 = false, int NQ = 0>
__device__ __forceinline__ void adjoint_sweep(const EfvArgs& a, const EfvShared<R, LV::NMU, DTHETA>& sm,
                                              const PairGeom<R>& geom, const double* cell64, int zi, int64_t beg,
                                              int64_t end,
                                              const R* D, R& fx, R& fy, R& fz, R* w, AccView<R> acc,
                                              bool own_acc) {
  constexpr int NMU = LV::NMU;
  PairStream<R> ps;
  int32_t j, img;
  typename PairGeom<R>::Load lj;
  ps.start(a, geom, beg, end);
  if constexpr (!CLOSE64 && (kPipeAdjointDtheta || !DTHETA)) {
    if (beg >= end) return;
    PairTerms<LV, R, DTHETA, NQ> cur;
    ps.step(a, geom, j, img, lj);
    cur.eval(a, sm, geom, zi, j, img, lj);
    for (int64_t p = beg; p < end; ++p) {
      PairTerms<LV, R, DTHETA, NQ> nxt;
      ps.step(a, geom, j, img, lj);
      nxt.eval(a, sm, geom, zi, j, img, lj);
      adjoint_pair<LV, R, DTHETA, G, NQ>(a, sm, zi, cur.j, cur.zj, cur.dx, cur.dy, cur.dz, cur.rinv, cur.f, cur.df,
                                          cur.q, D, fx, fy, fz, w, acc, own_acc);
      cur = nxt;
    }
    return;
  }
  while (ps.next(a, geom, j, img, lj)) {
    const int zj = lj.species;
    R dx, dy, dz;
    geom.vec(a, lj, img, dx, dy, dz);
    const R r2 = fmadd(dz, dz, fmadd(dy, dy, dx * dx));
    R rinv = rsqrt_r(r2);
    const R r = r2 * rinv;
    R f[NMU], df[NMU], q[DTHETA ? kMaxQ : 1];
    if constexpr (std::is_same<R, float>::value) {
      if (r < sm.rmin)
        close_pair_fp64<NMU, true, DTHETA>(a, cell64, geom.ci, j, img, zi, zj, dx, dy, dz, rinv, f, df, q);
      else
        radial<R, NMU, true, DTHETA, NQ>(sm.c + (zi * sm.S + zj) * sm.cstride, sm.nq, r, sm.mid, sm.scale, sm.rcut,
                                         f, df, q);
    } else {
      radial<R, NMU, true, DTHETA, NQ>(sm.c + (zi * sm.S + zj) * sm.cstride, sm.nq, r, sm.mid, sm.scale, sm.rcut, f,
                                       df, q);
    }
    adjoint_pair<LV, R, DTHETA, G, NQ>(a, sm, zi, j, zj, dx, dy, dz, rinv, f, df, q, D, fx, fy, fz, w, acc, own_acc);
  }
}

// Everything one centre atom contributes: its site energy (also stored in
// e_atom), its force terms (scattered), its virial terms (w) and, with
// DTHETA, its basis values and radial-coefficient gradient (shared
// accumulators).  `cell` holds the rows of its configuration's cell in the
// working precision, `cell64` in FP64.
// Every lane of the warp calls this (the basis values are summed across the
// warp right after the contraction, which frees their registers for the
// second sweep): a lane without an atom passes active = false and a valid
// atom index i, runs no pairs, writes nothing and contributes zeros (every
// basis function vanishes at zero moments).
// Levels with component groups (the interpreted contractions of levels 18
// and 20: 201 and 295 components) sweep the neighbours once per group, so
// that a group's moments, then its adjoints, stay in registers; the full
// vectors meet the interpreter once per atom.
// The contraction of a single-group level: the generated whole-DAG form
// (DAG) or the default for R (per graph in FP32).
template <class LV, bool DAG, class R, bool WANT_B, class MV, class BV>
__device__ __forceinline__ R contract_atom(MV M, const typename ScalarOf<R>::T* __restrict__ xi, R* D, BV B) {
  if constexpr (DAG)
    return LV::template contract_dag<R, WANT_B, MV, BV>(M, xi, D, B);
  else
    return LV::template contract<R, WANT_B, MV, BV>(M, xi, D, B);
}

template <class LV, class R, bool DTHETA, bool PHASE_SYNC = false, int NQ = 0, bool DAG = false>
__device__ __forceinline__ void efv_atom(const EfvArgs& a, const EfvShared<R, LV::NMU, DTHETA>& sm, int64_t i,
                                         bool active, const R* cell, const double* cell64, double& e_i, R* w) {
  constexpr int NMU = LV::NMU;
  static_assert(LV::NGROUPS == 1 || LV::NGROUPS == 2, "one or two component groups");
  PairGeom<R> geom;
  geom.load_centre(a, i, cell);
  const int zi = species_at(a.z, i, a.n_species);
  const int64_t beg = active ? __ldg(a.offsets + i) : 0, end = active ? __ldg(a.offsets + i + 1) : 0;
  R M[LV::NCOMP];
#pragma unroll
  for (int c = 0; c < LV::NCOMP; ++c) M[c] = R(0);
  if constexpr (LV::NGROUPS == 1) {
    moment_sweep<LV, R, DTHETA, -1, false, NQ>(a, sm, geom, cell64, zi, beg, end, M);
  } else {
    {
      R Mg[LV::NCOMP];
#pragma unroll
      for (int c = 0; c < LV::NCOMP; ++c) Mg[c] = R(0);
      moment_sweep<LV, R, DTHETA, 0>(a, sm, geom, cell64, zi, beg, end, Mg);
      LV::template store_group<0, R>(Mg, M, 1);
    }
    {
      R Mg[LV::NCOMP];
#pragma unroll
      for (int c = 0; c < LV::NCOMP; ++c) Mg[c] = R(0);
      moment_sweep<LV, R, DTHETA, 1>(a, sm, geom, cell64, zi, beg, end, Mg);
      LV::template store_group<1, R>(Mg, M, 1);
    }
  }
  R D[LV::NCOMP];
  if constexpr (PHASE_SYNC) __syncthreads();
  R ei;
  if constexpr (DTHETA && LV::NGROUPS == 1) {
    // dE/dxi: each basis value is summed across the warp as soon as the
    // contraction forms it, so that none of them stays live through the
    // reverse pass
    ei = contract_atom<LV, DAG, R, true, const R*, WarpBasisSink<R>>(
        M, sm.xi, D, WarpBasisSink<R>{sm.dxi, (int)(threadIdx.x & 31), active});
  } else if constexpr (!DTHETA && LV::NGROUPS == 1) {
    ei = contract_atom<LV, DAG, R, true, const R*, DiscardBasisSink<R>>(
        M, sm.xi, D, DiscardBasisSink<R>{sm.discard + (threadIdx.x >> 5), (threadIdx.x & 31) == 0});
  } else {
    R Bv[DTHETA ? LV::NBASIS : 1];
    ei = LV::template contract<R, DTHETA>(M, sm.xi, D, Bv);
    if (DTHETA) {
      // warp sums of the basis values (dE/dxi), in R: the block accumulator is
      // in R, and FP64 shuffles of 100+ values would occupy the FP64 pipe
      // longer than the atoms' own work on the mixed path
      const int lane = threadIdx.x & 31;
#pragma unroll
      for (int t = 0; t < (DTHETA ? LV::NBASIS : 1); ++t) {
        const R v = warp_sum_r(active ? Bv[t] : R(0));
        if (lane == 0) atomicAdd(sm.dxi + t, v);
      }
    }
  }
  if constexpr (PHASE_SYNC) __syncthreads();
  e_i = active ? a.species_energy[zi] + (double)ei : 0.0;
  if (active) a.e_atom[i] = e_i;

  R fx = R(0), fy = R(0), fz = R(0);
  // dE/dc contributions of this atom's pairs, summed per neighbour species in
  // thread-private memory and added to the block's shared accumulators once
  // per atom (per-pair shared atomics collide heavily between lanes)
  // (packed [zj][mu][k] with the runtime n_q, so only S NMU n_q entries are touched)
  constexpr int kAccS = 4;
  R acc_local[(DTHETA && sizeof(R) == 8) ? kAccS * NMU * kMaxQ : 1];
  const AccView<R> acc = (sizeof(R) == 4) ? AccView<R>{sm.acc ? sm.acc + threadIdx.x : nullptr, (int)blockDim.x}
                                          : AccView<R>{acc_local, 1};
  const bool own_acc = DTHETA && sm.S <= kAccS && acc.p != nullptr;
  if (own_acc) {
    for (int t = 0; t < sm.S * NMU * sm.nq; ++t) acc[t] = R(0);
  }
  if constexpr (LV::NGROUPS == 1) {
    adjoint_sweep<LV, R, DTHETA, -1, false, NQ>(a, sm, geom, cell64, zi, beg, end, D, fx, fy, fz, w, acc, own_acc);
  } else {
    {
      R Dg[LV::NCOMP];
      LV::template load_group<0, R>(D, 1, Dg);
      adjoint_sweep<LV, R, DTHETA, 0>(a, sm, geom, cell64, zi, beg, end, Dg, fx, fy, fz, w, acc, own_acc);
    }
    {
      R Dg[LV::NCOMP];
      LV::template load_group<1, R>(D, 1, Dg);
      adjoint_sweep<LV, R, DTHETA, 1>(a, sm, geom, cell64, zi, beg, end, Dg, fx, fy, fz, w, acc, own_acc);
    }
  }
  if (!active) return;
  if (own_acc) {
    for (int zj = 0; zj < sm.S; ++zj) {
      R* dst = sm.dc + (zi * sm.S + zj) * NMU * sm.nq;
      for (int t = 0; t < NMU * sm.nq; ++t) atomicAdd(dst + t, acc[zj * NMU * sm.nq + t]);
    }
  }
  scatter_force(a, i, fx, fy, fz);
  if (!isfinite(e_i) || !isfinite((double)fx) || !isfinite((double)fy) || !isfinite((double)fz))
    flag_status(a.status, MTP_ERR_NONFINITE);
  if (DTHETA) atomicAdd(sm.cnt + zi, 1);
}

// Block-wide FP64 reduction of the block's energy, virial and gradient into
// e_out[0], w_out[0..6) and theta_out (layout [ s | c[mu][k][zi][zj] | xi ]).
// Must be reached by every thread of the block.
constexpr unsigned kFlushEW = 1, kFlushDc = 2, kFlushDxi = 4, kFlushAll = 7;

template <class LV, class R, bool DTHETA>
__device__ __forceinline__ void efv_block_flush(const EfvShared<R, LV::NMU, DTHETA>& sm, double e_i, const R* w,
                                                double* e_out, double* w_out, double* theta_out,
                                                unsigned parts = kFlushAll) {
  constexpr int NMU = LV::NMU;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  double vals[7] = {e_i, (double)w[0], (double)w[1], (double)w[2], (double)w[3], (double)w[4], (double)w[5]};
#pragma unroll
  for (int t = 0; t < 7; ++t) vals[t] = warp_sum(vals[t]);
  if (lane == 0) {
#pragma unroll
    for (int t = 0; t < 7; ++t) sm.red[warp * 8 + t] = vals[t];
  }
  __syncthreads();
  if ((parts & kFlushEW) && threadIdx.x < 7) {
    double acc = 0.0;
    for (int wi = 0; wi < nwarps; ++wi) acc += sm.red[wi * 8 + threadIdx.x];
    if (threadIdx.x == 0) atomicAdd(e_out, acc);
    else atomicAdd(w_out + threadIdx.x - 1, acc);
  }
  if (DTHETA) {
    const int S = sm.S, SS = sm.SS, nq = sm.nq;
    if (parts & kFlushDxi)
      for (int t = threadIdx.x; t < S; t += blockDim.x) atomicAdd(theta_out + t, (double)sm.cnt[t]);
    if (parts & kFlushDc) {
      for (int t = threadIdx.x; t < SS * NMU * nq; t += blockDim.x) {
        const int p = t / (NMU * nq);
        const int mk = t % (NMU * nq);
        atomicAdd(theta_out + S + (int64_t)mk * SS + p, (double)sm.dc[t]);
      }
    }
    if (parts & kFlushDxi)
      for (int t = threadIdx.x; t < sm.m; t += blockDim.x)
        atomicAdd(theta_out + S + (int64_t)NMU * nq * SS + t, (double)sm.dxi[t]);
  }
}

template <class LV, class R, bool DTHETA, int NQ = 0>
__global__ void __launch_bounds__(kEfvFusedThreads) efv_kernel(const EfvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EfvShared<R, LV::NMU, DTHETA> sm;
  sm.setup(a, smem_raw);
  sm.zero_gradients();
  __syncthreads();
  const int64_t i = a.atom_begin + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e_i = 0.0;
  R w[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  const bool active = i < a.atom_end;
  // the block's warps meet between the neighbour sweeps and the contraction,
  // so that they run the same code at the same time (instruction cache); a
  // warp without atoms runs the phases on zero pairs
  efv_atom<LV, R, DTHETA, true, NQ>(a, sm, active ? i : a.atom_begin, active, cell_of<R>(a), a.cell, e_i, w);
  efv_block_flush<LV, R, DTHETA>(sm, e_i, w, a.e_total, a.virial, a.dtheta);
}

// Levels with component groups (interpreted contraction) and a scratch
// buffer a.mbuf run as three kernels: the interpreter's per-thread value
// arrays stream through local memory, which needs many resident warps, while
// the neighbour sweeps need many registers per thread.  a.mbuf holds the
// moment vectors of the atom range and then their adjoints, component-major:
// [2][c][atom - atom_begin].
template <class LV, class R>
__global__ void __launch_bounds__(kEfvThreads) split_moments_kernel(const EfvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EfvShared<R, LV::NMU, false> sm;
  sm.setup(a, smem_raw);
  __syncthreads();
  const int64_t n = a.atom_end - a.atom_begin;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = t < n;
  if (!__any_sync(0xffffffffu, active)) return;
  const int64_t i = a.atom_begin + (active ? t : 0);
  PairGeom<R> geom;
  geom.load_centre(a, i, cell_of<R>(a));
  const int zi = species_at(a.z, i, a.n_species);
  const int64_t beg = active ? __ldg(a.offsets + i) : 0, end = active ? __ldg(a.offsets + i + 1) : 0;
  R* buf = static_cast<R*>(a.mbuf) + (active ? t : 0);
  {
    R Mg[LV::NCOMP];
#pragma unroll
    for (int c = 0; c < LV::NCOMP; ++c) Mg[c] = R(0);
    moment_sweep<LV, R, false, 0, true>(a, sm, geom, a.cell, zi, beg, end, Mg);
    if (active) LV::template store_group<0, R>(Mg, buf, n);
  }
  {
    R Mg[LV::NCOMP];
#pragma unroll
    for (int c = 0; c < LV::NCOMP; ++c) Mg[c] = R(0);
    moment_sweep<LV, R, false, 1, true>(a, sm, geom, a.cell, zi, beg, end, Mg);
    if (active) LV::template store_group<1, R>(Mg, buf, n);
  }
}

template <class LV, class R, bool DTHETA>
__global__ void __launch_bounds__(kEfvThreads) split_contract_kernel(const EfvArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EfvShared<R, LV::NMU, DTHETA> sm;
  sm.setup(a, smem_raw);
  sm.zero_gradients();
  __syncthreads();
  const int64_t n = a.atom_end - a.atom_begin;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = t < n;
  double e_i = 0.0;
  const R w[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  if (__any_sync(0xffffffffu, active)) {
    const R* __restrict__ mrow = static_cast<const R*>(a.mbuf) + (active ? t : 0);
    R* __restrict__ drow = static_cast<R*>(a.mbuf) + (size_t)LV::NCOMP * n + (active ? t : 0);
    R V[LV::NVALUES], A[LV::NVALUES];
    R Bv[DTHETA ? LV::NBASIS : 1];
    for (int c = 0; c < LV::NCOMP; ++c) V[c] = active ? mrow[c * n] : R(0);
    const R ei = LV::template contract_values<R, DTHETA>(V, A, sm.xi, Bv);
    if (active)
      for (int c = 0; c < LV::NCOMP; ++c) drow[c * n] = A[c];
    if (DTHETA) {
      const int lane = threadIdx.x & 31;
#pragma unroll
      for (int u = 0; u < (DTHETA ? LV::NBASIS : 1); ++u) {
        const R v = warp_sum_r(active ? Bv[u] : R(0));
        if (lane == 0) atomicAdd(sm.dxi + u, v);
      }
    }
    if (active) {
      const int64_t i = a.atom_begin + t;
      const int zi = species_at(a.z, i, a.n_species);
      e_i = a.species_energy[zi] + (double)ei;
      a.e_atom[i] = e_i;
      if (!isfinite(e_i)) flag_status(a.status, MTP_ERR_NONFINITE);
      if (DTHETA) atomicAdd(sm.cnt + zi, 1);
    }
  }
  efv_block_flush<LV, R, DTHETA>(sm, e_i, w, a.e_total, a.virial, a.dtheta, kFlushEW | kFlushDxi);
}

template <class LV, class R, bool DTHETA>
__global__ void __launch_bounds__(kEfvThreads) split_adjoint_kernel(const EfvArgs a) {
  constexpr int NMU = LV::NMU;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  EfvShared<R, NMU, DTHETA> sm;
  sm.setup(a, smem_raw);
  sm.zero_gradients();
  __syncthreads();
  const int64_t n = a.atom_end - a.atom_begin;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = t < n;
  R w[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
  if (__any_sync(0xffffffffu, active)) {
    const int64_t i = a.atom_begin + (active ? t : 0);
    PairGeom<R> geom;
    geom.load_centre(a, i, cell_of<R>(a));
    const int zi = species_at(a.z, i, a.n_species);
    const int64_t beg = active ? __ldg(a.offsets + i) : 0, end = active ? __ldg(a.offsets + i + 1) : 0;
    const R* buf = static_cast<const R*>(a.mbuf) + (size_t)LV::NCOMP * n + (active ? t : 0);
    R fx = R(0), fy = R(0), fz = R(0);
    constexpr int kAccS = 4;
    R acc_local[(DTHETA && sizeof(R) == 8) ? kAccS * NMU * kMaxQ : 1];
    const AccView<R> acc = (sizeof(R) == 4) ? AccView<R>{sm.acc ? sm.acc + threadIdx.x : nullptr, (int)blockDim.x}
                                            : AccView<R>{acc_local, 1};
    const bool own_acc = DTHETA && sm.S <= kAccS && acc.p != nullptr;
    if (own_acc) {
      for (int u = 0; u < sm.S * NMU * sm.nq; ++u) acc[u] = R(0);
    }
    {
      R Dg[LV::NCOMP];
      LV::template load_group<0, R>(buf, n, Dg);
      adjoint_sweep<LV, R, DTHETA, 0, true>(a, sm, geom, a.cell, zi, beg, end, Dg, fx, fy, fz, w, acc, own_acc);
    }
    {
      R Dg[LV::NCOMP];
      LV::template load_group<1, R>(buf, n, Dg);
      adjoint_sweep<LV, R, DTHETA, 1, true>(a, sm, geom, a.cell, zi, beg, end, Dg, fx, fy, fz, w, acc, own_acc);
    }
    if (active) {
      if (own_acc) {
        for (int zj = 0; zj < sm.S; ++zj) {
          R* dst = sm.dc + (zi * sm.S + zj) * NMU * sm.nq;
          for (int u = 0; u < NMU * sm.nq; ++u) atomicAdd(dst + u, acc[zj * NMU * sm.nq + u]);
        }
      }
      scatter_force(a, i, fx, fy, fz);
      if (!isfinite((double)fx) || !isfinite((double)fy) || !isfinite((double)fz))
        flag_status(a.status, MTP_ERR_NONFINITE);
    }
  }
  efv_block_flush<LV, R, DTHETA>(sm, 0.0, w, a.e_total, a.virial, a.dtheta, kFlushEW | kFlushDc);
}

constexpr int kFixedQ = 8;

template <class K>
int set_smem(K kern, size_t bytes) {
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
      set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
      return MTP_ERR_CUDA;
    }
  }
  return MTP_OK;
}

template <class LV, class R, bool DTHETA>
int efv_split_launch(const EfvArgs& a, cudaStream_t stream) {
  const int SS = a.n_species * a.n_species;
  const int64_t n = a.atom_end - a.atom_begin;
  if (n <= 0) return MTP_OK;
  const unsigned grid = (unsigned)((n + kEfvThreads - 1) / kEfvThreads);
  const size_t b0 = efv_smem_bytes<R, LV::NMU, false>(SS, a.n_q, a.m);
  const size_t b1 = ((efv_smem_bytes<R, LV::NMU, DTHETA>(SS, a.n_q, a.m) + 15) & ~size_t(15)) +
                    efv_acc_bytes<R, LV::NMU, DTHETA>(a.n_species, a.n_q, kEfvThreads);
  int rc;
  // the contraction kernel has no dE/dc accumulators: without them its blocks
  // stay small, so that many warps hide the interpreter's local-memory traffic
  const size_t bc = efv_smem_bytes<R, LV::NMU, DTHETA>(SS, a.n_q, a.m);
  if ((rc = set_smem(split_moments_kernel<LV, R>, b0)) != MTP_OK) return rc;
  if ((rc = set_smem(split_contract_kernel<LV, R, DTHETA>, bc)) != MTP_OK) return rc;
  if ((rc = set_smem(split_adjoint_kernel<LV, R, DTHETA>, b1)) != MTP_OK) return rc;
  split_moments_kernel<LV, R><<<grid, kEfvThreads, b0, stream>>>(a);
  split_contract_kernel<LV, R, DTHETA><<<grid, kEfvThreads, bc, stream>>>(a);
  split_adjoint_kernel<LV, R, DTHETA><<<grid, kEfvThreads, b1, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("efv split kernels (level %d): %s", LV::LEVEL, cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  return MTP_OK;
}

template <class LV, class R, bool DTHETA>
int efv_launch_typed(const EfvArgs& a, cudaStream_t stream) {
  if constexpr (LV::NGROUPS > 1) {
    if (a.mbuf) return efv_split_launch<LV, R, DTHETA>(a, stream);
  }
  const int SS = a.n_species * a.n_species;
  const size_t bytes = ((efv_smem_bytes<R, LV::NMU, DTHETA>(SS, a.n_q, a.m) + 15) & ~size_t(15)) +
                       efv_acc_bytes<R, LV::NMU, DTHETA>(a.n_species, a.n_q, kEfvFusedThreads);
  auto kern = efv_kernel<LV, R, DTHETA>;
  // the mixed path of the single-group levels with the common radial basis
  // size n_q = 8 runs with n_q fixed at compile time
  if constexpr (std::is_same<R, float>::value && LV::NGROUPS == 1) {
    if (a.n_q == kFixedQ) kern = efv_kernel<LV, R, DTHETA, kFixedQ>;
  }
  if (bytes > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) {
      set_error("cudaFuncSetAttribute: %s", cudaGetErrorString(e));
      return MTP_ERR_CUDA;
    }
  }
  const int64_t n = a.atom_end - a.atom_begin;
  if (n <= 0) return MTP_OK;
  const unsigned grid = (unsigned)((n + kEfvFusedThreads - 1) / kEfvFusedThreads);
  kern<<<grid, kEfvFusedThreads, bytes, stream>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("efv kernel launch (level %d): %s", LV::LEVEL, cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  return MTP_OK;
}

template <class LV>
int efv_launch(const EfvArgs& a, int precision, bool want_dtheta, cudaStream_t stream) {
  if (precision == MTP_MIXED) {
    return want_dtheta ? efv_launch_typed<LV, float, true>(a, stream) : efv_launch_typed<LV, float, false>(a, stream);
  }
  return want_dtheta ? efv_launch_typed<LV, double, true>(a, stream) : efv_launch_typed<LV, double, false>(a, stream);
}

}  // namespace mtp
