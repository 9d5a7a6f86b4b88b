// Cell-list construction of the full periodic neighbour list.
//
// Atoms are binned in fractional coordinates.  Along axis k the cell has
// plane spacing h_k = 1 / |column k of H^-1|; a pair closer than R_cut
// differs by at most R_cut / h_k in fractional coordinate k, so with nb_k bins
// it lies at most R_k = floor(R_cut nb_k / h_k) + 1 bins away.  Periodic axes
// are searched over unwrapped bin offsets t in [b - R_k, b + R_k]; bin
// t mod nb_k together with the wrap q = floor(t / nb_k) gives each image of
// each candidate exactly once (several images for cells thinner than R_cut).
// The in/out decision is the exact FP64 expression of the list definition:
// d = (x_j + s) - x_i, s = (n1 a + n2 b) + n3 c, r^2 = (dx dx + dy dy) + dz dz,
// each operation separately rounded (explicit _rn intrinsics, no contraction),
// wherever an FP32 estimate with a proven error bound cannot decide it.
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "mtp_internal.cuh"

namespace mtp {

struct NbrGeom {
  double cell[9];
  float cellf[9];
  float rc2_hi;       // prefilter bound: rc^2 plus the worst FP32 rounding of r^2
  float rc2_lo;       // below it (and above rz2) a candidate is inside whatever the rounding
  float rz2;          // FP32 r^2 above which the exact r^2 is certainly positive
  double hinv[9];
  double origin[3];   // fractional origin of the bin grid (0 on periodic axes)
  double width[3];    // fractional width of one bin
  int nb[3];
  int reach[3];
  int pbc[3];
  double rc2;
};

// Order-preserving map of doubles onto unsigned integers (for atomic min/max).
__device__ __forceinline__ unsigned long long ordered_bits(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
static double unordered_bits(unsigned long long b) {
  const unsigned long long r = (b >> 63) ? (b & 0x7fffffffffffffffull) : ~b;
  double v;
  memcpy(&v, &r, sizeof(v));
  return v;
}

__global__ void wrap_kernel(const double* __restrict__ x, int64_t n, NbrGeom g, double* __restrict__ sw,
                            int* __restrict__ wrapcnt, unsigned long long* __restrict__ extent,
                            float4* __restrict__ xw, int* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long lo[3] = {~0ull, ~0ull, ~0ull}, hi[3] = {0ull, 0ull, 0ull};
  if (i < n) {
    const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
    if (!isfinite(px) || !isfinite(py) || !isfinite(pz)) atomicCAS(status, 0, MTP_ERR_NONFINITE);
    double sv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      double s = px * g.hinv[0 + k] + py * g.hinv[3 + k] + pz * g.hinv[6 + k];
      int w = 0;
      if (g.pbc[k]) {
        const double f = floor(s);
        w = (int)f;
        s -= f;
        if (s >= 1.0) { s -= 1.0; w += 1; }
        if (s < 0.0) s = 0.0;
      }
      sw[3 * i + k] = s;
      sv[k] = s;
      wrapcnt[3 * i + k] = w;
      lo[k] = hi[k] = ordered_bits(s);
    }
    // wrapped Cartesian position in FP32, for the distance prefilter
    xw[i] = make_float4((float)(sv[0] * g.cell[0] + sv[1] * g.cell[3] + sv[2] * g.cell[6]),
                        (float)(sv[0] * g.cell[1] + sv[1] * g.cell[4] + sv[2] * g.cell[7]),
                        (float)(sv[0] * g.cell[2] + sv[1] * g.cell[5] + sv[2] * g.cell[8]), 0.f);
  }
  // min/max of the fractional coordinates (used to lay bins over open axes)
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    for (int o = 16; o > 0; o >>= 1) {
      lo[k] = min(lo[k], __shfl_down_sync(0xffffffffu, lo[k], o));
      hi[k] = max(hi[k], __shfl_down_sync(0xffffffffu, hi[k], o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(extent + 2 * k, lo[k]);
      atomicMax(extent + 2 * k + 1, hi[k]);
    }
  }
}

__device__ __forceinline__ int bin_coord(double s, const NbrGeom& g, int k) {
  int b = (int)floor((s - g.origin[k]) / g.width[k]);
  return min(max(b, 0), g.nb[k] - 1);
}

__global__ void bin_count_kernel(const double* __restrict__ sw, int64_t n, NbrGeom g, int* __restrict__ bin_of,
                                 int* __restrict__ bin_count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b0 = bin_coord(sw[3 * i], g, 0), b1 = bin_coord(sw[3 * i + 1], g, 1), b2 = bin_coord(sw[3 * i + 2], g, 2);
  const int b = (b0 * g.nb[1] + b1) * g.nb[2] + b2;
  bin_of[i] = b;
  atomicAdd(bin_count + b, 1);
}

// Atoms in bin order, with their FP32 wrapped positions beside them (the
// candidate loops read both by slot, without a dependent gather).
__global__ void bin_fill_kernel(const int* __restrict__ bin_of, int64_t n, const int* __restrict__ bin_start,
                                int* __restrict__ cursor, const float4* __restrict__ xw, int* __restrict__ bin_atoms,
                                float4* __restrict__ bin_xw) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int b = bin_of[i];
  const int slot = bin_start[b] + atomicAdd(cursor + b, 1);
  bin_atoms[slot] = (int)i;
  bin_xw[slot] = xw[i];
}

__device__ __forceinline__ int floor_div(int t, int m) { return t >= 0 ? t / m : -((-t + m - 1) / m); }

// Visits every (j, n) within the cutoff of atom i; FILL writes them.  Along
// the last axis the searched bins of one (t0, t1) row are consecutive bin
// indices between wraps, so their atoms are one range of slots: the loop runs
// over such ranges (one per wrap q2) instead of bin by bin.
// A candidate passes to the exact FP64 test only if its FP32 squared distance
// (wrapped positions plus the bin wrap) is below rc2_hi, which exceeds R_cut^2
// by more than the FP32 rounding can move it, so no pair within the cutoff is
// dropped and the decision itself stays the exact FP64 expression.
template <bool FILL>
__global__ void pair_kernel(const double* __restrict__ x, const double* __restrict__ sw, const int* __restrict__ wrapcnt,
                            const float4* __restrict__ xw, int64_t n, NbrGeom g, const int* __restrict__ bin_start,
                            const int* __restrict__ bin_count, const int* __restrict__ bin_atoms,
                            const float4* __restrict__ bin_xw,
                            int* __restrict__ counts, const int64_t* __restrict__ offsets, int32_t* __restrict__ out_j,
                            int32_t* __restrict__ out_img, int* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
  const float4 pw = xw[i];
  const int wi[3] = {wrapcnt[3 * i], wrapcnt[3 * i + 1], wrapcnt[3 * i + 2]};
  const int bi[3] = {bin_coord(sw[3 * i], g, 0), bin_coord(sw[3 * i + 1], g, 1), bin_coord(sw[3 * i + 2], g, 2)};
  int found = 0;
  int64_t base = FILL ? offsets[i] : 0;
  for (int t0 = bi[0] - g.reach[0]; t0 <= bi[0] + g.reach[0]; ++t0) {
    int q0 = 0, c0 = t0;
    if (g.pbc[0]) { q0 = floor_div(t0, g.nb[0]); c0 = t0 - q0 * g.nb[0]; }
    else if (t0 < 0 || t0 >= g.nb[0]) continue;
    for (int t1 = bi[1] - g.reach[1]; t1 <= bi[1] + g.reach[1]; ++t1) {
      int q1 = 0, c1 = t1;
      if (g.pbc[1]) { q1 = floor_div(t1, g.nb[1]); c1 = t1 - q1 * g.nb[1]; }
      else if (t1 < 0 || t1 >= g.nb[1]) continue;
      int t2 = bi[2] - g.reach[2];
      int t2_hi = bi[2] + g.reach[2];
      if (!g.pbc[2]) {
        t2 = max(t2, 0);
        t2_hi = min(t2_hi, g.nb[2] - 1);
      }
      const int row = (c0 * g.nb[1] + c1) * g.nb[2];
      while (t2 <= t2_hi) {
        int q2 = 0, c2 = t2;
        if (g.pbc[2]) { q2 = floor_div(t2, g.nb[2]); c2 = t2 - q2 * g.nb[2]; }
        // bins c2 .. c2_end of this row share the wrap q2
        const int c2_end = min(g.nb[2] - 1, c2 + (t2_hi - t2));
        const int s_beg = bin_start[row + c2];
        const int s_end = bin_start[row + c2_end] + bin_count[row + c2_end];
        t2 += c2_end - c2 + 1;
        const float fq0 = (float)q0, fq1 = (float)q1, fq2 = (float)q2;
        const float shx = fq0 * g.cellf[0] + fq1 * g.cellf[3] + fq2 * g.cellf[6] - pw.x;
        const float shy = fq0 * g.cellf[1] + fq1 * g.cellf[4] + fq2 * g.cellf[7] - pw.y;
        const float shz = fq0 * g.cellf[2] + fq1 * g.cellf[5] + fq2 * g.cellf[8] - pw.z;
        for (int u = s_beg; u < s_end; ++u) {
          const float4 qw = bin_xw[u];
          const float fx = qw.x + shx, fy = qw.y + shy, fz = qw.z + shz;
          const float r2f = fx * fx + fy * fy + fz * fz;
          if (r2f >= g.rc2_hi) continue;
          const int j = bin_atoms[u];
          // image of j relative to the unwrapped positions
          const int n1 = q0 + wi[0] - wrapcnt[3 * j];
          const int n2 = q1 + wi[1] - wrapcnt[3 * j + 1];
          const int n3 = q2 + wi[2] - wrapcnt[3 * j + 2];
          bool inside = r2f < g.rc2_lo && r2f > g.rz2;   // decided by the FP32 bound
          if (!inside) {
            const double sx = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, g.cell[0]), __dmul_rn((double)n2, g.cell[3])),
                                        __dmul_rn((double)n3, g.cell[6]));
            const double sy = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, g.cell[1]), __dmul_rn((double)n2, g.cell[4])),
                                        __dmul_rn((double)n3, g.cell[7]));
            const double sz = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, g.cell[2]), __dmul_rn((double)n2, g.cell[5])),
                                        __dmul_rn((double)n3, g.cell[8]));
            const double dx = __dsub_rn(__dadd_rn(x[3 * j], sx), xi);
            const double dy = __dsub_rn(__dadd_rn(x[3 * j + 1], sy), yi);
            const double dz = __dsub_rn(__dadd_rn(x[3 * j + 2], sz), zi);
            const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
            inside = r2 < g.rc2 && r2 > 0.0;
          }
          if (inside) {
            if (n1 < -511 || n1 > 511 || n2 < -511 || n2 > 511 || n3 < -511 || n3 > 511) {
              atomicCAS(status, 0, MTP_ERR_NEIGHBOR_OVERFLOW);
              continue;
            }
            if (FILL) {
              out_j[base + found] = j;
              out_img[base + found] = pack_image(n1, n2, n3);
            }
            ++found;
          }
        }
      }
    }
  }
  if (!FILL) counts[i] = found;
  // FILL leaves the segment in search order; sort_rows_kernel orders it
}

// Canonical order of a list entry, (j, n1, n2, n3) lexicographic, as an
// unsigned key; every field is non-negative once biased.
__device__ __forceinline__ unsigned long long row_key(int32_t j, int32_t img) {
  const uint32_t u = (uint32_t)img;
  return ((unsigned long long)(uint32_t)j << 30) | ((unsigned long long)(u & 1023u) << 20) |
         ((unsigned long long)((u >> 10) & 1023u) << 10) | (unsigned long long)((u >> 20) & 1023u);
}
__device__ __forceinline__ void key_entry(unsigned long long key, int32_t& j, int32_t& img) {
  j = (int32_t)(key >> 30);
  const uint32_t n1 = (uint32_t)(key >> 20) & 1023u, n2 = (uint32_t)(key >> 10) & 1023u, n3 = (uint32_t)key & 1023u;
  img = (int32_t)(n1 | (n2 << 10) | (n3 << 20));
}

// Bitonic sort of one segment of at most 32 R entries held by a warp, entry
// e = 32 r + lane in register r of lane `lane` (padding: the largest key).
template <int R>
__device__ __forceinline__ void warp_sort_segment(int32_t* __restrict__ out_j, int32_t* __restrict__ out_img,
                                                  int64_t base, int cnt, int lane) {
  constexpr int E = 32 * R;
  unsigned long long v[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = 32 * r + lane;
    v[r] = e < cnt ? row_key(out_j[base + e], out_img[base + e]) : ~0ull;
  }
#pragma unroll
  for (int k = 2; k <= E; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j > 0; j >>= 1) {
      if (j >= 32) {
        const int rj = j >> 5;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if (r & rj) continue;
          const int e = 32 * r + lane;
          const unsigned long long a = v[r], b = v[r | rj];
          const bool asc = (e & k) == 0;
          v[r] = asc ? (a < b ? a : b) : (a < b ? b : a);
          v[r | rj] = asc ? (a < b ? b : a) : (a < b ? a : b);
        }
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int e = 32 * r + lane;
          const unsigned long long p = __shfl_xor_sync(0xffffffffu, v[r], j);
          const bool keep_min = ((e & k) == 0) == ((lane & j) == 0);
          v[r] = keep_min ? (v[r] < p ? v[r] : p) : (v[r] < p ? p : v[r]);
        }
      }
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int e = 32 * r + lane;
    if (e < cnt) {
      int32_t jj, im;
      key_entry(v[r], jj, im);
      out_j[base + e] = jj;
      out_img[base + e] = im;
    }
  }
}

// One warp per atom: its list segment into canonical order (j, n1, n2, n3).
// Segments of up to 256 entries are sorted in registers; longer ones (never
// at the densities here) by insertion, on lane 0.
__global__ void sort_rows_kernel(int64_t n, const int64_t* __restrict__ offsets, int32_t* __restrict__ out_j,
                                 int32_t* __restrict__ out_img) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;   // warp-uniform
  const int64_t base = offsets[i];
  const int64_t cnt64 = offsets[i + 1] - base;
  if (cnt64 <= 1) return;
  const int cnt = (int)cnt64;
  if (cnt64 <= 32) warp_sort_segment<1>(out_j, out_img, base, cnt, lane);
  else if (cnt64 <= 64) warp_sort_segment<2>(out_j, out_img, base, cnt, lane);
  else if (cnt64 <= 128) warp_sort_segment<4>(out_j, out_img, base, cnt, lane);
  else if (cnt64 <= 256) warp_sort_segment<8>(out_j, out_img, base, cnt, lane);
  else if (lane == 0) {
    for (int64_t p = 1; p < cnt64; ++p) {
      const int32_t jj = out_j[base + p], im = out_img[base + p];
      const unsigned long long kp = row_key(jj, im);
      int64_t q = p - 1;
      while (q >= 0 && row_key(out_j[base + q], out_img[base + q]) > kp) {
        out_j[base + q + 1] = out_j[base + q];
        out_img[base + q + 1] = out_img[base + q];
        --q;
      }
      out_j[base + q + 1] = jj;
      out_img[base + q + 1] = im;
    }
  }
}

__global__ void widen_counts(const int* __restrict__ c, int64_t n, int64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = c[i];
  if (i == n) out[n] = 0;
}

static void invert3(const double* m, double* inv) {
  const double a = m[0], b = m[1], c = m[2], d = m[3], e = m[4], f = m[5], gg = m[6], h = m[7], k = m[8];
  const double det = a * (e * k - f * h) - b * (d * k - f * gg) + c * (d * h - e * gg);
  inv[0] = (e * k - f * h) / det;
  inv[1] = (c * h - b * k) / det;
  inv[2] = (b * f - c * e) / det;
  inv[3] = (f * gg - d * k) / det;
  inv[4] = (a * k - c * gg) / det;
  inv[5] = (c * d - a * f) / det;
  inv[6] = (d * h - e * gg) / det;
  inv[7] = (b * gg - a * h) / det;
  inv[8] = (a * e - b * d) / det;
}

int build_neighbors(mtp_nlist* nl, const double* x, int64_t n, const double* cell, const int32_t* pbc, double r_cut,
                    cudaStream_t stream) {
  NbrGeom g;
  for (int k = 0; k < 9; ++k) g.cell[k] = cell[k];
  const double det = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) - cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) +
                     cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) {
    set_error("mtp_build_neighbors: cell is singular or not finite (det = %g)", det);
    return MTP_ERR_ARG;
  }
  invert3(cell, g.hinv);
  double h[3];
  for (int k = 0; k < 3; ++k) {
    // s = x H^-1 (x a row vector): column k of H^-1 maps x to s_k
    const double c0 = g.hinv[0 + k], c1 = g.hinv[3 + k], c2 = g.hinv[6 + k];
    h[k] = 1.0 / std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    g.pbc[k] = pbc[k] ? 1 : 0;
  }
  g.rc2 = r_cut * r_cut;
  for (int k = 0; k < 9; ++k) g.cellf[k] = (float)cell[k];

  for (int k = 0; k < 9; ++k) nl->cell[k] = cell[k];
  for (int k = 0; k < 3; ++k) nl->pbc[k] = g.pbc[k];
  nl->r_cut = r_cut;
  nl->n_atoms = n;

  const int T = 256;
  const unsigned blocks = (unsigned)((n + T - 1) / T);
  int rc;
  const int64_t n1 = std::max<int64_t>(n, 1);
  if ((rc = nl->wrapped.ensure(sizeof(float4) * n1 + sizeof(double) * 3 * n1 + sizeof(int) * 3 * n1 + 64)) != MTP_OK)
    return rc;
  float4* xw = nl->wrapped.as<float4>();
  double* sw = reinterpret_cast<double*>(xw + n1);
  int* wrapcnt = reinterpret_cast<int*>(sw + 3 * n1);
  unsigned long long* extent = reinterpret_cast<unsigned long long*>(
      (reinterpret_cast<uintptr_t>(wrapcnt + 3 * std::max<int64_t>(n, 1)) + 15) & ~uintptr_t(15));
  if ((rc = nl->status.ensure(sizeof(int) * 4)) != MTP_OK) return rc;
  int* status = nl->status.as<int>();
  MTP_TRY_CUDA(cudaMemsetAsync(status, 0, sizeof(int), stream));
  const unsigned long long ext_init[6] = {~0ull, 0ull, ~0ull, 0ull, ~0ull, 0ull};
  MTP_TRY_CUDA(cudaMemcpyAsync(extent, ext_init, sizeof(ext_init), cudaMemcpyHostToDevice, stream));
  if (n > 0) wrap_kernel<<<blocks, T, 0, stream>>>(x, n, g, sw, wrapcnt, extent, xw, status);
  MTP_TRY_CUDA(cudaGetLastError());
  unsigned long long ext_bits[6];
  int wrap_status = 0;
  MTP_TRY_CUDA(cudaMemcpyAsync(ext_bits, extent, sizeof(ext_bits), cudaMemcpyDeviceToHost, stream));
  MTP_TRY_CUDA(cudaMemcpyAsync(&wrap_status, status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  MTP_TRY_CUDA(cudaStreamSynchronize(stream));
  if (wrap_status == MTP_ERR_NONFINITE) {
    set_error("mtp_build_neighbors: non-finite position");
    return MTP_ERR_NONFINITE;
  }
  int64_t nbins = 1;
  for (int k = 0; k < 3; ++k) {
    if (g.pbc[k]) {
      // bins of about half the cutoff: a reach of 2 bins searches 5^3 bins of
      // width R_cut/2 (15.6 R_cut^3) instead of 3^3 bins of width R_cut (27 R_cut^3)
      g.nb[k] = std::max(1, (int)std::floor(2.0 * h[k] / r_cut));
      g.nb[k] = (int)std::min<int64_t>(g.nb[k], 1024);
      g.origin[k] = 0.0;
      g.width[k] = 1.0 / g.nb[k];
    } else {
      double lo = 0.0, hi = 0.0;
      if (n > 0) {
        lo = unordered_bits(ext_bits[2 * k]);
        hi = unordered_bits(ext_bits[2 * k + 1]);
      }
      const double w = r_cut / h[k];   // fractional width of one cutoff
      g.origin[k] = lo;
      g.width[k] = w;
      int64_t nbk = (int64_t)std::floor((hi - lo) / w) + 1;
      g.nb[k] = (int)std::max<int64_t>(1, std::min<int64_t>(nbk, 1024));
      if (nbk > 1024) g.width[k] = (hi - lo) / 1023.999;
    }
    g.reach[k] = (int)std::floor(r_cut * g.nb[k] / h[k] * (g.pbc[k] ? 1.0 : 0.0)) + 1;
    if (!g.pbc[k]) g.reach[k] = std::max(1, (int)std::ceil(r_cut / (g.width[k] * h[k])));
    nbins *= g.nb[k];
  }
  {
    // FP32 prefilter margin.  Along cell vector k the wrapped fractional
    // coordinate lies in [lo_k, hi_k] ([0, 1) on periodic axes) and the bin
    // wrap q_k is at most (reach_k + nb_k) / nb_k + 1 in magnitude, so every
    // position, shift and pair vector is below ext = sum_k |h_k| (span_k + q_k)
    // in size and each of the few FP32 roundings on the way is below
    // ext 2^-24 per component.
    double ext = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double len = std::sqrt(cell[3 * k] * cell[3 * k] + cell[3 * k + 1] * cell[3 * k + 1] +
                                   cell[3 * k + 2] * cell[3 * k + 2]);
      double span = 1.0;
      if (!g.pbc[k] && n > 0)
        span = std::max(std::fabs(unordered_bits(ext_bits[2 * k])), std::fabs(unordered_bits(ext_bits[2 * k + 1])));
      const double qmax = g.pbc[k] ? (double)(g.reach[k] + g.nb[k]) / g.nb[k] + 1.0 : 0.0;
      ext += len * (span + qmax + 1.0);
    }
    const double err = 8.0 * ext * std::ldexp(1.0, -24) * std::sqrt(3.0);
    g.rc2_hi = (float)((r_cut + 2.0 * err) * (r_cut + 2.0 * err) * (1.0 + 1e-5));
    // the same bound the other way: an FP32 distance below R_cut - 2 err (and
    // above 4 err) puts the exact one inside (0, R_cut), so the FP64 test is
    // needed only in the two shells of width ~4 err around 0 and R_cut
    const double lo = r_cut - 2.0 * err;
    g.rc2_lo = lo > 0.0 ? (float)(lo * lo * (1.0 - 1e-5)) : 0.0f;
    g.rz2 = (float)(16.0 * err * err * (1.0 + 1e-5)) + 1e-30f;
  }
  if ((rc = nl->bins.ensure(sizeof(int) * (2 * nbins + 1))) != MTP_OK) return rc;
  int* bin_count = nl->bins.as<int>();
  int* cursor = bin_count + nbins;
  if ((rc = nl->bin_start.ensure(sizeof(int) * (nbins + 1))) != MTP_OK) return rc;
  int* bin_start = nl->bin_start.as<int>();
  const size_t bin_xw_off = (sizeof(int) * 2 * (size_t)std::max<int64_t>(n, 1) + 15) & ~size_t(15);
  if ((rc = nl->bin_atoms.ensure(bin_xw_off + sizeof(float4) * (size_t)std::max<int64_t>(n, 1))) != MTP_OK) return rc;
  int* bin_of = nl->bin_atoms.as<int>();
  int* bin_atoms = bin_of + std::max<int64_t>(n, 1);
  float4* bin_xw = reinterpret_cast<float4*>(reinterpret_cast<char*>(nl->bin_atoms.ptr) + bin_xw_off);
  MTP_TRY_CUDA(cudaMemsetAsync(bin_count, 0, sizeof(int) * 2 * nbins, stream));
  if (n > 0) bin_count_kernel<<<blocks, T, 0, stream>>>(sw, n, g, bin_of, bin_count);
  MTP_TRY_CUDA(cudaGetLastError());
  size_t tmp_bytes = 0;
  MTP_TRY_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, bin_count, bin_start, (int)nbins, stream));
  size_t tmp2 = 0;
  MTP_TRY_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tmp2, (int64_t*)nullptr, (int64_t*)nullptr, (int)(n + 1), stream));
  tmp_bytes = std::max(tmp_bytes, tmp2);
  if ((rc = nl->counts.ensure(sizeof(int) * std::max<int64_t>(n, 1) + sizeof(int64_t) * (n + 2) + tmp_bytes + 64)) !=
      MTP_OK)
    return rc;
  int* counts = nl->counts.as<int>();
  int64_t* counts64 = reinterpret_cast<int64_t*>((reinterpret_cast<uintptr_t>(counts + std::max<int64_t>(n, 1)) + 15) &
                                                 ~uintptr_t(15));
  void* tmp = counts64 + n + 2;
  MTP_TRY_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, bin_count, bin_start, (int)nbins, stream));
  if (n > 0) bin_fill_kernel<<<blocks, T, 0, stream>>>(bin_of, n, bin_start, cursor, xw, bin_atoms, bin_xw);
  MTP_TRY_CUDA(cudaGetLastError());
  if (n > 0)
    pair_kernel<false><<<blocks, T, 0, stream>>>(x, sw, wrapcnt, xw, n, g, bin_start, bin_count, bin_atoms, bin_xw, counts, nullptr,
                                                 nullptr, nullptr, status);
  MTP_TRY_CUDA(cudaGetLastError());
  if ((rc = nl->offsets.ensure(sizeof(int64_t) * (n + 1))) != MTP_OK) return rc;
  int64_t* offsets = nl->offsets.as<int64_t>();
  widen_counts<<<(unsigned)((n + 1 + T - 1) / T), T, 0, stream>>>(counts, n, counts64);
  MTP_TRY_CUDA(cudaGetLastError());
  MTP_TRY_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, counts64, offsets, (int)(n + 1), stream));
  int64_t total = 0;
  int st = 0;
  MTP_TRY_CUDA(cudaMemcpyAsync(&total, offsets + n, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
  MTP_TRY_CUDA(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, stream));
  MTP_TRY_CUDA(cudaStreamSynchronize(stream));
  if (st != 0) {
    set_error("mtp_build_neighbors: a neighbour image exceeds +-511 cells (cell too thin for the cutoff)");
    return MTP_ERR_NEIGHBOR_OVERFLOW;
  }
  nl->n_pairs = total;
  if ((rc = nl->nbr_j.ensure(sizeof(int32_t) * std::max<int64_t>(total, 1))) != MTP_OK) return rc;
  if ((rc = nl->nbr_img.ensure(sizeof(int32_t) * std::max<int64_t>(total, 1))) != MTP_OK) return rc;
  if (n > 0) {
    pair_kernel<true><<<blocks, T, 0, stream>>>(x, sw, wrapcnt, xw, n, g, bin_start, bin_count, bin_atoms, bin_xw, nullptr, offsets,
                                                nl->nbr_j.as<int32_t>(), nl->nbr_img.as<int32_t>(), status);
    MTP_TRY_CUDA(cudaGetLastError());
    sort_rows_kernel<<<(unsigned)((32 * n + T - 1) / T), T, 0, stream>>>(n, offsets, nl->nbr_j.as<int32_t>(),
                                                                        nl->nbr_img.as<int32_t>());
  }
  MTP_TRY_CUDA(cudaGetLastError());
  return MTP_OK;
}

}  // namespace mtp
