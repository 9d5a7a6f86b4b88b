// Extrapolation grade: gamma_i = max_k |(b_i A^-1)_k| (neighbourhood mode) and
// gamma_cfg = max_k |((sum_i b_i) A_cfg^-1)_k| (configuration mode), with the
// selection and break thresholds of paper Sec. 2.1 / Sec. 2.3.
//
// Basis rows are FP64: on active sets drawn from near-perfect lattices the
// product b_i A^-1 cancels by a factor sum_j |b_ij A_jk| / gamma_i of about
// 5e7 (median over a sigma = 0.15 A BCC box against a sigma = 0.05 A pool),
// so FP32 basis values cannot decide a flag.
//
// Two methods for the neighbourhood-mode product:
//   MTP_GRADE_TENSOR (default): the BF16 tensor cores with error-free slicing
//     (grade_tc.cu); rows within max(5% of a threshold, the slicing bound) of
//     a threshold are re-checked by the FP64 kernel below on a compacted list.
//   MTP_GRADE_FP64: every row through the FP64 kernel below.
// In both, each FP64 result carries the bound eps_i = kGradeRelErr *
// sum_j |b_ij| max_k |A_jk|; a row whose FP64 grade lies within eps_i of a
// threshold is counted as ambiguous (its flag is still the FP64 comparison).
//
// gemm_grade_kernel: 64 rows x all m columns per block of 256 threads (in
// column blocks of 128), K in blocks of 16 staged in shared memory, 4 x 8
// FP64 accumulators per thread,
// fused row maximum, bound, flags and the running maximum grade; rows come
// either contiguously or from an index list.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "mtp_internal.cuh"

namespace mtp {

constexpr double kGradeRelErr = 1e-12;
constexpr int kGemmBM = 64, kGemmBK = 16, kGemmBN = 128;

// Row r of the product is row `src` of `rows` (stride ld), entry j read at
// column cols[j] when cols is given (else j): the configuration mode over the
// parameter gradient grades a subset of its columns.
__global__ void __launch_bounds__(256) gemm_grade_kernel(const double* __restrict__ rows, int64_t ld,
                                                         const int32_t* __restrict__ cols, int64_t n, int m,
                                                         const double* __restrict__ ainv,
                                                         const double* __restrict__ amax, double tau_sel,
                                                         double tau_brk, double* __restrict__ gamma,
                                                         uint8_t* __restrict__ flags,
                                                         unsigned long long* __restrict__ gmax_bits,
                                                         unsigned long long* __restrict__ n_ambiguous,
                                                         const int32_t* __restrict__ list,
                                                         const unsigned* __restrict__ list_n) {
  __shared__ double As[kGemmBK][kGemmBM + 1];
  __shared__ double Bs[kGemmBK][kGemmBN];
  __shared__ double red[kGemmBM][17];
  const int tid = threadIdx.x;
  const int ty = tid / 16, tx = tid % 16;
  const int64_t row0 = (int64_t)blockIdx.x * kGemmBM;
  if (list) {
    n = (int64_t)*list_n;   // rows are list[0 .. *list_n)
    if (row0 >= n) return;  // uniform over the block
  }
  double rmax[4] = {0.0, 0.0, 0.0, 0.0};
  for (int cb = 0; cb < m; cb += kGemmBN) {   // column blocks of A^-1 (one for m <= 128)
    double acc[4][8];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) acc[r][c] = 0.0;
    for (int kb = 0; kb < m; kb += kGemmBK) {
#pragma unroll
      for (int t = 0; t < (kGemmBM * kGemmBK) / 256; ++t) {
        const int e = tid + 256 * t;
        const int rr = e / kGemmBK, kk = e % kGemmBK;
        const int64_t gr = row0 + rr;
        const int64_t src = (gr < n && list) ? (int64_t)list[gr] : gr;
        const int col = kb + kk;
        As[kk][rr] = (gr < n && col < m) ? rows[src * ld + (cols ? cols[col] : col)] : 0.0;
      }
#pragma unroll
      for (int t = 0; t < (kGemmBK * kGemmBN) / 256; ++t) {
        const int e = tid + 256 * t;
        const int kk = e / kGemmBN, cc = e % kGemmBN;
        Bs[kk][cc] = (kb + kk < m && cb + cc < m) ? ainv[(int64_t)(kb + kk) * m + cb + cc] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kGemmBK; ++kk) {
        double av[4], bv[8];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[r] = As[kk][ty * 4 + r];
#pragma unroll
        for (int c = 0; c < 8; ++c) bv[c] = Bs[kk][tx + 16 * c];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 8; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 8; ++c) rmax[r] = fmax(rmax[r], fabs(acc[r][c]));
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) red[ty * 4 + r][tx] = rmax[r];
  __syncthreads();
  if (tid < kGemmBM) {
    int64_t gr = row0 + tid;
    if (gr < n) {
      if (list) gr = list[gr];
      double g = 0.0;
      for (int t = 0; t < 16; ++t) g = fmax(g, red[tid][t]);
      double bound = 0.0;
      for (int j = 0; j < m; ++j) bound = fma(fabs(rows[gr * ld + (cols ? cols[j] : j)]), amax[j], bound);
      bound *= kGradeRelErr;
      gamma[gr] = g;
      flags[gr] = (uint8_t)((g > tau_sel ? 1 : 0) | (g > tau_brk ? 2 : 0));
      if (fabs(g - tau_sel) <= bound || fabs(g - tau_brk) <= bound) atomicAdd(n_ambiguous, 1ull);
      atomicMax(gmax_bits, (unsigned long long)__double_as_longlong(g));
    }
  }
}

// max_k |A_jk| for every row j.
__global__ void row_absmax_kernel(const double* __restrict__ a, int m, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  double mx = 0.0;
  for (int k = 0; k < m; ++k) mx = fmax(mx, fabs(a[(int64_t)j * m + k]));
  out[j] = mx;
}

// Configuration mode: gamma_cfg = max_k |(bsum A_cfg^-1)_k| and its bound.
__global__ void cfg_grade_kernel(const double* __restrict__ bsum, const double* __restrict__ acfg, int m,
                                 double* __restrict__ out) {
  __shared__ double smax[256], sbound[256];
  double mx = 0.0, bd = 0.0;
  for (int k = threadIdx.x; k < m; k += blockDim.x) {
    double g = 0.0, b = 0.0;
    for (int j = 0; j < m; ++j) {
      g = fma(bsum[j], acfg[(int64_t)j * m + k], g);
      b = fma(fabs(bsum[j]), fabs(acfg[(int64_t)j * m + k]), b);
    }
    mx = fmax(mx, fabs(g));
    bd = fmax(bd, b);
  }
  smax[threadIdx.x] = mx;
  sbound[threadIdx.x] = bd;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
      sbound[threadIdx.x] = fmax(sbound[threadIdx.x], sbound[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = smax[0];
    out[1] = kGradeRelErr * sbound[0];
  }
}

// total += *count (one thread).
__global__ void add_count_kernel(unsigned long long* total, const unsigned* count) { *total += *count; }

}  // namespace mtp

using namespace mtp;

namespace {

size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

}  // namespace

extern "C" int mtp_compute_grade(mtp_handle* h, const mtp_nlist* nl, const double* x, const int32_t* z, int64_t n,
                                 const double* cell, const double* a_inv, const double* a_inv_cfg, double tau_sel,
                                 double tau_brk, int64_t chunk_atoms, int32_t method, double* gamma, uint8_t* flags,
                                 double* gamma_max, double* gamma_cfg, int64_t* n_ambiguous, int64_t* n_rechecked,
                                 void* stream) {
  if (!h || !nl || !cell || (n > 0 && (!x || !z))) {
    set_error("mtp_compute_grade: NULL argument");
    return MTP_ERR_ARG;
  }
  if (n != nl->n_atoms) {
    set_error("mtp_compute_grade: n_atoms = %lld but the list holds %lld", (long long)n, (long long)nl->n_atoms);
    return MTP_ERR_ARG;
  }
  if (!a_inv && !a_inv_cfg) {
    set_error("mtp_compute_grade: neither a neighbourhood nor a configuration active set was given");
    return MTP_ERR_ARG;
  }
  if (a_inv && (!gamma || !flags)) {
    set_error("mtp_compute_grade: neighbourhood mode needs gamma and flags outputs");
    return MTP_ERR_ARG;
  }
  if (!(tau_sel > 0.0) || !(tau_brk >= tau_sel)) {
    set_error("mtp_compute_grade: thresholds must satisfy 0 < tau_sel <= tau_brk");
    return MTP_ERR_ARG;
  }
  if (chunk_atoms < 0) {
    set_error("mtp_compute_grade: chunk_atoms < 0");
    return MTP_ERR_ARG;
  }
  if (method != MTP_GRADE_TENSOR && method != MTP_GRADE_FP64) {
    set_error("mtp_compute_grade: unknown method %d", (int)method);
    return MTP_ERR_ARG;
  }
  if (!h->ops->rows) {
    set_error("mtp_compute_grade: level %d has no basis-row kernel", h->level);
    return MTP_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int m = h->m;
  const bool tensor = a_inv && method == MTP_GRADE_TENSOR;
  if (tensor && m > kTcMaxBasis) {
    set_error("mtp_compute_grade: the tensor-core method supports m <= %d (m = %d); use MTP_GRADE_FP64", kTcMaxBasis,
              m);
    return MTP_ERR_UNSUPPORTED;
  }
  const int64_t chunk = chunk_atoms > 0 ? std::min<int64_t>(chunk_atoms, std::max<int64_t>(n, 1))
                                        : std::min<int64_t>(std::max<int64_t>(n, 1), 262144);
  int rc;
  // scratch: head [gmax bits, ambiguous count, cfg(2), rechecked, list count, status] | amax [m] | bsum [m] |
  //          rows [chunk][m] | tensor-core method: colmax, dexp, fexp, fmax, Y slices, erow, gamma bits, list, X slices
  const size_t head = 8;
  size_t off = sizeof(double) * (head + 2 * (size_t)m + (size_t)chunk * m);
  size_t o_colmax = 0, o_dexp = 0, o_fexp = 0, o_fmax = 0, o_ys = 0, o_erow = 0, o_gbits = 0, o_list = 0, o_xs = 0;
  if (tensor) {
    o_colmax = off = align256(off);
    off += sizeof(unsigned long long) * kTcMaxBasis;
    o_dexp = off = align256(off);
    off += sizeof(int) * kTcMaxBasis;
    o_fexp = off = align256(off);
    off += sizeof(int) * kTcMaxBasis;
    o_fmax = off = align256(off);
    off += sizeof(int) * 4;
    o_ys = off = align256(off);
    off += tc_y_bytes();
    o_erow = off = align256(off);
    off += sizeof(int) * (size_t)chunk;
    o_gbits = off = align256(off);
    off += sizeof(unsigned long long) * (size_t)chunk;
    o_list = off = align256(off);
    off += sizeof(int32_t) * (size_t)chunk;
    o_xs = off = align256(off);
    off += tc_x_bytes(chunk);
  }
  if ((rc = h->grade.ensure(off)) != MTP_OK) return rc;
  unsigned char* raw = h->grade.as<unsigned char>();
  double* base = h->grade.as<double>();
  unsigned long long* gmax_bits = reinterpret_cast<unsigned long long*>(base);
  unsigned long long* n_amb = gmax_bits + 1;
  double* cfg_out = base + 2;
  unsigned long long* n_rchk = gmax_bits + 4;
  unsigned* list_n = reinterpret_cast<unsigned*>(base + 5);
  int* tc_status = reinterpret_cast<int*>(base + 6);
  double* amax = base + head;
  double* bsum = amax + m;
  double* rows = bsum + m;
  MTP_TRY_CUDA(cudaMemsetAsync(base, 0, sizeof(double) * (head + 2 * (size_t)m), s));
  if (a_inv) {
    row_absmax_kernel<<<(m + 127) / 128, 128, 0, s>>>(a_inv, m, amax);
    MTP_TRY_CUDA(cudaGetLastError());
  }
  EfvArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_atoms = n;
  a.offsets = nl->offsets.as<int64_t>();
  a.nbr_j = nl->nbr_j.as<int32_t>();
  a.nbr_img = nl->nbr_img.as<int32_t>();
  a.x = x;
  a.z = z;
  for (int k = 0; k < 9; ++k) {
    a.cell[k] = cell[k];
    a.cellf[k] = (float)cell[k];
  }
  a.n_species = h->n_species;
  a.n_q = h->n_q;
  a.n_mu = h->n_mu;
  a.m = m;
  a.r_min = h->r_min;
  a.r_cut = h->r_cut;
  a.radial_d = h->radial_d.as<double>();
  a.xi_d = h->xi_d.as<double>();
  a.status = h->status.as<int>();
  for (int64_t b = 0; b < n; b += chunk) {
    const int64_t cnt = std::min<int64_t>(chunk, n - b);
    a.atom_begin = b;
    a.atom_end = b + cnt;
    if ((rc = h->ops->rows(a, nullptr, cnt, rows, m, a_inv_cfg ? bsum : nullptr, s)) != MTP_OK) return rc;
    if (tensor) {
      auto* colmax = reinterpret_cast<unsigned long long*>(raw + o_colmax);
      auto* dexp = reinterpret_cast<int*>(raw + o_dexp);
      auto* fexp = reinterpret_cast<int*>(raw + o_fexp);
      auto* fmax = reinterpret_cast<int*>(raw + o_fmax);
      auto* ys = reinterpret_cast<uint16_t*>(raw + o_ys);
      auto* erow = reinterpret_cast<int*>(raw + o_erow);
      auto* gbits = reinterpret_cast<unsigned long long*>(raw + o_gbits);
      auto* list = reinterpret_cast<int32_t*>(raw + o_list);
      auto* xs = reinterpret_cast<uint16_t*>(raw + o_xs);
      if ((rc = tc_prepare(rows, cnt, m, a_inv, amax, colmax, ys, fexp, dexp, fmax, xs, erow, tc_status, s)) !=
          MTP_OK)
        return rc;
      if ((rc = tc_gemm(xs, ys, fexp, erow, cnt, gbits, tc_status, nullptr, s)) != MTP_OK) return rc;
      MTP_TRY_CUDA(cudaMemsetAsync(list_n, 0, sizeof(unsigned), s));
      if ((rc = tc_finalize(gbits, cnt, erow, fmax, tau_sel, tau_brk, gamma + b, flags + b, gmax_bits, list, list_n,
                            s)) != MTP_OK)
        return rc;
      gemm_grade_kernel<<<(unsigned)((cnt + kGemmBM - 1) / kGemmBM), 256, 0, s>>>(
          rows, m, nullptr, cnt, m, a_inv, amax, tau_sel, tau_brk, gamma + b, flags + b, gmax_bits, n_amb, list,
          list_n);
      MTP_TRY_CUDA(cudaGetLastError());
      add_count_kernel<<<1, 1, 0, s>>>(n_rchk, list_n);
      MTP_TRY_CUDA(cudaGetLastError());
    } else if (a_inv) {
      gemm_grade_kernel<<<(unsigned)((cnt + kGemmBM - 1) / kGemmBM), 256, 0, s>>>(
          rows, m, nullptr, cnt, m, a_inv, amax, tau_sel, tau_brk, gamma + b, flags + b, gmax_bits, n_amb, nullptr,
          nullptr);
      MTP_TRY_CUDA(cudaGetLastError());
    }
  }
  if (a_inv_cfg) {
    cfg_grade_kernel<<<1, 256, 0, s>>>(bsum, a_inv_cfg, m, cfg_out);
    MTP_TRY_CUDA(cudaGetLastError());
  }
  double hostbuf[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  MTP_TRY_CUDA(cudaMemcpyAsync(hostbuf, base, sizeof(double) * 8, cudaMemcpyDeviceToHost, s));
  MTP_TRY_CUDA(cudaStreamSynchronize(s));
  unsigned long long gbits_h, amb, rchk;
  std::memcpy(&gbits_h, &hostbuf[0], sizeof(gbits_h));
  std::memcpy(&amb, &hostbuf[1], sizeof(amb));
  std::memcpy(&rchk, &hostbuf[4], sizeof(rchk));
  int tcs;
  std::memcpy(&tcs, &hostbuf[6], sizeof(tcs));
  if (tcs == MTP_ERR_TIMEOUT) {
    set_error("mtp_compute_grade: a wait inside the tensor-core grade kernel gave up");
    return MTP_ERR_TIMEOUT;
  }
  double gmax;
  std::memcpy(&gmax, &gbits_h, sizeof(gmax));
  if (a_inv_cfg && std::fabs(hostbuf[2] - tau_sel) <= hostbuf[3]) ++amb;
  if (a_inv_cfg && std::fabs(hostbuf[2] - tau_brk) <= hostbuf[3]) ++amb;
  if (gamma_max) *gamma_max = a_inv ? gmax : 0.0;
  if (gamma_cfg) *gamma_cfg = a_inv_cfg ? hostbuf[2] : 0.0;
  if (n_ambiguous) *n_ambiguous = (int64_t)amb;
  if (n_rechecked) *n_rechecked = (int64_t)rchk;
  if (!std::isfinite(gmax) || (a_inv_cfg && !std::isfinite(hostbuf[2])) || tcs == MTP_ERR_NONFINITE) {
    set_error("mtp_compute_grade: non-finite grade");
    return MTP_ERR_NONFINITE;
  }
  const double worst = std::max(a_inv ? gmax : 0.0, a_inv_cfg ? hostbuf[2] : 0.0);
  return worst > tau_brk ? MTP_STATUS_BREAK : MTP_OK;
}

// Verification hook for the tensor-core product (see mtp.h).
extern "C" int mtp_grade_tc_selftest(const uint16_t* xs, const uint16_t* ys, const int32_t* fexp, const int32_t* erow,
                                     int64_t n_rows, float* acc, uint64_t* gamma_bits, void* stream) {
  if (n_rows < 0 || (n_rows > 0 && (!xs || !ys || !fexp || !erow || !gamma_bits))) {
    set_error("mtp_grade_tc_selftest: NULL argument");
    return MTP_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int* status = nullptr;
  MTP_TRY_CUDA(cudaMalloc(&status, sizeof(int)));
  int st = 0;
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), s);
  int rc = e == cudaSuccess ? tc_gemm(xs, ys, fexp, erow, n_rows, reinterpret_cast<unsigned long long*>(gamma_bits),
                                      status, acc, s)
                            : MTP_ERR_CUDA;
  if (rc == MTP_OK) {
    e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error("mtp_grade_tc_selftest: %s", cudaGetErrorString(e));
      rc = MTP_ERR_CUDA;
    }
  }
  cudaFree(status);
  if (rc != MTP_OK) return rc;
  if (st != 0) {
    set_error(st == MTP_ERR_TIMEOUT ? "mtp_grade_tc_selftest: a device-side wait gave up"
                                    : "mtp_grade_tc_selftest: device status %d", st);
    return st;
  }
  return MTP_OK;
}

// Grade of caller-given rows (configuration mode over the full parameter
// gradient, see mtp.h): the FP64 row-max product with its error bound.
extern "C" int mtp_grade_rows(const double* rows, int64_t n_rows, int64_t ld, const int32_t* cols, int32_t m,
                              const double* a_inv, double tau_sel, double tau_brk, double* gamma, uint8_t* flags,
                              double* gamma_max, int64_t* n_ambiguous, void* stream) {
  if (n_rows < 0 || m < 1 || (n_rows > 0 && (!rows || !a_inv || !gamma || !flags)) || (!cols && ld < m) || ld < 1) {
    set_error("mtp_grade_rows: invalid argument");
    return MTP_ERR_ARG;
  }
  if (!(tau_sel > 0.0) || !(tau_brk >= tau_sel)) {
    set_error("mtp_grade_rows: thresholds must satisfy 0 < tau_sel <= tau_brk");
    return MTP_ERR_ARG;
  }
  if (m > 16384) {
    set_error("mtp_grade_rows: m = %d exceeds 16384", (int)m);
    return MTP_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // scratch: gmax bits, ambiguous count, then max_k |A^-1_jk| [m]
  void* scratch = nullptr;
  MTP_TRY_CUDA(cudaMalloc(&scratch, sizeof(double) * (2 + (size_t)m)));
  unsigned long long* gmax_bits = static_cast<unsigned long long*>(scratch);
  unsigned long long* n_amb = gmax_bits + 1;
  double* amax = reinterpret_cast<double*>(gmax_bits + 2);
  unsigned long long host[2] = {0ull, 0ull};
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long) * 2, s);
  if (e == cudaSuccess) {
    row_absmax_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(a_inv, m, amax);
    if (n_rows > 0)
      gemm_grade_kernel<<<(unsigned)((n_rows + kGemmBM - 1) / kGemmBM), 256, 0, s>>>(
          rows, ld, cols, n_rows, m, a_inv, amax, tau_sel, tau_brk, gamma, flags, gmax_bits, n_amb, nullptr, nullptr);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host, scratch, sizeof(host), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(scratch);
  if (e != cudaSuccess) {
    set_error("mtp_grade_rows: %s", cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  double g;
  std::memcpy(&g, &host[0], sizeof(g));
  if (gamma_max) *gamma_max = g;
  if (n_ambiguous) *n_ambiguous = (int64_t)host[1];
  if (!std::isfinite(g)) {
    set_error("mtp_grade_rows: non-finite grade");
    return MTP_ERR_NONFINITE;
  }
  return g > tau_brk ? MTP_STATUS_BREAK : MTP_OK;
}
