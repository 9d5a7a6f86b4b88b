// Active-set selection by MaxVol, and FP64 basis rows for its pool.
//
// The paper's active learning compares each neighbourhood (or configuration)
// with an active set of basis rows and selects those whose extrapolation
// grade exceeds a threshold (Sec. 2.1, Sec. 2.3); the active set itself is
// the MaxVol submatrix of a pool of rows (Goreinov et al. 2010, as in the
// MLIP package the paper builds on).  With P the pool [n_pool][m] and A = P[I]
// the active rows:
//   C = P A^-1;  (i, k) = argmax |C_ik| (first in row-major order);
//   stop when |C_ik| <= 1 + delta, else I[k] = i and repeat.
// Replacing row k of A by p_i changes A^-1 and C by rank-one (Sherman-Morrison)
// updates: with w = (c_i - e_k) / C_ik,
//   A^-1 <- A^-1 - (A^-1 e_k) w,   C <- C - (C e_k) w.
// Updates accumulate rounding, so C and A^-1 are recomputed from scratch
// (Gauss-Jordan with partial pivoting, then the product) every kRefresh
// swaps and before the stopping test is accepted.
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "mtp_internal.cuh"

namespace mtp {

constexpr int kMvThreads = 256;
constexpr int kRefresh = 32;

// aug = [P[rows] | I] ([m][2m]) for Gauss-Jordan.
__global__ void mv_gather_kernel(const double* __restrict__ pool, const int32_t* __restrict__ rows, int m,
                                 double* __restrict__ aug) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * 2 * m) return;
  const int r = (int)(t / (2 * m)), c = (int)(t % (2 * m));
  aug[t] = c < m ? pool[(int64_t)rows[r] * m + c] : (c - m == r ? 1.0 : 0.0);
}

// Gauss-Jordan elimination with partial pivoting on aug [m][2m] by one block:
// per column the pivot is the first largest |aug[r][col]|, r >= col; the pivot
// row is divided by the pivot and subtracted, times aug[r][col], from every
// other row.  Each operation is rounded separately.  The right half becomes
// A^-1.  *singular = 1 if a pivot is zero.
__global__ void mv_gauss_jordan_kernel(double* __restrict__ aug, int m, int* __restrict__ singular) {
  __shared__ double s_val[kMvThreads];
  __shared__ int s_idx[kMvThreads];
  __shared__ int s_piv;
  extern __shared__ double s_f[];   // [m] elimination factors
  const int w = 2 * m;
  for (int col = 0; col < m; ++col) {
    double best = -1.0;
    int bi = m;
    for (int r = col + threadIdx.x; r < m; r += blockDim.x) {
      const double v = fabs(aug[(int64_t)r * w + col]);
      if (v > best) { best = v; bi = r; }
    }
    s_val[threadIdx.x] = best;
    s_idx[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) {
        const double v = s_val[threadIdx.x + o];
        const int j = s_idx[threadIdx.x + o];
        if (v > s_val[threadIdx.x] || (v == s_val[threadIdx.x] && j < s_idx[threadIdx.x])) {
          s_val[threadIdx.x] = v;
          s_idx[threadIdx.x] = j;
        }
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      s_piv = s_idx[0];
      if (!(s_val[0] > 0.0)) *singular = 1;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv >= m || !(s_val[0] > 0.0)) return;   // block-uniform
    if (piv != col)
      for (int c = threadIdx.x; c < w; c += blockDim.x) {
        const double t = aug[(int64_t)col * w + c];
        aug[(int64_t)col * w + c] = aug[(int64_t)piv * w + c];
        aug[(int64_t)piv * w + c] = t;
      }
    __syncthreads();
    const double p = aug[(int64_t)col * w + col];
    __syncthreads();
    for (int c = threadIdx.x; c < w; c += blockDim.x) aug[(int64_t)col * w + c] = __ddiv_rn(aug[(int64_t)col * w + c], p);
    for (int r = threadIdx.x; r < m; r += blockDim.x) s_f[r] = aug[(int64_t)r * w + col];
    __syncthreads();
    // one thread per column, down the column (coalesced across the warp).
    // Columns left of col are unit vectors and columns whose pivot-row entry
    // is zero are unchanged by the update (x - f * 0 = x exactly), so only
    // the others are visited; every update keeps its separate roundings.
    for (int c = col + threadIdx.x; c < w; c += blockDim.x) {
      const double pc = aug[(int64_t)col * w + c];
      if (pc == 0.0) continue;
      for (int r = 0; r < m; ++r) {
        const double f = s_f[r];
        if (r != col && f != 0.0) aug[(int64_t)r * w + c] = __dsub_rn(aug[(int64_t)r * w + c], __dmul_rn(f, pc));
      }
    }
    __syncthreads();
  }
}

__global__ void mv_extract_inverse_kernel(const double* __restrict__ aug, int m, double* __restrict__ a_inv) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)m * m) return;
  const int r = (int)(t / m), c = (int)(t % m);
  a_inv[t] = aug[(int64_t)r * 2 * m + m + c];
}

// C = P A^-1: 64 rows x 32 columns per block, K in steps of 32 through shared memory.
constexpr int kMvBM = 64, kMvBN = 32, kMvBK = 32;
__global__ void __launch_bounds__(kMvThreads) mv_product_kernel(const double* __restrict__ pool, int64_t n, int m,
                                                                const double* __restrict__ a_inv, double* __restrict__ c) {
  __shared__ double sp[kMvBM][kMvBK + 1];
  __shared__ double sa[kMvBK][kMvBN + 1];
  const int64_t r0 = (int64_t)blockIdx.x * kMvBM;
  const int c0 = blockIdx.y * kMvBN;
  const int tx = threadIdx.x % kMvBN, ty = threadIdx.x / kMvBN;   // 32 x 8 threads, 8 rows each
  double acc[kMvBM / 8];
#pragma unroll
  for (int u = 0; u < kMvBM / 8; ++u) acc[u] = 0.0;
  for (int k0 = 0; k0 < m; k0 += kMvBK) {
    for (int t = threadIdx.x; t < kMvBM * kMvBK; t += kMvThreads) {
      const int rr = t / kMvBK, kk = t % kMvBK;
      sp[rr][kk] = (r0 + rr < n && k0 + kk < m) ? pool[(r0 + rr) * m + k0 + kk] : 0.0;
    }
    for (int t = threadIdx.x; t < kMvBK * kMvBN; t += kMvThreads) {
      const int kk = t / kMvBN, cc = t % kMvBN;
      sa[kk][cc] = (k0 + kk < m && c0 + cc < m) ? a_inv[(int64_t)(k0 + kk) * m + c0 + cc] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kMvBK; ++kk) {
      const double b = sa[kk][tx];
#pragma unroll
      for (int u = 0; u < kMvBM / 8; ++u) acc[u] = fma(sp[ty + 8 * u][kk], b, acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < kMvBM / 8; ++u) {
    const int64_t r = r0 + ty + 8 * u;
    if (r < n && c0 + tx < m) c[r * m + c0 + tx] = acc[u];
  }
}

// Device-side step state of mtp_maxvol (so that a run of swaps needs no host
// round trip): st[0] stop decided, st[1] swaps made, st[2] swaps since the
// last refresh, st[3] non-finite C, st[4] this step swaps; sel = (i, k).
enum { kMvDone = 0, kMvIt = 1, kMvSince = 2, kMvBad = 3, kMvAct = 4, kMvState = 8 };

// Largest |C| with the first flat index among equal values: per-block
// candidates, then one block over the candidates (nothing once a stop is
// decided).
__device__ __forceinline__ void mv_better(double& v, long long& i, double v2, long long i2) {
  if (v2 > v || (v2 == v && i2 < i)) {
    v = v2;
    i = i2;
  }
}

__global__ void mv_argmax_kernel(const double* __restrict__ c, long long total, double* __restrict__ bv,
                                 long long* __restrict__ bi, const int* __restrict__ st) {
  if (st[kMvDone]) return;   // grid-uniform
  __shared__ double sv[kMvThreads];
  __shared__ long long si[kMvThreads];
  double v = -1.0;
  long long idx = total;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    double a = fabs(c[t]);
    if (a != a) a = INFINITY;   // NaN: reported as non-finite by the host
    mv_better(v, idx, a, t);
  }
  sv[threadIdx.x] = v;
  si[threadIdx.x] = idx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) mv_better(sv[threadIdx.x], si[threadIdx.x], sv[threadIdx.x + o], si[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bv[blockIdx.x] = sv[0];
    bi[blockIdx.x] = si[0];
  }
}

__global__ void mv_argmax_final_kernel(const double* __restrict__ bv, const long long* __restrict__ bi, int nb,
                                       double* __restrict__ out_v, long long* __restrict__ out_i,
                                       const int* __restrict__ st) {
  if (st[kMvDone]) return;
  __shared__ double sv[kMvThreads];
  __shared__ long long si[kMvThreads];
  double v = -1.0;
  long long idx = LLONG_MAX;
  for (int t = threadIdx.x; t < nb; t += blockDim.x) mv_better(v, idx, bv[t], bi[t]);
  sv[threadIdx.x] = v;
  si[threadIdx.x] = idx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) mv_better(sv[threadIdx.x], si[threadIdx.x], sv[threadIdx.x + o], si[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *out_v = sv[0];
    *out_i = si[0];
  }
}

// The MaxVol decision on the argmax (v, flat index): stop when v <= 1 +
// delta or max_iter swaps are made, else swap pool row i into slot k.
__global__ void mv_decide_kernel(const double* __restrict__ best_v, const long long* __restrict__ best_i, int m,
                                 double delta, int max_iter, int* __restrict__ st, long long* __restrict__ sel,
                                 int32_t* __restrict__ rows) {
  st[kMvAct] = 0;
  if (st[kMvDone]) return;
  const double v = *best_v;
  if (!isfinite(v)) {
    st[kMvBad] = 1;
    st[kMvDone] = 1;
    return;
  }
  if (v <= 1.0 + delta || st[kMvIt] >= max_iter) {
    st[kMvDone] = 1;
    return;
  }
  const long long flat = *best_i;
  const long long i = flat / m;
  const int k = (int)(flat % m);
  sel[0] = i;
  sel[1] = k;
  rows[k] = (int32_t)i;
  st[kMvIt] += 1;
  st[kMvSince] += 1;
  st[kMvAct] = 1;
}

// Snapshot before a swap of row k for pool row i: u = C[:, k] (n), w = (c_i - e_k) / C_ik (m),
// q = A^-1[:, k] (m).  Nothing when the step made no swap.
__global__ void mv_snapshot_kernel(const double* __restrict__ c, int64_t n, int m, const double* __restrict__ a_inv,
                                   const long long* __restrict__ sel, const int* __restrict__ st,
                                   double* __restrict__ u, double* __restrict__ w, double* __restrict__ q) {
  if (!st[kMvAct]) return;
  const int64_t i = sel[0];
  const int k = (int)sel[1];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) u[t] = c[t * m + k];
  if (t < m) {
    const double cik = c[i * m + k];
    w[t] = (c[i * m + t] - (t == k ? 1.0 : 0.0)) / cik;
    q[t] = a_inv[t * m + k];
  }
}

// C -= u w (n x m), A^-1 -= q w (m x m).  Nothing when the step made no swap.
__global__ void mv_rank1_kernel(double* __restrict__ c, int64_t n, int m, double* __restrict__ a_inv,
                                const double* __restrict__ u, const double* __restrict__ w,
                                const double* __restrict__ q, const int* __restrict__ st) {
  if (!st[kMvAct]) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nc = n * m;
  if (t < nc) {
    const int64_t r = t / m;
    const int col = (int)(t % m);
    c[t] = fma(-u[r], w[col], c[t]);
  } else if (t < nc + (int64_t)m * m) {
    const int64_t s = t - nc;
    const int r = (int)(s / m), col = (int)(s % m);
    a_inv[s] = fma(-q[r], w[col], a_inv[s]);
  }
}

namespace {

struct MvScratch {
  double* aug;       // [m][2m]
  double* c;         // [n][m]
  double* u;         // [n]
  double* w;         // [m]
  double* q;         // [m]
  double* bv;        // [nb]
  long long* bi;     // [nb]
  double* best_v;    // [1]
  long long* best_i; // [1]
  int32_t* rows;     // [m] the current active rows (device copy, updated by mv_decide_kernel)
  int* singular;     // [1]
  int* st;           // [kMvState] step state
  long long* sel;    // [2] (i, k) of the step's swap
  int nb;
};

// A^-1 of P[rows] into a_inv and C = P A^-1 (rows: sc.rows); MTP_ERR_ARG if singular.
int mv_refresh(const double* pool, int64_t n, int m, double* a_inv, MvScratch& sc, cudaStream_t s) {
  MTP_TRY_CUDA(cudaMemsetAsync(sc.singular, 0, sizeof(int), s));
  const int64_t na = (int64_t)m * 2 * m;
  mv_gather_kernel<<<(unsigned)((na + kMvThreads - 1) / kMvThreads), kMvThreads, 0, s>>>(pool, sc.rows, m, sc.aug);
  mv_gauss_jordan_kernel<<<1, kMvThreads, sizeof(double) * m, s>>>(sc.aug, m, sc.singular);
  mv_extract_inverse_kernel<<<(unsigned)(((int64_t)m * m + kMvThreads - 1) / kMvThreads), kMvThreads, 0, s>>>(sc.aug, m,
                                                                                                            a_inv);
  dim3 grid((unsigned)((n + kMvBM - 1) / kMvBM), (unsigned)((m + kMvBN - 1) / kMvBN));
  mv_product_kernel<<<grid, kMvThreads, 0, s>>>(pool, n, m, a_inv, sc.c);
  MTP_TRY_CUDA(cudaGetLastError());
  int sing = 0;
  MTP_TRY_CUDA(cudaMemcpyAsync(&sing, sc.singular, sizeof(int), cudaMemcpyDeviceToHost, s));
  MTP_TRY_CUDA(cudaStreamSynchronize(s));
  if (sing) {
    set_error("mtp_maxvol: the active rows are linearly dependent (zero pivot)");
    return MTP_ERR_ARG;
  }
  return MTP_OK;
}

// One MaxVol step on the device: argmax of |C|, the decision, and (if it
// swaps) the rank-one updates of C and A^-1.
int mv_step(int64_t n, int m, double delta, int max_iter, double* a_inv, MvScratch& sc, cudaStream_t s) {
  const long long total = (long long)n * m;
  mv_argmax_kernel<<<sc.nb, kMvThreads, 0, s>>>(sc.c, total, sc.bv, sc.bi, sc.st);
  mv_argmax_final_kernel<<<1, kMvThreads, 0, s>>>(sc.bv, sc.bi, sc.nb, sc.best_v, sc.best_i, sc.st);
  mv_decide_kernel<<<1, 1, 0, s>>>(sc.best_v, sc.best_i, m, delta, max_iter, sc.st, sc.sel, sc.rows);
  const unsigned gs = (unsigned)((std::max<int64_t>(n, m) + kMvThreads - 1) / kMvThreads);
  mv_snapshot_kernel<<<gs, kMvThreads, 0, s>>>(sc.c, n, m, a_inv, sc.sel, sc.st, sc.u, sc.w, sc.q);
  const int64_t tot = (int64_t)n * m + (int64_t)m * m;
  mv_rank1_kernel<<<(unsigned)((tot + kMvThreads - 1) / kMvThreads), kMvThreads, 0, s>>>(sc.c, n, m, a_inv, sc.u,
                                                                                         sc.w, sc.q, sc.st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_error("mtp_maxvol: %s", cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  return MTP_OK;
}

}  // namespace
}  // namespace mtp

extern "C" {

int mtp_maxvol(const double* pool, int64_t n_pool, int32_t m, int32_t* rows, double delta, int32_t max_iter,
               double* a_inv, int32_t* iterations, void* stream) {
  using namespace mtp;
  if (!pool || !rows || !a_inv || m <= 0 || n_pool < m || max_iter < 0 || !(delta >= 0.0) || !std::isfinite(delta)) {
    set_error("mtp_maxvol: invalid argument (need pool, rows, a_inv, 0 < m <= n_pool, delta >= 0, max_iter >= 0)");
    return MTP_ERR_ARG;
  }
  if ((int64_t)n_pool * m > ((int64_t)1 << 40) || m > 4096) {
    set_error("mtp_maxvol: pool too large (n_pool m <= 2^40 and m <= 4096)");
    return MTP_ERR_ARG;
  }
  std::vector<char> seen((size_t)n_pool, 0);
  for (int k = 0; k < m; ++k) {
    if (rows[k] < 0 || rows[k] >= n_pool || seen[(size_t)rows[k]]) {
      set_error("mtp_maxvol: initial rows must be %d distinct indices in [0, %lld)", m, (long long)n_pool);
      return MTP_ERR_ARG;
    }
    seen[(size_t)rows[k]] = 1;
  }
  cudaStream_t s = (cudaStream_t)stream;
  MvScratch sc;
  sc.nb = (int)std::min<int64_t>(4 * 152, ((int64_t)n_pool * m + kMvThreads - 1) / kMvThreads);
  const size_t n = (size_t)n_pool, mm = (size_t)m;
  const size_t bytes = sizeof(double) * (2 * mm * mm + n * mm + n + 2 * mm + (size_t)sc.nb + 1) +
                       sizeof(long long) * ((size_t)sc.nb + 1 + 2) + sizeof(int32_t) * mm +
                       sizeof(int) * (1 + kMvState) + 256;
  DevBuf buf;
  int rc = buf.ensure(bytes);
  if (rc != MTP_OK) return rc;
  double* d = buf.as<double>();
  sc.aug = d;
  sc.c = sc.aug + 2 * mm * mm;
  sc.u = sc.c + n * mm;
  sc.w = sc.u + n;
  sc.q = sc.w + mm;
  sc.bv = sc.q + mm;
  sc.best_v = sc.bv + sc.nb;
  sc.bi = reinterpret_cast<long long*>(sc.best_v + 1);
  sc.best_i = sc.bi + sc.nb;
  sc.sel = sc.best_i + 1;
  sc.rows = reinterpret_cast<int32_t*>(sc.sel + 2);
  sc.singular = reinterpret_cast<int*>(sc.rows + mm);
  sc.st = sc.singular + 1;

  // The swaps run on the device (mv_step); the host waits once per run of
  // up to kRefresh - since steps, then refreshes C and A^-1 where the
  // sequential algorithm would: after kRefresh swaps, and when a stop was
  // decided on updated rather than freshly computed C.
  int st[kMvState] = {0};
  MTP_TRY_CUDA(cudaMemcpyAsync(sc.rows, rows, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
  MTP_TRY_CUDA(cudaMemsetAsync(sc.st, 0, sizeof(int) * kMvState, s));
  if ((rc = mv_refresh(pool, n_pool, m, a_inv, sc, s)) != MTP_OK) {
    buf.release();
    return rc;
  }
  while (true) {
    for (int b = st[kMvSince]; b < kRefresh && rc == MTP_OK; ++b) rc = mv_step(n_pool, m, delta, max_iter, a_inv, sc, s);
    if (rc != MTP_OK) break;
    if (cudaMemcpyAsync(st, sc.st, sizeof(int) * kMvState, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
      set_error("mtp_maxvol: %s", cudaGetErrorString(cudaGetLastError()));
      rc = MTP_ERR_CUDA;
      break;
    }
    if (st[kMvBad]) {
      set_error("mtp_maxvol: non-finite entry in P A^-1");
      rc = MTP_ERR_NONFINITE;
      break;
    }
    if (st[kMvDone] && st[kMvSince] == 0) break;   // decided on freshly computed C
    if (!st[kMvDone] && st[kMvSince] < kRefresh) continue;
    // a stop on updated C, or kRefresh swaps since the last refresh
    if ((rc = mv_refresh(pool, n_pool, m, a_inv, sc, s)) != MTP_OK) break;
    st[kMvDone] = 0;
    st[kMvSince] = 0;
    if (cudaMemcpyAsync(sc.st, st, sizeof(int) * kMvState, cudaMemcpyHostToDevice, s) != cudaSuccess) {
      set_error("mtp_maxvol: %s", cudaGetErrorString(cudaGetLastError()));
      rc = MTP_ERR_CUDA;
      break;
    }
  }
  std::vector<int32_t> cur((size_t)m);
  if (rc == MTP_OK) {
    if (cudaMemcpyAsync(cur.data(), sc.rows, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s) != cudaSuccess) rc = MTP_ERR_CUDA;
  }
  cudaStreamSynchronize(s);
  buf.release();
  if (rc != MTP_OK) return rc;
  std::memcpy(rows, cur.data(), sizeof(int32_t) * m);
  if (iterations) *iterations = st[kMvIt];
  return MTP_OK;
}

int mtp_compute_basis_rows(mtp_handle* h, const mtp_nlist* nl, const double* x, const int32_t* z, int64_t n,
                           const double* cell, double* rows, void* stream) {
  using namespace mtp;
  if (!h || !nl || !cell || (n > 0 && (!x || !z || !rows))) {
    set_error("mtp_compute_basis_rows: NULL argument");
    return MTP_ERR_ARG;
  }
  if (n != nl->n_atoms) {
    set_error("mtp_compute_basis_rows: n_atoms = %lld but the list holds %lld", (long long)n, (long long)nl->n_atoms);
    return MTP_ERR_ARG;
  }
  if (!h->ops->rows) {
    set_error("mtp_compute_basis_rows: level %d has no basis-row kernel", h->level);
    return MTP_ERR_UNSUPPORTED;
  }
  if (n == 0) return MTP_OK;
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
  a.m = h->m;
  a.r_min = h->r_min;
  a.r_cut = h->r_cut;
  a.radial_d = h->radial_d.as<double>();
  a.xi_d = h->xi_d.as<double>();
  a.status = h->status.as<int>();
  a.atom_begin = 0;
  a.atom_end = n;
  return h->ops->rows(a, nullptr, n, rows, h->m, nullptr, (cudaStream_t)stream);
}

}  // extern "C"
