// Tensor-core extrapolation grade: gamma_i = max_k |(b_i A^-1)_k| (paper
// Sec. 2.1 and Sec. 2.3, neighbourhood mode) on the BF16 tensor cores with
// FP32 accumulation, exact to the FP64 level by error-free splitting.
//
// Why splitting.  On active sets drawn from near-perfect lattices the product
// b_i A^-1 cancels: sum_j |b_ij A^-1_jk| exceeds gamma_i by ~5e7 (median) to
// ~4e8.  A single BF16 or TF32 product therefore cannot decide a flag.  The
// operands are instead written as short sums of BF16 "slices" whose pairwise
// products the tensor core forms exactly (Ozaki, Ogita, Oishi and Rump 2012:
// error-free transformation of a matrix product into products of
// lower-precision matrices):
//
//   1. Column balancing (exact, powers of two): C = b A^-1 = (b D)(D^-1 A^-1)
//      with d_j = 2^((ilogb max_k|A^-1_jk| - ilogb max_i|b_ij|) / 2).
//   2. Row/column scaling: x_ij = b_ij d_j 2^-e_i with |x| <= 1 per row,
//      y_jk = A^-1_jk / d_j 2^-f_k with |y| <= 1 per column.
//   3. Slices: x = sum_{s=1..7} 2^-8s X_s + rho, each X_s an integer matrix
//      with |X_1| <= 256 and |X_s| <= 128 (s >= 2), |rho| <= 2^-57; the same
//      for y with Y_t.  Integers of at most 8 significant bits are exact in
//      BF16.
//   4. Groups: G_d = sum_{s+t=d} X_s Y_t for d = 2..8 (28 products of
//      128 x 64 x 128 per tile and column half; the products of one X slice
//      with consecutive Y slices are single MMAs of up to 256 columns, since
//      their accumulators are adjacent in Tensor Memory and the Y slices of a
//      half form one 448-row operand: 80 MMA instructions per tile instead
//      of 224).  Every product of two slices
//      is an integer below 2^16 and every partial sum of a group stays below
//      2^24 for d <= 7 (|X_1 Y_1| <= 2^16 per term, the later slices at most
//      half as large each), so the FP32 accumulation in Tensor Memory is exact;
//      G_8 may round by one unit of 2^-64.
//   5. Epilogue: T = sum_d G_d 2^(56-8d) in int64 (exact; |T| <= 115 2^56),
//      gamma = max_k |T_k| 2^(e_i + f_k - 56), compared exactly on
//      (exponent, normalised mantissa) pairs.
//
// Error bound per element, in units of 2^(e_i + f_k): slice remainders
// 2 * 2^-57, omitted pairs s + t >= 9 at most 1.53 * 2^-56, per term j; over
// m <= 115 terms and with the int64 truncation of G_8: below 2^-47.8.  Hence
// |gamma - gamma_exact| <= 2^(e_i + F - 47) + 2^-52 gamma with F = max_k f_k.
// Rows whose grade lies within max(0.05 tau, bound) of a threshold are
// re-checked in FP64: a fixed band of 5% around each threshold, widened to
// the bound where that is larger.
//
// Kernel layout (tc_grade_kernel): one CTA per SM, persistent over 128-row
// tiles, one column half (64 of the padded 128 columns) per CTA.  Shared
// memory holds the 7 Y slices of the half (7 x 16 KB, loaded once by bulk
// copies) and three X slice buffers (3 x 32 KB, streamed by 1-D bulk copies
// through the TMA engine).  Warp 0: copy producer; warp 1: Tensor Memory
// allocation and the MMA issuer (one thread); warps 2-17: epilogue, four
// warps per TMEM lane quarter (a warp may read only the lanes of its
// quarter), 16 of the 64 columns each, one TMEM lane (tile row) per thread.
// Seven FP32 accumulators of 64 columns occupy 448 of the 512 TMEM columns,
// so the epilogue of a tile and the MMAs of the next do not overlap; more
// epilogue warps shorten the epilogue instead (262,144 rows: 0.454 ms with 4,
// 0.361 with 8, 0.331 with 16).  Operands use the no-swizzle K-major
// canonical layout (8-row x 16-byte core matrices).
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "mtp_internal.cuh"
#include "tc_ptx.cuh"

namespace mtp {

namespace {

constexpr int kTcM = 128;                 // tile rows (TMEM lanes)
constexpr int kTcN = 64;                  // output columns per CTA
constexpr int kTcK = 128;                 // padded basis size
constexpr int kTcS = kTcSlices;           // slices per operand
constexpr int kTcDmax = 8;                // slice pairs with s + t <= kTcDmax
constexpr int kTcNacc = kTcDmax - 1;      // accumulators G_2 .. G_8
constexpr uint32_t kXBytes = kTcM * kTcK * 2;   // one X slice tile, BF16
constexpr uint32_t kYBytes = kTcN * kTcK * 2;   // one Y slice half, BF16
constexpr int kXBufs = 3;
constexpr int kTcEpiWarps = 16;           // four per TMEM lane quarter, 16 columns each
constexpr int kTcThreads = 64 + 32 * kTcEpiWarps;
constexpr uint32_t kTmemCols = 512;
constexpr uint64_t kTcTimeoutNs = 1000000000ull;  // 1 s per wait
// Limit of the pipeline waits (producer, MMA issuer, epilogue); the drain
// waits at the end (for copies and MMAs already issued) always allow
// kTcTimeoutNs, so a block never exits with work of its own in flight.
static uint64_t g_tc_wait_ns = kTcTimeoutNs;

// X slice layout (BF16 elements) inside one [128 rows][128 K] tile:
// element (i, j) at (j / 8) * 1024 + (i / 8) * 64 + (i % 8) * 8 + j % 8,
// i.e. core matrices of 8 rows x 16 bytes, LBO (K direction) 2048 bytes,
// SBO (row groups) 128 bytes.
constexpr uint32_t kXLbo = 2048, kXSbo = 128;
// Y slices of a half: one [448 rows][128 K] operand, row kg = 64 t + k for
// column k of slice t: element (kg, j) at (j / 8) * 3584 + (kg / 8) * 64 +
// (kg % 8) * 8 + j % 8, i.e. core matrices of 8 rows x 16 bytes, LBO (K
// direction) 7168 bytes, SBO (row groups) 128 bytes.
constexpr uint32_t kYRows = kTcS * kTcN;                       // 448
constexpr uint32_t kYLbo = (kYRows / 8) * 128, kYSbo = 128;   // 7168, 128

__host__ __device__ __forceinline__ int64_t x_elem(int i, int j) {
  return (int64_t)(j >> 3) * 1024 + (i >> 3) * 64 + (i & 7) * 8 + (j & 7);
}
__host__ __device__ __forceinline__ int64_t y_elem(int kg, int j) {
  return (int64_t)(j >> 3) * (kYRows * 8) + (kg >> 3) * 64 + (kg & 7) * 8 + (j & 7);
}

// Shared-memory map of tc_grade_kernel (bytes).
constexpr uint32_t kSmX = 0;
constexpr uint32_t kSmY = kSmX + kXBufs * kXBytes;          // 98304
constexpr uint32_t kSmBar = kSmY + kTcS * kYBytes;          // 212992
constexpr int kNumBars = 4 + 2 * kXBufs;   // y_full, x_full[kXBufs], x_empty[kXBufs], acc_full, acc_empty, drain
constexpr uint32_t kSmSlot = kSmBar + 8 * kNumBars;         // TMEM base address
constexpr uint32_t kSmAbort = kSmSlot + 4;
constexpr uint32_t kSmFexp = kSmAbort + 4;                  // int [64]
constexpr uint32_t kSmTotal = kSmFexp + 4 * kTcN;
// The block takes the whole 227 KB a block may have: one block per SM (the
// 512 TMEM columns are this block's alone), and every operand descriptor,
// whichever of its two strides the hardware applies to rows or to K, stays
// inside the allocation (worst cases: X buffer 2 at 65,536 + 59,648 =
// 125,184 bytes; Y slice 6 at 196,608 + 14,336 + 7,424 = 218,368 bytes).
constexpr uint32_t kSmAlloc = 232448;
static_assert(kSmTotal <= kSmAlloc, "shared-memory map exceeds the allocation");
// furthest byte an operand descriptor could reach with its strides swapped:
// last X buffer, last K step, 16 row groups at LBO and 2 K core matrices at SBO
static_assert(kSmX + (kXBufs - 1) * kXBytes + (kTcK / 16 - 1) * 2 * kXLbo + 15 * kXLbo + kXSbo + 128 <= kSmAlloc,
              "X operand descriptors may leave the allocation");
// Y operands (runs of up to 4 slices starting at slice 0 or 4), last K step:
// row groups at SBO, the second K core matrix at LBO; inside the Y region
static_assert(kSmY + (kTcK / 16 - 1) * 2 * kYLbo + (4 * kTcN / 8 - 1) * kYSbo + kYLbo + 128 <= kSmBar,
              "Y operand (slices 0-3) leaves the Y region");
static_assert(kSmY + 4 * (kTcN / 8) * kYSbo + (kTcK / 16 - 1) * 2 * kYLbo + (3 * kTcN / 8 - 1) * kYSbo + kYLbo +
                      128 <= kSmBar,
              "Y operand (slices 4-6) leaves the Y region");

constexpr int kBadRow = INT_MAX;   // erow sentinel: non-finite basis row

// BF16 encoding of an integer |q| <= 256 (at most 8 significant bits, so
// exact): the integer enters the mantissa of 1.5 * 2^23 (exact for
// |q| < 2^22, no conversion instruction) and the upper 16 bits of the FP32
// value are its BF16 encoding.
__device__ __forceinline__ uint32_t bf16_of_int(int q) {
  return __float_as_uint(__int_as_float(0x4B400000 + q) - 12582912.0f) >> 16;
}

// floor(log2 |b|) from the IEEE fields (b finite and nonzero).
__device__ __forceinline__ int ilog2_bits(long long bits) {
  const int E = (int)((bits >> 52) & 0x7FF);
  if (E != 0) return E - 1023;
  const long long M = bits & 0xFFFFFFFFFFFFFll;
  return (63 - __clzll(M)) - 1074;
}

// F = round(b 2^shift) as an integer (halves away from zero), straight from
// the IEEE fields; the caller guarantees |b| 2^shift <= 2^56.
__device__ __forceinline__ long long fixed_round(double b, int shift) {
  const long long bits = __double_as_longlong(b);
  const int E = (int)((bits >> 52) & 0x7FF);
  long long M = bits & 0xFFFFFFFFFFFFFll;
  int ex = -1074;
  if (E != 0) {
    M |= 1ll << 52;
    ex = E - 1075;
  }
  const int sh = ex + shift;   // |F| = M 2^sh
  long long F;
  if (sh >= 0) F = M << sh;
  else if (sh > -63) F = (M + (1ll << (-sh - 1))) >> (-sh);
  else F = 0;
  return bits < 0 ? -F : F;
}

// Balanced base-256 digits of F (|F| <= 2^56): F = sum_{s=1..7} q_s 2^(8(7-s)),
// q_7..q_2 in [-128, 127] (the digit of least weight first), |q_1| <= 256;
// returned as BF16 encodings, q[s-1] for slice s.
__device__ __forceinline__ void balanced_digits(long long F, uint32_t (&q)[kTcSlices]) {
#pragma unroll
  for (int s = kTcSlices - 1; s >= 1; --s) {
    const int dig = (int)((F + 128) & 255) - 128;
    q[s] = bf16_of_int(dig);
    F = (F - dig) >> 8;   // exact: F - dig is a multiple of 256
  }
  q[0] = bf16_of_int((int)F);
}

__device__ __forceinline__ void set_status(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

}  // namespace

// ---------------------------------------------------------------------------
// Column maxima of |b| over the chunk's rows (bit patterns of non-negative
// doubles order like the values).
__global__ void tc_colmax_kernel(const double* __restrict__ rows, int64_t n, int m,
                                 unsigned long long* __restrict__ colmax) {
  const int j = threadIdx.x;
  if (j >= m) return;
  double v = 0.0;
  for (int64_t r = blockIdx.x; r < n; r += gridDim.x) v = fmax(v, fabs(rows[r * m + j]));
  atomicMax(colmax + j, (unsigned long long)__double_as_longlong(v));
}

// Balancing exponents d_j = (ilogb max_k|A^-1_jk| - ilogb max_i|b_ij|) / 2
// (one thread per basis function j).
__global__ void tc_dexp_kernel(const double* __restrict__ amax, const unsigned long long* __restrict__ colmax, int m,
                               int* __restrict__ dexp) {
  const int j = threadIdx.x;
  if (j >= kTcK) return;
  int d = 0;
  if (j < m) {
    const double bm = __longlong_as_double((long long)colmax[j]);
    const double am = amax[j];
    if (bm > 0.0 && am > 0.0 && isfinite(bm) && isfinite(am)) d = (ilogb(am) - ilogb(bm)) / 2;
  }
  dexp[j] = d;
}

// Column exponent f_k (|A^-1_jk| 2^(-d_j - f_k) < 1 for all j) and the BF16
// slices of y_jk = A^-1_jk 2^(-d_j - f_k), written as [half][448 x 128] in
// the Y layout.  One block per column k, one thread per row j.
__global__ void __launch_bounds__(kTcK) tc_prep_y_kernel(const double* __restrict__ a_inv, int m,
                                                         const int* __restrict__ dexp, uint16_t* __restrict__ ys,
                                                         int* __restrict__ fexp, int* __restrict__ fmax_out,
                                                         int* status) {
  __shared__ int s_lg;
  const int k = blockIdx.x, j = threadIdx.x;
  if (j == 0) s_lg = INT_MIN;
  __syncthreads();
  double v = 0.0;
  bool finite = true;
  if (k < m && j < m) {
    v = a_inv[(int64_t)j * m + k];
    finite = isfinite(v);
    if (!finite) v = 0.0;
    if (v != 0.0) atomicMax(&s_lg, ilog2_bits(__double_as_longlong(v)) - dexp[j]);
  }
  if (!finite) set_status(status, MTP_ERR_NONFINITE);
  __syncthreads();
  const int f = (s_lg == INT_MIN) ? 0 : s_lg + 1;
  if (j == 0) {
    fexp[k] = f;
    if (k < m) atomicMax(fmax_out, f);
  }
  long long F = 0;
  if (v != 0.0) F = fixed_round(v, 56 - dexp[j] - f);
  uint32_t q[kTcS];
  balanced_digits(F, q);
  const int half = k / kTcN, kl = k % kTcN;
#pragma unroll
  for (int s = 0; s < kTcS; ++s)
    ys[(int64_t)half * (kYRows * kTcK) + y_elem(s * kTcN + kl, j)] = (uint16_t)q[s];
}

// Row exponents e_i and the BF16 slices of x = b D 2^-e, written as
// [tile][s][128 x 128] in the X layout.  One thread per tile row; rows beyond
// n (the ragged last tile) get zero slices.
__global__ void __launch_bounds__(kTcM) tc_split_x_kernel(const double* __restrict__ rows, int64_t n, int m,
                                                          const int* __restrict__ dexp, uint16_t* __restrict__ xs,
                                                          int* __restrict__ erow) {
  __shared__ int s_dexp[kTcK];
  const int il = threadIdx.x;
  s_dexp[il] = dexp[il];
  __syncthreads();
  const int64_t tile = blockIdx.x;
  const int64_t r = tile * kTcM + il;
  const bool valid = r < n;
  const double* row = rows + r * m;
  int e = 0;
  bool bad = false;
  if (valid) {
    // e_i = 1 + max_j floor(log2 |b_ij 2^d_j|), so that |x_ij| < 1
    int mx = INT_MIN;
    for (int j = 0; j < m; ++j) {
      const long long bits = __double_as_longlong(row[j]);
      if (((bits >> 52) & 0x7FF) == 0x7FF) bad = true;
      if ((bits & 0x7FFFFFFFFFFFFFFFll) != 0) mx = max(mx, ilog2_bits(bits) + s_dexp[j]);
    }
    e = (mx == INT_MIN || bad) ? 0 : mx + 1;
    erow[r] = bad ? kBadRow : e;
  }
  uint16_t* base = xs + tile * (int64_t)kTcS * (kTcM * kTcK);
  for (int jc = 0; jc < kTcK / 8; ++jc) {
    uint32_t q[8][kTcS];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int j = jc * 8 + u;
      long long F = 0;
      if (valid && !bad && j < m) {
        const double v = row[j];
        if (v != 0.0) F = fixed_round(v, s_dexp[j] - e + 56);
      }
      balanced_digits(F, q[u]);
    }
#pragma unroll
    for (int s = 0; s < kTcS; ++s) {
      *reinterpret_cast<uint4*>(base + (int64_t)s * (kTcM * kTcK) + x_elem(il, jc * 8)) =
          make_uint4(q[0][s] | (q[1][s] << 16), q[2][s] | (q[3][s] << 16), q[4][s] | (q[5][s] << 16),
                     q[6][s] | (q[7][s] << 16));
    }
  }
}

// ---------------------------------------------------------------------------
struct TcGemmArgs {
  const uint16_t* xs;
  const uint16_t* ys;
  const int* fexp;
  const int* erow;
  int64_t n_rows;
  int n_tiles;
  unsigned long long* gbits;   // [n_rows], zeroed: atomicMax of gamma bits over the two halves
  int* status;
  float* dbg;                  // nullable: raw accumulators [n_tiles*128][2][7][64]
  uint64_t wait_ns;            // limit of each pipeline wait
};

__global__ void __launch_bounds__(kTcThreads, 1) tc_grade_kernel(const TcGemmArgs p) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = blockIdx.x & 1;
  const int cta = blockIdx.x >> 1, n_cta = gridDim.x >> 1;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kSmBar);
  uint32_t* slot = reinterpret_cast<uint32_t*>(sm + kSmSlot);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(sm + kSmAbort);
  int* s_fexp = reinterpret_cast<int*>(sm + kSmFexp);
  const uint32_t y_sm = tc::smem_addr(sm + kSmY);
  const uint32_t x_sm = tc::smem_addr(sm + kSmX);
  const uint32_t b_yfull = tc::smem_addr(&bars[0]);
  const uint32_t b_xfull0 = tc::smem_addr(&bars[1]);
  const uint32_t b_xempty0 = tc::smem_addr(&bars[1 + kXBufs]);
  const uint32_t b_accfull = tc::smem_addr(&bars[1 + 2 * kXBufs]);
  const uint32_t b_accempty = tc::smem_addr(&bars[2 + 2 * kXBufs]);
  const uint32_t b_drain = tc::smem_addr(&bars[3 + 2 * kXBufs]);

  if (threadIdx.x == 0) {
    tc::mbar_init(b_yfull, 1);
    for (int b = 0; b < kXBufs; ++b) {
      tc::mbar_init(b_xfull0 + 8 * b, 1);
      tc::mbar_init(b_xempty0 + 8 * b, 1);
    }
    tc::mbar_init(b_accfull, 1);
    tc::mbar_init(b_accempty, 32 * kTcEpiWarps);
    tc::mbar_init(b_drain, 1);
    *abort_flag = 0;
    tc::mbar_init_fence();
  }
  for (int t = threadIdx.x; t < kTcN; t += blockDim.x) s_fexp[t] = p.fexp[half * kTcN + t];
  if (warp == 1) {
    tc::tmem_alloc(tc::smem_addr(slot), kTmemCols);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- producer: Y slices once, then X slices per (tile, s) ----
      bool ok = true;
      tc::mbar_arrive_expect_tx(b_yfull, kTcS * kYBytes);
      for (int t = 0; t < kTcS; ++t)
        tc::bulk_g2s(y_sm + t * kYBytes, p.ys + (int64_t)(half * kTcS + t) * (kTcN * kTcK), kYBytes, b_yfull);
      int it = 0;
      for (int tile = cta; ok && tile < p.n_tiles; tile += n_cta) {
        for (int s = 0; s < kTcS; ++s, ++it) {
          const int buf = it % kXBufs;
          const uint32_t ph = (uint32_t)(it / kXBufs) & 1u;
          if (!tc::mbar_wait(b_xempty0 + 8 * buf, ph ^ 1u, abort_flag, p.wait_ns)) {
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(b_xfull0 + 8 * buf, kXBytes);
          tc::bulk_g2s(x_sm + buf * kXBytes, p.xs + ((int64_t)tile * kTcS + s) * (kTcM * kTcK), kXBytes,
                       b_xfull0 + 8 * buf);
        }
      }
      if (!ok) {
        *abort_flag = 1;
        set_status(p.status, MTP_ERR_TIMEOUT);
      }
      // no copy may still be in flight when the block exits
      int never = 0;
      tc::mbar_wait(b_yfull, 0u, &never, kTcTimeoutNs);
      for (int k = (it > kXBufs ? it - kXBufs : 0); k < it; ++k)
        tc::mbar_wait(b_xfull0 + 8 * (k % kXBufs), (uint32_t)(k / kXBufs) & 1u, &never, kTcTimeoutNs);
      if (ok)
        for (int k = (it > kXBufs ? it - kXBufs : 0); k < it; ++k)
          tc::mbar_wait(b_xempty0 + 8 * (k % kXBufs), (uint32_t)(k / kXBufs) & 1u, abort_flag, kTcTimeoutNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer ----
      // instruction descriptors for runs of 1..4 Y slices (N = 64..256)
      constexpr uint32_t idesc1 = tc::idesc_bf16_f32(kTcM, kTcN), idesc2 = tc::idesc_bf16_f32(kTcM, 2 * kTcN),
                         idesc3 = tc::idesc_bf16_f32(kTcM, 3 * kTcN), idesc4 = tc::idesc_bf16_f32(kTcM, 4 * kTcN);
      bool ok = tc::mbar_wait(b_yfull, 0u, abort_flag, p.wait_ns);
      tc::fence_after_sync();
      int it = 0, tcount = 0;
      for (int tile = cta; ok && tile < p.n_tiles; tile += n_cta, ++tcount) {
        if (!tc::mbar_wait(b_accempty, ((uint32_t)tcount & 1u) ^ 1u, abort_flag, p.wait_ns)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        for (int s = 0; s < kTcS; ++s, ++it) {
          const int buf = it % kXBufs;
          const uint32_t ph = (uint32_t)(it / kXBufs) & 1u;
          if (!tc::mbar_wait(b_xfull0 + 8 * buf, ph, abort_flag, p.wait_ns)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t xa = x_sm + buf * kXBytes;
          // X_s Y_t for t = 0 .. 6 - s, as runs of up to 4 consecutive Y
          // slices: accumulators G_{s+t} .. are adjacent TMEM columns
          for (int t0 = 0; t0 <= kTcDmax - 2 - s; t0 += 4) {
            const int cnt = min(4, kTcDmax - 1 - s - t0);
            const uint32_t idesc = cnt == 4 ? idesc4 : cnt == 3 ? idesc3 : cnt == 2 ? idesc2 : idesc1;
            const uint32_t d_tmem = tmem + (uint32_t)((s + t0) * kTcN);
            const uint32_t yb = y_sm + (uint32_t)t0 * (kTcN / 8) * kYSbo;
#pragma unroll
            for (int kk = 0; kk < kTcK / 16; ++kk) {
              tc::mma_bf16(d_tmem, tc::smem_desc(xa + kk * 2 * kXLbo, kXLbo, kXSbo),
                           tc::smem_desc(yb + kk * 2 * kYLbo, kYLbo, kYSbo), idesc, !(s == 0 && kk == 0));
            }
          }
          tc::mma_commit(b_xempty0 + 8 * buf);
        }
        if (!ok) break;
        tc::mma_commit(b_accfull);
      }
      if (!ok) {
        *abort_flag = 1;
        set_status(p.status, MTP_ERR_TIMEOUT);
      }
      // every MMA issued has completed before Tensor Memory is released
      int never = 0;
      tc::mma_commit(b_drain);
      tc::mbar_wait(b_drain, 0u, &never, kTcTimeoutNs);
    }
  } else {
    // ---- epilogue: thread = TMEM lane = tile row ----
    const int q = warp & 3;   // TMEM lane quarter this warp may access
    const int c_lo = ((warp - 2) / 4) * (kTcN * 4 / kTcEpiWarps);   // its columns: c_lo .. c_lo + 15
    const int rl = q * 32 + lane;
    const uint32_t lane_base = tmem + ((uint32_t)(q * 32) << 16);
    int tcount = 0;
    for (int tile = cta; tile < p.n_tiles; tile += n_cta, ++tcount) {
      if (!tc::mbar_wait(b_accfull, (uint32_t)tcount & 1u, abort_flag, p.wait_ns)) {
        *abort_flag = 1;
        set_status(p.status, MTP_ERR_TIMEOUT);
        break;
      }
      tc::fence_after_sync();
      const int64_t row = (int64_t)tile * kTcM + rl;
      const bool valid = row < p.n_rows;
      const int e_i = valid ? p.erow[row] : 0;
      int best_e = INT_MIN;
      unsigned long long best_m = 0ull;
      for (int c0 = c_lo; c0 < c_lo + kTcN * 4 / kTcEpiWarps; c0 += 8) {
        uint32_t v[kTcNacc][8];
#pragma unroll
        for (int a = 0; a < kTcNacc; ++a) tc::tmem_ld8(lane_base + (uint32_t)(a * kTcN + c0), v[a]);
        tc::tmem_ld_wait();
#pragma unroll
        for (int a = 0; a < kTcNacc; ++a) tc::reg_fence(v[a]);
        if (p.dbg && valid) {
          float* dst = p.dbg + ((row * 2 + half) * kTcNacc) * kTcN + c0;
#pragma unroll
          for (int a = 0; a < kTcNacc; ++a)
#pragma unroll
            for (int cc = 0; cc < 8; ++cc) dst[a * kTcN + cc] = __uint_as_float(v[a][cc]);
        }
#pragma unroll
        for (int cc = 0; cc < 8; ++cc) {
          long long T = 0;
#pragma unroll
          for (int a = 0; a < kTcNacc - 1; ++a)   // G_2 .. G_7: exact integers below 2^24
            T += (long long)__float2int_rn(__uint_as_float(v[a][cc])) * (1ll << (40 - 8 * a));
          T += (long long)(__float2int_rn(__uint_as_float(v[kTcNacc - 1][cc])) >> 8);   // G_8 / 2^8, floor
          const unsigned long long u = (unsigned long long)(T < 0 ? -T : T);
          if (u != 0ull) {
            const int lz = __clzll((long long)u);
            const unsigned long long mant = u << lz;
            const int ex = s_fexp[c0 + cc] - lz;
            if (ex > best_e || (ex == best_e && mant > best_m)) {
              best_e = ex;
              best_m = mant;
            }
          }
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(b_accempty);
      if (valid) {
        double g = 0.0;
        if (e_i == kBadRow) g = __longlong_as_double(0x7ff8000000000000ll);
        else if (best_m != 0ull) g = ldexp((double)best_m, best_e + e_i - 56);
        atomicMax(p.gbits + row, (unsigned long long)__double_as_longlong(g));
      }
    }
  }
  __syncthreads();
  if (warp == 1) {
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, kTmemCols);
  }
}

// Per-row decision: grades clear of both thresholds by more than
// max(0.05 tau, bound) take their flags here; the others are listed for the
// FP64 re-check.  List appends and the running maximum are aggregated per
// warp (one atomic each).
__global__ void __launch_bounds__(256) tc_finalize_kernel(const unsigned long long* __restrict__ gbits, int64_t n,
                                                          const int* __restrict__ erow,
                                                          const int* __restrict__ fexp_max, double tau_sel,
                                                          double tau_brk, double* __restrict__ gamma,
                                                          uint8_t* __restrict__ flags,
                                                          unsigned long long* __restrict__ gmax_bits,
                                                          int32_t* __restrict__ list, unsigned* __restrict__ list_n) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const bool in = r < n;
  double g = 0.0;
  bool near = false;
  if (in) {
    g = __longlong_as_double((long long)gbits[r]);
    const int e = erow[r];
    gamma[r] = g;
    // 2^(e + F - 47) + 2^-52 g; exponents clamped to the normal range
    const int pe = (e == kBadRow) ? -1023 : max(-1022, min(1023, e + *fexp_max - 47));
    const double bound = (pe <= -1023) ? 0.0 : __longlong_as_double((long long)(pe + 1023) << 52) + g * 0x1p-52;
    near = !isfinite(g) || fabs(g - tau_sel) <= fmax(0.05 * tau_sel, bound) ||
           fabs(g - tau_brk) <= fmax(0.05 * tau_brk, bound);
    if (!near) flags[r] = (uint8_t)((g > tau_sel ? 1 : 0) | (g > tau_brk ? 2 : 0));
  }
  const unsigned listed = __ballot_sync(0xffffffffu, in && near);
  if (listed) {
    const int leader = __ffs(listed) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(list_n, (unsigned)__popc(listed));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (in && near) list[base + __popc(listed & ((1u << lane) - 1u))] = (int32_t)r;
  }
  double gm = (in && !near) ? g : 0.0;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) gm = fmax(gm, __shfl_down_sync(0xffffffffu, gm, o));
  if (lane == 0 && gm > 0.0) atomicMax(gmax_bits, (unsigned long long)__double_as_longlong(gm));
}

// ---------------------------------------------------------------------------
// Host launchers.

static int sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return 1;
  return n;
}

size_t tc_x_bytes(int64_t n_rows) { return (size_t)((n_rows + kTcM - 1) / kTcM) * kTcS * kXBytes; }
size_t tc_y_bytes() { return (size_t)2 * kTcS * kYBytes; }

#define MTP_TC_CHECK(what)                                              \
  do {                                                                  \
    cudaError_t e_ = cudaGetLastError();                                \
    if (e_ != cudaSuccess) {                                            \
      set_error("%s: %s", what, cudaGetErrorString(e_));                \
      return MTP_ERR_CUDA;                                              \
    }                                                                   \
  } while (0)

int tc_prepare(const double* rows, int64_t n, int m, const double* a_inv, const double* amax,
               unsigned long long* colmax, uint16_t* ys, int* fexp, int* dexp, int* fmax, uint16_t* xs, int* erow,
               int* status, cudaStream_t s) {
  if (m > kTcK) {
    set_error("tensor-core grade: m = %d exceeds %d", m, kTcK);
    return MTP_ERR_UNSUPPORTED;
  }
  if (n <= 0) return MTP_OK;
  MTP_TRY_CUDA(cudaMemsetAsync(colmax, 0, sizeof(unsigned long long) * kTcK, s));
  const int grid = (int)std::min<int64_t>(n, 4 * (int64_t)sm_count());
  tc_colmax_kernel<<<grid, kTcK, 0, s>>>(rows, n, m, colmax);
  MTP_TC_CHECK("tc_colmax_kernel");
  tc_dexp_kernel<<<1, kTcK, 0, s>>>(amax, colmax, m, dexp);
  MTP_TC_CHECK("tc_dexp_kernel");
  MTP_TRY_CUDA(cudaMemsetAsync(fmax, 0x80, sizeof(int), s));   // INT_MIN-like start for the maximum
  tc_prep_y_kernel<<<kTcK, kTcK, 0, s>>>(a_inv, m, dexp, ys, fexp, fmax, status);
  MTP_TC_CHECK("tc_prep_y_kernel");
  const int64_t tiles = (n + kTcM - 1) / kTcM;
  tc_split_x_kernel<<<(unsigned)tiles, kTcM, 0, s>>>(rows, n, m, dexp, xs, erow);
  MTP_TC_CHECK("tc_split_x_kernel");
  return MTP_OK;
}

int tc_gemm(const uint16_t* xs, const uint16_t* ys, const int* fexp, const int* erow, int64_t n,
            unsigned long long* gbits, int* status, float* dbg, cudaStream_t s) {
  if (n <= 0) return MTP_OK;
  const int64_t tiles = (n + kTcM - 1) / kTcM;
  if (tiles > INT_MAX / 2) {
    set_error("tensor-core grade: %lld rows exceed one launch", (long long)n);
    return MTP_ERR_ARG;
  }
  static bool attr_done = false;
  if (!attr_done) {
    cudaError_t e = cudaFuncSetAttribute(tc_grade_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmAlloc);
    if (e != cudaSuccess) {
      set_error("cudaFuncSetAttribute(tc_grade_kernel): %s", cudaGetErrorString(e));
      return MTP_ERR_CUDA;
    }
    attr_done = true;
  }
  MTP_TRY_CUDA(cudaMemsetAsync(gbits, 0, sizeof(unsigned long long) * (size_t)n, s));
  TcGemmArgs p;
  p.xs = xs;
  p.ys = ys;
  p.fexp = fexp;
  p.erow = erow;
  p.n_rows = n;
  p.n_tiles = (int)tiles;
  p.gbits = gbits;
  p.status = status;
  p.dbg = dbg;
  p.wait_ns = g_tc_wait_ns;
  const int per_half = (int)std::min<int64_t>(tiles, std::max(1, sm_count() / 2));
  tc_grade_kernel<<<2 * per_half, kTcThreads, kSmAlloc, s>>>(p);
  MTP_TC_CHECK("tc_grade_kernel");
  return MTP_OK;
}

int tc_finalize(const unsigned long long* gbits, int64_t n, const int* erow, const int* fmax, double tau_sel,
                double tau_brk, double* gamma, uint8_t* flags, unsigned long long* gmax_bits, int32_t* list,
                unsigned* list_n, cudaStream_t s) {
  if (n <= 0) return MTP_OK;
  tc_finalize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(gbits, n, erow, fmax, tau_sel, tau_brk, gamma,
                                                                  flags, gmax_bits, list, list_n);
  MTP_TC_CHECK("tc_finalize_kernel");
  return MTP_OK;
}

}  // namespace mtp

extern "C" int mtp_set_wait_limit(int64_t ns) {
  mtp::g_tc_wait_ns = ns < 0 ? mtp::kTcTimeoutNs : (uint64_t)ns;
  return MTP_OK;
}
