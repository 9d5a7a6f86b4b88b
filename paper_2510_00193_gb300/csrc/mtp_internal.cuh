// Internal definitions of the GB300 MTP library (not part of the C-ABI).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "mtp.h"

namespace mtp {

void set_error(const char* fmt, ...);

#define MTP_TRY_CUDA(call)                                                                      \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess) {                                                                    \
      mtp::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return e_ == cudaErrorMemoryAllocation ? MTP_ERR_OOM : MTP_ERR_CUDA;                      \
    }                                                                                           \
  } while (0)

// Device buffer that only grows.
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
  int ensure(size_t want);
  void release();
  template <class T> T* as() const { return static_cast<T*>(ptr); }
};

constexpr int kMaxSpecies = 16;
constexpr int kMaxQ = 16;
constexpr int kImageBias = 512;  // image components are stored as n + 512 in 10 bits each

__host__ __device__ inline int32_t pack_image(int n1, int n2, int n3) {
  return (int32_t)(((uint32_t)(n1 + kImageBias)) | ((uint32_t)(n2 + kImageBias) << 10) |
                   ((uint32_t)(n3 + kImageBias) << 20));
}
__host__ __device__ inline void unpack_image(int32_t p, int& n1, int& n2, int& n3) {
  uint32_t u = (uint32_t)p;
  n1 = (int)(u & 1023u) - kImageBias;
  n2 = (int)((u >> 10) & 1023u) - kImageBias;
  n3 = (int)((u >> 20) & 1023u) - kImageBias;
}

// Species index of atom i as the kernels use it: a value outside 0..S-1
// (reported through the status word by the entry point's checks) is read as
// species 0, so that no table lookup leaves its array.
__device__ __forceinline__ int species_at(const int32_t* z, int64_t i, int S) {
  const int v = __ldg(z + i);
  return (unsigned)v < (unsigned)S ? v : 0;
}

// Everything an energy/force launch needs, passed by value.
struct EfvArgs {
  int64_t atom_begin, atom_end, n_atoms;
  const int64_t* offsets;
  const int32_t* nbr_j;
  const int32_t* nbr_img;
  const double* x;          // FP64 path
  const long long* xq;      // mixed path: 32.32 fixed-point fractional coordinates [N][3]
  const int32_t* z;
  double cell[9];
  float cellf[9];
  int n_species, n_q, n_mu, m;
  double r_min, r_cut;
  const double* species_energy;
  const double* radial_d;   // [n_mu][n_q][S][S]
  const double* xi_d;
  const float* radial_f;
  const float* xi_f;
  double* e_atom;
  double* forces;
  float* forces_f;          // mixed path: FP32 force accumulator [N][3], converted at the end
  double* virial;
  double* e_total;
  double* dtheta;           // nullable
  int* status;
  void* mbuf;               // levels with component groups: moment and adjoint scratch
                            // [2][NCOMP][atom_end - atom_begin] in the working precision (nullptr: one fused kernel)
};

using EfvLaunch = int (*)(const EfvArgs&, int precision, bool want_dtheta, cudaStream_t);
// FP64 basis rows of listed atoms (list == nullptr: atoms atom_begin..), optional FP64 column sums.
using RowsLaunch = int (*)(const EfvArgs&, const int32_t* list, int64_t n_rows, double* rows, int64_t ld,
                           double* bsum, cudaStream_t);

struct BatchArgs;
using BatchLaunch = int (*)(const BatchArgs&, int precision, bool want_dtheta, int threads, cudaStream_t);
struct TangentArgs;
using TangentLaunch = int (*)(const TangentArgs&, int precision, cudaStream_t);

struct LevelEntry {
  int level;
  EfvLaunch efv;
  RowsLaunch rows;
  BatchLaunch batch;
  TangentLaunch tangent;
  int split_comps;   // components per atom of the EfvArgs::mbuf scratch (0: the level needs none)
  EfvLaunch team;    // warp-per-atom energy/force kernel (levels without component groups)
};

const LevelEntry* find_level(int level);

// Tensor-core grade (grade_tc.cu).
constexpr int kTcSlices = 7;      // BF16 slices per operand
constexpr int kTcMaxBasis = 128;  // padded basis size of the tensor-core product
size_t tc_x_bytes(int64_t n_rows);
size_t tc_y_bytes();
int tc_prepare(const double* rows, int64_t n, int m, const double* a_inv, const double* amax,
               unsigned long long* colmax, uint16_t* ys, int* fexp, int* dexp, int* fmax, uint16_t* xs, int* erow,
               int* status, cudaStream_t s);
int tc_gemm(const uint16_t* xs, const uint16_t* ys, const int* fexp, const int* erow, int64_t n,
            unsigned long long* gbits, int* status, float* dbg, cudaStream_t s);
int tc_finalize(const unsigned long long* gbits, int64_t n, const int* erow, const int* fmax, double tau_sel,
                double tau_brk, double* gamma, uint8_t* flags, unsigned long long* gmax_bits, int32_t* list,
                unsigned* list_n, cudaStream_t s);

}  // namespace mtp

struct mtp_handle {
  int device = 0;
  int level = 0, n_species = 0, n_q = 0, n_mu = 0, m = 0, n_comp = 0;
  double r_min = 0, r_cut = 0;
  int64_t n_params = 0;
  const mtp::LevelEntry* ops = nullptr;
  std::vector<double> h_species, h_radial, h_xi;
  mtp::DevBuf species, radial_d, xi_d, radial_f, xi_f, status;
  mtp::DevBuf xq;        // fixed-point positions scratch
  mtp::DevBuf forces_f;  // FP32 force accumulator (mixed path)
  mtp::DevBuf grade;     // grade scratch: counters, row maxima, column sums, FP64 basis rows
  mtp::DevBuf mbuf;      // moment/adjoint scratch of levels whose contraction is interpreted
  int efv_variant = 0;   // 0: tuned or by size, 1: thread per atom, 2: warp per atom
  int8_t tuned[2][64] = {};   // [precision][floor(log2 N)]: 0 untuned, else the faster variant
};

struct mtp_nlist {
  int device = 0;
  int64_t n_atoms = 0, n_pairs = 0;
  double r_cut = 0;
  double cell[9] = {0};
  int pbc[3] = {0, 0, 0};
  mtp::DevBuf offsets, nbr_j, nbr_img;
  mtp::DevBuf counts, bins, bin_start, bin_atoms, wrapped, status;
};
