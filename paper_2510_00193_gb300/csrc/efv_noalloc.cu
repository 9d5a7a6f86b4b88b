// mtp_compute_efv_noalloc: the mixed-precision energy/force/virial evaluation
// without any device allocation inside the call.
//
// Why it exists.  mtp_compute_efv keeps its fixed-point position scratch in a
// buffer owned by the handle and grows it with cudaMalloc when a larger
// configuration arrives.  Some callers cannot let a library allocate at step
// time: an MD engine that lays out all of its device memory once at start-up
// under a fixed budget, or a time-stepping loop where the device-wide
// synchronisation that cudaMalloc implies would stall the other streams.
// This entry point uses a fixed scratch array compiled into the library
// instead; the caller still provides every input and output array.
//
// The scratch.  g_noalloc_scratch below is a file-scope __device__ array
// sized for kNoAllocMaxAtoms atoms: 32 bytes of fixed-point position and 12
// bytes of FP32 force accumulator per atom (2.75 MiB in all).  Every GPU that
// loads this library holds it until the process exits.  Host code cannot use
// the array's name as a device address (in host code it names a host-side
// stand-in), so the first call on each device looks the address up with
// cudaGetSymbolAddress, with that device current, and caches it.  Make that
// first call on a device before any stream capture starts.
//
// Levels 18 and 20.  mtp_compute_efv runs these levels as three kernels
// (moment sweep, contraction, adjoint sweep) through a moment scratch buffer
// that it allocates; with no buffer to hand, this entry point runs them as the
// one fused kernel (per-group neighbour sweeps, interpreted contraction in
// local memory), which gives the same results but is about 3.4x slower at
// level 20.
//
// Sharing.  All calls on a device share the one array and it keeps whatever
// the previous call wrote.  Each call overwrites the positions of all its
// atoms before reading them and clears the force accumulator of its atoms
// before adding to it.  Calls that overlap on the GPU (different streams or
// host threads at once) race on the array; issue them one after another.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "mtp_internal.cuh"

namespace mtp {

constexpr int64_t kNoAllocMaxAtoms = 65536;
constexpr int kNoAllocMaxDevices = 64;

// [4 * kNoAllocMaxAtoms] int64 positions, then [3 * kNoAllocMaxAtoms] floats
static __device__ __align__(256) long long g_noalloc_scratch[4 * kNoAllocMaxAtoms + 3 * kNoAllocMaxAtoms / 2];

__global__ void fixed_point_kernel(const double* __restrict__ x, const int32_t* __restrict__ z, int64_t n,
                                   double h0, double h1, double h2, double h3, double h4, double h5, double h6,
                                   double h7, double h8, int S, long long* __restrict__ out, int* __restrict__ status);
__global__ void forces_to_fp64_kernel(const float* __restrict__ f, int64_t n3, double* __restrict__ out);

static std::mutex g_noalloc_mutex;
static long long* g_noalloc_address[kNoAllocMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once).
static int noalloc_scratch(long long** out) {
  int dev = 0;
  MTP_TRY_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("mtp_compute_efv_noalloc: device %d is beyond the %d devices this entry point tracks", dev,
              kNoAllocMaxDevices);
    return MTP_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_address[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      set_error("mtp_compute_efv_noalloc: cudaGetSymbolAddress of the scratch array failed: %s",
                cudaGetErrorString(e));
      return MTP_ERR_CUDA;
    }
    g_noalloc_address[dev] = static_cast<long long*>(p);
  }
  *out = g_noalloc_address[dev];
  return MTP_OK;
}

}  // namespace mtp

using namespace mtp;

extern "C" int mtp_compute_efv_noalloc(mtp_handle* h, const mtp_nlist* nl, const double* x, const int32_t* z,
                                       int64_t n, const double* cell, int64_t chunk_atoms, double* e_atom,
                                       double* forces, double* virial, double* e_total, void* stream) {
  if (!h || !nl || !cell || !e_atom || !forces || !virial || !e_total || (n > 0 && (!x || !z))) {
    set_error("mtp_compute_efv_noalloc: NULL argument");
    return MTP_ERR_ARG;
  }
  if (n < 0 || n > kNoAllocMaxAtoms) {
    set_error("mtp_compute_efv_noalloc: %lld atoms, but the built-in scratch holds at most %lld; use "
              "mtp_compute_efv for larger configurations",
              (long long)n, (long long)kNoAllocMaxAtoms);
    return MTP_ERR_ARG;
  }
  if (n != nl->n_atoms) {
    set_error("mtp_compute_efv_noalloc: n_atoms = %lld but the list holds %lld", (long long)n,
              (long long)nl->n_atoms);
    return MTP_ERR_ARG;
  }
  if (chunk_atoms < 0) {
    set_error("mtp_compute_efv_noalloc: chunk_atoms < 0");
    return MTP_ERR_ARG;
  }
  const double det = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) -
                     cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) + cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
  if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) {
    set_error("mtp_compute_efv_noalloc: singular or non-finite cell");
    return MTP_ERR_ARG;
  }
  long long* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc != MTP_OK) return rc;

  cudaStream_t s = (cudaStream_t)stream;
  float* forces_f = reinterpret_cast<float*>(scratch + 4 * kNoAllocMaxAtoms);
  MTP_TRY_CUDA(cudaMemsetAsync(virial, 0, sizeof(double) * 6, s));
  MTP_TRY_CUDA(cudaMemsetAsync(e_total, 0, sizeof(double), s));
  if (n == 0) return MTP_OK;

  double hi[9];
  hi[0] = (cell[4] * cell[8] - cell[5] * cell[7]) / det;
  hi[1] = (cell[2] * cell[7] - cell[1] * cell[8]) / det;
  hi[2] = (cell[1] * cell[5] - cell[2] * cell[4]) / det;
  hi[3] = (cell[5] * cell[6] - cell[3] * cell[8]) / det;
  hi[4] = (cell[0] * cell[8] - cell[2] * cell[6]) / det;
  hi[5] = (cell[2] * cell[3] - cell[0] * cell[5]) / det;
  hi[6] = (cell[3] * cell[7] - cell[4] * cell[6]) / det;
  hi[7] = (cell[1] * cell[6] - cell[0] * cell[7]) / det;
  hi[8] = (cell[0] * cell[4] - cell[1] * cell[3]) / det;
  fixed_point_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, z, n, hi[0], hi[1], hi[2], hi[3], hi[4], hi[5],
                                                                 hi[6], hi[7], hi[8], h->n_species, scratch,
                                                                 h->status.as<int>());
  MTP_TRY_CUDA(cudaGetLastError());
  MTP_TRY_CUDA(cudaMemsetAsync(forces_f, 0, sizeof(float) * 3 * (size_t)n, s));

  EfvArgs a;
  std::memset(&a, 0, sizeof(a));
  a.n_atoms = n;
  a.offsets = nl->offsets.as<int64_t>();
  a.nbr_j = nl->nbr_j.as<int32_t>();
  a.nbr_img = nl->nbr_img.as<int32_t>();
  a.x = x;
  a.xq = scratch;
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
  a.species_energy = h->species.as<double>();
  a.radial_d = h->radial_d.as<double>();
  a.xi_d = h->xi_d.as<double>();
  a.radial_f = h->radial_f.as<float>();
  a.xi_f = h->xi_f.as<float>();
  a.e_atom = e_atom;
  a.forces = forces;
  a.forces_f = forces_f;
  a.virial = virial;
  a.e_total = e_total;
  a.dtheta = nullptr;
  a.status = h->status.as<int>();
  const int64_t chunk = chunk_atoms > 0 ? chunk_atoms : n;
  for (int64_t b = 0; b < n; b += chunk) {
    a.atom_begin = b;
    a.atom_end = b + chunk < n ? b + chunk : n;
    rc = h->ops->efv(a, MTP_MIXED, false, s);
    if (rc != MTP_OK) return rc;
  }
  forces_to_fp64_kernel<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(forces_f, 3 * n, forces);
  MTP_TRY_CUDA(cudaGetLastError());
  return MTP_OK;
}
