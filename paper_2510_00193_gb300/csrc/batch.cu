// Batches of small periodic configurations: one neighbour list over all of
// them, and one persistent launch for energies, forces, virials and dE/dtheta
// of every configuration (the per-atom work is the single-configuration code).
//
// mtp_batch_create: per configuration, the exact FP64 list of every (j, n)
// with |x_j + n.H - x_i| < R_cut, the same decision expression as the single
// list; images are enumerated per pair over the box of n that the fractional
// difference allows, with j outermost and n1, n2, n3 ascending, which is the
// canonical order directly.
#include <cuda_runtime.h>
#include <cub/device/device_scan.cuh>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "batch_kernel.cuh"
#include "mtp_internal.cuh"

struct mtp_batch {
  int device = 0;
  int32_t n_cfg = 0;
  int64_t n_atoms = 0;
  int threads = 64;            // atoms per block of the persistent launch
  int32_t n_items = 0;
  std::vector<int64_t> h_off;
  std::vector<double> h_cells;
  mtp::DevBuf off, cells, items_cfg, items_begin, items_count, queue;
  mtp_nlist nl;
  mtp::DevBuf xq, forces_f, frac, work, eatom;
};

namespace mtp {

__global__ void batch_frac_kernel(const double* __restrict__ x, const int64_t* __restrict__ off, int n_cfg,
                                  const double* __restrict__ hinv, int64_t n, double* __restrict__ s,
                                  int32_t* __restrict__ cfg_of) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int lo = 0, hi = n_cfg - 1;
  while (lo < hi) {  // last configuration whose first atom <= i
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  const double* h = hinv + 9 * (int64_t)lo;
  const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
  s[3 * i] = px * h[0] + py * h[3] + pz * h[6];
  s[3 * i + 1] = px * h[1] + py * h[4] + pz * h[7];
  s[3 * i + 2] = px * h[2] + py * h[5] + pz * h[8];
  cfg_of[i] = lo;
}

// Fixed-point fractional coordinates with each atom's own cell (mixed path).
__global__ void batch_fixed_point_kernel(const double* __restrict__ s, const int32_t* __restrict__ z, int64_t n,
                                         int S, long long* __restrict__ out, int* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double k = 4294967296.0;
  const double s0 = s[3 * i], s1 = s[3 * i + 1], s2 = s[3 * i + 2];
  const int zi = z[i];
  const bool z_ok = zi >= 0 && zi < S;
  if (!z_ok) atomicCAS(status, 0, MTP_ERR_ARG);
  out[4 * i + 3] = z_ok ? (long long)zi : 0ll;   // out-of-range species read as 0 (reported above)
  if (!(fabs(s0) < 2147483647.0 && fabs(s1) < 2147483647.0 && fabs(s2) < 2147483647.0)) {
    atomicCAS(status, 0, MTP_ERR_NONFINITE);   // stored as the origin: no kernel reads undefined coordinates
    out[4 * i] = out[4 * i + 1] = out[4 * i + 2] = 0ll;
    return;
  }
  out[4 * i] = __double2ll_rn(s0 * k);
  out[4 * i + 1] = __double2ll_rn(s1 * k);
  out[4 * i + 2] = __double2ll_rn(s2 * k);
}

struct BatchNbrArgs {
  const double* x;
  const double* s;           // fractional coordinates [N][3]
  const int32_t* cfg_of;     // [N]
  const int64_t* off;        // [n_cfg + 1]
  const double* cells;       // [n_cfg][9]
  const double* reach;       // [n_cfg][3]: R_cut / plane spacing, with margin
  int pbc[3];
  double rc2;
  int64_t n;
  int* counts;
  const int64_t* offsets;
  int32_t* out_j;
  int32_t* out_img;
  int* status;
};

template <bool FILL>
__global__ void batch_pairs_kernel(const BatchNbrArgs g) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int c = g.cfg_of[i];
  const double* H = g.cells + 9 * (int64_t)c;
  const double* w = g.reach + 3 * (int64_t)c;
  const double xi = g.x[3 * i], yi = g.x[3 * i + 1], zi = g.x[3 * i + 2];
  const double si0 = g.s[3 * i], si1 = g.s[3 * i + 1], si2 = g.s[3 * i + 2];
  int found = 0;
  const int64_t base = FILL ? g.offsets[i] : 0;
  for (int64_t j = g.off[c]; j < g.off[c + 1]; ++j) {
    const double d0 = g.s[3 * j] - si0, d1 = g.s[3 * j + 1] - si1, d2 = g.s[3 * j + 2] - si2;
    // |d_k + n_k| <= R_cut / h_k for every image within the cutoff
    const int a0 = g.pbc[0] ? (int)ceil(-d0 - w[0]) : 0, b0 = g.pbc[0] ? (int)floor(-d0 + w[0]) : 0;
    const int a1 = g.pbc[1] ? (int)ceil(-d1 - w[1]) : 0, b1 = g.pbc[1] ? (int)floor(-d1 + w[1]) : 0;
    const int a2 = g.pbc[2] ? (int)ceil(-d2 - w[2]) : 0, b2 = g.pbc[2] ? (int)floor(-d2 + w[2]) : 0;
    for (int n1 = a0; n1 <= b0; ++n1)
      for (int n2 = a1; n2 <= b1; ++n2)
        for (int n3 = a2; n3 <= b2; ++n3) {
          const double sx = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, H[0]), __dmul_rn((double)n2, H[3])),
                                      __dmul_rn((double)n3, H[6]));
          const double sy = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, H[1]), __dmul_rn((double)n2, H[4])),
                                      __dmul_rn((double)n3, H[7]));
          const double sz = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, H[2]), __dmul_rn((double)n2, H[5])),
                                      __dmul_rn((double)n3, H[8]));
          const double dx = __dsub_rn(__dadd_rn(g.x[3 * j], sx), xi);
          const double dy = __dsub_rn(__dadd_rn(g.x[3 * j + 1], sy), yi);
          const double dz = __dsub_rn(__dadd_rn(g.x[3 * j + 2], sz), zi);
          const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
          if (r2 < g.rc2 && r2 > 0.0) {
            if (n1 < -511 || n1 > 511 || n2 < -511 || n2 > 511 || n3 < -511 || n3 > 511) {
              atomicCAS(g.status, 0, MTP_ERR_NEIGHBOR_OVERFLOW);
              continue;
            }
            if (FILL) {
              g.out_j[base + found] = (int32_t)j;
              g.out_img[base + found] = pack_image(n1, n2, n3);
            }
            ++found;
          }
        }
  }
  if (!FILL) g.counts[i] = found;
}

__global__ void widen_counts_batch(const int* __restrict__ c, int64_t n, int64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = c[i];
  if (i == n) out[n] = 0;
}

__global__ void forces_to_fp64_kernel(const float* __restrict__ f, int64_t n3, double* __restrict__ out);

static void invert3_host(const double* m, double* inv) {
  const double det = m[0] * (m[4] * m[8] - m[5] * m[7]) - m[1] * (m[3] * m[8] - m[5] * m[6]) +
                     m[2] * (m[3] * m[7] - m[4] * m[6]);
  inv[0] = (m[4] * m[8] - m[5] * m[7]) / det;
  inv[1] = (m[2] * m[7] - m[1] * m[8]) / det;
  inv[2] = (m[1] * m[5] - m[2] * m[4]) / det;
  inv[3] = (m[5] * m[6] - m[3] * m[8]) / det;
  inv[4] = (m[0] * m[8] - m[2] * m[6]) / det;
  inv[5] = (m[2] * m[3] - m[0] * m[5]) / det;
  inv[6] = (m[3] * m[7] - m[4] * m[6]) / det;
  inv[7] = (m[1] * m[6] - m[0] * m[7]) / det;
  inv[8] = (m[0] * m[4] - m[1] * m[3]) / det;
}

// Work items of at most `threads` atoms, each inside one configuration,
// largest first (the persistent blocks then finish close together).
static int build_items(mtp_batch* b, int threads) {
  std::vector<int32_t> cfg, cnt;
  std::vector<int64_t> beg;
  for (int32_t c = 0; c < b->n_cfg; ++c)
    for (int64_t a = b->h_off[c]; a < b->h_off[c + 1]; a += threads) {
      cfg.push_back(c);
      beg.push_back(a);
      cnt.push_back((int32_t)std::min<int64_t>(threads, b->h_off[c + 1] - a));
    }
  std::vector<size_t> order(cfg.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](size_t p, size_t q) { return cnt[p] > cnt[q]; });
  std::vector<int32_t> c2(cfg.size()), n2(cfg.size());
  std::vector<int64_t> b2(cfg.size());
  for (size_t k = 0; k < order.size(); ++k) {
    c2[k] = cfg[order[k]];
    b2[k] = beg[order[k]];
    n2[k] = cnt[order[k]];
  }
  const size_t n = std::max<size_t>(1, c2.size());
  int rc;
  if ((rc = b->items_cfg.ensure(sizeof(int32_t) * n)) || (rc = b->items_begin.ensure(sizeof(int64_t) * n)) ||
      (rc = b->items_count.ensure(sizeof(int32_t) * n)) || (rc = b->queue.ensure(sizeof(int32_t) * 4)))
    return rc;
  MTP_TRY_CUDA(cudaMemcpy(b->items_cfg.ptr, c2.data(), sizeof(int32_t) * c2.size(), cudaMemcpyHostToDevice));
  MTP_TRY_CUDA(cudaMemcpy(b->items_begin.ptr, b2.data(), sizeof(int64_t) * b2.size(), cudaMemcpyHostToDevice));
  MTP_TRY_CUDA(cudaMemcpy(b->items_count.ptr, n2.data(), sizeof(int32_t) * n2.size(), cudaMemcpyHostToDevice));
  b->n_items = (int32_t)c2.size();
  b->threads = threads;
  return MTP_OK;
}

}  // namespace mtp

using namespace mtp;

extern "C" {

void mtp_batch_free(mtp_batch* b) {
  if (!b) return;
  for (DevBuf* d : {&b->off, &b->cells, &b->items_cfg, &b->items_begin, &b->items_count, &b->queue, &b->xq,
                    &b->forces_f, &b->frac, &b->work, &b->eatom, &b->nl.offsets, &b->nl.nbr_j, &b->nl.nbr_img,
                    &b->nl.status})
    d->release();
  delete b;
}

int mtp_batch_create(mtp_handle* h, int32_t n_cfg, const int64_t* atom_off, const double* cells, const int32_t* pbc,
                     const double* x, int32_t atoms_per_block, mtp_batch** out, void* stream) {
  if (!h || !atom_off || !cells || !pbc || !out || n_cfg < 1) {
    set_error("mtp_batch_create: invalid argument");
    return MTP_ERR_ARG;
  }
  *out = nullptr;
  if (atom_off[0] != 0) {
    set_error("mtp_batch_create: atom_off[0] must be 0");
    return MTP_ERR_ARG;
  }
  for (int32_t c = 0; c < n_cfg; ++c)
    if (atom_off[c + 1] < atom_off[c]) {
      set_error("mtp_batch_create: atom_off must be non-decreasing");
      return MTP_ERR_ARG;
    }
  const int64_t n = atom_off[n_cfg];
  if (n > 0 && !x) {
    set_error("mtp_batch_create: NULL positions");
    return MTP_ERR_ARG;
  }
  if (n > 2147483647LL) {
    set_error("mtp_batch_create: too many atoms");
    return MTP_ERR_ARG;
  }
  if (atoms_per_block != 0 && (atoms_per_block < 32 || atoms_per_block > 256 || atoms_per_block % 32)) {
    set_error("mtp_batch_create: atoms_per_block must be 0 or a multiple of 32 in 32..256");
    return MTP_ERR_ARG;
  }
  mtp_batch* b = new (std::nothrow) mtp_batch();
  if (!b) {
    set_error("mtp_batch_create: out of host memory");
    return MTP_ERR_OOM;
  }
  cudaGetDevice(&b->device);
  b->n_cfg = n_cfg;
  b->n_atoms = n;
  b->h_off.assign(atom_off, atom_off + n_cfg + 1);
  b->h_cells.assign(cells, cells + 9 * (size_t)n_cfg);
  std::vector<double> hinv(9 * (size_t)n_cfg), reach(3 * (size_t)n_cfg);
  for (int32_t c = 0; c < n_cfg; ++c) {
    const double* H = cells + 9 * (size_t)c;
    const double det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                       H[2] * (H[3] * H[7] - H[4] * H[6]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) {
      mtp_batch_free(b);
      set_error("mtp_batch_create: cell of configuration %d is singular", c);
      return MTP_ERR_ARG;
    }
    invert3_host(H, &hinv[9 * (size_t)c]);
    for (int k = 0; k < 3; ++k) {
      const double* hv = &hinv[9 * (size_t)c];
      const double len = std::sqrt(hv[k] * hv[k] + hv[3 + k] * hv[3 + k] + hv[6 + k] * hv[6 + k]);
      reach[3 * (size_t)c + k] = h->r_cut * len * (1.0 + 1e-9) + 1e-9;   // R_cut / plane spacing
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  int rc;
  const size_t nn = (size_t)std::max<int64_t>(n, 1);
  if ((rc = b->off.ensure(sizeof(int64_t) * (n_cfg + 1))) || (rc = b->cells.ensure(sizeof(double) * 9 * n_cfg)) ||
      (rc = b->frac.ensure(sizeof(double) * 3 * nn + sizeof(int32_t) * nn)) ||
      (rc = b->work.ensure(sizeof(double) * (9 + 3) * n_cfg + sizeof(int) * nn + sizeof(int64_t) * (nn + 2) + 64))) {
    mtp_batch_free(b);
    return rc;
  }
  double* hinv_d = b->work.as<double>();
  double* reach_d = hinv_d + 9 * (size_t)n_cfg;
  int* counts = reinterpret_cast<int*>(reach_d + 3 * (size_t)n_cfg);
  int64_t* counts64 = reinterpret_cast<int64_t*>(
      (reinterpret_cast<uintptr_t>(counts + nn) + 15) & ~uintptr_t(15));
  double* sfrac = b->frac.as<double>();
  int32_t* cfg_of = reinterpret_cast<int32_t*>(sfrac + 3 * nn);
  cudaError_t e = cudaSuccess;
  if (!e) e = cudaMemcpy(b->off.ptr, atom_off, sizeof(int64_t) * (n_cfg + 1), cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(b->cells.ptr, cells, sizeof(double) * 9 * n_cfg, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(hinv_d, hinv.data(), sizeof(double) * 9 * n_cfg, cudaMemcpyHostToDevice);
  if (!e) e = cudaMemcpy(reach_d, reach.data(), sizeof(double) * 3 * n_cfg, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    mtp_batch_free(b);
    set_error("mtp_batch_create: copy failed: %s", cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  const unsigned blocks = (unsigned)((n + 127) / 128);
  if (n > 0) {
    batch_frac_kernel<<<blocks, 128, 0, s>>>(x, b->off.as<int64_t>(), n_cfg, hinv_d, n, sfrac, cfg_of);
  }
  BatchNbrArgs g;
  std::memset(&g, 0, sizeof(g));
  g.x = x;
  g.s = sfrac;
  g.cfg_of = cfg_of;
  g.off = b->off.as<int64_t>();
  g.cells = b->cells.as<double>();
  g.reach = reach_d;
  for (int k = 0; k < 3; ++k) g.pbc[k] = pbc[k] ? 1 : 0;
  g.rc2 = h->r_cut * h->r_cut;
  g.n = n;
  g.counts = counts;
  if ((rc = b->nl.status.ensure(sizeof(int) * 4)) != MTP_OK) {
    mtp_batch_free(b);
    return rc;
  }
  g.status = b->nl.status.as<int>();
  cudaMemsetAsync(g.status, 0, sizeof(int), s);
  if (n > 0) batch_pairs_kernel<false><<<blocks, 128, 0, s>>>(g);
  if ((rc = b->nl.offsets.ensure(sizeof(int64_t) * (n + 1))) != MTP_OK) {
    mtp_batch_free(b);
    return rc;
  }
  widen_counts_batch<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(counts, n, counts64);
  size_t tmp_bytes = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, counts64, b->nl.offsets.as<int64_t>(), (int)(n + 1), s);
  DevBuf tmp;
  if ((rc = tmp.ensure(tmp_bytes + 16)) != MTP_OK) {
    mtp_batch_free(b);
    return rc;
  }
  cub::DeviceScan::ExclusiveSum(tmp.ptr, tmp_bytes, counts64, b->nl.offsets.as<int64_t>(), (int)(n + 1), s);
  int64_t total = 0;
  int st = 0;
  e = cudaMemcpyAsync(&total, b->nl.offsets.as<int64_t>() + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaMemcpyAsync(&st, g.status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (!e) e = cudaStreamSynchronize(s);
  tmp.release();
  if (e != cudaSuccess) {
    mtp_batch_free(b);
    set_error("mtp_batch_create: neighbour count failed: %s", cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  if (st != 0) {
    mtp_batch_free(b);
    set_error("mtp_batch_create: a neighbour image exceeds +-511 cells");
    return MTP_ERR_NEIGHBOR_OVERFLOW;
  }
  b->nl.n_atoms = n;
  b->nl.n_pairs = total;
  b->nl.r_cut = h->r_cut;
  if ((rc = b->nl.nbr_j.ensure(sizeof(int32_t) * std::max<int64_t>(total, 1))) ||
      (rc = b->nl.nbr_img.ensure(sizeof(int32_t) * std::max<int64_t>(total, 1)))) {
    mtp_batch_free(b);
    return rc;
  }
  g.offsets = b->nl.offsets.as<int64_t>();
  g.out_j = b->nl.nbr_j.as<int32_t>();
  g.out_img = b->nl.nbr_img.as<int32_t>();
  if (n > 0) batch_pairs_kernel<true><<<blocks, 128, 0, s>>>(g);
  e = cudaGetLastError();
  if (!e) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    mtp_batch_free(b);
    set_error("mtp_batch_create: neighbour fill failed: %s", cudaGetErrorString(e));
    return MTP_ERR_CUDA;
  }
  if ((rc = b->xq.ensure(sizeof(long long) * 4 * nn)) || (rc = b->forces_f.ensure(sizeof(float) * 3 * nn)) ||
      (rc = b->eatom.ensure(sizeof(double) * nn)) ||
      (rc = build_items(b, atoms_per_block ? atoms_per_block : 64))) {
    mtp_batch_free(b);
    return rc;
  }
  *out = b;
  return MTP_OK;
}

int mtp_batch_nlist(const mtp_batch* b, const mtp_nlist** nl) {
  if (!b || !nl) {
    set_error("mtp_batch_nlist: NULL argument");
    return MTP_ERR_ARG;
  }
  *nl = &b->nl;
  return MTP_OK;
}

int mtp_compute_batch(mtp_handle* h, const mtp_batch* b, const double* x, const int32_t* z, int32_t precision,
                      double* e_cfg, double* e_atom, double* forces, double* virial, double* dtheta, void* stream) {
  if (!h || !b || !e_cfg || !forces || !virial || (b->n_atoms > 0 && (!x || !z))) {
    set_error("mtp_compute_batch: NULL argument");
    return MTP_ERR_ARG;
  }
  if (precision != MTP_FP64 && precision != MTP_MIXED) {
    set_error("mtp_compute_batch: precision must be MTP_FP64 or MTP_MIXED");
    return MTP_ERR_ARG;
  }
  if (!h->ops->batch) {
    set_error("mtp_compute_batch: level %d has no batch kernel", h->level);
    return MTP_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = b->n_atoms;
  MTP_TRY_CUDA(cudaMemsetAsync(e_cfg, 0, sizeof(double) * b->n_cfg, s));
  MTP_TRY_CUDA(cudaMemsetAsync(virial, 0, sizeof(double) * 6 * b->n_cfg, s));
  if (dtheta) MTP_TRY_CUDA(cudaMemsetAsync(dtheta, 0, sizeof(double) * h->n_params * b->n_cfg, s));
  MTP_TRY_CUDA(cudaMemsetAsync(b->queue.ptr, 0, sizeof(int32_t), s));
  if (precision == MTP_FP64 || n == 0) MTP_TRY_CUDA(cudaMemsetAsync(forces, 0, sizeof(double) * 3 * n, s));
  if (n == 0) return MTP_OK;
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  EfvArgs& e = a.base;
  e.n_atoms = n;
  e.offsets = b->nl.offsets.as<int64_t>();
  e.nbr_j = b->nl.nbr_j.as<int32_t>();
  e.nbr_img = b->nl.nbr_img.as<int32_t>();
  e.x = x;
  e.z = z;
  e.n_species = h->n_species;
  e.n_q = h->n_q;
  e.n_mu = h->n_mu;
  e.m = h->m;
  e.r_min = h->r_min;
  e.r_cut = h->r_cut;
  e.species_energy = h->species.as<double>();
  e.radial_d = h->radial_d.as<double>();
  e.xi_d = h->xi_d.as<double>();
  e.radial_f = h->radial_f.as<float>();
  e.xi_f = h->xi_f.as<float>();
  e.forces = forces;
  e.status = h->status.as<int>();
  e.e_atom = e_atom ? e_atom : b->eatom.as<double>();
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (precision == MTP_MIXED) {
    // fractional coordinates of the current positions, then fixed point
    double* hinv_d = reinterpret_cast<double*>(b->work.ptr);
    double* sfrac = reinterpret_cast<double*>(b->frac.ptr);
    int32_t* cfg_of = reinterpret_cast<int32_t*>(sfrac + 3 * n);
    batch_frac_kernel<<<blocks, 256, 0, s>>>(x, b->off.as<int64_t>(), b->n_cfg, hinv_d, n, sfrac, cfg_of);
    batch_fixed_point_kernel<<<blocks, 256, 0, s>>>(sfrac, z, n, h->n_species, b->xq.as<long long>(), e.status);
    MTP_TRY_CUDA(cudaGetLastError());
    e.xq = b->xq.as<long long>();
    e.forces_f = b->forces_f.as<float>();
    MTP_TRY_CUDA(cudaMemsetAsync(e.forces_f, 0, sizeof(float) * 3 * n, s));
  }
  a.item_cfg = b->items_cfg.as<int32_t>();
  a.item_begin = b->items_begin.as<int64_t>();
  a.item_count = b->items_count.as<int32_t>();
  a.n_items = b->n_items;
  a.queue = b->queue.as<int32_t>();
  a.cells = b->cells.as<double>();
  a.e_cfg = e_cfg;
  a.virial_cfg = virial;
  a.dtheta_cfg = dtheta;
  a.n_params = h->n_params;
  int rc = h->ops->batch(a, precision, dtheta != nullptr, b->threads, s);
  if (rc != MTP_OK) return rc;
  if (precision == MTP_MIXED) {
    forces_to_fp64_kernel<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(e.forces_f, 3 * n, forces);
    MTP_TRY_CUDA(cudaGetLastError());
  }
  return MTP_OK;
}

int mtp_batch_tune(mtp_handle* h, mtp_batch* b, const double* x, const int32_t* z, int32_t precision,
                   int32_t want_dtheta, int32_t* chosen, double* e_cfg, double* forces, double* virial,
                   double* dtheta, void* stream) {
  if (!h || !b) {
    set_error("mtp_batch_tune: NULL argument");
    return MTP_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0, e1;
  MTP_TRY_CUDA(cudaEventCreate(&e0));
  MTP_TRY_CUDA(cudaEventCreate(&e1));
  const int cand[] = {32, 64, 128, 256};
  int best = b->threads;
  float best_ms = 1e30f;
  int rc = MTP_OK;
  for (int t : cand) {
    if ((rc = build_items(b, t)) != MTP_OK) break;
    for (int rep = 0; rep < 2 && rc == MTP_OK; ++rep)   // warm-up
      rc = mtp_compute_batch(h, b, x, z, precision, e_cfg, nullptr, forces, virial, want_dtheta ? dtheta : nullptr,
                             stream);
    if (rc != MTP_OK) break;
    cudaEventRecord(e0, s);
    for (int rep = 0; rep < 3 && rc == MTP_OK; ++rep)
      rc = mtp_compute_batch(h, b, x, z, precision, e_cfg, nullptr, forces, virial, want_dtheta ? dtheta : nullptr,
                             stream);
    cudaEventRecord(e1, s);
    if (rc != MTP_OK) break;
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != MTP_OK) return rc;
  if ((rc = build_items(b, best)) != MTP_OK) return rc;
  if (chosen) *chosen = best;
  return MTP_OK;
}

}  // extern "C"
