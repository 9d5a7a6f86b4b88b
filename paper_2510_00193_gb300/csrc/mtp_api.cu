// C-ABI entry points of the GB300 MTP library (declared in include/mtp.h).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "mtp_internal.cuh"
#include "mtp_tables.h"
#include "tangent_kernel.cuh"

namespace mtp {

static thread_local char g_err[1024] = "";

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int DevBuf::ensure(size_t want) {
  if (want <= bytes && ptr) return MTP_OK;
  release();
  cudaError_t e = cudaMalloc(&ptr, want);
  if (e != cudaSuccess) {
    ptr = nullptr;
    bytes = 0;
    set_error("cudaMalloc(%zu bytes): %s", want, cudaGetErrorString(e));
    return MTP_ERR_OOM;
  }
  bytes = want;
  return MTP_OK;
}

void DevBuf::release() {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
  bytes = 0;
}

static const tables::LevelTable* find_table(int level) {
  for (int k = 0; k < tables::kNumLevels; ++k)
    if (tables::kLevels[k].level == level) return &tables::kLevels[k];
  return nullptr;
}

int build_neighbors(mtp_nlist* nl, const double* x, int64_t n, const double* cell, const int32_t* pbc, double r_cut,
                    cudaStream_t stream);

// x (FP64) -> 32.32 fixed-point fractional coordinates s = x H^-1 (not
// wrapped: the pair difference plus the image is then exact), species in slot 3.
__global__ void fixed_point_kernel(const double* __restrict__ x, const int32_t* __restrict__ z, int64_t n,
                                   double h0, double h1, double h2, double h3, double h4, double h5, double h6,
                                   double h7, double h8, int S, long long* __restrict__ out, int* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double px = x[3 * i], py = x[3 * i + 1], pz = x[3 * i + 2];
  const double s0 = px * h0 + py * h3 + pz * h6;
  const double s1 = px * h1 + py * h4 + pz * h7;
  const double s2 = px * h2 + py * h5 + pz * h8;
  const double k = 4294967296.0;
  const double lim = 2147483647.0;
  const int zi = z[i];
  const bool z_ok = zi >= 0 && zi < S;
  if (!z_ok) atomicCAS(status, 0, MTP_ERR_ARG);
  out[4 * i + 3] = z_ok ? (long long)zi : 0ll;   // out-of-range species read as 0 (reported above)
  if (!(fabs(s0) < lim && fabs(s1) < lim && fabs(s2) < lim)) {
    // non-finite (or absurdly far) position: reported, stored as the origin so
    // that no kernel reads undefined coordinates
    atomicCAS(status, 0, MTP_ERR_NONFINITE);
    out[4 * i] = out[4 * i + 1] = out[4 * i + 2] = 0ll;
    return;
  }
  out[4 * i] = __double2ll_rn(s0 * k);
  out[4 * i + 1] = __double2ll_rn(s1 * k);
  out[4 * i + 2] = __double2ll_rn(s2 * k);
}

// Mixed path: the FP32 force accumulator converted to the FP64 output.
__global__ void forces_to_fp64_kernel(const float* __restrict__ f, int64_t n3, double* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n3) out[k] = (double)f[k];
}

__global__ void species_check_kernel(const int32_t* __restrict__ z, int64_t n, int S, int* __restrict__ status) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n && (z[i] < 0 || z[i] >= S)) atomicCAS(status, 0, MTP_ERR_ARG);
}

}  // namespace mtp

using namespace mtp;

namespace mtp {
// Below this many atoms an untuned handle takes the warp-per-atom kernel.
constexpr int64_t kTeamDefaultAtoms = 2048;
}  // namespace mtp

extern "C" {

const char* mtp_last_error(void) { return g_err; }

int mtp_basis_info(int32_t level, int32_t* m, int32_t* n_mu, int32_t* n_comp, int32_t* n_graph) {
  const tables::LevelTable* t = find_table(level);
  if (!t) {
    set_error("mtp_basis_info: level %d is not built into this library", level);
    return MTP_ERR_UNSUPPORTED;
  }
  if (m) *m = t->m;
  if (n_mu) *n_mu = t->nmu;
  if (n_comp) *n_comp = t->ncomp;
  if (n_graph) *n_graph = t->ngraph;
  return MTP_OK;
}

int mtp_basis_table(int32_t level, int32_t which, int64_t* buf, int64_t* len) {
  const tables::LevelTable* t = find_table(level);
  if (!t) {
    set_error("mtp_basis_table: level %d is not built into this library", level);
    return MTP_ERR_UNSUPPORTED;
  }
  if (!len) {
    set_error("mtp_basis_table: len is NULL");
    return MTP_ERR_ARG;
  }
  const int64_t* src;
  int64_t n;
  switch (which) {
    case 0: src = t->graphs; n = t->ngraphs_len; break;
    case 1: src = t->bases; n = t->nbases_len; break;
    case 2: src = t->poly; n = t->npoly_len; break;
    case 3: src = t->comps; n = t->ncomps_len; break;
    default: set_error("mtp_basis_table: which must be 0..3"); return MTP_ERR_ARG;
  }
  if (!buf) {
    *len = n;
    return MTP_OK;
  }
  if (*len < n) {
    set_error("mtp_basis_table: buffer holds %lld entries, %lld needed", (long long)*len, (long long)n);
    return MTP_ERR_ARG;
  }
  std::memcpy(buf, src, sizeof(int64_t) * n);
  *len = n;
  return MTP_OK;
}

int mtp_load_params(const mtp_params_desc* d, mtp_handle** out) {
  if (!d || !out) {
    set_error("mtp_load_params: NULL argument");
    return MTP_ERR_ARG;
  }
  *out = nullptr;
  const tables::LevelTable* t = find_table(d->level);
  const LevelEntry* ops = find_level(d->level);
  if (!t || !ops) {
    set_error("mtp_load_params: level %d is not built into this library", d->level);
    return MTP_ERR_UNSUPPORTED;
  }
  if (d->n_species < 1 || d->n_species > kMaxSpecies) {
    set_error("mtp_load_params: n_species = %d outside 1..%d", d->n_species, kMaxSpecies);
    return MTP_ERR_ARG;
  }
  if (d->n_q < 1 || d->n_q > kMaxQ) {
    set_error("mtp_load_params: n_q = %d outside 1..%d", d->n_q, kMaxQ);
    return MTP_ERR_ARG;
  }
  if (!(d->r_min >= 0.0) || !(d->r_cut > d->r_min) || !std::isfinite(d->r_cut)) {
    set_error("mtp_load_params: need 0 <= r_min < r_cut (got %g, %g)", d->r_min, d->r_cut);
    return MTP_ERR_ARG;
  }
  if (d->m != t->m) {
    set_error("mtp_load_params: m = %lld but level %d has %d basis functions", (long long)d->m, d->level, t->m);
    return MTP_ERR_ARG;
  }
  if (!d->species_energy || !d->radial || !d->xi) {
    set_error("mtp_load_params: NULL coefficient array");
    return MTP_ERR_ARG;
  }
  mtp_handle* h = new (std::nothrow) mtp_handle();
  if (!h) {
    set_error("mtp_load_params: out of host memory");
    return MTP_ERR_OOM;
  }
  cudaGetDevice(&h->device);
  h->level = d->level;
  h->n_species = d->n_species;
  h->n_q = d->n_q;
  h->n_mu = t->nmu;
  h->m = t->m;
  h->n_comp = t->ncomp;
  h->r_min = d->r_min;
  h->r_cut = d->r_cut;
  h->ops = ops;
  const int S = d->n_species;
  const int64_t nrad = (int64_t)h->n_mu * d->n_q * S * S;
  h->n_params = S + nrad + h->m;
  h->h_species.assign(d->species_energy, d->species_energy + S);
  h->h_radial.assign(d->radial, d->radial + nrad);
  h->h_xi.assign(d->xi, d->xi + h->m);
  for (double v : h->h_radial)
    if (!std::isfinite(v)) { delete h; set_error("mtp_load_params: non-finite radial coefficient"); return MTP_ERR_ARG; }
  for (double v : h->h_xi)
    if (!std::isfinite(v)) { delete h; set_error("mtp_load_params: non-finite xi"); return MTP_ERR_ARG; }
  std::vector<float> rf(h->h_radial.begin(), h->h_radial.end()), xf(h->h_xi.begin(), h->h_xi.end());
  int rc;
  if ((rc = h->species.ensure(sizeof(double) * S)) || (rc = h->radial_d.ensure(sizeof(double) * nrad)) ||
      (rc = h->xi_d.ensure(sizeof(double) * h->m)) || (rc = h->radial_f.ensure(sizeof(float) * nrad)) ||
      (rc = h->xi_f.ensure(sizeof(float) * h->m)) || (rc = h->status.ensure(sizeof(int) * 4))) {
    delete h;
    return rc;
  }
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMemcpy(h->species.ptr, h->h_species.data(), sizeof(double) * S, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->radial_d.ptr, h->h_radial.data(), sizeof(double) * nrad, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->xi_d.ptr, h->h_xi.data(), sizeof(double) * h->m, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->radial_f.ptr, rf.data(), sizeof(float) * nrad, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(h->xi_f.ptr, xf.data(), sizeof(float) * h->m, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(h->status.ptr, 0, sizeof(int) * 4);
  if (e != cudaSuccess) {
    set_error("mtp_load_params: copy to device failed: %s", cudaGetErrorString(e));
    delete h;
    return MTP_ERR_CUDA;
  }
  *out = h;
  return MTP_OK;
}

}  // extern "C"

namespace mtp {
// theta = [ s (S) | c (n_rad, [mu][k][zi][zj]) | xi (m) ] -> the handle's FP64
// and FP32 parameter copies; a non-finite entry sets the status word.
__global__ void set_theta_kernel(const double* __restrict__ theta, int S, int64_t nrad, int m,
                                 double* __restrict__ species, double* __restrict__ radial_d,
                                 double* __restrict__ xi_d, float* __restrict__ radial_f, float* __restrict__ xi_f,
                                 int* __restrict__ status) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t n = S + nrad + m;
  if (t >= n) return;
  const double v = theta[t];
  if (!isfinite(v)) atomicCAS(status, 0, MTP_ERR_NONFINITE);
  if (t < S) {
    species[t] = v;
  } else if (t < S + nrad) {
    radial_d[t - S] = v;
    radial_f[t - S] = (float)v;
  } else {
    xi_d[t - S - nrad] = v;
    xi_f[t - S - nrad] = (float)v;
  }
}
}  // namespace mtp

extern "C" {

int mtp_set_theta(mtp_handle* h, const double* theta_dev, void* stream) {
  using namespace mtp;
  if (!h || !theta_dev) {
    set_error("mtp_set_theta: invalid argument");
    return MTP_ERR_ARG;
  }
  const int S = h->n_species;
  const int64_t nrad = (int64_t)h->n_mu * h->n_q * S * S;
  set_theta_kernel<<<(unsigned)((h->n_params + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      theta_dev, S, nrad, h->m, h->species.as<double>(), h->radial_d.as<double>(), h->xi_d.as<double>(),
      h->radial_f.as<float>(), h->xi_f.as<float>(), h->status.as<int>());
  MTP_TRY_CUDA(cudaGetLastError());
  return MTP_OK;
}

void mtp_free(mtp_handle* h) {
  if (!h) return;
  h->species.release();
  h->radial_d.release();
  h->xi_d.release();
  h->radial_f.release();
  h->xi_f.release();
  h->status.release();
  h->xq.release();
  h->forces_f.release();
  h->grade.release();
  h->mbuf.release();
  delete h;
}

int mtp_param_count(const mtp_handle* h, int64_t* n) {
  if (!h || !n) {
    set_error("mtp_param_count: NULL argument");
    return MTP_ERR_ARG;
  }
  *n = h->n_params;
  return MTP_OK;
}

int mtp_build_neighbors(mtp_handle* h, const double* x, int64_t n, const double* cell, const int32_t* pbc,
                        mtp_nlist** inout, void* stream) {
  if (!h || !inout || !cell || !pbc || (n > 0 && !x) || n < 0) {
    set_error("mtp_build_neighbors: invalid argument");
    return MTP_ERR_ARG;
  }
  if (n > 2147483647LL) {
    set_error("mtp_build_neighbors: %lld atoms exceed the int32 index range", (long long)n);
    return MTP_ERR_ARG;
  }
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(cell[k])) {
      set_error("mtp_build_neighbors: non-finite cell");
      return MTP_ERR_ARG;
    }
  mtp_nlist* nl = *inout;
  bool created = false;
  if (!nl) {
    nl = new (std::nothrow) mtp_nlist();
    if (!nl) {
      set_error("mtp_build_neighbors: out of host memory");
      return MTP_ERR_OOM;
    }
    created = true;
  }
  cudaGetDevice(&nl->device);
  int rc = build_neighbors(nl, x, n, cell, pbc, h->r_cut, (cudaStream_t)stream);
  if (rc != MTP_OK) {
    if (created) mtp_free_nlist(nl);
    return rc;
  }
  *inout = nl;
  return MTP_OK;
}

int mtp_nlist_info(const mtp_nlist* nl, int64_t* n_atoms, int64_t* n_pairs) {
  if (!nl) {
    set_error("mtp_nlist_info: NULL list");
    return MTP_ERR_ARG;
  }
  if (n_atoms) *n_atoms = nl->n_atoms;
  if (n_pairs) *n_pairs = nl->n_pairs;
  return MTP_OK;
}

}  // extern "C"

namespace mtp {
__global__ void unpack_images_kernel(const int32_t* __restrict__ img, int64_t p, int32_t* __restrict__ out) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= p) return;
  int a, b, c;
  unpack_image(img[k], a, b, c);
  out[3 * k] = a;
  out[3 * k + 1] = b;
  out[3 * k + 2] = c;
}
}  // namespace mtp

extern "C" {

int mtp_nlist_copy(const mtp_nlist* nl, int64_t* offsets, int32_t* j, int32_t* img, void* stream) {
  if (!nl || !offsets || !j || !img) {
    set_error("mtp_nlist_copy: NULL argument");
    return MTP_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  MTP_TRY_CUDA(cudaMemcpyAsync(offsets, nl->offsets.ptr, sizeof(int64_t) * (nl->n_atoms + 1), cudaMemcpyDeviceToDevice, s));
  if (nl->n_pairs > 0) {
    MTP_TRY_CUDA(cudaMemcpyAsync(j, nl->nbr_j.ptr, sizeof(int32_t) * nl->n_pairs, cudaMemcpyDeviceToDevice, s));
    unpack_images_kernel<<<(unsigned)((nl->n_pairs + 255) / 256), 256, 0, s>>>(nl->nbr_img.as<int32_t>(), nl->n_pairs, img);
    MTP_TRY_CUDA(cudaGetLastError());
  }
  return MTP_OK;
}

void mtp_free_nlist(mtp_nlist* nl) {
  if (!nl) return;
  nl->offsets.release();
  nl->nbr_j.release();
  nl->nbr_img.release();
  nl->counts.release();
  nl->bins.release();
  nl->bin_start.release();
  nl->bin_atoms.release();
  nl->wrapped.release();
  nl->status.release();
  delete nl;
}

int mtp_compute_efv(mtp_handle* h, const mtp_nlist* nl, const double* x, const int32_t* z, int64_t n,
                    const double* cell, int32_t precision, int64_t chunk_atoms, double* e_atom, double* forces,
                    double* virial, double* e_total, double* dtheta, void* stream) {
  if (!h || !nl || !cell || !e_atom || !forces || !virial || !e_total || (n > 0 && (!x || !z))) {
    set_error("mtp_compute_efv: NULL argument");
    return MTP_ERR_ARG;
  }
  if (n != nl->n_atoms) {
    set_error("mtp_compute_efv: n_atoms = %lld but the list holds %lld", (long long)n, (long long)nl->n_atoms);
    return MTP_ERR_ARG;
  }
  if (precision != MTP_FP64 && precision != MTP_MIXED) {
    set_error("mtp_compute_efv: precision must be MTP_FP64 or MTP_MIXED");
    return MTP_ERR_ARG;
  }
  if (chunk_atoms < 0) {
    set_error("mtp_compute_efv: chunk_atoms < 0");
    return MTP_ERR_ARG;
  }
  {
    const double det = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) -
                       cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) +
                       cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) {
      set_error("mtp_compute_efv: singular or non-finite cell (det = %g)", det);
      return MTP_ERR_ARG;
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (precision == MTP_FP64 || n == 0) MTP_TRY_CUDA(cudaMemsetAsync(forces, 0, sizeof(double) * 3 * (size_t)n, s));
  MTP_TRY_CUDA(cudaMemsetAsync(virial, 0, sizeof(double) * 6, s));
  MTP_TRY_CUDA(cudaMemsetAsync(e_total, 0, sizeof(double), s));
  if (dtheta) MTP_TRY_CUDA(cudaMemsetAsync(dtheta, 0, sizeof(double) * h->n_params, s));
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
  a.species_energy = h->species.as<double>();
  a.radial_d = h->radial_d.as<double>();
  a.xi_d = h->xi_d.as<double>();
  a.radial_f = h->radial_f.as<float>();
  a.xi_f = h->xi_f.as<float>();
  a.e_atom = e_atom;
  a.forces = forces;
  a.virial = virial;
  a.e_total = e_total;
  a.dtheta = dtheta;
  a.status = h->status.as<int>();
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (precision == MTP_MIXED) {
    int rc = h->xq.ensure(sizeof(long long) * 4 * (size_t)n);
    if (rc != MTP_OK) return rc;
    double det = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) - cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) +
                 cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
    if (!(std::fabs(det) > 0.0)) {
      set_error("mtp_compute_efv: singular cell");
      return MTP_ERR_ARG;
    }
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
    fixed_point_kernel<<<blocks, 256, 0, s>>>(x, z, n, hi[0], hi[1], hi[2], hi[3], hi[4], hi[5], hi[6], hi[7], hi[8],
                                              h->n_species, h->xq.as<long long>(), a.status);
    MTP_TRY_CUDA(cudaGetLastError());
    a.xq = h->xq.as<long long>();
    if ((rc = h->forces_f.ensure(sizeof(float) * 3 * (size_t)n)) != MTP_OK) return rc;
    a.forces_f = h->forces_f.as<float>();
    MTP_TRY_CUDA(cudaMemsetAsync(a.forces_f, 0, sizeof(float) * 3 * (size_t)n, s));
  } else {
    species_check_kernel<<<blocks, 256, 0, s>>>(z, n, h->n_species, a.status);
    MTP_TRY_CUDA(cudaGetLastError());
  }
  const int64_t chunk = chunk_atoms > 0 ? chunk_atoms : n;
  // energy/force kernel: one thread per atom, or one warp per atom (small
  // systems); forced by mtp_set_efv_variant, else the tuned choice for this
  // size (mtp_efv_tune), else by size
  int variant = h->efv_variant;
  if (variant == 0) {
    const int bucket = std::min(63, (int)std::floor(std::log2((double)std::max<int64_t>(n, 1))));
    variant = h->tuned[precision == MTP_MIXED ? 1 : 0][bucket];
    if (variant == 0) variant = n <= kTeamDefaultAtoms ? 2 : 1;
  }
  if (h->ops->split_comps > 0 && n > 0 && variant == 1) {
    // moment/adjoint scratch of the split kernels (levels with an interpreted
    // contraction), bounded by the chunk as the paper's chunk size bounds memory
    const size_t bytes = 2 * (size_t)h->ops->split_comps * (size_t)std::min<int64_t>(chunk, n) *
                         (precision == MTP_MIXED ? sizeof(float) : sizeof(double));
    int rc = h->mbuf.ensure(bytes);
    if (rc != MTP_OK) return rc;
    a.mbuf = h->mbuf.ptr;
  }
  for (int64_t b = 0; b < n; b += chunk) {
    a.atom_begin = b;
    a.atom_end = b + chunk < n ? b + chunk : n;
    int rc = variant == 2 ? h->ops->team(a, precision, dtheta != nullptr, s)
                          : h->ops->efv(a, precision, dtheta != nullptr, s);
    if (rc != MTP_OK) return rc;
  }
  if (precision == MTP_MIXED) {
    forces_to_fp64_kernel<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(a.forces_f, 3 * n, forces);
    MTP_TRY_CUDA(cudaGetLastError());
  }
  return MTP_OK;
}

int mtp_set_efv_variant(mtp_handle* h, int32_t variant) {
  if (!h || variant < 0 || variant > 2) {
    set_error("mtp_set_efv_variant: variant must be 0 (auto), 1 (thread per atom) or 2 (warp per atom)");
    return MTP_ERR_ARG;
  }
  h->efv_variant = variant;
  return MTP_OK;
}

int mtp_efv_tune(mtp_handle* h, const mtp_nlist* nl, const double* x, const int32_t* z, int64_t n,
                 const double* cell, int32_t precision, int32_t* chosen, float* ms_out, void* stream) {
  if (!h || !nl || n <= 0 || (precision != MTP_FP64 && precision != MTP_MIXED)) {
    set_error("mtp_efv_tune: invalid argument");
    return MTP_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int saved = h->efv_variant;
  const int n_var = 2;
  double* buf = nullptr;
  MTP_TRY_CUDA(cudaMalloc(&buf, sizeof(double) * (4 * (size_t)n + 8)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float best = 0.f, t[2] = {0.f, 0.f};
  int win = 1, rc = MTP_OK;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) rc = MTP_ERR_CUDA;
  for (int v = 1; rc == MTP_OK && v <= n_var; ++v) {
    h->efv_variant = v;
    for (int rep = 0; rc == MTP_OK && rep < 4; ++rep) {   // one warm-up, three timed
      if (rep == 1 && cudaEventRecord(e0, s) != cudaSuccess) rc = MTP_ERR_CUDA;
      if (rc == MTP_OK)
        rc = mtp_compute_efv(h, nl, x, z, n, cell, precision, 0, buf, buf + n, buf + 4 * n, buf + 4 * n + 6, nullptr,
                             stream);
    }
    if (rc == MTP_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                         cudaEventElapsedTime(&t[v - 1], e0, e1) != cudaSuccess))
      rc = MTP_ERR_CUDA;
    if (rc == MTP_OK && (v == 1 || t[v - 1] < best)) {
      best = t[v - 1];
      win = v;
    }
  }
  h->efv_variant = saved;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (rc != MTP_OK) {
    if (rc == MTP_ERR_CUDA) set_error("mtp_efv_tune: timing failed");
    return rc;
  }
  const int bucket = std::min(63, (int)std::floor(std::log2((double)n)));
  h->tuned[precision == MTP_MIXED ? 1 : 0][bucket] = (int8_t)win;
  if (chosen) *chosen = win;
  if (ms_out) {
    ms_out[0] = t[0] / 3.f;
    ms_out[1] = n_var > 1 ? t[1] / 3.f : 0.f;
  }
  return MTP_OK;
}

int mtp_device_status(mtp_handle* h, void* stream) {
  if (!h) {
    set_error("mtp_device_status: NULL handle");
    return MTP_ERR_ARG;
  }
  int st = 0;
  cudaStream_t s = (cudaStream_t)stream;
  MTP_TRY_CUDA(cudaMemcpyAsync(&st, h->status.ptr, sizeof(int), cudaMemcpyDeviceToHost, s));
  MTP_TRY_CUDA(cudaMemsetAsync(h->status.ptr, 0, sizeof(int), s));
  MTP_TRY_CUDA(cudaStreamSynchronize(s));
  if (st != 0) {
    set_error(st == MTP_ERR_NONFINITE ? "device status: non-finite position, energy or force"
                                      : "device status: species index out of range");
  }
  return st;
}

}  // extern "C"

namespace mtp {
static int fill_efv_args(mtp_handle* h, const mtp_nlist* nl, const double* x, const int32_t* z, int64_t n,
                         const double* cell, EfvArgs& a) {
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
  a.species_energy = h->species.as<double>();
  a.radial_d = h->radial_d.as<double>();
  a.xi_d = h->xi_d.as<double>();
  a.radial_f = h->radial_f.as<float>();
  a.xi_f = h->xi_f.as<float>();
  a.status = h->status.as<int>();
  return MTP_OK;
}
}  // namespace mtp

extern "C" int mtp_compute_efv_tangent(mtp_handle* h, const mtp_nlist* nl, const double* x, const int32_t* z,
                                       int64_t n, const double* cell, int32_t precision, const double* v,
                                       double* dtheta_tan, double* force_tan, void* stream) {
  if (!h || !nl || !cell || !dtheta_tan || (n > 0 && (!x || !z || !v))) {
    set_error("mtp_compute_efv_tangent: NULL argument");
    return MTP_ERR_ARG;
  }
  if (n != nl->n_atoms) {
    set_error("mtp_compute_efv_tangent: n_atoms = %lld but the list holds %lld", (long long)n,
              (long long)nl->n_atoms);
    return MTP_ERR_ARG;
  }
  if (precision != MTP_FP64 && precision != MTP_MIXED) {
    set_error("mtp_compute_efv_tangent: precision must be MTP_FP64 or MTP_MIXED");
    return MTP_ERR_ARG;
  }
  if (!h->ops->tangent) {
    set_error("mtp_compute_efv_tangent: level %d has no tangent kernel", h->level);
    return MTP_ERR_UNSUPPORTED;
  }
  cudaStream_t s = (cudaStream_t)stream;
  MTP_TRY_CUDA(cudaMemsetAsync(dtheta_tan, 0, sizeof(double) * h->n_params, s));
  if (force_tan) MTP_TRY_CUDA(cudaMemsetAsync(force_tan, 0, sizeof(double) * 3 * (size_t)n, s));
  if (n == 0) return MTP_OK;
  TangentArgs t;
  std::memset(&t, 0, sizeof(t));
  fill_efv_args(h, nl, x, z, n, cell, t.base);
  t.v = v;
  t.dtheta_tan = dtheta_tan;
  t.force_tan = force_tan;
  if (precision == MTP_MIXED) {
    int rc = h->xq.ensure(sizeof(long long) * 4 * (size_t)n);
    if (rc != MTP_OK) return rc;
    double det = cell[0] * (cell[4] * cell[8] - cell[5] * cell[7]) - cell[1] * (cell[3] * cell[8] - cell[5] * cell[6]) +
                 cell[2] * (cell[3] * cell[7] - cell[4] * cell[6]);
    if (!(std::fabs(det) > 0.0)) {
      set_error("mtp_compute_efv_tangent: singular cell");
      return MTP_ERR_ARG;
    }
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
                                                                   hi[6], hi[7], hi[8], h->n_species,
                                                                   h->xq.as<long long>(), t.base.status);
    MTP_TRY_CUDA(cudaGetLastError());
    t.base.xq = h->xq.as<long long>();
  }
  t.base.atom_begin = 0;
  t.base.atom_end = n;
  if (h->ops->split_comps > 0 && n > 0) {
    // dual moments and adjoints of the split tangent kernels: 2 x components x atoms (value, tangent) pairs
    const size_t bytes = 4 * (size_t)h->ops->split_comps * (size_t)n *
                         (precision == MTP_MIXED ? sizeof(float) : sizeof(double));
    int rc = h->mbuf.ensure(bytes);
    if (rc != MTP_OK) return rc;
    t.base.mbuf = h->mbuf.ptr;
  }
  return h->ops->tangent(t, precision, s);
}
