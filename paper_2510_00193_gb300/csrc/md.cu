// On-device molecular dynamics with the MTP forces: velocity-Verlet (NVE)
// steps with a skin neighbour list that is filtered to the exact cutoff list
// every step.
//
// The paper measures the potential inside LAMMPS molecular dynamics: 100
// steps of 1 fs per run, throughput in atom-timesteps per second (Sec. 2.2,
// Fig. 3), and its examples run 1 fs MD (Sec. 3); the pair style receives a
// neighbour list from the MD engine (Sec. 2.3).  Here one step is
//   v += (dt/2) F/m;  x += dt v            (md_kick_drift_kernel)
//   exact list of x from the skin list     (md_filter_kernel, scan, md_compact_kernel)
//   F, E_pot = MTP(x)                      (the energy/force kernels)
//   v += (dt/2) F/m;  E_kin = sum m v^2/2  (md_kick_kernel)
// The skin list holds every pair within R_cut + skin of the positions at its
// last build; while no atom has moved more than skin/2 since then, it holds
// every pair within R_cut now.  The filter decides each listed pair with the
// same FP64 expression as the neighbour build (so the exact list equals a
// fresh build, entry for entry and in order), after an FP32 estimate whose
// rigorous error bound settles all pairs that are not within rounding
// distance of the cutoff.
#include <cub/device/device_scan.cuh>

#include <cmath>
#include <cstring>
#include <new>

#include "mtp_internal.cuh"

namespace mtp {

int build_neighbors(mtp_nlist* nl, const double* x, int64_t n, const double* cell, const int32_t* pbc, double r_cut,
                    cudaStream_t stream);

// LAMMPS metal units: 1 amu A^2 / ps^2 = 1.0364269e-4 eV; 1 eV/A^3 = 1.602176634e6 bar.
constexpr double kMvv2e = 1.0364269e-4;
constexpr double kEvA3ToBar = 1.602176634e6;

struct MdMass {
  double inv_m[kMaxSpecies];   // 1 / (m kMvv2e): eV/A -> A/ps^2
  double half_m[kMaxSpecies];  // m kMvv2e / 2: (A/ps)^2 -> eV
};

struct MdFilterGeom {
  double cell[9];
  float cellf[9];
  float hmax[3];   // max_c |H_kc| (FP32, rounded up)
  double rc2;
  float rc2_lo, rc2_hi;   // FP32 neighbours of R_cut^2: rc2_lo <= R_cut^2 <= rc2_hi
};

__global__ void md_kick_drift_kernel(double* __restrict__ x, double* __restrict__ v, const double* __restrict__ f,
                                     const int32_t* __restrict__ z, MdMass mm, double dt, int64_t n,
                                     const double* __restrict__ xref, double half_skin2, float4* __restrict__ xf,
                                     int* __restrict__ flags) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double a = mm.inv_m[min(max(z[i], 0), kMaxSpecies - 1)] * 0.5 * dt;   // species checked by the force pass
  double p[3];
  double d2 = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double vc = v[3 * i + c] + a * f[3 * i + c];
    v[3 * i + c] = vc;
    p[c] = x[3 * i + c] + dt * vc;
    x[3 * i + c] = p[c];
    const double u = p[c] - xref[3 * i + c];
    d2 += u * u;
  }
  if (!(d2 <= half_skin2)) atomicOr(flags, 1);   // moved beyond half the skin (or not finite)
  const double amax = fmax(fabs(p[0]), fmax(fabs(p[1]), fabs(p[2])));
  xf[i] = make_float4((float)p[0], (float)p[1], (float)p[2], __double2float_ru(amax));
}

__global__ void md_float_positions_kernel(const double* __restrict__ x, int64_t n, float4* __restrict__ xf) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double p0 = x[3 * i], p1 = x[3 * i + 1], p2 = x[3 * i + 2];
  const double amax = fmax(fabs(p0), fmax(fabs(p1), fabs(p2)));
  xf[i] = make_float4((float)p0, (float)p1, (float)p2, __double2float_ru(amax));
}

// Is the listed pair (i, j, image) within the cutoff now?  FP32 estimate of
// r^2 with a bound on its error, then, only where the bound cannot decide,
// the exact FP64 expression of the neighbour build:
//   s = (n1 a + n2 b) + n3 c,  d = (x_j + s) - x_i,  r^2 = (dx dx + dy dy) + dz dz,
// every operation rounded separately; keep iff 0 < r^2 < R_cut^2.
// Error of the estimate (u = 2^-24, A = max |x| of the atom, rounded up,
// S = sum_k |n_k| max_c |H_kc|): each FP32 pair-vector component is within
// delta = 8 u (A_i + A_j + S) of the exact one (two position roundings, the
// cell rounding, three roundings in the shift and two in the difference, each
// at most u times a magnitude below A_i + A_j + S), so
// |r^2_32 - r^2| <= 2 delta (|dx| + |dy| + |dz|) + 3 delta^2 + 4 u r^2_32;
// the bound is taken 1.25x and the last term 8 u r^2_32 (covering the bound's
// own FP32 evaluation and the rounding of r^2_32 +- bound).
__device__ __forceinline__ bool md_keep_pair(const double* __restrict__ x, const float4* __restrict__ xf,
                                             const MdFilterGeom& g, int64_t i, float4 pi, int32_t j, int32_t img) {
  int n1, n2, n3;
  unpack_image(img, n1, n2, n3);
  const float4 pj = xf[j];
  const float f1 = (float)n1, f2 = (float)n2, f3 = (float)n3;
  const float sx = fmaf(f3, g.cellf[6], fmaf(f2, g.cellf[3], f1 * g.cellf[0]));
  const float sy = fmaf(f3, g.cellf[7], fmaf(f2, g.cellf[4], f1 * g.cellf[1]));
  const float sz = fmaf(f3, g.cellf[8], fmaf(f2, g.cellf[5], f1 * g.cellf[2]));
  const float dx = (pj.x + sx) - pi.x, dy = (pj.y + sy) - pi.y, dz = (pj.z + sz) - pi.z;
  const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  const float S = fabsf(f1) * g.hmax[0] + fabsf(f2) * g.hmax[1] + fabsf(f3) * g.hmax[2];
  const float delta = 4.76837158203125e-7f * (pi.w + pj.w + S);   // 8 * 2^-24
  const float bound =
      1.25f * (2.0f * delta * (fabsf(dx) + fabsf(dy) + fabsf(dz)) + 3.0f * delta * delta) + 4.76837158203125e-7f * r2;
  if (r2 + bound < g.rc2_lo && r2 - bound > 0.0f) return true;
  if (r2 - bound > g.rc2_hi) return false;
  const double ex = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, g.cell[0]), __dmul_rn((double)n2, g.cell[3])),
                              __dmul_rn((double)n3, g.cell[6]));
  const double ey = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, g.cell[1]), __dmul_rn((double)n2, g.cell[4])),
                              __dmul_rn((double)n3, g.cell[7]));
  const double ez = __dadd_rn(__dadd_rn(__dmul_rn((double)n1, g.cell[2]), __dmul_rn((double)n2, g.cell[5])),
                              __dmul_rn((double)n3, g.cell[8]));
  const double ddx = __dsub_rn(__dadd_rn(x[3 * (int64_t)j], ex), x[3 * i]);
  const double ddy = __dsub_rn(__dadd_rn(x[3 * (int64_t)j + 1], ey), x[3 * i + 1]);
  const double ddz = __dsub_rn(__dadd_rn(x[3 * (int64_t)j + 2], ez), x[3 * i + 2]);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
  return d2 < g.rc2 && d2 > 0.0;
}

// One warp per atom: the lanes test 32 consecutive listed pairs at a time
// (coalesced list reads) and a ballot keeps the kept ones in list order,
// packed at the start of the atom's skin-list segment of tmp_j / tmp_img;
// counts[i] = their number (the warp of i = n writes counts[n] = 0 for the
// scan).
__global__ void md_filter_kernel(const double* __restrict__ x, const float4* __restrict__ xf, int64_t n, MdFilterGeom g,
                                 const int64_t* __restrict__ off, const int32_t* __restrict__ nj,
                                 const int32_t* __restrict__ nimg, int64_t* __restrict__ counts,
                                 int32_t* __restrict__ tmp_j, int32_t* __restrict__ tmp_img) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i == n && lane == 0) counts[n] = 0;
  if (i >= n) return;   // warp-uniform
  const float4 pi = xf[i];
  const int64_t beg = off[i], end = off[i + 1];
  int64_t w = beg;
  for (int64_t k0 = beg; k0 < end; k0 += 32) {
    const int64_t k = k0 + lane;
    bool keep = false;
    int32_t j = 0, im = 0;
    if (k < end) {
      j = nj[k];
      im = nimg[k];
      keep = md_keep_pair(x, xf, g, i, pi, j, im);
    }
    const unsigned mask = __ballot_sync(0xffffffffu, keep);
    if (keep) {
      const int64_t pos = w + __popc(mask & ((1u << lane) - 1u));
      tmp_j[pos] = j;
      tmp_img[pos] = im;
    }
    w += __popc(mask);
  }
  if (lane == 0) counts[i] = w - beg;
}

// One warp per atom: moves the kept pairs of atom i from its skin-list
// segment to out_off[i] in the exact list.
__global__ void md_compact_kernel(int64_t n, const int64_t* __restrict__ off, const int64_t* __restrict__ out_off,
                                  const int32_t* __restrict__ tmp_j, const int32_t* __restrict__ tmp_img,
                                  int32_t* __restrict__ out_j, int32_t* __restrict__ out_img) {
  const int lane = threadIdx.x & 31;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= n) return;
  const int64_t src = off[i], dst = out_off[i], cnt = out_off[i + 1] - dst;
  for (int64_t k = lane; k < cnt; k += 32) {
    out_j[dst + k] = tmp_j[src + k];
    out_img[dst + k] = tmp_img[src + k];
  }
}

__global__ void md_kick_kernel(double* __restrict__ v, const double* __restrict__ f, const int32_t* __restrict__ z,
                               MdMass mm, double dt, int64_t n, double* __restrict__ e_kin) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double ke = 0.0;
  if (i < n) {
    const int zi = min(max(z[i], 0), kMaxSpecies - 1);   // species checked by the force pass
    const double a = mm.inv_m[zi] * 0.5 * dt;
    double vv = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double vc = v[3 * i + c] + a * f[3 * i + c];
      v[3 * i + c] = vc;
      vv += vc * vc;
    }
    ke = mm.half_m[zi] * vv;
  }
  if (!e_kin) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ke += __shfl_down_sync(0xffffffffu, ke, o);
  __shared__ double part[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) part[warp] = ke;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += part[k];
    atomicAdd(e_kin, s);
  }
}

// Isotropic cell scaling of the Berendsen barostat: x *= mu and the
// reference positions of the skin list too (the displacement check then
// measures the motion relative to the affinely scaled build positions).
__global__ void md_scale_kernel(double* __restrict__ x, double* __restrict__ xref, double mu, int64_t n3) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n3) return;
  x[t] *= mu;
  xref[t] *= mu;
}

// Selection record of the in-run grade: selected[i] |= flags[i] (bit 0
// above the selection threshold, bit 1 above the break threshold at some
// evaluation) and counts[0] += atoms above the selection threshold now.
__global__ void md_select_kernel(const uint8_t* __restrict__ flags, int64_t n, uint8_t* __restrict__ selected,
                                 unsigned long long* __restrict__ count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool sel = i < n && (flags[i] & 1u);
  if (i < n && selected) selected[i] |= flags[i];
  const unsigned b = __ballot_sync(0xffffffffu, sel);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, (unsigned long long)__popc(b));
}

}  // namespace mtp

struct mtp_md {
  int device = 0;
  int64_t n_atoms = 0;
  double cell[9] = {0};
  int32_t pbc[3] = {0, 0, 0};
  double skin = 0, r_cut = 0;
  int64_t since_build = 0;
  int64_t rebuilds = 0;             // skin-list builds since creation (the first included)
  mtp_nlist* skin_list = nullptr;   // R_cut + skin, at the positions xref
  mtp_nlist* exact = nullptr;       // R_cut, at the current positions
  mtp::DevBuf xref;                 // positions at the last skin-list build [N][3]
  mtp::DevBuf xf;                   // FP32 positions and max |x| [N] float4
  mtp::DevBuf counts;               // int64 [N + 1] and the scan's temporary storage
  mtp::DevBuf tmp;                  // kept pairs at their skin-list positions: j, then image [2][P_skin]
  size_t scan_bytes = 0;
  mtp::DevBuf e_atom, small;        // site energies [N]; virial [6], E_pot [1], flags [1]
  mtp::MdFilterGeom geom;
  int64_t steps_total = 0;          // steps run since creation
  double scale_since_build = 1.0;   // product of barostat scale factors since the last skin-list build
  // in-run extrapolation grade (mtp_md_set_grade)
  const double* a_inv = nullptr;
  int32_t grade_every = 0, grade_method = 0;
  double tau_sel = 0, tau_brk = 0;
  uint8_t* selected = nullptr;
  mtp::DevBuf gamma, flags, sel_count;
  int64_t grade_evals = 0, n_selected_last = 0;
  double gamma_max_last = 0.0;
  // Berendsen barostat (mtp_md_set_barostat)
  double p_target = 0, tau_p = 0, modulus = 10.0;
  double pressure_last = 0.0;
  double bulk_modulus() const { return modulus; }
};

namespace {

using mtp::set_error;

void free_nlist_only(mtp_nlist* nl) {
  if (nl) mtp_free_nlist(nl);
}

// Cell-dependent parts of the filter geometry (the neighbour-list image
// shifts are n.H with the current H).
void md_set_cell(mtp_md* md, const double* cell) {
  mtp::MdFilterGeom& g = md->geom;
  for (int k = 0; k < 9; ++k) {
    md->cell[k] = cell[k];
    g.cell[k] = cell[k];
    g.cellf[k] = (float)cell[k];
  }
  for (int k = 0; k < 3; ++k) {
    double hm = 0.0;
    for (int c = 0; c < 3; ++c) hm = std::max(hm, std::fabs(cell[3 * k + c]));
    g.hmax[k] = (float)(hm * (1.0 + 1e-6));
  }
  if (md->exact)
    for (int k = 0; k < 9; ++k) md->exact->cell[k] = cell[k];
}

int md_filter(mtp_md* md, const double* x, cudaStream_t s) {
  using namespace mtp;
  const int64_t n = md->n_atoms;
  if (n == 0) return MTP_OK;
  const int T = 256;   // 8 atoms (warps) per block; n + 1 warps for the filter pass
  const unsigned blocks = (unsigned)((32 * (n + 1) + T - 1) / T);
  int64_t* counts = md->counts.as<int64_t>();
  void* tmp = reinterpret_cast<char*>(md->counts.ptr) + ((sizeof(int64_t) * (n + 1) + 255) & ~size_t(255));
  mtp_nlist* sl = md->skin_list;
  mtp_nlist* ex = md->exact;
  const int64_t cap = std::max<int64_t>(sl->n_pairs, 1);
  int32_t* tmp_j = md->tmp.as<int32_t>();
  int32_t* tmp_img = tmp_j + cap;
  md_filter_kernel<<<blocks, T, 0, s>>>(x, md->xf.as<float4>(), n, md->geom, sl->offsets.as<int64_t>(),
                                        sl->nbr_j.as<int32_t>(), sl->nbr_img.as<int32_t>(), counts, tmp_j, tmp_img);
  MTP_TRY_CUDA(cudaGetLastError());
  size_t tb = md->scan_bytes;
  MTP_TRY_CUDA(cub::DeviceScan::ExclusiveSum(tmp, tb, counts, ex->offsets.as<int64_t>(), (int)(n + 1), s));
  md_compact_kernel<<<blocks, T, 0, s>>>(n, sl->offsets.as<int64_t>(), ex->offsets.as<int64_t>(), tmp_j, tmp_img,
                                         ex->nbr_j.as<int32_t>(), ex->nbr_img.as<int32_t>());
  MTP_TRY_CUDA(cudaGetLastError());
  return MTP_OK;
}

int md_read_flags(mtp_md* md, cudaStream_t s, int* flags) {
  int* dflags = reinterpret_cast<int*>(md->small.as<double>() + 7);
  MTP_TRY_CUDA(cudaMemcpyAsync(flags, dflags, sizeof(int), cudaMemcpyDeviceToHost, s));
  MTP_TRY_CUDA(cudaStreamSynchronize(s));
  return MTP_OK;
}

int md_rebuild(mtp_handle* h, mtp_md* md, const double* x, cudaStream_t s) {
  using namespace mtp;
  const int64_t n = md->n_atoms;
  int rc = build_neighbors(md->skin_list, x, n, md->cell, md->pbc, md->r_cut + md->skin, s);
  if (rc != MTP_OK) return rc;
  md->skin_list->n_atoms = n;
  mtp_nlist* ex = md->exact;
  ex->n_atoms = n;
  ex->r_cut = md->r_cut;
  for (int k = 0; k < 9; ++k) ex->cell[k] = md->cell[k];
  for (int k = 0; k < 3; ++k) ex->pbc[k] = md->pbc[k];
  const int64_t cap = std::max<int64_t>(md->skin_list->n_pairs, 1);
  if ((rc = ex->offsets.ensure(sizeof(int64_t) * (n + 1))) != MTP_OK) return rc;
  if ((rc = ex->nbr_j.ensure(sizeof(int32_t) * cap)) != MTP_OK) return rc;
  if ((rc = ex->nbr_img.ensure(sizeof(int32_t) * cap)) != MTP_OK) return rc;
  if ((rc = md->tmp.ensure(2 * sizeof(int32_t) * cap)) != MTP_OK) return rc;
  ex->n_pairs = -1;   // known after the next synchronising query
  if (n > 0) {
    MTP_TRY_CUDA(cudaMemcpyAsync(md->xref.ptr, x, sizeof(double) * 3 * n, cudaMemcpyDeviceToDevice, s));
    md_float_positions_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, md->xf.as<float4>());
    MTP_TRY_CUDA(cudaGetLastError());
  }
  int* dflags = reinterpret_cast<int*>(md->small.as<double>() + 7);
  MTP_TRY_CUDA(cudaMemsetAsync(dflags, 0, sizeof(int), s));
  md->since_build = 0;
  md->rebuilds += 1;
  md->scale_since_build = 1.0;
  (void)h;
  return md_filter(md, x, s);
}

}  // namespace

extern "C" {

int mtp_md_create(mtp_handle* h, const double* x, int64_t n, const double* cell, const int32_t* pbc, double skin,
                  mtp_md** out, void* stream) {
  using namespace mtp;
  if (!h || !out || !cell || !pbc || n < 0 || (n > 0 && !x)) {
    set_error("mtp_md_create: invalid argument");
    return MTP_ERR_ARG;
  }
  if (!(skin >= 0.0) || !std::isfinite(skin)) {
    set_error("mtp_md_create: skin must be finite and >= 0 (got %g)", skin);
    return MTP_ERR_ARG;
  }
  if (n > 2147483647LL) {
    set_error("mtp_md_create: %lld atoms exceed the int32 index range", (long long)n);
    return MTP_ERR_ARG;
  }
  for (int k = 0; k < 9; ++k)
    if (!std::isfinite(cell[k])) {
      set_error("mtp_md_create: non-finite cell");
      return MTP_ERR_ARG;
    }
  mtp_md* md = new (std::nothrow) mtp_md();
  if (!md) {
    set_error("mtp_md_create: out of host memory");
    return MTP_ERR_OOM;
  }
  md->skin_list = new (std::nothrow) mtp_nlist();
  md->exact = new (std::nothrow) mtp_nlist();
  if (!md->skin_list || !md->exact) {
    mtp_md_free(md);
    set_error("mtp_md_create: out of host memory");
    return MTP_ERR_OOM;
  }
  cudaGetDevice(&md->device);
  md->skin_list->device = md->exact->device = md->device;
  md->n_atoms = n;
  md->skin = skin;
  md->r_cut = h->r_cut;
  for (int k = 0; k < 3; ++k) md->pbc[k] = pbc[k] ? 1 : 0;
  md_set_cell(md, cell);
  MdFilterGeom& g = md->geom;
  g.rc2 = h->r_cut * h->r_cut;
  g.rc2_lo = g.rc2_hi = (float)g.rc2;
  if ((double)g.rc2_lo > g.rc2) g.rc2_lo = std::nextafter(g.rc2_lo, 0.0f);
  if ((double)g.rc2_hi < g.rc2) g.rc2_hi = std::nextafter(g.rc2_hi, 3.0e38f);
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n1 = std::max<int64_t>(n, 1);
  int rc;
  size_t scan = 0;
  if (cub::DeviceScan::ExclusiveSum(nullptr, scan, (int64_t*)nullptr, (int64_t*)nullptr, (int)(n1 + 1), s) !=
      cudaSuccess) {
    mtp_md_free(md);
    set_error("mtp_md_create: scan sizing failed");
    return MTP_ERR_CUDA;
  }
  md->scan_bytes = scan;
  if ((rc = md->xref.ensure(sizeof(double) * 3 * n1)) != MTP_OK || (rc = md->xf.ensure(sizeof(float4) * n1)) != MTP_OK ||
      (rc = md->counts.ensure(((sizeof(int64_t) * (n1 + 1) + 255) & ~size_t(255)) + scan + 256)) != MTP_OK ||
      (rc = md->e_atom.ensure(sizeof(double) * n1)) != MTP_OK ||
      (rc = md->small.ensure(sizeof(double) * 12)) != MTP_OK) {
    mtp_md_free(md);
    return rc;
  }
  if ((rc = md_rebuild(h, md, x, s)) != MTP_OK) {
    mtp_md_free(md);
    return rc;
  }
  *out = md;
  return MTP_OK;
}

int mtp_md_rebuild(mtp_handle* h, mtp_md* md, const double* x, void* stream) {
  if (!h || !md || (md->n_atoms > 0 && !x)) {
    mtp::set_error("mtp_md_rebuild: invalid argument");
    return MTP_ERR_ARG;
  }
  return md_rebuild(h, md, x, (cudaStream_t)stream);
}

int mtp_md_nlist(mtp_md* md, const mtp_nlist** nl, void* stream) {
  if (!md || !nl) {
    mtp::set_error("mtp_md_nlist: invalid argument");
    return MTP_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  int64_t total = 0;
  if (md->n_atoms > 0) {
    MTP_TRY_CUDA(cudaMemcpyAsync(&total, md->exact->offsets.as<int64_t>() + md->n_atoms, sizeof(int64_t),
                                 cudaMemcpyDeviceToHost, s));
    MTP_TRY_CUDA(cudaStreamSynchronize(s));
  }
  md->exact->n_pairs = total;
  *nl = md->exact;
  return MTP_OK;
}

int mtp_md_status(mtp_md* md, int64_t* steps_since_build, int64_t* rebuilds, void* stream) {
  if (!md) {
    mtp::set_error("mtp_md_status: invalid argument");
    return MTP_ERR_ARG;
  }
  if (steps_since_build) *steps_since_build = md->since_build;
  if (rebuilds) *rebuilds = md->rebuilds;
  int flags = 0;
  int rc = md_read_flags(md, (cudaStream_t)stream, &flags);
  if (rc != MTP_OK) return rc;
  if (flags) {
    mtp::set_error("mtp_md: an atom moved more than skin/2 since the last list build; pairs may be missing "
                   "(rebuild more often or use a larger skin)");
    return MTP_ERR_STALE_LIST;
  }
  return MTP_OK;
}

int mtp_md_run(mtp_handle* h, mtp_md* md, double* x, double* v, const int32_t* z, const double* mass, double dt,
               int32_t n_steps, int32_t rebuild_every, int32_t precision, double* forces, double* e_pot,
               double* e_kin, void* stream) {
  using namespace mtp;
  if (!h || !md || !mass || n_steps < 0 ||
      (md->n_atoms > 0 && (!x || !v || !z || !forces))) {
    set_error("mtp_md_run: invalid argument");
    return MTP_ERR_ARG;
  }
  if (precision != MTP_FP64 && precision != MTP_MIXED) {
    set_error("mtp_md_run: precision must be MTP_FP64 or MTP_MIXED");
    return MTP_ERR_ARG;
  }
  if (!std::isfinite(dt)) {
    set_error("mtp_md_run: dt is not finite");
    return MTP_ERR_ARG;
  }
  MdMass mm;
  for (int k = 0; k < kMaxSpecies; ++k) mm.inv_m[k] = mm.half_m[k] = 0.0;
  for (int k = 0; k < h->n_species; ++k) {
    if (!(mass[k] > 0.0) || !std::isfinite(mass[k])) {
      set_error("mtp_md_run: mass of species %d must be positive and finite", k);
      return MTP_ERR_ARG;
    }
    mm.inv_m[k] = 1.0 / (mass[k] * kMvv2e);
    mm.half_m[k] = 0.5 * mass[k] * kMvv2e;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = md->n_atoms;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  double* small = md->small.as<double>();
  int* dflags = reinterpret_cast<int*>(small + 7);
  const bool npt = md->tau_p > 0.0;
  const bool graded = md->a_inv && md->grade_every > 0;
  int rc;
  for (int32_t step = 0; step < n_steps; ++step) {
    // half the skin, less what the barostat has compressed the cell by since
    // the last build: a pair beyond R_cut + skin then was at least
    // s (R_cut + skin) - 2 max|dx| away now (s the scale factor since the build)
    const double reach = md->scale_since_build * (md->r_cut + md->skin) - md->r_cut;
    const double half_skin = reach > 0.0 ? 0.5 * reach : 0.0;
    const double half_skin2 = half_skin * half_skin;
    if (rebuild_every > 0 && md->since_build >= rebuild_every) {
      int flags = 0;
      if ((rc = md_read_flags(md, s, &flags)) != MTP_OK) return rc;
      if (flags) return mtp_md_status(md, nullptr, nullptr, stream);
      if ((rc = md_rebuild(h, md, x, s)) != MTP_OK) return rc;
    }
    if (n > 0) {
      md_kick_drift_kernel<<<blocks, 256, 0, s>>>(x, v, forces, z, mm, dt, n, md->xref.as<double>(), half_skin2,
                                                  md->xf.as<float4>(), dflags);
      MTP_TRY_CUDA(cudaGetLastError());
    }
    bool rebuilt = false;
    if (rebuild_every < 0) {
      // displacement check of this step's positions: rebuild before the list is used
      int flags = 0;
      if ((rc = md_read_flags(md, s, &flags)) != MTP_OK) return rc;
      if (flags) {
        if ((rc = md_rebuild(h, md, x, s)) != MTP_OK) return rc;   // filters too
        rebuilt = true;
      }
    }
    if (!rebuilt && (rc = md_filter(md, x, s)) != MTP_OK) return rc;
    double* ep = e_pot ? e_pot + step : small + 6;
    rc = mtp_compute_efv(h, md->exact, x, z, n, md->cell, precision, 0, md->e_atom.as<double>(), forces, small, ep,
                         nullptr, stream);
    if (rc != MTP_OK) return rc;
    double* ek = e_kin ? e_kin + step : (npt ? small + 8 : nullptr);
    if (ek) MTP_TRY_CUDA(cudaMemsetAsync(ek, 0, sizeof(double), s));
    if (n > 0) {
      md_kick_kernel<<<blocks, 256, 0, s>>>(v, forces, z, mm, dt, n, ek);
      MTP_TRY_CUDA(cudaGetLastError());
    }
    md->since_build += 1;
    md->steps_total += 1;
    bool stop = false;
    if (graded && md->steps_total % md->grade_every == 0) {
      // extrapolation grade of this step's configuration (the positions and
      // exact list the forces were computed with), before any cell scaling
      double gmax = 0.0;
      rc = mtp_compute_grade(h, md->exact, x, z, n, md->cell, md->a_inv, nullptr, md->tau_sel, md->tau_brk, 0,
                             md->grade_method, md->gamma.as<double>(), md->flags.as<uint8_t>(), &gmax, nullptr,
                             nullptr, nullptr, stream);
      if (rc < 0) return rc;
      stop = rc == MTP_STATUS_BREAK;
      unsigned long long* cnt = md->sel_count.as<unsigned long long>();
      unsigned long long hc = 0;
      MTP_TRY_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), s));
      if (n > 0) {
        md_select_kernel<<<blocks, 256, 0, s>>>(md->flags.as<uint8_t>(), n, md->selected, cnt);
        MTP_TRY_CUDA(cudaGetLastError());
      }
      MTP_TRY_CUDA(cudaMemcpyAsync(&hc, cnt, sizeof(hc), cudaMemcpyDeviceToHost, s));
      MTP_TRY_CUDA(cudaStreamSynchronize(s));
      md->grade_evals += 1;
      md->gamma_max_last = gmax;
      md->n_selected_last = (int64_t)hc;
    }
    if (npt) {
      // Berendsen barostat, isotropic: P = (2 E_kin + tr W) / (3 V), then
      // x, the reference positions and the cell scale by
      // mu = (1 - dt / tau_p (P_target - P) / B)^(1/3)
      double hv[9];
      MTP_TRY_CUDA(cudaMemcpyAsync(hv, small, sizeof(double) * 9, cudaMemcpyDeviceToHost, s));
      MTP_TRY_CUDA(cudaStreamSynchronize(s));
      const double* H = md->cell;
      const double vol = std::fabs(H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                                   H[2] * (H[3] * H[7] - H[4] * H[6]));
      const double p_bar = (2.0 * hv[8] + hv[0] + hv[1] + hv[2]) / (3.0 * vol) * kEvA3ToBar;
      md->pressure_last = p_bar;
      const double mu3 = 1.0 - dt / md->tau_p * (md->p_target - p_bar) / md->bulk_modulus();
      if (!(mu3 > 0.0) || !std::isfinite(mu3)) {
        set_error("mtp_md_run: barostat scale factor^3 = %g (pressure %g bar); use a longer tau_p", mu3, p_bar);
        return MTP_ERR_NONFINITE;
      }
      const double mu = std::cbrt(mu3);
      double hn[9];
      for (int k = 0; k < 9; ++k) hn[k] = H[k] * mu;
      md_set_cell(md, hn);
      md->scale_since_build *= mu;
      if (n > 0) {
        md_scale_kernel<<<(unsigned)((3 * n + 255) / 256), 256, 0, s>>>(x, md->xref.as<double>(), mu, 3 * n);
        MTP_TRY_CUDA(cudaGetLastError());
      }
    }
    if (stop) return MTP_STATUS_BREAK;
  }
  if (rebuild_every > 0) return mtp_md_status(md, nullptr, nullptr, stream);
  return MTP_OK;
}

int mtp_md_set_grade(mtp_handle* h, mtp_md* md, const double* a_inv_dev, int32_t every, double tau_sel,
                     double tau_brk, int32_t method, uint8_t* selected_dev) {
  using namespace mtp;
  if (!h || !md) {
    set_error("mtp_md_set_grade: invalid argument");
    return MTP_ERR_ARG;
  }
  if (!a_inv_dev || every <= 0) {   // off
    md->a_inv = nullptr;
    md->grade_every = 0;
    md->selected = nullptr;
    return MTP_OK;
  }
  if (!(tau_sel > 0.0) || !(tau_brk >= tau_sel)) {
    set_error("mtp_md_set_grade: thresholds must satisfy 0 < tau_sel <= tau_brk");
    return MTP_ERR_ARG;
  }
  if (method != MTP_GRADE_TENSOR && method != MTP_GRADE_FP64) {
    set_error("mtp_md_set_grade: unknown method %d", (int)method);
    return MTP_ERR_ARG;
  }
  const int64_t n1 = std::max<int64_t>(md->n_atoms, 1);
  int rc;
  if ((rc = md->gamma.ensure(sizeof(double) * n1)) != MTP_OK || (rc = md->flags.ensure(n1)) != MTP_OK ||
      (rc = md->sel_count.ensure(sizeof(unsigned long long))) != MTP_OK)
    return rc;
  md->a_inv = a_inv_dev;
  md->grade_every = every;
  md->tau_sel = tau_sel;
  md->tau_brk = tau_brk;
  md->grade_method = method;
  md->selected = selected_dev;
  return MTP_OK;
}

int mtp_md_set_barostat(mtp_md* md, double p_target_bar, double tau_p_ps, double bulk_modulus_bar) {
  if (!md) {
    mtp::set_error("mtp_md_set_barostat: invalid argument");
    return MTP_ERR_ARG;
  }
  if (!(tau_p_ps > 0.0)) {   // off
    md->tau_p = 0.0;
    return MTP_OK;
  }
  if (!std::isfinite(p_target_bar) || !std::isfinite(tau_p_ps) || !(bulk_modulus_bar > 0.0) ||
      !std::isfinite(bulk_modulus_bar)) {
    mtp::set_error("mtp_md_set_barostat: need finite p_target, tau_p > 0 and bulk modulus > 0");
    return MTP_ERR_ARG;
  }
  md->p_target = p_target_bar;
  md->tau_p = tau_p_ps;
  md->modulus = bulk_modulus_bar;
  return MTP_OK;
}

int mtp_md_info(const mtp_md* md, int64_t* steps_total, int64_t* grade_evals, double* gamma_max_last,
                int64_t* n_selected_last, double* pressure_last_bar, double* cell) {
  if (!md) {
    mtp::set_error("mtp_md_info: invalid argument");
    return MTP_ERR_ARG;
  }
  if (steps_total) *steps_total = md->steps_total;
  if (grade_evals) *grade_evals = md->grade_evals;
  if (gamma_max_last) *gamma_max_last = md->gamma_max_last;
  if (n_selected_last) *n_selected_last = md->n_selected_last;
  if (pressure_last_bar) *pressure_last_bar = md->pressure_last;
  if (cell)
    for (int k = 0; k < 9; ++k) cell[k] = md->cell[k];
  return MTP_OK;
}

void mtp_md_free(mtp_md* md) {
  if (!md) return;
  free_nlist_only(md->skin_list);
  free_nlist_only(md->exact);
  md->xref.release();
  md->xf.release();
  md->counts.release();
  md->tmp.release();
  md->e_atom.release();
  md->small.release();
  md->gamma.release();
  md->flags.release();
  md->sel_count.release();
  delete md;
}

}  // extern "C"
