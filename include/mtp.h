/*
 * C-ABI of the GB300 Moment Tensor Potential library (libmtp_gb300.so).
 *
 * The library evaluates the Moment Tensor Potential (MTP) that the paper
 * accelerates inside LAMMPS: site energies, forces, the virial (stress), the
 * parameter gradient and the active-learning extrapolation grade (paper
 * Sec. 2.1: inference yields energies, forces and stresses; Sec. 2.1 and
 * Sec. 2.3: configuration- and neighbourhood-mode grades with a selection and
 * a break threshold).  The model itself is the published MTP the paper cites
 * (Shapeev 2016; MLIP-2/MLIP-3):
 *
 *   E_i = s[z_i] + sum_alpha xi_alpha B_alpha(i),  E = sum_i E_i,
 *   B_alpha: products of full contractions of the moment tensors
 *   M_{mu,nu}(i) = sum_j f_mu(|r_ij|) rhat_ij^{(x) nu},
 *   f_mu(r) = sum_k c[mu][k][z_i][z_j] T_k(xi(r)) (R_cut - r)^2.
 *
 * Conventions shared by every entry point
 *   - Units: Angstrom, eV, eV/Angstrom (LAMMPS "metal"); species are 0-based.
 *   - A cell is 9 doubles on the HOST, row-major, rows are the lattice vectors
 *     a, b, c; pbc[3] on the HOST, nonzero = periodic along that vector.
 *   - Positions x are [N][3] doubles in DEVICE memory, Cartesian, anywhere in
 *     space (they need not be wrapped into the cell).
 *   - Every array argument is owned by the caller and must stay valid until
 *     the work queued on `stream` has finished.  `stream` is a cudaStream_t
 *     passed as void* (NULL = legacy default stream).  Calls are asynchronous
 *     unless stated otherwise.
 *   - The library owns handles, neighbour lists and its internal scratch.
 *     A handle must not be used by two host threads or two streams at once.
 *   - Every function returns an mtp_status and never aborts; on failure
 *     mtp_last_error() gives a message (thread-local).
 *   - Virial order: xx, yy, zz, xy, xz, yz; W = -dE/d(strain), the LAMMPS
 *     pressure-virial convention.
 *   - Parameter vector theta (for gradients): [ s (S) | c (n_mu*n_q*S*S, in
 *     [mu][k][z_i][z_j] order) | xi (m) ].
 */
#ifndef MTP_GB300_H
#define MTP_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mtp_handle mtp_handle;
typedef struct mtp_nlist mtp_nlist;

typedef enum {
  MTP_OK = 0,
  MTP_STATUS_BREAK = 1,            /* grade above the break threshold (paper Sec. 2.3) */
  MTP_ERR_ARG = -1,                /* invalid argument (message says which) */
  MTP_ERR_CUDA = -2,               /* a CUDA call failed */
  MTP_ERR_OOM = -3,                /* device allocation failed */
  MTP_ERR_NEIGHBOR_OVERFLOW = -4,  /* a neighbour image lies beyond +-511 cells */
  MTP_ERR_NONFINITE = -5,          /* NaN/Inf in inputs or results */
  MTP_ERR_TIMEOUT = -6,            /* a device-side wait gave up */
  MTP_ERR_UNSUPPORTED = -7,        /* level not compiled into this library */
  MTP_ERR_STALE_LIST = -8          /* MD: an atom moved more than skin/2 since the list build */
} mtp_status;

typedef enum { MTP_FP64 = 0, MTP_MIXED = 1 } mtp_precision;

/* Potential parameters, all HOST pointers, copied by mtp_load_params. */
typedef struct {
  int32_t level;                 /* MTP level L (even, 2..20 compiled into the library) */
  int32_t n_species;             /* S >= 1 */
  int32_t n_q;                   /* radial basis size, 1..16 */
  double r_min, r_cut;           /* radial basis interval, 0 <= r_min < r_cut */
  const double* species_energy;  /* [S] */
  const double* radial;          /* [n_mu][n_q][S][S]; n_mu = (L - 2) / 4 + 1 */
  const double* xi;              /* [m] in the library's basis order (mtp_basis_table) */
  int64_t m;                     /* must equal the basis size of the level */
} mtp_params_desc;

/* Basis of a level, host only (no GPU needed).
 * Enumeration: all products of connected contraction graphs of moment tensors
 * with total level <= L, level(M_{mu,nu}) = 2 + 4 mu + nu, minus functions
 * linearly dependent on earlier ones.  m: basis size; n_mu: radial functions;
 * n_comp: symmetric moment components per atom; n_graph: connected graphs. */
int mtp_basis_info(int32_t level, int32_t* m, int32_t* n_mu, int32_t* n_comp, int32_t* n_graph);

/* Host-only export of the basis tables for bit-exact comparison.
 * which = 0: graphs, per graph: nv, mu[nv], e[nv(nv-1)/2] (upper triangle, row-major);
 * which = 1: basis functions, per function: n_factors, graph indices;
 * which = 2: per graph: n_terms, then per term: integer coefficient and per
 *            vertex (mu, a, b, c): the graph as a polynomial of the symmetric
 *            components M_mu[a,b,c] = sum_j f_mu rhat_x^a rhat_y^b rhat_z^c;
 * which = 3: moment components in kernel order, (mu, a, b, c) each.
 * Call with buf = NULL to get the length in *len; otherwise *len is the
 * capacity of buf on input and the number written on output. */
int mtp_basis_table(int32_t level, int32_t which, int64_t* buf, int64_t* len);

/* Copies the parameters to the current CUDA device.  *out receives a new
 * handle (free with mtp_free).  Fails with MTP_ERR_UNSUPPORTED for a level
 * this library was not built for, MTP_ERR_ARG if desc->m differs from the
 * basis size or a value is out of range. */
int mtp_load_params(const mtp_params_desc* desc, mtp_handle** out);
void mtp_free(mtp_handle* h);
/* Number of entries of theta (see the header comment). */
int mtp_param_count(const mtp_handle* h, int64_t* n_params);
/* Replaces the handle's parameters by theta_dev (DEVICE [n_params] FP64, the
 * theta layout of the header comment), queued on `stream`: later work on the
 * handle evaluates the new potential (the training loop of the paper's
 * MLIP-3 workflow changes theta between evaluations; Sec. 2.1).  A non-finite
 * entry is recorded in the device status word (mtp_device_status).
 * Asynchronous; theta_dev must stay valid until the copy has run. */
int mtp_set_theta(mtp_handle* h, const double* theta_dev, void* stream);

/* Full neighbour list (paper Sec. 2.3 needs a neighbour list; this one is
 * full, not half): every (j, n) with r_ij = x_j + n.H - x_i and
 * 0 < |r_ij|^2 < R_cut^2, n an image vector (zero on open axes), self images
 * included.  The squared distance is decided in FP64 as (dx*dx + dy*dy) +
 * dz*dz with d = (x_j + s) - x_i and s = (n1 a + n2 b) + n3 c, every
 * operation rounded separately.  Per atom the entries are sorted by
 * (j, n1, n2, n3).  R_cut comes from the handle.
 * *inout: NULL to create a list, or an existing list to rebuild in place
 * (its storage grows when needed).  Synchronises `stream` (the pair count
 * sizes the list).  MTP_ERR_NEIGHBOR_OVERFLOW if an image exceeds +-511. */
int mtp_build_neighbors(mtp_handle* h, const double* x_dev, int64_t n_atoms, const double* cell,
                        const int32_t* pbc, mtp_nlist** inout, void* stream);
int mtp_nlist_info(const mtp_nlist* nl, int64_t* n_atoms, int64_t* n_pairs);
/* Copies the list to caller DEVICE arrays: offsets [N+1] (int64), j [P]
 * (int32), images [P][3] (int32). */
int mtp_nlist_copy(const mtp_nlist* nl, int64_t* offsets_dev, int32_t* j_dev, int32_t* img_dev, void* stream);
void mtp_free_nlist(mtp_nlist* nl);

/* Energies, forces, virial and (optionally) dE/dtheta for one configuration.
 * x_dev [N][3], z_dev [N] (int32 species); nl built for these atoms (positions
 * may have moved since, the list is used as is).  cell: host [9], the current
 * cell (image shifts are n.H with this H).
 * precision: MTP_FP64, or MTP_MIXED (radial basis, moments, contractions and
 * the adjoint in FP32; pair vectors from 32.32 fixed-point fractional
 * coordinates; forces accumulated by FP32 atomics in a library-owned [N][3]
 * buffer and converted to FP64 once; site energies, the total energy, the
 * virial and dE/dtheta reduced in FP64 (per-thread and per-block partial sums
 * of the virial and dE/dtheta are FP32)).  Mixed-precision error: a site's
 * energy error grows with sum_alpha |xi_alpha B_alpha(i)|, the conditioning
 * of its basis sum (FP32 rounding times that sum).
 * chunk_atoms: centre atoms per launch (the chunk size of paper Sec. 2.3); 0 = all.
 * Outputs (DEVICE, overwritten): e_atom [N], forces [N][3], virial [6],
 * e_total [1]; dEdtheta [n_params] or NULL to skip the parameter gradient. */
int mtp_compute_efv(mtp_handle* h, const mtp_nlist* nl, const double* x_dev, const int32_t* z_dev,
                    int64_t n_atoms, const double* cell, int32_t precision, int64_t chunk_atoms,
                    double* e_atom_dev, double* forces_dev, double* virial_dev, double* e_total_dev,
                    double* dEdtheta_dev, void* stream);

/* Kernel for mtp_compute_efv (same results within rounding):
 *   1: one thread per centre atom (the thread-parallel variant, for large
 *      systems; paper Sec. 2.1, Table 1);
 *   2: one warp per centre atom, the warp's lanes sharing the atom's pairs
 *      (the block-parallel variant for small systems and high levels, paper
 *      Sec. 2.1, Table 1, Sec. 4); at levels 18 and 20 the warp also shares
 *      the interpreted contraction, level by level of its records;
 *   0 (default): the variant mtp_efv_tune measured faster for the atom count's
 *      power-of-two size class, else warp per atom up to 2048 atoms. */
int mtp_set_efv_variant(mtp_handle* h, int32_t variant);
/* Times both variants on this configuration (one warm-up and three timed
 * evaluations each, CUDA events on `stream`) and records the faster for its
 * precision and power-of-two size class in the handle.  chosen (HOST,
 * nullable): 1 or 2; ms (HOST [2], nullable): mean ms per evaluation of
 * each.  Allocates scratch outputs for
 * the call; synchronises `stream`. */
int mtp_efv_tune(mtp_handle* h, const mtp_nlist* nl, const double* x_dev, const int32_t* z_dev, int64_t n_atoms,
                 const double* cell, int32_t precision, int32_t* chosen, float* ms, void* stream);

/* Directional second derivatives, for the parameter gradient of a loss on
 * forces (double backward): with v_dev (DEVICE [N][3]) a direction of the
 * positions, dtheta_tan_dev [n_params] = d/dt dE/dtheta (x + t v) and
 * force_tan_dev [N][3] (nullable) = d/dt F(x + t v) = -H v.  For a
 * force-matching loss l = (1/3N) sum |F - F_t|^2 with v = F - F_t,
 * dl/dtheta = -(2/3N) dtheta_tan.  Forward-mode (dual-number) evaluation of
 * the energy/force code; species-energy entries are zero.  Asynchronous. */
int mtp_compute_efv_tangent(mtp_handle* h, const mtp_nlist* nl, const double* x_dev, const int32_t* z_dev,
                            int64_t n_atoms, const double* cell, int32_t precision, const double* v_dev,
                            double* dtheta_tan_dev, double* force_tan_dev, void* stream);

/* Extrapolation grade (paper Sec. 2.1: configuration and neighbourhood mode
 * with a selection and a break threshold; Sec. 2.3: select above tau_sel,
 * halt above tau_brk).  With b_i the basis row of atom i (the m basis
 * functions B_alpha of its neighbourhood):
 *   neighbourhood mode: gamma_i = max_k |(b_i A^-1)_k|, flags_i bit 0 =
 *     gamma_i > tau_sel, bit 1 = gamma_i > tau_brk;
 *   configuration mode: gamma_cfg = max_k |((sum_i b_i) A_cfg^-1)_k|.
 * a_inv_dev / a_inv_cfg_dev: DEVICE, m x m row-major FP64 inverses of the
 * active sets (either may be NULL, not both).  Basis rows are FP64;
 * chunk_atoms bounds the row scratch (0 = 262144).
 * method (neighbourhood mode):
 *   MTP_GRADE_TENSOR: the product on the BF16 tensor cores (tcgen05) by
 *     error-free splitting of both FP64 operands into 7 BF16 slices each
 *     (exact FP32 accumulation of every slice group), grade error at most
 *     2^-47 max|b_i D| max|D^-1 A^-1| + 2^-52 gamma_i for a power-of-two
 *     column balancing D; rows within max(5% of a threshold, that bound) of
 *     either threshold are re-checked in FP64 and take the FP64 grade and
 *     flags.  Needs m <= 128 (MTP_ERR_UNSUPPORTED otherwise).
 *   MTP_GRADE_FP64: every product in FP64 on the CUDA cores.
 * Outputs: gamma_dev [N] FP64 and flags_dev [N] uint8 (DEVICE, neighbourhood
 * mode); gamma_max, gamma_cfg, n_ambiguous, n_rechecked on the HOST
 * (nullable): n_ambiguous counts FP64 grades within their FP64 error bound of
 * a threshold, n_rechecked the rows the tensor-core method sent to FP64.
 * Synchronises `stream`.  Returns MTP_STATUS_BREAK when the largest grade
 * exceeds tau_brk, MTP_OK otherwise, or an error code (MTP_ERR_TIMEOUT if a
 * device-side wait of the tensor-core kernel gave up). */
typedef enum { MTP_GRADE_TENSOR = 0, MTP_GRADE_FP64 = 1 } mtp_grade_method;
int mtp_compute_grade(mtp_handle* h, const mtp_nlist* nl, const double* x_dev, const int32_t* z_dev,
                      int64_t n_atoms, const double* cell, const double* a_inv_dev, const double* a_inv_cfg_dev,
                      double tau_sel, double tau_brk, int64_t chunk_atoms, int32_t method, double* gamma_dev,
                      uint8_t* flags_dev, double* gamma_max, double* gamma_cfg, int64_t* n_ambiguous,
                      int64_t* n_rechecked, void* stream);

/* Grade of caller-given rows against an active set: gamma_r = max_k
 * |(b_r A^-1)_k|, with b_r = (rows_dev[r ld + c_0], ..., rows_dev[r ld +
 * c_{m-1}]), c_j = cols_dev[j] (DEVICE int32 [m]) or j when cols_dev is NULL
 * (then ld >= m); rows_dev DEVICE FP64 with row stride ld; a_inv_dev (DEVICE
 * [m][m] FP64) the inverse of the active set; flags_dev bit 0 = gamma_r >
 * tau_sel, bit 1 = gamma_r > tau_brk; all in FP64 (the kernel of
 * MTP_GRADE_FP64).  This is the configuration mode of the grade over the full
 * parameter gradient (paper Sec. 2.1; MLIP's configuration mode): b_r =
 * dE/dtheta of configuration r (from mtp_compute_efv or mtp_compute_batch,
 * ld = n_params) restricted to a set of linearly independent columns.  The
 * full gradient always has at least n_mu (n_mu + 1) / 2 exact linear
 * relations (E is
 * unchanged to first order when f_mu gains a multiple of f_nu, nu <= mu, and
 * xi compensates), so an active set over every column is singular; the
 * columns are chosen once, on the pool the active set is drawn from.
 * Outputs gamma_dev [n_rows], flags_dev [n_rows] (DEVICE); gamma_max and
 * n_ambiguous (HOST, nullable; the count of grades within 1e-12 sum_j |b_rj|
 * max_k |A^-1_jk| of a threshold).  m <= 16384.  Allocates 8 (m + 2) bytes of
 * scratch for the call; synchronises `stream`.  Returns MTP_STATUS_BREAK when
 * the largest grade exceeds tau_brk. */
int mtp_grade_rows(const double* rows_dev, int64_t n_rows, int64_t ld, const int32_t* cols_dev, int32_t m,
                   const double* a_inv_dev, double tau_sel, double tau_brk, double* gamma_dev, uint8_t* flags_dev,
                   double* gamma_max, int64_t* n_ambiguous, void* stream);

/* Verification hook for the tensor-core grade product (same kernel as
 * MTP_GRADE_TENSOR; the paper has no counterpart, it exists so that tests can
 * check the tensor-core arithmetic bit for bit).  Inputs, all DEVICE:
 *   xs_dev: BF16 bit patterns, [ceil(n_rows/128)][7][128 x 128] X slices in
 *     the kernel's operand layout: element (row i, column j) of a tile at
 *     (j/8)*1024 + (i/8)*64 + (i%8)*8 + j%8;
 *   ys_dev: [2][448 x 128] Y slices, per column half one operand whose row
 *     kg = 64 t + k is column k of slice t: element (kg, row j) at
 *     (j/8)*3584 + (kg/8)*64 + (kg%8)*8 + j%8;
 *   fexp_dev [128] column exponents, erow_dev [n_rows] row exponents.
 * Outputs (DEVICE): acc_dev (nullable) [n_rows][2][7][64] FP32 slice-group
 * sums G_d = sum_{s+t=d} X_s Y_t for d = 2..8 per column half;
 * gamma_bits_dev [n_rows] the FP64 bit patterns of the grades.
 * Synchronises `stream`; MTP_ERR_TIMEOUT if a device-side wait gave up
 * (mtp_set_wait_limit). */
int mtp_grade_tc_selftest(const uint16_t* xs_dev, const uint16_t* ys_dev, const int32_t* fexp_dev,
                          const int32_t* erow_dev, int64_t n_rows, float* acc_dev, uint64_t* gamma_bits_dev,
                          void* stream);

/* Limit, in nanoseconds, of each pipeline wait of the tensor-core grade
 * kernel (mbarrier waits between its copy, MMA and epilogue roles) for the
 * launches that follow; ns < 0 restores the default of 1 s.  A wait that runs
 * out sets MTP_ERR_TIMEOUT: the kernel then stops issuing work, waits (up to
 * 1 s, whatever this limit) for the copies and MMAs it has already issued,
 * frees its Tensor Memory and returns, so the context stays usable.  The
 * paper has no counterpart; the setting exists so that the timeout path can be
 * exercised by a test.  Process-wide, not thread-safe against concurrent
 * launches. */
int mtp_set_wait_limit(int64_t ns);

/* Batches of many small periodic configurations (for example thousands of
 * 8..256-atom cells), evaluated in one persistent launch.
 * mtp_batch_create: atom_off (HOST, n_cfg + 1, atom_off[0] = 0) splits the
 * concatenated atoms into configurations; cells (HOST, n_cfg x 9, rows a, b,
 * c per configuration); pbc (HOST, 3, for all); x_dev the positions used to
 * build the per-configuration neighbour lists (same definition and order as
 * mtp_build_neighbors, indices global).  atoms_per_block: 32..256 (multiple
 * of 32) or 0 for 64; mtp_batch_tune can pick it by timing.  Synchronises. */
typedef struct mtp_batch mtp_batch;
int mtp_batch_create(mtp_handle* h, int32_t n_cfg, const int64_t* atom_off, const double* cells,
                     const int32_t* pbc, const double* x_dev, int32_t atoms_per_block, mtp_batch** out,
                     void* stream);
/* The batch's combined neighbour list (owned by the batch). */
int mtp_batch_nlist(const mtp_batch* b, const mtp_nlist** nl);
/* Energies, forces, virials and (optionally) dE/dtheta of every
 * configuration.  Work items (configuration, up to atoms_per_block atoms) are
 * taken from a device counter by a grid of (SM count x resident blocks)
 * blocks.  Outputs (DEVICE, overwritten): e_cfg [n_cfg], e_atom [N] (or
 * NULL), forces [N][3], virial [n_cfg][6], dEdtheta [n_cfg][n_params] (or
 * NULL).  Asynchronous; allocates nothing. */
int mtp_compute_batch(mtp_handle* h, const mtp_batch* b, const double* x_dev, const int32_t* z_dev,
                      int32_t precision, double* e_cfg_dev, double* e_atom_dev, double* forces_dev,
                      double* virial_dev, double* dEdtheta_dev, void* stream);
/* Times mtp_compute_batch with 32, 64, 128 and 256 atoms per block (CUDA
 * events, after warm-up) and keeps the fastest (*chosen).  The outputs are
 * scratch for the trial runs.  Synchronises. */
int mtp_batch_tune(mtp_handle* h, mtp_batch* b, const double* x_dev, const int32_t* z_dev, int32_t precision,
                   int32_t want_dtheta, int32_t* chosen, double* e_cfg_dev, double* forces_dev,
                   double* virial_dev, double* dEdtheta_dev, void* stream);
void mtp_batch_free(mtp_batch* b);

/* Same evaluation as mtp_compute_efv with precision MTP_MIXED and no
 * parameter gradient, but the call allocates no device memory: its
 * scratch (fixed-point positions and an FP32 force accumulator) is a
 * 2.75 MiB array built into the library, so
 * n_atoms may be at most 65536 (larger n fails with MTP_ERR_ARG; use
 * mtp_compute_efv then).  For callers that must not have a library allocate
 * during a step: an MD engine that sets its whole device-memory budget at
 * start-up, or a loop where cudaMalloc's device-wide synchronisation would
 * stall other streams.  The paper has no counterpart; this entry point exists
 * for such callers only.  The first call on each device looks up the scratch
 * array's device address (cudaGetSymbolAddress, with that device current);
 * make that first call before any stream capture starts.  All calls on a
 * device share the scratch array, so calls that overlap on the GPU race:
 * issue them one after another.  Levels 18 and 20 run here as one fused
 * kernel (mtp_compute_efv splits them into three kernels through a scratch
 * buffer it allocates): same results, about 3.4x slower at level 20.
 * Arguments and outputs as mtp_compute_efv. */
int mtp_compute_efv_noalloc(mtp_handle* h, const mtp_nlist* nl, const double* x_dev, const int32_t* z_dev,
                            int64_t n_atoms, const double* cell, int64_t chunk_atoms, double* e_atom_dev,
                            double* forces_dev, double* virial_dev, double* e_total_dev, void* stream);

/* FP64 basis rows b_i = (B_1(i) .. B_m(i)) of every atom (the rows the
 * extrapolation grade multiplies by A^-1; paper Sec. 2.1), e.g. to build an
 * active-set pool for mtp_maxvol.  rows_dev: DEVICE [N][m] FP64, row-major,
 * in the library's basis order.  Asynchronous. */
int mtp_compute_basis_rows(mtp_handle* h, const mtp_nlist* nl, const double* x_dev, const int32_t* z_dev,
                           int64_t n_atoms, const double* cell, double* rows_dev, void* stream);

/* Active-set selection by MaxVol (Goreinov et al. 2010), the selection behind
 * the active set A of the extrapolation grade (paper Sec. 2.1 and Sec. 2.3:
 * configurations whose grade exceeds the selection threshold are selected for
 * the active set).  pool_dev: DEVICE [n_pool][m] FP64 rows; rows: HOST [m]
 * distinct pool indices, on entry the initial active rows, on return the
 * selected ones (rows[k] is the pool row in position k of A).  Repeats
 *   C = P A^-1, (i, k) = argmax |C_ik| (first in row-major order),
 *   stop if |C_ik| <= 1 + delta (or after max_iter swaps), else rows[k] = i,
 * with rank-one (Sherman-Morrison) updates of C and A^-1 and a fresh
 * Gauss-Jordan inverse (partial pivoting) every 32 swaps and before a stop is
 * accepted.  a_inv_dev: DEVICE [m][m] FP64, on return the inverse of the final
 * active rows.  iterations: HOST (nullable), the number of swaps.
 * m <= 4096.  MTP_ERR_ARG for invalid or duplicate rows or a singular active set,
 * MTP_ERR_NONFINITE for non-finite entries.  Allocates its scratch
 * (8 (n_pool m + 2 m^2) bytes and a little more) for the call; synchronises
 * `stream` once per swap. */
int mtp_maxvol(const double* pool_dev, int64_t n_pool, int32_t m, int32_t* rows, double delta, int32_t max_iter,
               double* a_inv_dev, int32_t* iterations, void* stream);

/* On-device molecular dynamics: velocity-Verlet (NVE) steps with the MTP
 * forces.  The paper measures the potential inside LAMMPS molecular dynamics
 * (100 steps of 1 fs per run, atom-timesteps per second: Sec. 2.2, Fig. 3;
 * 1 fs MD in the examples of Sec. 3), with the neighbour list the MD engine
 * hands to the pair style (Sec. 2.3).  One step is
 *   v += (dt/2) F/m,  x += dt v,  F = -dE/dx at the new x,  v += (dt/2) F/m.
 * Units: LAMMPS metal (x in A, v in A/ps, dt in ps, masses in amu, energies in
 * eV; 1 amu A^2/ps^2 = 1.0364269e-4 eV).
 * Neighbours: a skin list of every pair within R_cut + skin of the positions at
 * its last build; every step it is filtered to the exact R_cut list of the
 * current positions with the FP64 decision of mtp_build_neighbors (same
 * entries in the same order as a fresh build, as long as no atom has moved more
 * than skin/2 since the skin list was built).  Positions are never wrapped, so
 * the image vectors of the skin list stay valid between builds.
 *
 * mtp_md_create: builds the skin list of x_dev [N][3] (DEVICE) in the cell
 * (host [9]) with pbc (host [3]) and the exact list; the cell changes only
 * under the barostat (mtp_md_set_barostat; mtp_md_info returns it).
 * Synchronises `stream`.  Free with mtp_md_free. */
typedef struct mtp_md mtp_md;
int mtp_md_create(mtp_handle* h, const double* x_dev, int64_t n_atoms, const double* cell, const int32_t* pbc,
                  double skin, mtp_md** out, void* stream);
/* Rebuilds the skin list (and the exact list) at the positions x_dev.
 * Synchronises `stream`. */
int mtp_md_rebuild(mtp_handle* h, mtp_md* md, const double* x_dev, void* stream);
/* The exact neighbour list of the current positions (owned by md, valid until
 * the next call on md); usable with mtp_compute_efv, mtp_compute_grade and
 * mtp_nlist_copy.  Synchronises `stream` (it reads the pair count). */
int mtp_md_nlist(mtp_md* md, const mtp_nlist** nl, void* stream);
/* MTP_ERR_STALE_LIST if an atom has moved more than skin/2 from its position
 * at the last skin-list build (the exact lists since then may miss pairs),
 * else MTP_OK; *steps_since_build (HOST, nullable) counts the steps run on the
 * current skin list, *rebuilds (HOST, nullable) the skin-list builds since
 * creation (the first included).  Synchronises `stream`. */
int mtp_md_status(mtp_md* md, int64_t* steps_since_build, int64_t* rebuilds, void* stream);
/* Runs n_steps velocity-Verlet steps in place on x_dev and v_dev ([N][3]
 * DEVICE, FP64).  forces_dev [N][3] (DEVICE) holds on entry the forces at
 * x_dev (from mtp_compute_efv on the exact list, or from the previous
 * mtp_md_run) and on return the forces at the final positions.  mass: HOST
 * [S] in amu.  precision: MTP_FP64 or MTP_MIXED for the forces (the
 * integration itself is FP64).  e_pot_dev / e_kin_dev: DEVICE [n_steps]
 * (nullable), the potential and kinetic energy after each step.
 * rebuild_every < 0: after each drift the displacement check is read (one
 * synchronisation per step) and the skin list is rebuilt at once when an atom
 * has moved more than skin/2, so no step uses an incomplete list (the LAMMPS
 * default of checking every step).
 * rebuild_every > 0: the skin list is rebuilt after every rebuild_every steps
 * (the displacement check is read before each rebuild and at the end, which
 * synchronises; MTP_ERR_STALE_LIST stops the run).  rebuild_every = 0: no
 * rebuild and no synchronisation (the call only queues work, so it can be
 * captured in a CUDA graph once a first call has sized the scratch); check
 * with mtp_md_status. */
int mtp_md_run(mtp_handle* h, mtp_md* md, double* x_dev, double* v_dev, const int32_t* z_dev, const double* mass,
               double dt, int32_t n_steps, int32_t rebuild_every, int32_t precision, double* forces_dev,
               double* e_pot_dev, double* e_kin_dev, void* stream);
/* Extrapolation control inside mtp_md_run (paper Sec. 2.3: the grade is
 * evaluated every X steps of the MD run; configurations above the selection
 * threshold are kept for the active set and a grade above the break threshold
 * halts the run).  After every `every`-th step (counted since creation) the
 * neighbourhood grade of the current configuration is computed as
 * mtp_compute_grade does (a_inv_dev: DEVICE m x m FP64 inverse of the active
 * set, kept by reference; method MTP_GRADE_TENSOR or MTP_GRADE_FP64);
 * selected_dev (DEVICE [N] uint8, nullable) accumulates each atom's flags by
 * bitwise or (bit 0: grade above tau_sel, bit 1: above tau_brk at some
 * evaluation).  When the largest grade exceeds tau_brk, mtp_md_run returns
 * MTP_STATUS_BREAK right after that step (positions, velocities and forces
 * are those of the completed step).  Each evaluation synchronises the stream.
 * a_inv_dev = NULL or every <= 0 switches the grade off.  Allocates the
 * grade outputs (12 bytes per atom) once. */
int mtp_md_set_grade(mtp_handle* h, mtp_md* md, const double* a_inv_dev, int32_t every, double tau_sel,
                     double tau_brk, int32_t method, uint8_t* selected_dev);
/* Berendsen barostat for NPT runs (the paper's examples run NPT MD, Sec. 3),
 * isotropic: after each step the pressure P = (2 E_kin + W_xx + W_yy + W_zz) /
 * (3 V) (bar, from the FP64 virial of the step's forces) sets
 * mu = (1 - (dt / tau_p) (p_target - P) / bulk_modulus)^(1/3), and the
 * positions, the cell and the skin list's reference positions are scaled by
 * mu (the LAMMPS fix press/berendsen form, "iso" coupling; bulk modulus in
 * bar, LAMMPS default 10).  The skin criterion accounts for the compression
 * since the last build.  Each step then reads the pressure on the host (one
 * synchronisation per step).  tau_p_ps <= 0 switches it off (NVE). */
int mtp_md_set_barostat(mtp_md* md, double p_target_bar, double tau_p_ps, double bulk_modulus_bar);
/* Host-side record of the run (all nullable): steps run since creation,
 * grade evaluations, the largest grade and the number of atoms above tau_sel
 * at the last evaluation, the last barostat pressure (bar) and the current
 * cell (HOST [9]). */
int mtp_md_info(const mtp_md* md, int64_t* steps_total, int64_t* grade_evals, double* gamma_max_last,
                int64_t* n_selected_last, double* pressure_last_bar, double* cell);
void mtp_md_free(mtp_md* md);

/* Device status word of the handle: the first device-side error recorded
 * since the last call (non-finite site energy or force, ...), then cleared.
 * Synchronises `stream`. */
int mtp_device_status(mtp_handle* h, void* stream);

/* Human-readable message for the last failure on this thread. */
const char* mtp_last_error(void);

/* Measurement aid (no counterpart in the paper): the FMA throughput of the
 * current device, the denominator of the arithmetic roofline of the
 * energy/force kernels.  kind 0: FP32 fma; 1: FP64 fma; 2: packed FP32 pairs
 * (fma.rn.f32x2).  A kernel of blocks_per_sm (1..32) blocks of 256 threads
 * per SM runs iters x 16 x 8 dependent-in-8-chains multiply-adds per thread
 * once to warm up and once under CUDA events on the legacy default stream.
 * flops_per_s (HOST): 2 x multiply-adds / elapsed time; ms (HOST): elapsed
 * time.  Allocates and frees a small output buffer; synchronises the
 * device's default stream; changes no device setting. */
int mtp_probe_fma(int32_t kind, int64_t iters, int32_t blocks_per_sm, double* flops_per_s, double* ms);

#ifdef __cplusplus
}
#endif
#endif /* MTP_GB300_H */
