/*
 * pmchwt.h -- C ABI of the GB300 proxy fast direct solver for 2-D Helmholtz
 * transmission scattering by many disjoint inclusions in the PMCHWT (Omit)
 * formulation (Y. Matsumoto, arXiv 2603.09381).
 *
 * Conventions
 *  - Every call returns pm_status; PM_OK == 0.  On any other status the call
 *    has produced no partial output, and pm_last_error() returns a message
 *    (thread-local, valid until the next call on the same thread).
 *  - Complex numbers are pm_c64 {re, im}, layout-compatible with complex128.
 *  - Unknowns and equations are ordered per inclusion, in input order.
 *    Inclusion j with n_j nodes owns 2 n_j consecutive entries:
 *      unknowns  phi_j = [q_j (n_j); u_j (n_j)]          (paper Sec. 2.2, phi_i)
 *      equations       = [u-equation rows; q-equation rows],
 *      plane-wave RHS f_j = [-u^I_j; -q^I_j]             (paper Sec. 2.2, f_i)
 *    where u is the total field on the boundary and q = (1/eps) du/dn its
 *    scaled normal derivative (paper Sec. 2.1, eqs. pressure and flux),
 *    N = sum_j 2 n_j.  Matrices and multi-RHS blocks are column-major.
 *  - Handles are owned by the library and released with the *_free calls
 *    (NULL-safe).  Factor handles are immutable after pm_factorize.
 *  - All compute runs on the current CUDA device; there is no CPU fallback.
 *    If no CUDA device is present the calls fail with PM_ERR_CUDA.
 */
#ifndef PMCHWT_H
#define PMCHWT_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PM_OK = 0,
  PM_ERR_INVALID_ARG = 1,   /* bad pointer, size, shape or option */
  PM_ERR_OOM = 2,           /* device or host allocation failed */
  PM_ERR_CUDA = 3,          /* CUDA runtime error (message names the call) */
  PM_ERR_SINGULAR = 4,      /* exactly singular pivot in an LU, or R A^{-1} L singular */
  PM_ERR_NOT_CONVERGED = 5, /* PM_MIXED: refinement stopped above refine_tol after max_refine steps */
  PM_ERR_TIMEOUT = 6,       /* a bounded device wait ran out (tensor-core completion, chained solve) */
  PM_ERR_GEOMETRY = 7,      /* inclusions not on a grid, two in one cell, ... */
  PM_ERR_UNSUPPORTED = 8    /* valid input the library does not handle yet */
} pm_status;

typedef struct { double re, im; } pm_c64;

enum { PM_CIRCLE = 0, PM_ELLIPSE = 1, PM_STAR = 2, PM_FOURIER = 3 };
enum { PM_FP64 = 0, PM_MIXED = 1 };

/* One inclusion (paper Sec. 2.1: Omega_j with smooth boundary Gamma_j).
 * Boundary x(t) = (cx, cy) + Rot(rot) rho(t), t in [0, 2 pi), counter-clockwise:
 *   PM_CIRCLE : prm[0] = a;                     rho = a (cos t, sin t)
 *   PM_ELLIPSE: prm[0] = a, prm[1] = b;         rho = (a cos t, b sin t)
 *   PM_STAR   : prm[0] = r0, prm[1] = e, prm[2] = p;  r(t) = r0 (1 + e cos(p t))
 *   PM_FOURIER: prm[0] = r0, prm[1..5] = a_2..a_6, prm[6..10] = phi_2..phi_6;
 *               r(t) = r0 (1 + sum_m a_m cos(m t + phi_m)),  rho = r(t) (cos t, sin t)
 * n_nodes: Nystrom nodes t_l = 2 pi l / n (paper Sec. 2.2), even, 16..4096.
 * k_in: interior wavenumber k^- (eps^- = (k^-/k^+)^2, eps^+ = 1); Re k_in > 0,
 * Im k_in >= 0 (a lossy interior), else PM_ERR_INVALID_ARG. */
typedef struct {
  int32_t shape;
  double cx, cy, rot;
  double prm[16];
  int32_t n_nodes;
  pm_c64 k_in;
} pm_inclusion;

/* m inclusions on a grid of spacing `spacing` (paper Sec. 4: inclusions on a
 * regular grid, each one a leaf cell), or with spacing = 0 anywhere (Sec.
 * 4.4's general arrangements): the quadtree then covers the bounding square
 * of the centres, deep enough (up to 20 levels) for one centre per finest
 * cell, a leaf's proxy circle around its inclusion and a parent's around its
 * cell; the near lists keep every inclusion with a node inside a box's proxy
 * circle.  Inclusions must not overlap.  k_out = k^+ = omega (eps^+ = 1). */
typedef struct {
  int32_t m;
  const pm_inclusion* inc;
  double k_out;
  int32_t grid_nx, grid_ny;
  double spacing;
} pm_problem;

typedef struct pm_geometry pm_geometry;
typedef struct pm_factor pm_factor;

/* Factorization options.
 * tol: CPQR threshold epsilon; a column is kept while |R_jj| > tol |R_11|
 *      (paper Sec. 3, adaptive rank).  Must be in (0, 1).
 * proxy_factor: proxy circle radius / cell radius (> 1; default 1.5).
 * proxy_points: points on every proxy circle; 0 selects
 *      p = max(32, 8 ceil((2 k^+ R_p + ceil(ln(1/tol)/ln(proxy_factor)))/8)).
 * precision: PM_FP64 (everything complex128), or PM_MIXED: the levels are
 *      factored in complex64 with ID threshold max(tol, low_tol) and serve as a
 *      preconditioner, and pm_solve refines the solution against the
 *      complex128 operator (no counterpart in the paper).  The top-level
 *      system is assembled in complex128 and factored in complex64 (its
 *      rounding stays far below the levels' ID threshold); PM_FLAG_TOP_FP64
 *      factors it in complex128.  pm_factorize assembles the dense
 *      complex128 operator on a low-priority stream concurrently with the
 *      complex64 factorization, from the end of the leaf level's assembly
 *      (one persistent CTA of 128 threads per SM);
 *      PM_FLAG_OPERATOR_AFTER assembles it after the factorization instead
 *      (pm_factor_batch always does).
 * stream: cudaStream_t to run on, or NULL for the default stream.
 * flags: PM_FLAG_PROFILE records per-kernel timings.  PM_MIXED writes the
 *      complex128 operator out densely (N^2 x 16 bytes) when it fits in 60% of
 *      the free device memory, the dense operators of all live factorizations
 *      of the process stay within 40% of the device, and sum n_j <= 65535, so
 *      that each refinement step is one matrix product (else, or with
 *      PM_FLAG_NO_DENSE_OPERATOR, the operator is applied on the fly).  PM_MIXED reduces every complex64 ID
 *      input with at least twice as many rows as candidate columns to its
 *      triangular factor (unpivoted Householder QR) before the pivoted QR;
 *      PM_FLAG_NO_QR_FIRST pivots on the full input instead.  Each trailing
 *      update of that QR, Q^H C = C - V (T^H (V^H C)), forms V^H C per block
 *      of 256 rows on the FP32 CUDA cores, sums the blocks in a fixed order,
 *      and applies C -= V Y on the tensor cores (3xTF32, FP32 accuracy; a
 *      64-term real accumulation per tile); PM_FLAG_QR_CUDA_CORES applies it
 *      on the CUDA cores instead.  PM_FLAG_TENSOR_CORES moves the whole
 *      update to pm_gemm_c32's kernel, whose FP32 accumulation over the full
 *      row count adds enough rounding error to raise the ranks at the
 *      complex64 threshold.
 *      Confirming residual (PM_MIXED with the dense operator): by default the
 *      residual that ends the refinement comes from a float-float product of
 *      the stored operator whose sums are folded into FP64 every 16 columns
 *      (worst-case error ~9e-13 of sum_j |a_ij| |x_j| per row, below that of
 *      a sequential FP64 sum); PM_FLAG_FP64_CONFIRM forms it with the FP64
 *      product instead.  PM_FLAG_FF_CONFIRM names the default and changes
 *      nothing.  PM_FLAG_NO_AUTOTUNE: the call tunes no batched-GEMM tile
 *      shape (classes tuned before keep their choice; see pm_autotune_table).
 *      Solve graphs: the compressed inverse (PM_FP64) and the mixed
 *      preconditioner are launch sequences fixed by the factorization; the
 *      second time a factor applies one for a given right-hand-side count it
 *      captures the launches into a CUDA graph (kept with the factor) and
 *      replays it from then on; PM_FLAG_NO_GRAPHS (or PM_FLAG_PROFILE) keeps
 *      every application eager.  Solves of one factor are serialised.
 * refine_tol: PM_MIXED: stop refining once every column's relative residual
 *      ||b - A x|| / ||b|| <= refine_tol (0 -> 1e-10).  Intermediate residuals
 *      may come from FP32 or float-float products of the stored operator;
 *      the residual that ends the refinement is formed by the folded
 *      float-float product (or, with PM_FLAG_FP64_CONFIRM, in complex128).
 * max_refine: PM_MIXED: refinement steps at most (0 -> 10); not reaching
 *      refine_tol returns PM_ERR_NOT_CONVERGED.
 * low_tol: PM_MIXED: ID threshold of the complex64 levels (0 -> 5e-6).
 * rank_model: NULL, or a trained predictor on the device (float32:
 *      PM_MLP_NPARAM weights, then 8 feature means and 8 feature scales) whose
 *      two outputs per box and index group are the ID rank / n_g and the
 *      fraction of the rule's proxy count the box needs.  Ranks: the CPQR of
 *      every level runs up to the median predicted rank before its first rank
 *      check (host synchronisation) instead of checking every 16 steps; IDs
 *      whose rank exceeds the prediction continue under the regular checks.
 *      Proxy counts (when proxy_points = 0): each box gets
 *      max(16, 8 ceil(s p_rule / 8)) points, s = min(1, max(0.25, predicted
 *      fraction + 0.1)); in PM_FP64 every box below the rule is judged by the
 *      held-out check below, and a box that fails is redone with the rule's
 *      count (pm_stats.proxy_fallbacks); in PM_MIXED the refinement against
 *      the complex128 operator judges the result (the check runs only with
 *      PM_FLAG_PROXY_CHECK).
 * proxy_scale: 0 or 1 -> the rule's proxy count; s in (0, 1) -> every box
 *      gets max(16, 8 ceil(s p_rule / 8)) points (proxy_points = 0 only).
 *      With PM_FLAG_PROXY_CHECK every ID is then checked a posteriori on a
 *      held-out ring: the box's proxy count of points on the proxy circle,
 *      turned by half their spacing; with H the kernel block between that
 *      ring and the ID's candidates, the check passes when
 *      ||H_J - H_S T||_F <= 200 tol ||H||_F (S the skeleton, J the rest,
 *      T the interpolation matrix).  No counterpart in the paper.
 * formulation: PM_FORM_* (0: PMCHWT (Omit)).  PMCHWT (All) and Burton-Miller
 *      need proxies for the interior kernel as well: PMCHWT (All) uses two
 *      families of proxy densities (exterior and interior kernel), Burton-
 *      Miller its own entries with the proxy circle as an inclusion; the
 *      closed-form proxy count then uses max(k+, k-).  These run in PM_FP64
 *      with one real interior wavenumber for all inclusions (else
 *      PM_ERR_UNSUPPORTED).  For every formulation pm_solve takes the PMCHWT
 *      right-hand side [-u^I; -q^I] and returns [q; u] per inclusion
 *      (Burton-Miller maps it to [-(u^I + alpha q^I); 0] and reorders its
 *      [u; q] unknowns).
 * scratch_gb: device memory for the ID inputs of one step of the levels
 *      (0 -> 35% of the memory free when the step starts).  A level whose
 *      boxes need more runs in consecutive chunks of boxes, each within the
 *      budget (pm_stats.level_chunks); results do not depend on the chunks.
 * debug_flags: 0 in normal use.  Host-side fault injection for tests of the
 *      failure paths (no counterpart in the paper); every injected fault is a
 *      plain write of zeros or a changed host decision, never a device fault:
 *      PM_DEBUG_SINGULAR_BLOCK zeroes the first leaf box's self block before
 *        its LU (-> PM_ERR_SINGULAR, "diagonal block");
 *      PM_DEBUG_SINGULAR_COMPRESSED zeroes R_b A_bb^{-1} L_b of the first leaf
 *        box before its inversion (-> PM_ERR_SINGULAR, the failure that
 *        Sec. 3 shows for the simplified Burton-Miller system);
 *      PM_DEBUG_UNDERPREDICT replaces every predicted rank by 1 (with a
 *        rank_model): every ID falls back to the adaptive checks, and the
 *        factorization is unchanged;
 *      PM_DEBUG_TC_NO_ARRIVE makes the tensor-core kernels (the QR update's
 *        C -= V Y by default, pm_gemm_c32's with PM_FLAG_TENSOR_CORES) wait,
 *        with a short bound, on a barrier that nothing arrives at before
 *        they issue any work (-> PM_ERR_TIMEOUT);
 *      PM_DEBUG_SOLVE_NO_FLAG makes the chained top-level triangular solves
 *        (one launch per triangle, used for at most 8 right-hand sides) wait,
 *        with a 1 ms bound, on a flag that nothing sets before any work
 *        (-> PM_ERR_TIMEOUT from pm_solve / pm_solve_ex). */
typedef struct {
  double tol;
  double proxy_factor;
  int32_t proxy_points;
  int32_t precision;
  void* stream;
  uint32_t flags;
  double refine_tol;
  int32_t max_refine;
  double low_tol;
  const float* rank_model;
  uint32_t debug_flags;
  double proxy_scale;
  int32_t formulation;
  double scratch_gb;
} pm_factor_opts;
/* Boundary integral formulations (paper Sec. 2.1): PMCHWT (Omit), eq.
 * pmchwt_omit_bie, the default; PMCHWT (All), eq. pmchwt_all_bie (interior
 * potentials kept in the off-diagonal blocks); Burton-Miller, eq. bm_bie
 * (alpha = i/k+), and its simplified form without the off-diagonal interior
 * terms, which the fast solver cannot use: its R A^{-1} L is singular
 * (Sec. 3), reported as PM_ERR_SINGULAR. */
enum { PM_FORM_OMIT = 0, PM_FORM_ALL = 1, PM_FORM_BM = 2, PM_FORM_BM_SIMPLIFIED = 3 };
enum {
  PM_DEBUG_SINGULAR_BLOCK = 1,
  PM_DEBUG_SINGULAR_COMPRESSED = 2,
  PM_DEBUG_UNDERPREDICT = 4,
  PM_DEBUG_TC_NO_ARRIVE = 8,
  PM_DEBUG_SOLVE_NO_FLAG = 16
};

/* Outcome of a refined solve (PM_MIXED): steps taken, the final largest
 * relative residual over the right-hand sides (-1 when not refined) and the
 * residual after each of the first 16 steps. */
typedef struct {
  int32_t iterations;
  double residual;
  double history[16];
} pm_solve_info;

/* Statistics of a factorization (filled by pm_factor_stats). */
typedef struct {
  int32_t levels;           /* compressed levels L (0: a single inclusion, dense) */
  int32_t N;                /* unknowns 2 sum n_j */
  int32_t K;                /* size of the top-level dense system */
  int32_t skeleton[16];     /* sum of box ranks per level, index = level (1..L) */
  double ms_assemble, ms_id, ms_schur, ms_top, ms_total;   /* factor phase times */
  int32_t cpqr_launches;    /* CPQR elimination-step launches */
  int32_t rank_checks;      /* device-to-host rank checks (host synchronisations) */
  int32_t predictor_fallbacks;  /* IDs whose rank exceeded the predicted bound */
  double ms_level[16];      /* wall time of each compressed level (index = level) */
  int32_t graph_captures;   /* solve graphs captured so far (one per kind and right-hand-side count) */
  int32_t graph_launches;   /* solve graph replays so far */
  int32_t proxy_checked;    /* boxes whose IDs ran the held-out proxy check */
  int32_t proxy_fallbacks;  /* boxes redone with the rule's proxy count after failing it */
  int64_t id_rows;          /* sum over all IDs of their input rows (near + proxy), the work measure of the IDs */
  int32_t level_chunks;     /* chunks of boxes the levels ran in (one per level when the scratch fits) */
} pm_stats;

/* Build node geometry on the device (paper Sec. 2.2) and the quadtree
 * (paper Sec. 3 / Sec. 4: each inclusion a leaf cell, Morton order).
 * The problem struct and its inclusion array are copied; the caller keeps
 * ownership.  Errors: PM_ERR_INVALID_ARG (m < 1, bad shape, odd n_nodes ...),
 * PM_ERR_GEOMETRY (two inclusions rounding to one grid cell). */
pm_status pm_build_geometry(const pm_problem* prob, pm_geometry** out);

/* Number of unknowns N = 2 sum n_j. */
pm_status pm_geometry_size(const pm_geometry* g, int32_t* N, int32_t* total_nodes);

/* Copy node data to caller buffers (host): xy (2 x total_nodes, interleaved x,y),
 * nrm (interleaved unit outward normals), w (trapezoid weights (2 pi/n)|x'|).
 * Any pointer may be NULL. */
pm_status pm_geometry_nodes(const pm_geometry* g, double* xy, double* nrm, double* w);

/* Plane-wave right-hand sides (paper Sec. 4: u^I = exp(i k^+ d.x)), one column
 * per angle: rhs is N x nrhs column-major, on the device if on_device = 1
 * (caller-owned, e.g. a torch tensor's data_ptr), else on the host. */
pm_status pm_plane_wave_rhs(const pm_geometry* g, const double* angles, int32_t nrhs, pm_c64* rhs,
                            int32_t on_device);

/* Factor the PMCHWT (Omit) system (paper Sec. 2.2, eq. pmchwt_omit_bie) with
 * the multilevel proxy / interpolative-decomposition fast direct solver
 * (paper Sec. 3): self blocks, proxy IDs per cell (exterior kernel only),
 * compressed blocks A~_i = (R_i A_ii^{-1} L_i)^{-1}, recursive merge, top LU.
 * Errors: PM_ERR_INVALID_ARG, PM_ERR_OOM, PM_ERR_CUDA, PM_ERR_SINGULAR,
 * PM_ERR_TIMEOUT (opt-in tensor-core path only), PM_ERR_UNSUPPORTED. */
pm_status pm_factorize(const pm_geometry* g, const pm_factor_opts* opts, pm_factor** out);

/* Solve A phi = rhs for nrhs right-hand sides (paper Sec. 3: eq. compressed and
 * the recovery formula).  rhs and phi are N x nrhs column-major, device
 * pointers on the current device if on_device = 1 (anything else, e.g. a
 * host pointer, -> PM_ERR_INVALID_ARG before any launch), else host
 * pointers; they may alias.  A right-hand side with a NaN or infinite entry
 * -> PM_ERR_INVALID_ARG, phi untouched.  PM_MIXED factors refine the
 * solution (PM_ERR_NOT_CONVERGED if refine_tol is not reached).  With at
 * most 8 right-hand sides the top-level triangular solves run as one chained
 * launch per triangle whose cross-block waits are bounded: PM_ERR_TIMEOUT if
 * one ran out (phi then invalid; the factor stays usable). */
pm_status pm_solve(const pm_factor* f, const pm_c64* rhs, int32_t nrhs, pm_c64* phi, int32_t on_device);

/* pm_solve that also reports the refinement outcome (info may be NULL). */
pm_status pm_solve_ex(const pm_factor* f, const pm_c64* rhs, int32_t nrhs, pm_c64* phi, int32_t on_device,
                      pm_solve_info* info);

/* Many independent problems (no counterpart in the paper; the paper factors
 * one system at a time).  pm_factor_batch splits g[0..count) into `workers`
 * groups (0 -> 4; each problem, in descending order of N^1.5, joins the group
 * with the least work so far).  The problems of a group are factored
 * together in shared launches: one gather, one batched QR / CPQR step, one
 * batched LU and GEMM per phase for all of their boxes, step s taking level
 * L_i - s of every problem i (leaves first, whatever the depths), then all
 * top-level systems in one batched LU; each group runs on its own host
 * thread and CUDA stream, so groups overlap.  workers = count gives one
 * problem per group (no shared launches).  Every problem's result equals
 * its pm_factorize.  out[i] receives each handle (all NULL on error).
 * opts->stream is ignored and PM_FLAG_PROFILE cleared; the returned handles
 * run later pm_solve calls on the default stream.
 * pm_solve_batch solves each factor for its own right-hand sides rhs[i] ->
 * phi[i] (N_i x nrhs each) with `workers` host threads (0 -> 8), one CUDA
 * stream each. */
pm_status pm_factor_batch(const pm_geometry* const* g, int32_t count, const pm_factor_opts* opts, pm_factor** out,
                          int32_t workers);
pm_status pm_solve_batch(const pm_factor* const* f, int32_t count, const pm_c64* const* rhs, int32_t nrhs,
                         pm_c64* const* phi, int32_t on_device, int32_t workers);

pm_status pm_factor_stats(const pm_factor* f, pm_stats* out);

/* Skeleton (selected) global row / column indices of one box, for inspection.
 * level in 1..L, box in Morton order of that level; rows/cols receive up to
 * cap entries each; *k receives the box rank. */
pm_status pm_factor_skeleton(const pm_factor* f, int32_t level, int32_t box, int32_t* rows, int32_t* cols,
                             int32_t cap, int32_t* k);

/* Entries of the PMCHWT (Omit) matrix between inclusions (trapezoid rule,
 * exterior kernel only, paper Sec. 2.2): out[i + j M] = A(rows[i], cols[j])
 * for global indices on different inclusions (same-inclusion pairs give 0).
 * Host arrays; M x N complex output. */
pm_status pm_matrix_entries(const pm_geometry* g, const int32_t* rows, int32_t M, const int32_t* cols,
                            int32_t Ncols, pm_c64* out);

/* The self block A_jj (2 n_j x 2 n_j, column-major) of inclusion j
 * (paper Sec. 2.2: Kress log-split quadrature for S, D, D*; Maue's form of N). */
pm_status pm_self_block(const pm_geometry* g, int32_t j, pm_c64* out);

/* Fields represented by a boundary solution phi (N x nrhs, [q_j; u_j] per
 * inclusion, as pm_solve returns it): Green's representation over all
 * boundaries with the trapezoid rule, u^s(x) = sum_j int [dG/dn_y u -
 * G eps+ q] ds, G = (i/4) H0(k+ |x - y|) (the incident wave adds nothing
 * outside the inclusions).  No counterpart in the paper's text, which uses
 * the boundary solutions only; the paper's Sec. 4.3 frequency study reuses
 * them.
 * pm_far_field: the far-field pattern u_inf(xhat), u^s(x) = e^{i k r}/sqrt(r)
 *      (u_inf + O(1/r)), at directions xhat = (cos a, sin a) for the ndir
 *      host angles: out[d + c ndir].
 * pm_scattered_field: u^s at npts host points (xy: x, y pairs), which must
 *      lie outside the inclusions and a few node spacings from every
 *      boundary for trapezoid accuracy: out[p + c npts].
 * phi and out are device pointers of the geometry's device if on_device = 1,
 * else host buffers.  Errors: PM_ERR_INVALID_ARG (NULL, sizes, non-finite
 * directions or points, host pointer for on_device = 1), PM_ERR_CUDA. */
pm_status pm_far_field(const pm_geometry* g, const pm_c64* phi, int32_t nrhs, int32_t on_device, const double* angles,
                       int32_t ndir, pm_c64* out);
pm_status pm_scattered_field(const pm_geometry* g, const pm_c64* phi, int32_t nrhs, int32_t on_device,
                             const double* xy, int32_t npts, pm_c64* out);

/* Per-kernel timing of a factorization made with flags & PM_FLAG_PROFILE
 * (no counterpart in the paper; measurement aid).  CUDA events bracket every
 * launch on the factorization's stream.  `work` is the algorithmic work of
 * all launches: real flops for cpqr_step, interp_solve, lu_*, getrs,
 * gemm_batched, qr_update32, dense_matvec64 and dense_offdiag64 (164 per node
 * pair); bytes for cpqr_step32 (one read and write of every trailing entry);
 * matrix entries for gather_entries; node pairs for self_pointwise.  Names
 * ending in 32 are the complex64 instances.  Writes up to cap entries, *count = number available. */
typedef struct {
  char name[32];
  int32_t launches;
  double ms;
  double work;
} pm_kernel_stat;
enum {
  PM_FLAG_PROFILE = 1,
  PM_FLAG_NO_DENSE_OPERATOR = 2,
  PM_FLAG_NO_QR_FIRST = 4,
  PM_FLAG_TENSOR_CORES = 8,
  PM_FLAG_FF_CONFIRM = 16,
  PM_FLAG_FP64_CONFIRM = 32,
  PM_FLAG_NO_AUTOTUNE = 64,
  PM_FLAG_NO_GRAPHS = 128,
  PM_FLAG_PROXY_CHECK = 256,
  PM_FLAG_QR_CUDA_CORES = 512,
  PM_FLAG_TOP_FP64 = 1024,
  PM_FLAG_OPERATOR_AFTER = 2048
};
pm_status pm_factor_profile(const pm_factor* f, pm_kernel_stat* out, int32_t cap, int32_t* count);

/* ---- learned ID-rank predictor (no counterpart in the paper) ----------------
 * An MLP 8 -> 64 -> 64 -> 2 (tanh) maps features of a box and index group
 * (log n_g, log W of the row and column ID inputs, k+ r_cell, log10 tol,
 * log2 of the box's inclusions, the group, mean k-/k+) to the adaptive ranks
 * of its row and column IDs divided by n_g.  Parameters: one flat array of
 * PM_MLP_NPARAM numbers (row-major W1 64x8, b1, W2 64x64, b2, W3 2x64, b3).
 * Loss (1/B) sum (1 + lam [y < t]) (y - t)^2; Adam.  All pointers except
 * the host arrays of pm_factor_rank_data / pm_mlp_train's X, T and
 * loss_history are device pointers; dtype 0 = float32, 1 = float64. */
enum { PM_MLP_NPARAM = 4866 };
/* Training samples recorded by a factorization, two per box (index groups
 * 0, 1), in level order L..1 and Morton order: X (count x 8) the features,
 * T (count x 2) = (max(row rank, column rank) / n_g, proxy count used / the
 * rule's count), host buffers. */
pm_status pm_factor_rank_data(const pm_factor* f, float* X, float* T, int32_t cap, int32_t* count);
/* For the same samples: the held-out check's ratio ||H_J - H_S T|| /
 * (tol ||H||) of the box (largest over its four IDs; -1 where it did not run)
 * and whether the box was redone with the rule's proxy count (0 / 1). */
pm_status pm_factor_proxy_data(const pm_factor* f, float* ratio, int32_t* redone, int32_t cap, int32_t* count);
pm_status pm_mlp_forward(int32_t dtype, const void* theta, int32_t B, const void* X, void* Y, void* stream);
/* loss (1 value) and gradient (PM_MLP_NPARAM) of a batch, overwritten. */
pm_status pm_mlp_loss_grad(int32_t dtype, const void* theta, int32_t B, const void* X, const void* T, double lam,
                           void* grad, void* loss, void* stream);
pm_status pm_mlp_adam_step(int32_t dtype, void* theta, const void* grad, void* m, void* v, int32_t t, double lr,
                           double b1, double b2, double eps, void* stream);
/* Train float32 parameters in place: epochs of shuffled minibatches (splitmix64
 * with `seed`), Adam (b1 0.9, b2 0.999, eps 1e-8).  X, T: device, row-major
 * nsamples x 8 / x 2 (features already standardised); loss_history: host,
 * one mean loss per epoch, or NULL. */
pm_status pm_mlp_train(void* theta, int32_t nsamples, const float* X, const float* T, int32_t epochs, int32_t batch,
                       double lr, double lam, uint64_t seed, double* loss_history, void* stream);

/* The batched-GEMM autotuner's choices (no counterpart in the paper).  The
 * complex GEMMs of the factorization and the solve run one kernel over a list
 * of products; its output tile is chosen per class of batch (device, complex
 * size in bytes, ceil log2 of the largest m, of the largest n, of the mean k,
 * of the number of products) among 32x32, 64x64, 64x32, 128x8 and 64x16.
 * The first batch of a class whose outputs are write-only times every shape
 * once (CUDA events, after a warm-up launch) and keeps the fastest; the
 * choice is cached per process.  All shapes accumulate over k in the same
 * order, so the choice changes no result.  Writes up to cap entries (ms: the
 * measured time of each shape in the order above), *count = entries known. */
typedef struct {
  int32_t device, complex_bytes, log2_m, log2_n, log2_k, log2_count;
  int32_t tm, tn;      /* chosen output tile */
  float ms[8];
  int64_t uses;        /* batches of the class run so far */
} pm_tune_entry;
pm_status pm_autotune_table(pm_tune_entry* out, int32_t cap, int32_t* count);

/* Number of CUDA kernel launches this library has made in this process
 * (no counterpart in the paper; measurement aid). */
pm_status pm_launch_counter(uint64_t* out);

/* Complex64 product on the tensor cores: the tcgen05 kernel (kind::tf32
 * with each FP32 operand split into two tf32 parts, three products, FP32
 * accumulation in tensor memory) that the complex64 QR updates can use,
 * exported so that its numerics can be checked on their own.  No counterpart
 * in the paper.  C = alpha op(A) op(B) + beta C with column-major DEVICE
 * buffers of interleaved (re, im) floats: op(A) is m x k, A itself (lda >= m)
 * or with conj_a != 0 the conjugate transpose of a stored k x m matrix
 * (lda >= k); op(B) is k x n, B (ldb >= k) or with conj_b the conjugate
 * transpose of a stored n x k matrix (ldb >= n); C is m x n (ldc >= m).
 * alpha, beta: host pointers to (re, im).  Runs on `stream` (NULL: default
 * stream) and returns once it has finished.  PM_ERR_TIMEOUT: a wait on the
 * tensor cores ran out (about a second); C is then undefined. */
pm_status pm_gemm_c32(int32_t m, int32_t n, int32_t k, const void* A, int32_t lda, int32_t conj_a, const void* B,
                      int32_t ldb, int32_t conj_b, void* C, int32_t ldc, const float* alpha, const float* beta,
                      void* stream);

/* The self block A_jj, like pm_self_block, without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot let the library call cudaMalloc / cudaFree, because those calls may
 * synchronise the device while the caller has work in flight, or because the
 * caller runs under its own device-memory manager or a fixed budget.
 *   out: caller-owned DEVICE buffer of (2 n_j)^2 pm_c64, column-major,
 *        on the current device, which must be the device the geometry was
 *        built on; fully overwritten.  A host pointer or another device's
 *        memory -> PM_ERR_INVALID_ARG before any launch.
 * Scratch lives in a file-scope device array of 4 MiB + 64 KiB that every GPU
 * loading the library holds until the process exits; it limits n_j to 256
 * (larger n_j -> PM_ERR_INVALID_ARG, nothing written).  The first call on a
 * device looks up that array's device address; make it before any stream
 * capture.  The address is cached for the life of the process: it does not
 * survive cudaDeviceReset or a reset of the primary context by the host
 * application (call no further pm_self_block_noalloc after one).  Calls share the array and return only when their work on the
 * default stream has finished, so calls overlapping on the GPU (e.g. from
 * several host threads at once) race and must be serialised by the caller. */
pm_status pm_self_block_noalloc(const pm_geometry* g, int32_t j, pm_c64* out);

/* Peak arithmetic rates of the current device, measured by the library's
 * own loop of independent fused multiply-adds (no counterpart in the paper;
 * the denominators of the roofline fractions of the FP64 and FP32 kernels).
 * which = 0: FP64 FMA, 1: FP32 FMA.  Runs about `ms_target` milliseconds on
 * the default stream; *tflops receives 2 flops per FMA over the event time,
 * *sm_mhz (may be NULL) the SM clock the loop ran at (clock64 cycles of the
 * longest CTA over that time), so that the rate can be scaled to another
 * clock.  Errors: PM_ERR_INVALID_ARG (which, ms_target outside (0, 10000],
 * NULL tflops), PM_ERR_CUDA. */
pm_status pm_measure_peak(int32_t which, double ms_target, double* tflops, double* sm_mhz);

/* Device memory the library keeps for reuse (no counterpart in the paper).
 * Blocks that freed factors, solves and scratch arenas give back stay cached
 * per device (at most 45% of its memory), each until the stream that used it
 * has finished, and serve later requests of up to 1.5x their size: repeated
 * factorizations of a problem then neither map nor unmap their memory again
 * (cudaFree of a 69 GB operator alone takes 25 ms on GB300).  A request that
 * cudaMalloc cannot meet first releases the device's cached blocks.
 * pm_release_cached_memory waits for and frees every cached block of every
 * device; *bytes (may be NULL) receives the bytes freed.  Errors: none
 * (PM_OK also without a GPU). */
pm_status pm_release_cached_memory(int64_t* bytes);

void pm_factor_free(pm_factor* f);
void pm_geometry_free(pm_geometry* g);
const char* pm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
