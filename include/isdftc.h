/*
 * isdftc -- C ABI of the B300 (sm_103a) ISDF-xTC kernel library.
 *
 * The library builds the ISDF-compressed transcorrelated two-body kernels of
 * "Interpolative Separable Density-Fitting for Transcorrelated Hamiltonians"
 * (Liao, Cheng, Dobrautz, Zhu, Alavi): orbitals on a molecular grid,
 * pivoted-Cholesky interpolation points, the least-squares auxiliary fit,
 * the Jastrow kernels u^(1),c and u^(3), and the xTC density contraction.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers owned by the caller, dense and
 *     row-major in the layout stated per argument; nothing is freed or
 *     retained by the library.  Small parameter structs are host memory and
 *     are copied by value during the call.
 *   - The library allocates no device memory.  Each call that needs scratch
 *     takes a caller workspace (ws, ws_bytes, 256-byte aligned); the matching
 *     *_workspace() function returns the bytes needed.  A too-small workspace
 *     is ISDF_E_ARG.
 *   - Work is enqueued on `stream` (a cudaStream_t, NULL = legacy default).
 *     Calls that report a host-side result (n_mu_out, jitter, energies) or
 *     that check the device error word synchronise `stream` before
 *     returning; this is stated per call.
 *   - Every call returns an isdf_status; isdf_last_error() gives a message
 *     for the last failure on the calling thread.
 *   - One device (the current one); no host fallback exists.
 */
#ifndef ISDFTC_H
#define ISDFTC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* isdf_stream_t; /* == cudaStream_t */

typedef enum {
  ISDF_OK = 0,
  ISDF_E_ARG = 1,        /* invalid argument, size or workspace */
  ISDF_E_NOT_PD = 2,     /* Gram Cholesky failed after the last jitter retry */
  ISDF_E_RANK = 3,       /* numerical rank exhausted before n_mu points (informational) */
  ISDF_E_NONFINITE = 4,  /* NaN or Inf found by a call that synchronises (stated per
                            call); the asynchronous calls propagate them */
  ISDF_E_TIMEOUT = 5,    /* a bounded device wait expired; the kernel returned early */
  ISDF_E_CUDA = 6,       /* CUDA runtime error */
  ISDF_E_UNSUPPORTED = 7 /* option combination not implemented */
} isdf_status;

typedef enum {
  ISDF_PREC_FP64 = 0,   /* FP64 on CUDA cores (the FP64 GPU path) */
  ISDF_PREC_BF16X3 = 1, /* tcgen05 BF16, 2-limb split (hi*hi + hi*lo + lo*hi), FP32 accumulation */
  ISDF_PREC_BF16X6 = 2, /* tcgen05 BF16, 3-limb split (6 products), FP32 accumulation */
  ISDF_PREC_FP32 = 3,   /* FP32 on CUDA cores (adjoint) */
  ISDF_PREC_TF32X3 = 4  /* W build, radial correlator: stage 1 on tcgen05 kind::tf32 with
                           2-limb TF32 operands (3 products), FP32 accumulation; stage 2 as
                           ISDF_PREC_BF16X6 */
} isdf_precision;

/* Contracted Cartesian Gaussian basis (device arrays).  Function f is
 *   chi_f(r) = sum_k coefs[f][k] (x-X_f)^a (y-Y_f)^b (z-Z_f)^c exp(-exps[f][k] |r-R_f|^2)
 * with (a,b,c) = powers[f]. */
typedef struct {
  int32_t n_bf;
  int32_t n_prim;
  const double* center;  /* [n_bf][3] bohr */
  const int32_t* powers; /* [n_bf][3] */
  const double* exps;    /* [n_bf][n_prim] */
  const double* coefs;   /* [n_bf][n_prim], normalisation folded in */
} isdf_basis;

#define ISDF_MAX_NUC 64
#define ISDF_MAX_TYPES 4
#define ISDF_MAX_TERMS 32

/* Boys-Handy correlator (Sec. II.B, Eqs. bh-scaled and bh-u):
 *   u(i,j) = sum_I sum_k coef[type(I)][k] [A_iI^m A_jI^n + A_jI^m A_iI^n] E_ij^o
 *            + cusp * E_ij / (2 d)
 * with A_iI = b_I r_iI / (1 + b_I r_iI), E_ij = d r_ij / (1 + d r_ij) and
 * (m,n,o) = mno[k].  The cusp line is the cusp-normalised (0,0,1) term
 * (slope du/dr_ij -> 1/2).  n_terms = 0 with cusp = 1 is the radial
 * electron-electron correlator u(r) = r / (2 (1 + d r)).
 * One-body nuclear-cusp term (Eq. tau-def): when some chi_a[t] != 0,
 *   u(i,j) += [chi(r_i) + chi(r_j)] / (n_elec - 1),
 *   chi(r) = sum_I chi_a[t] r_iI / (1 + chi_b[t] r_iI),  t = nuc_type[I]
 * (the paper cites chi's form without stating it; chi_a[t] = -Z_t gives the
 * electron-nucleus cusp slope).  It adds grad chi(r_g)/(n_elec - 1) to K_c(g,g')
 * for every g' != g; the self pair stays 0.  Host struct.  Calls return
 * ISDF_E_ARG for d <= 0, counts or exponents out of range, non-finite
 * positions, d or coefficients, b_t <= 0 when n_terms > 0, and, with chi on,
 * n_elec < 2, n_nuc = 0 or chi_b[t] <= 0. */
typedef struct {
  int32_t n_nuc;
  int32_t n_types;
  int32_t n_terms;
  int32_t cusp;
  double d;
  double nuc_xyz[ISDF_MAX_NUC][3];
  int32_t nuc_type[ISDF_MAX_NUC];
  double b[ISDF_MAX_TYPES];
  int32_t mno[ISDF_MAX_TERMS][3];
  double coef[ISDF_MAX_TYPES][ISDF_MAX_TERMS];
  double chi_a[ISDF_MAX_TYPES];  /* one-body term amplitude per type (0 = off) */
  double chi_b[ISDF_MAX_TYPES];  /* its scale beta per type */
  int32_t n_elec;                /* electrons N of Eq. tau-def (used with chi on) */
} isdf_jastrow;

/* Options of the kernel build and the fit (host struct; NULL = defaults;
 * a zero field takes its default). */
typedef struct {
  int32_t precision;  /* isdf_precision; default ISDF_PREC_BF16X3 */
  int32_t kchunk;     /* stage 1: inner-grid points the tensor core accumulates into
                         its FP32 chunk sum before the epilogue folds that sum into
                         the IEEE-rounded FP32 running sum (also in tensor memory;
                         the tile is written to FP64 once); rounded up to a multiple
                         of 32; 0 = default (384; 128 for ISDF_PREC_TF32X3) */
  int32_t s2_kchunk;  /* fold interval of stage 2; 0 = default (256) */
  int32_t sync_check; /* 1 (default): synchronise the stream on return and report
                         device-side errors (expired bounded waits, CUDA errors) */
  int32_t debug_flags;/* bit 0: the stage-1 producer skips its first arrival, so
                         the consumer's bounded wait expires (fault-path test);
                         bit 1: with ISDF_PREC_BF16X3, the radial correlator's
                         stage 1 runs on single CTAs (128-row tiles) instead of
                         CTA pairs (256-row tiles; always used for BF16X6) */
  float* stage_ms;    /* host [2] or NULL: when set (with sync_check), the device
                         times of stage 1 and stage 2, measured with CUDA events
                         on `stream` around the two kernels */
  double jitter_init; /* isdf_fit: Tikhonov shift of the first retry, relative to
                         max(diag) of the Gram (the first attempt has none);
                         0 = default 1e-14 (Sec. IV.B leaves it unstated) */
  double jitter_growth;   /* factor per further retry; 0 = default 10 */
  int32_t max_jitter_tries; /* retries after the unshifted attempt; 0 = default 8,
                               negative = none (an indefinite Gram returns
                               ISDF_E_NOT_PD at once) */
  int32_t wait_limit_ms;  /* tc_kernel_build: bound of every device-side wait of
                             its tensor-core kernels, in ms; 0 = default 2000;
                             larger values are clamped to 60000 */
  int32_t fit_mode;       /* isdf_fit: 0 = FP64 on CUDA cores (default); 1 = the
                             right-hand-side GEMMs and the triangular solves as
                             FP64 products emulated on the tensor cores
                             (isdf_dgemm_emulated; workspace from
                             isdf_fit_workspace_mode) */
} isdf_options;

const char* isdf_last_error(void);
int isdf_abi_version(void);
/* Number of CUDA kernels this library has launched in the process so far
 * (a diagnostic counter; host side, monotone). */
uint64_t isdf_kernel_launches(void);

/* ---------------------------------------------------------------------------
 * Orbitals and gradients on the grid (Alg. 2 step 2).
 *   phi[p][g]     = sum_f mo_coef[f][p] chi_f(r_g)
 *   dphi[c][p][g] = sum_f mo_coef[f][p] d_c chi_f(r_g)
 * mo_coef [n_bf][n_orb]; grid_xyz [n_g][3]; phi [n_orb][n_g];
 * dphi [3][n_orb][n_g].  FP64.  Asynchronous. */
size_t isdf_eval_orbitals_workspace(int n_bf, int64_t n_g);
int isdf_eval_orbitals(const isdf_basis* basis, const double* mo_coef, int n_orb,
                       const double* grid_xyz, int64_t n_g, double* phi, double* dphi,
                       void* ws, size_t ws_bytes, isdf_stream_t stream);
/* The same with mode 0 (= isdf_eval_orbitals: FP64 GEMMs on CUDA cores) or
 * mode 1: the four contractions C^T chi as the emulated FP64 products of
 * isdf_dgemm_emulated (error within (n_bf + 4) 2^-52 2^(e_p + e_g) per value,
 * 2^e the powers of two above max_f|C_fp| and max_f|chi_f(g)|).  The workspace query takes n_orb for mode 1. */
size_t isdf_eval_orbitals_workspace_mode(int n_bf, int64_t n_g, int n_orb, int mode);
int isdf_eval_orbitals_mode(const isdf_basis* basis, const double* mo_coef, int n_orb,
                            const double* grid_xyz, int64_t n_g, double* phi, double* dphi,
                            int mode, void* ws, size_t ws_bytes, isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Interpolation points by weighted pivoted Cholesky (Alg. 1; gradient branch
 * and pivot fusion of Sec. II.D; matrix-free form of Sec. IV.B).
 *   scalar   S(g,h) = (w_g w_h) (sum_p phi_p(g) phi_p(h))^2
 *   gradient S(g,h) = (w_g w_h) (sum_p phi_p(g) phi_p(h)) (sum_{c,p} dphi_cp(g) dphi_cp(h))
 * FP64 with every sum accumulated by fused multiply-add in a fixed order
 * (p ascending; c outer), argmax ties broken by the lowest grid index, and
 * d_g* = 0 after each step, so the indices are reproducible bit for bit.
 * mode 0 = fused: alternate scalar / gradient steps (scalar first), append
 *          each new point, stop at n_mu points;
 * mode 1 = scalar channel only; mode 2 = gradient channel only.
 * A channel stops when its pivot d_g* <= 64 eps max_g d_g(initial).
 * pivots [n_mu] int32 (append order) receives *n_mu_out entries.  Returns
 * ISDF_E_RANK (with *n_mu_out < n_mu) when both channels stopped early, and
 * ISDF_E_NONFINITE (before any step) when phi, dphi or w hold a NaN or Inf.
 * Synchronises `stream`. */
size_t isdf_points_workspace(int64_t n_g, int n_mu);
int isdf_points(const double* phi, const double* dphi, const double* w, int64_t n_g,
                int n_orb, int n_mu, int mode, int32_t* pivots, int* n_mu_out, void* ws,
                size_t ws_bytes, isdf_stream_t stream);

/* The paper's pivot fusion (Sec. II.D, pivot-fusion paragraph): the scalar
 * channel runs to rank n_ch_phi, then the gradient channel to rank n_ch_grad,
 * each on its own with the arithmetic and tie rule of isdf_points, and the
 * interpolation set is their union -- the scalar pivots in order, then each
 * gradient pivot not already present.  The union size is an outcome:
 * *n_mu_out <= n_ch_phi + n_ch_grad.  pivots: device int32 with room for
 * n_ch_phi + n_ch_grad entries.  n_ch_phi, n_ch_grad >= 0 with a positive
 * sum.  Returns ISDF_E_RANK (pivots still valid) when a channel stopped before
 * its rank, ISDF_E_NONFINITE (before any step) when phi, dphi or w hold a NaN
 * or Inf.  Synchronises `stream`. */
size_t isdf_points_fixed_rank_workspace(int64_t n_g, int n_ch_phi, int n_ch_grad);
int isdf_points_fixed_rank(const double* phi, const double* dphi, const double* w, int64_t n_g,
                           int n_orb, int n_ch_phi, int n_ch_grad, int32_t* pivots,
                           int* n_mu_out, void* ws, size_t ws_bytes, isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Least-squares ISDF fit (Eq. isdf-rho and the normal equations of Sec. II.D).
 *   G[mu][g] = sum_p phi_p(r_mu) phi_p(r_g)
 *   scalar:     (G_PP o G_PP) xi = G o G
 *   gradient c: (dG^c_PP o G_PP) xi~^c = dG^c o G,  dG^c[mu][g] = sum_p d_c phi_p(r_mu) d_c phi_p(r_g)
 * FP64 Cholesky with adaptive Tikhonov retry (Sec. IV.B): lambda = 0, then
 * jitter_init max(diag) times jitter_growth per retry, at most
 * max_jitter_tries retries (options; NULL = 1e-14, 10, 8); the lambda used
 * per system is written to jitter_used (host [4], may be NULL).
 * pivots [n_mu] (distinct grid indices in [0, n_g), as isdf_points returns
 * them); xi [n_mu][n_g]; xi_grad [3][n_mu][n_g].  Synchronises `stream`.
 * Errors: ISDF_E_ARG when a pivot index lies outside [0, n_g) (checked on the
 * device before any solve; such an index is never dereferenced);
 * ISDF_E_NONFINITE when phi or dphi hold a NaN or Inf, or the solutions
 * overflow; ISDF_E_NOT_PD if a system stays indefinite.
 * With options->fit_mode = 1 the right-hand sides G, dG^c and the two
 * triangular solves (by blocks of 128 with inverted diagonal blocks) run as
 * the emulated FP64 products of isdf_dgemm_emulated; the Grams and their
 * Cholesky factors stay FP64 on CUDA cores. */
size_t isdf_fit_workspace(int64_t n_g, int n_orb, int n_mu);
/* Workspace for fit_mode 0 (= isdf_fit_workspace) or 1 (adds the emulated
 * products' digit planes: 16 (n_g + 64) max(n_orb, 128) bytes and less); 0 for
 * another mode. */
size_t isdf_fit_workspace_mode(int64_t n_g, int n_orb, int n_mu, int fit_mode);
int isdf_fit(const double* phi, const double* dphi, int64_t n_g, int n_orb,
             const int32_t* pivots, int n_mu, double* xi, double* xi_grad,
             double* jitter_used, const isdf_options* options, void* ws, size_t ws_bytes,
             isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * FP64 matrix product emulated on the BF16 tensor cores (not in the paper; the
 * fit's FP64 solves otherwise set the step time on B300, whose FP64 rate is
 * ~1 TFLOP/s):  C = alpha A B + beta C, beta 0 or 1, A [M][K] (row stride lda),
 * B [K][N] (ldb), C [M][N] (ldc), all FP64 row-major on the device.
 * Each row of A and column of B is scaled by a power of two and cut into eight
 * signed 7-bit digits held exactly in BF16; the 36 digit products of weight
 * >= 2^-63 are summed exactly in FP32 per weight (at most 128 inner terms per
 * tensor-core run) and combined exactly in 64-bit integers, up to 8 runs of one
 * output tile in turn, before one rounding to FP64; longer K is split over CTAs
 * whose results are added with FP64 atomics.  Error within (K + 4) 2^-52 2^(e_m + e_n) per element, 2^e_m the power
 * of two above max_k|A_mk| and 2^e_n that above max_k|B_kn|.
 * A NaN or Inf in A or B gives undefined values in C.  Asynchronous. */
size_t isdf_dgemm_emulated_workspace(int64_t M, int64_t N, int64_t K);
int isdf_dgemm_emulated(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                        const double* B, int64_t ldb, double alpha, double beta, double* C,
                        int64_t ldc, void* ws, size_t ws_bytes, isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Jastrow kernels of the ISDF K integrals (Eqs. K1-isdf and K3-isdf):
 *   W[c][mu][nu] = sum_{g in [g_begin,g_end)} sum_{g'} w_g w_g' xi~^c_mu(g) xi_nu(g') K_c(g,g')  c = x,y,z
 *   W[3][mu][nu] = sum_{g in [g_begin,g_end)} sum_{g'} w_g w_g' xi_mu(g)   xi_nu(g') K_sq(g,g')
 * with K_c = d u / d r_{g,c} (electron 1 at r_g) and K_sq = sum_c K_c^2, both
 * generated on the fly; the self pair g = g' contributes 0.  Computed as
 *   calG[c][nu][g - g_begin] = sum_g' w_g' xi_nu(g') K_c(g,g')   (calG of Sec. III.B)
 *   W[c] = (w xi~^c) calG[c]^T, W[3] = (w xi) calG[3]^T   over the slice.
 * The outer-grid slice [g_begin, g_end) gives additive partial kernels.
 * grid_xyz [n_g][3]; w [n_g]; xi [n_mu][n_g]; xi_grad [3][n_mu][n_g];
 * W [4][n_mu][n_mu] FP64 (overwritten); calG [4][n_mu][g_end-g_begin] FP64
 * (overwritten; required).  With sync_check (default) the call returns
 * ISDF_E_NONFINITE when W holds a NaN or Inf (every input value reaches W).
 * ISDF_PREC_FP64 takes any correlator.  The
 * tensor-core precisions take the radial correlator (n_terms = 0, cusp = 1,
 * no one-body term) and, on the multi-centre generator, correlators with the
 * one-body term and those whose terms have m, n <= 3, o <= 4 and at most two
 * distinct E exponents o among the terms with (m, n) != (0, 0), both on CTA
 * pairs, with the nucleus count limited by shared memory (ISDF_E_ARG beyond
 * it; 12 centres with the benzene configuration's term set use 206 KB).
 * Synchronises `stream` when options->sync_check (default).
 * The workspace query takes the correlator (NULL: the largest layout the
 * call accepts). */
size_t tc_kernel_build_workspace(int64_t n_g, int n_mu, int64_t g_begin, int64_t g_end,
                                 int precision, const isdf_jastrow* jas);
int tc_kernel_build(const double* grid_xyz, const double* w, const double* xi,
                    const double* xi_grad, int64_t n_g, int n_mu, int64_t g_begin,
                    int64_t g_end, const isdf_jastrow* jas, const isdf_options* options,
                    double* W, double* calG, void* ws, size_t ws_bytes,
                    isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * tc_kernel_build with xi and xi_grad in HOST memory (Sec. II.D grid-batched
 * streaming with depth-one prefetch; the doubly-blocked bra/ket grid loops of
 * Sec. IV.C): W over the whole grid as
 *   W[c] = sum_{bra batches b} (w xi~^c)_b [ sum_{ket batches k} calG^c_{b,k} ]^T,
 *   calG^c_{b,k}[nu][g] = sum_{g' in k} w_g' xi_nu(g') K_c(g, g'),
 * with batches of `bra` outer and `ket` inner points (ket a multiple of 32).
 * Each ket batch of xi is copied to the device (cudaMemcpy2DAsync on a stream
 * of the call) while stage 1 runs on the previous one, and each bra batch of
 * xi~ and xi while the bra batch's stage 1 runs; xi_host [n_mu][n_g] and
 * xi_grad_host [3][n_mu][n_g] should be pinned (page-locked) for the copies to
 * overlap.  Device memory: the grid, w and the per-point coordinate and
 * nucleus tables, two ket batches and one bra batch of FP64 xi, the bra
 * batch's calG and the limb operands (the workspace query gives the bytes);
 * none of it grows with n_g beyond the per-point tables.  The ket loop re-reads
 * xi from the host once per bra batch.  Tensor-core precisions only
 * (ISDF_E_ARG for FP64); otherwise as tc_kernel_build (same correlators,
 * options, error codes); synchronises `stream`.  W [4][n_mu][n_mu] device FP64
 * (overwritten). */
size_t tc_kernel_build_streamed_workspace(int64_t n_g, int n_mu, int64_t bra, int64_t ket,
                                          int precision, const isdf_jastrow* jas);
int tc_kernel_build_streamed(const double* grid_xyz, const double* w, const double* xi_host,
                             const double* xi_grad_host, int64_t n_g, int n_mu, int64_t bra,
                             int64_t ket, const isdf_jastrow* jas, const isdf_options* options,
                             double* W, void* ws, size_t ws_bytes, isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Adjoint of the Jastrow kernels with respect to the correlator parameters
 * (not in the paper).  For the seed Wbar [4][n_mu][n_mu] and
 *   L(theta) = sum_c <Wbar^c, W^c(theta)>      (W of tc_kernel_build, full grid)
 * writes dtheta[j] = dL/dtheta_j for theta = (d, b_0, c_0 .. c_{K-1}):
 *   dL/dtheta_j = sum_{g != g'} sum_{c<3} (M^c + 2 M^sq K_c)(g,g') dK_c(g,g')/dtheta_j
 *   M^c(g,g') = [(w xi~^c)^T Wbar^c (w xi)]_{g g'},  M^sq with w xi and Wbar^sq,
 * recomputing the M tiles from the factors (nothing of size n_g^2 is stored).
 * The one-body term (isdf_jastrow chi) has no parameter in theta; it enters
 * through K_c in the M^sq factor.
 * One nucleus type and at most 30 free terms (else ISDF_E_UNSUPPORTED);
 * precision ISDF_PREC_FP64 (M tiles and pair arithmetic in FP64 on CUDA
 * cores; asynchronous) or ISDF_PREC_FP32: the M tiles of each outer slice of
 * up to 2048 points as one split-BF16 tcgen05 GEMM (three limbs, FP32
 * accumulation folded every 256 mu, FP64 output slab [4][slice][n_g] in the
 * workspace), the pair arithmetic in FP32; it synchronises `stream` at the end
 * and returns ISDF_E_TIMEOUT if a bounded wait of the GEMM expired.  The
 * reduction is FP64.  dtheta: device [2 + n_terms] FP64 (overwritten). */
size_t tc_kernel_adjoint_workspace(int64_t n_g, int n_mu, int n_nuc, int precision);
int tc_kernel_adjoint(const double* grid_xyz, const double* w, const double* xi,
                      const double* xi_grad, int64_t n_g, int n_mu, const isdf_jastrow* jas,
                      const double* Wbar, int precision, double* dtheta, void* ws,
                      size_t ws_bytes, isdf_stream_t stream);

/* tc_kernel_adjoint restricted to the outer points g in [g_begin, g_end) (all
 * inner points g'): the derivative of L over W built on that outer slice
 * (tc_kernel_build with the same slice).  The sums are additive over slices.
 * Same workspace as tc_kernel_adjoint; ISDF_E_ARG for an empty or out-of-range
 * slice. */
int tc_kernel_adjoint_range(const double* grid_xyz, const double* w, const double* xi,
                            const double* xi_grad, int64_t n_g, int n_mu, int64_t g_begin,
                            int64_t g_end, const isdf_jastrow* jas, const double* Wbar,
                            int precision, double* dtheta, void* ws, size_t ws_bytes,
                            isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Learned interpolation-point proposer (not in the paper).  A network
 * s = W3 relu(W2 relu(W1 x + b1) + b2) + b3 (8 -> 128 -> 128 -> 1) scores grid
 * points; the highest-scoring kappa N_mu points form a candidate set on which
 * the plain pivoted Cholesky (isdf_points) runs; the scalar-channel fit error
 * decides between the result and the plain selection, which stays the fallback.
 * params: device FP32 [isdf_mlp_n_params()] laid out W1 [128][8], b1 [128],
 * W2 [128][128], b2 [128], W3 [128], b3; the forward uses their BF16
 * roundings.  Layers 1 and 3 run in FP32 on CUDA cores; the 128 x 128 layer
 * products (z2, and in the backward d1 and the W2/W1 weight gradients) run on
 * the tcgen05 tensor cores with FP32 values in two BF16 limbs (three products)
 * and FP32 accumulation.  A bounded wait of those kernels that expires (2 s)
 * writes NaN into the first score of the CTA's first tile (forward) or adds
 * NaN to *loss (backward). */
int isdf_mlp_n_params(void);

/* Per-point features feat [n_g][8] (FP32): log10 of the scalar and gradient
 * pivot diagonals w^2 rho^2 and w^2 rho tau (Alg. 1, Sec. II.D), of w, rho =
 * sum_p phi_p^2 and tau = sum_{c,p} (d_c phi_p)^2 (each / 10), the distances to
 * the two nearest nuclei / 5, and log10(r_1 + 1e-3).  nuc_xyz: HOST
 * [n_nuc][3] (n_nuc <= ISDF_MAX_NUC).  Asynchronous. */
int isdf_mlp_features(const double* phi, const double* dphi, const double* w,
                      const double* grid_xyz, int64_t n_g, int n_orb, const double* nuc_xyz,
                      int n_nuc, float* feat, isdf_stream_t stream);

/* scores[n] = network(feat[n][8]).  Asynchronous. */
int isdf_mlp_forward(const float* params, const float* feat, int64_t n, float* scores,
                     isdf_stream_t stream);

/* Adds to grad [n_params] the gradient of (1/n_total) sum over these n points of
 * the weighted binary cross-entropy pos_w y softplus(-s) + (1 - y) softplus(s)
 * (labels y in {0, 1}), and adds the unnormalised loss sum to *loss (device
 * FP64).  Gradients pass through the BF16 rounding unchanged.  Asynchronous. */
int isdf_mlp_backward(const float* params, const float* feat, const float* labels, int64_t n,
                      float pos_w, int64_t n_total, float* grad, double* loss,
                      isdf_stream_t stream);

/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected with the
 * 1-based step count) on params with moments m, v [n_params].  Asynchronous. */
int isdf_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
                  isdf_stream_t stream);

/* out[k] = indices of the k highest scores (ties by lowest index), ascending.
 * Asynchronous. */
int isdf_mlp_topk(const float* scores, int64_t n, int k, int32_t* out, isdf_stream_t stream);

/* isdf_points (fused mode) on the candidate points cand[n_cand] only (distinct
 * grid indices in [0, n_g)); pivots receive grid indices.  Synchronises
 * `stream`; ISDF_E_RANK and ISDF_E_NONFINITE as isdf_points; ISDF_E_ARG when
 * a candidate index lies outside [0, n_g) (checked on the device before any
 * step; such an index is never dereferenced). */
size_t isdf_points_restricted_workspace(int n_cand, int n_orb, int n_mu);
int isdf_points_restricted(const double* phi, const double* dphi, const double* w, int64_t n_g,
                           int n_orb, const int32_t* cand, int n_cand, int n_mu, int32_t* pivots,
                           int* n_mu_out, void* ws, size_t ws_bytes, isdf_stream_t stream);

/* Scalar-channel ISDF fit error of a pivot set over the whole grid:
 *   *eps = sum_g w_g^2 [(sum_p phi_p^2)^2 - sum_mu xi_mu(g) G_{mu g}^2] / sum_g w_g^2 (sum_p phi_p^2)^2
 * with xi from the FP64 normal equations of Eq. isdf-rho (the weighted
 * Frobenius residual).  pivots: device [n_mu], distinct indices in [0, n_g)
 * (ISDF_E_ARG otherwise, checked on the device; such an index is never
 * dereferenced).  eps host.  ISDF_E_NONFINITE when phi or w hold a NaN or Inf
 * or eps is not finite.  Synchronises `stream`. */
size_t isdf_fit_error_workspace(int64_t n_g, int n_orb, int n_mu);
int isdf_fit_error(const double* phi, const double* w, int64_t n_g, int n_orb,
                   const int32_t* pivots, int n_mu, double* eps, void* ws, size_t ws_bytes,
                   isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * xTC density contraction, Terms 1 and 4 (Sec. III.B, Eq. delta-u-dx-kernels):
 *   G_nu  = sum_{i < n_occ} phi_i(r_nu)^2          (closed-shell HF projector)
 *   w~_g  = w_g sum_l G_l xi_l(g)
 *   D4    = sum_g w~_g sum_c calG^c_mu calG^c_nu
 *   H_gc  = sum_l G_l calG^c_{l g},  V_{nu g} = sum_c H_gc calG^c_{nu g}
 *   D1    = sum_g w_g xi_mu(g) V_{nu g},   D = D4 + 2 D1
 * and, when X_packed is not NULL, Terms 2 and 3 in the low-rank projector
 * form with the occupied fields A^s_{a,g,c} = sum_nu C^a_s(nu) calG^c_{nu g}
 * and rho~^s_a(g) = sum_nu C^a_s(nu) xi_nu(g):
 *   X_{qs mu} = sum_g w_g [ xi_mu(g) sum_{a,c} A^s_{a,c} A^q_{a,c}
 *                          + sum_c calG^c_{mu g} sum_a (rho~^s_a A^q_{a,c} + A^s_{a,c} rho~^q_a) ]
 *   for q <= s < n_orb_x, packed row s(s+1)/2 + q.
 * phi_piv [n_mu][n_orb] = phi_p(r_mu); 1 <= n_occ <= n_orb; xi [n_mu][n_g];
 * w [n_g]; calG [>=3][n_mu][n_g] FP64; D [n_mu][n_mu] FP64;
 * X_packed [n_orb_x (n_orb_x + 1) / 2][n_mu] FP64 or NULL.
 * precision: ISDF_PREC_FP64 (CUDA-core FP64 GEMMs) or ISDF_PREC_BF16X3 /
 * ISDF_PREC_BF16X6 (the D4 and D1 contractions and the two GEMM families of
 * X as split-BF16 tcgen05 GEMMs with FP32 accumulation folded every 256 inner
 * points, X always with three limbs; the element-wise parts in FP64);
 * ISDF_PREC_TF32X3 is accepted and runs as ISDF_PREC_BF16X3 (these GEMMs have
 * no TF32 form).
 * Asynchronous for FP64.  The tensor-core precisions synchronise `stream`
 * after the D and X contractions to read the pipeline's wait-status word and
 * return ISDF_E_TIMEOUT if a bounded wait expired, or ISDF_E_NONFINITE if D
 * or X holds a NaN or Inf. */
size_t xtc_density_contract_workspace(int64_t n_g, int n_mu, int n_orb, int n_occ,
                                      int n_orb_x, int precision);
int xtc_density_contract(const double* phi_piv, int n_orb, int n_occ, const double* xi,
                         const double* w, const double* calG, int64_t n_g, int n_mu,
                         double* D, double* X_packed, int n_orb_x, int precision, void* ws,
                         size_t ws_bytes, isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Closed-shell test energies from the factors (Eqs. K-recombine-final,
 * xtc-deltah, xtc-const), occupied block only:
 *   K = 1/2 P12 [K1 - K1swap + K3],  DeltaU = -P12 [C D C - C X]
 *   out[0] = E_K  = sum_{ij} (2 K^{ij}_{ij} - K^{ij}_{ji})
 *   out[1] = E_dU = sum_{ij} (2 DeltaU^{ij}_{ij} - DeltaU^{ij}_{ji})
 *   out[2] = E0   = -2/3 sum_i Delta h_ii   (without nuclear repulsion)
 * W [4][n_mu][n_mu]; D [n_mu][n_mu]; X_packed as above with n_orb_x >= n_occ;
 * phi_piv [n_mu][n_orb]; dphi_piv [3][n_mu][n_orb]; out host [3].  FP64.
 * Synchronises `stream`; ISDF_E_NONFINITE when an energy is NaN or Inf. */
size_t tc_energies_workspace(int n_mu, int n_occ);
int tc_energies(const double* W, const double* D, const double* X_packed,
                const double* phi_piv, const double* dphi_piv, int n_mu, int n_orb,
                int n_occ, double* out, void* ws, size_t ws_bytes, isdf_stream_t stream);

/* The energies call above without a workspace argument, for callers that
 * cannot allocate device memory: code running inside another framework's
 * memory pool (cudaMalloc may synchronise the device and fragments a pool it
 * does not own) and latency-critical loops that must not block on an
 * allocator.  The paper has no counterpart; this is an interface convenience.
 * Arguments, layouts and results are those of tc_energies.  Its scratch is a
 * fixed 16 MiB device array inside the library (held by every GPU that loads
 * the library until exit); sizes needing more (6 n_mu n_occ^2 + 4 n_occ^4
 * doubles plus alignment) return ISDF_E_ARG.  The first call on a device looks
 * up the array's device address with that device current, and looks it up
 * again in a new context of the device (after a cudaDeviceReset); make that
 * first call before any stream capture.  All calls share the array: calls
 * that overlap on the GPU (other streams or host threads) race.  No device
 * memory is allocated.  Synchronises `stream`. */
int tc_energies_noalloc(const double* W, const double* D, const double* X_packed,
                        const double* phi_piv, const double* dphi_piv, int n_mu, int n_orb,
                        int n_occ, double* out, isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Assembly of the xTC Hamiltonian's corrections over every orbital index
 * (final assembly of Sec. III.B and the assembly subsection after it).
 *
 * Two-body panels (Eqs. K-recombine-final and deltaU-four): with the
 * composite indices (p,r) = p n_orb + r and (q,s) = q n_orb + s,
 *   K_panel [pr_end - pr_begin][n_orb^2]:  K_panel[(p,r) - pr_begin][(q,s)] = K^{pq}_{rs}
 *   dU_panel (same shape):                 DeltaU^{pq}_{rs}
 * for the rows pr_begin <= (p,r) < pr_end (either output may be NULL), from
 *   K  = 1/2 P12 [K1 - K1swap + K3],  K1^{pq}_{rs} = sum_c sum_{mu nu} phi_p(mu) d_c phi_r(mu)
 *        u1^c_{mu nu} phi_q(nu) phi_s(nu),  K3 with u3 and C^p_r(mu) = phi_p(mu) phi_r(mu),
 *   DeltaU = -P12 [ sum C^p_r(mu) D_{mu nu} C^q_s(nu) - sum_mu C^p_r(mu) X_{qs mu} ],
 *   P12 T^{pq}_{rs} = T^{pq}_{rs} + T^{qp}_{sr}.
 * A panel is two GEMMs of inner dimension 4 n_mu and 2 n_mu over all n_orb^2
 * columns, streamed panel by panel as in the paper's cost analysis (Sec. IV.C).
 * W [4][n_mu][n_mu]; D [n_mu][n_mu]; X_packed [n_orb (n_orb + 1) / 2][n_mu] (the
 * full X, n_orb_x = n_orb); phi_piv [n_mu][n_orb]; dphi_piv [3][n_mu][n_orb].
 * precision: ISDF_PREC_FP64 (CUDA-core FP64 GEMMs) or ISDF_PREC_BF16X3 /
 * ISDF_PREC_BF16X6 (the two panel GEMMs as split-BF16 tcgen05 GEMMs with FP32
 * accumulation folded every 256 terms, three limbs for either precision since
 * these products cancel strongly; the left factors in FP64).  FP64 is
 * asynchronous; the tensor-core precisions synchronise `stream` and return
 * ISDF_E_TIMEOUT if a bounded wait expired.  0 <= pr_begin < pr_end <= n_orb^2. */
size_t tc_two_body_panel_workspace(int n_mu, int n_orb, int64_t rows, int precision);
int tc_two_body_panel(const double* W, const double* D, const double* X_packed,
                      const double* phi_piv, const double* dphi_piv, int n_mu, int n_orb,
                      int64_t pr_begin, int64_t pr_end, int precision, double* K_panel,
                      double* dU_panel, void* ws, size_t ws_bytes, isdf_stream_t stream);

/* One-body increment, xTC Fock correction and constant for every orbital pair
 * (Eqs. xtc-deltah, xtc-fock, xtc-const), closed shell with the first n_occ
 * orbitals occupied:
 *   delta_h[p][q] = -1/2 sum_{o<n_occ} (2 DeltaU^{po}_{qo} - DeltaU^{po}_{oq})
 *   fock[p][q]    = delta_h[p][q] + sum_{i<n_occ} (2 W^{pi}_{qi} - W^{pi}_{iq}),
 *                   W = -K + DeltaU (not symmetrised)
 *   *e0           = -2/3 sum_{i<n_occ} delta_h[i][i]   (nuclear repulsion not included)
 * computed without forming four-index tensors (contractions of the occupied
 * projector on the pivots with W, D and X: O(n_mu^2 n_orb) work, FP64).
 * Inputs as tc_two_body_panel (X_packed is the full X); delta_h, fock: device
 * [n_orb][n_orb] FP64; e0: host scalar or NULL.  Asynchronous when e0 is
 * NULL; otherwise synchronises `stream` and returns ISDF_E_NONFINITE for a
 * NaN or Inf E0. */
size_t tc_xtc_one_body_workspace(int n_mu, int n_orb);
int tc_xtc_one_body(const double* W, const double* D, const double* X_packed,
                    const double* phi_piv, const double* dphi_piv, int n_mu, int n_orb, int n_occ,
                    double* delta_h, double* fock, double* e0, void* ws, size_t ws_bytes,
                    isdf_stream_t stream);

/* Gather phi_p(r_mu) and d_c phi_p(r_mu): phi_piv [n_mu][n_orb],
 * dphi_piv [3][n_mu][n_orb] (dphi_piv may be NULL); pivots: device [n_mu],
 * indices in [0, n_g).  Asynchronous, so an index outside [0, n_g) cannot be
 * reported: it is never dereferenced and its rows are written as quiet NaN,
 * which the synchronising calls downstream report as ISDF_E_NONFINITE. */
int isdf_gather_pivots(const double* phi, const double* dphi, int64_t n_g, int n_orb,
                       const int32_t* pivots, int n_mu, double* phi_piv, double* dphi_piv,
                       isdf_stream_t stream);

/* ---------------------------------------------------------------------------
 * Reference-variance VMC optimisation of the correlator (Sec. II.C, Eqs. Eloc,
 * var-loss and gn).  Trial function Psi_T = exp(tau) Phi_0: Phi_0 the
 * closed-shell determinant of the first n_occ orbitals (columns of mo_coef),
 * electrons 0 .. n_occ-1 spin up and n_occ .. 2 n_occ-1 spin down; tau =
 * sum_{i<j} u(r_i, r_j) with u of isdf_jastrow (cusp, free terms, one-body
 * term).  The nuclei of the Hamiltonian are the correlator's (jas->nuc_xyz)
 * with charges[I] (host [n_nuc]).  walkers: device [n_walkers][2 n_occ][3]
 * bohr.  theta = (d, b_0 .. b_{T-1}, coef[t][k] row-major), P = 1 + T + T K
 * (isdf_vmc_n_params).  Limits: 1 <= n_occ <= 64, and the per-walker tables
 * must fit one CTA's shared memory (ISDF_E_ARG otherwise).  FP64 throughout.
 *
 * isdf_vmc_local_energy: E[w] = E_loc of Eq. Eloc,
 *   E_loc = -1/2 sum_i [lap_i Phi_0/Phi_0 + 2 grad_i tau . grad_i Phi_0/Phi_0
 *                       + lap_i tau + |grad_i tau|^2] + V,
 *   V = sum_{i<j} 1/r_ij - sum_{i,I} Z_I/r_iI + sum_{I<J} Z_I Z_J/R_IJ,
 * with the correlator's parameters from theta (device [P]) or, when theta is
 * NULL, from jas.  dE (device [P][n_walkers] or NULL): dE_loc/dtheta; the d and
 * b_t rows by central differences of step fd_step, the coefficient rows exact
 * (E_loc is quadratic in them).  b_t rows are 0 when the correlator has no
 * free terms.  A singular determinant gives NaN energies.  Asynchronous. */
int isdf_vmc_n_params(const isdf_jastrow* jas);
size_t isdf_vmc_local_energy_workspace(int n_bf, int n_occ, int64_t n_walkers,
                                       const isdf_jastrow* jas);
int isdf_vmc_local_energy(const isdf_basis* basis, const double* mo_coef, int n_orb, int n_occ,
                          const double* walkers, int64_t n_walkers, const isdf_jastrow* jas,
                          const double* charges, const double* theta, double fd_step, double* E,
                          double* dE, void* ws, size_t ws_bytes, isdf_stream_t stream);

/* n_steps Metropolis sweeps on |Phi_0|^2 (the sample does not depend on the
 * correlator).  Sweep s moves electrons i = 0 .. 2 n_occ-1 in turn:
 *   r' = r_i + sigma normals[s][i][w][0..2],
 *   accepted when uniforms[s][i][w] < (Phi_0(R')/Phi_0(R))^2,
 * the ratio taken against the walker's inverse determinant, which an accepted
 * move updates by Sherman-Morrison (each call starts from a fresh inversion).
 * normals device [n_steps][2 n_occ][n_walkers][3], uniforms device
 * [n_steps][2 n_occ][n_walkers] (the random numbers are inputs); walkers are
 * updated in place; *accepted (device int64) = accepted moves of this call.
 * Asynchronous. */
int isdf_vmc_sample(const isdf_basis* basis, const double* mo_coef, int n_orb, int n_occ,
                    double* walkers, int64_t n_walkers, const double* normals,
                    const double* uniforms, int n_steps, double sigma, int64_t* accepted,
                    isdf_stream_t stream);

/* One Gauss-Newton step of Eq. gn on the clipped objective of Eq. var-loss:
 *   m, dev = mean and mean absolute deviation of E; E~ = clip(E, m - 5 dev, m + 5 dev);
 *   r_k = E~_k - mean(E~); var = sum r_k^2 / (n - 1);
 *   dr = d r / d theta with clipped energies following their bound
 *        (d(m +- 5 dev), d dev = mean(sign(E - m) (dE - dm)));
 *   C = dr dr^T / n + lambda I;  step = -eta C^-1 (2/(n-1) dr r).
 * E device [n_walkers], dE device [n_par][n_walkers]; step device [n_par];
 * stats device [4] = (mean(E~), var, m, dev); theta device [n_par] or NULL:
 * theta += step when the factorisation succeeds.  Synchronises `stream`;
 * ISDF_E_NOT_PD when C is not positive definite (lambda = 0 with a rank-
 * deficient Jacobian).  The paper adapts lambda without stating the rule; the
 * Python front end's vmc_optimize takes a step only when the clipped variance
 * at the new theta is lower (then lambda /= 3), else keeps theta and sets
 * lambda *= 10. */
size_t isdf_vmc_gn_step_workspace(int64_t n_walkers, int n_par);
/* The objective of Eq. var-loss alone: stats device [4] as isdf_vmc_gn_step.
 * Asynchronous. */
int isdf_vmc_objective(const double* E, int64_t n_walkers, double* stats, isdf_stream_t stream);
/* Polyak-Ruppert averaging of the parameters (Sec. II.C: the production
 * correlator averages the stationary tail of the refinement trajectory):
 * avg[p] += (theta[p] - avg[p]) / k for the k-th averaged iterate (k >= 1; k = 1
 * copies theta without reading avg, so avg needs no initial value).  theta, avg:
 * device [n_par].  Asynchronous. */
int isdf_vmc_polyak(const double* theta, double* avg, int n_par, int64_t k, isdf_stream_t stream);
int isdf_vmc_gn_step(const double* E, const double* dE, int64_t n_walkers, int n_par,
                     double lambda, double eta, double* theta, double* step, double* stats,
                     void* ws, size_t ws_bytes, isdf_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* ISDFTC_H */
