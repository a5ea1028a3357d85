// extern "C" entry points of libisdftc (declared in include/isdftc.h).
#include <stdarg.h>

#include <cmath>

#include <atomic>

#include "common.cuh"
#include "jastrow.cuh"

namespace isdf {

static thread_local char g_err[1024] = "";
static std::atomic<uint64_t> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// implemented in the kernel translation units
size_t eval_orbitals_ws(int n_bf, int64_t n_g, int mode, int n_orb_max);
int eval_orbitals(const isdf_basis*, const double*, int, const double*, int64_t, double*, double*,
                  int, void*, size_t, cudaStream_t);
size_t points_ws(int64_t n_g, int n_mu);
int points(const double*, const double*, const double*, int64_t, int, int, int, int32_t*, int*,
           void*, size_t, cudaStream_t);
size_t points_ranks_ws(int64_t n_g, int n_phi, int n_grad);
int points_ranks(const double*, const double*, const double*, int64_t, int, int, int, int32_t*,
                 int*, void*, size_t, cudaStream_t);
size_t fit_ws(int64_t, int, int, int);
int fit(const double*, const double*, int64_t, int, const int32_t*, int, double*, double*,
        double*, double, double, int, int, void*, size_t, cudaStream_t);
size_t em_dgemm_ws(int64_t, int64_t, int64_t);
int em_dgemm(int64_t, int64_t, int64_t, const double*, int64_t, int64_t, const double*, int64_t,
             int64_t, double, bool, double*, int64_t, void*, size_t, cudaStream_t);
int gather_pivots(const double*, const double*, int64_t, int, const int32_t*, int, double*,
                  double*, cudaStream_t);
size_t wbuild_fp64_ws(int64_t n_g, const isdf_jastrow* J);
int wbuild_fp64(const double*, const double*, const double*, const double*, int64_t, int, int64_t,
                int64_t, const isdf_jastrow&, double*, double*, int, void*, size_t, cudaStream_t);
size_t wbuild_tc_ws(int64_t, int, int64_t, int64_t, int, const isdf_jastrow*);
int wbuild_tc(const double*, const double*, const double*, const double*, int64_t, int, int64_t,
              int64_t, const isdf_jastrow&, const isdf_options&, double*, double*, void*, size_t,
              cudaStream_t);
size_t wbuild_streamed_ws(int64_t, int, int64_t, int64_t, int, const isdf_jastrow*);
int wbuild_streamed(const double*, const double*, const double*, const double*, int64_t, int,
                    int64_t, int64_t, const isdf_jastrow&, const isdf_options&, double*, void*,
                    size_t, cudaStream_t);
size_t xtc_ws(int64_t, int, int, int, int, int);
int xtc(const double*, int, int, const double*, const double*, const double*, int64_t, int,
        double*, double*, int, int, void*, size_t, cudaStream_t);
size_t energies_ws(int, int);
int energies(const double*, const double*, const double*, const double*, const double*, int, int,
             int, double*, void*, size_t, cudaStream_t);
size_t adjoint_ws(int64_t, int, int, int);
int adjoint(const double*, const double*, const double*, const double*, int64_t, int64_t, int64_t,
            int, const isdf_jastrow&, const double*, int, double*, void*, size_t, cudaStream_t);
int mlp_n_params();
int mlp_features(const double*, const double*, const double*, const double*, int64_t, int,
                 const double*, int, float*, cudaStream_t);
int mlp_forward(const float*, const float*, int64_t, float*, cudaStream_t);
int mlp_backward(const float*, const float*, const float*, int64_t, float, int64_t, float*, double*,
                 cudaStream_t);
int mlp_adam(float*, const float*, float*, float*, int, float, cudaStream_t);
int mlp_topk(const float*, int64_t, int, int32_t*, cudaStream_t);
size_t points_restricted_ws(int, int, int);
int points_restricted(const double*, const double*, const double*, int64_t, int, const int32_t*,
                      int, int, int32_t*, int*, void*, size_t, cudaStream_t);
size_t fit_error_ws(int64_t, int, int);
int fit_error(const double*, const double*, int64_t, int, const int32_t*, int, double*, void*,
              size_t, cudaStream_t);
int energies_noalloc(const double*, const double*, const double*, const double*, const double*,
                     int, int, int, double*, cudaStream_t);
size_t xtc_one_body_ws(int, int);
int xtc_one_body(const double*, const double*, const double*, const double*, const double*, int, int,
                 int, double*, double*, double*, void*, size_t, cudaStream_t);
size_t xtc_panel_ws(int, int, int64_t, int);
int xtc_panel(const double*, const double*, const double*, const double*, const double*, int, int,
              int64_t, int64_t, int, double*, double*, void*, size_t, cudaStream_t);

int vmc_n_params(const isdf_jastrow&);
size_t vmc_local_energy_ws(int, int, int64_t, const isdf_jastrow&);
int vmc_local_energy(const isdf_basis*, const double*, int, int, const double*, int64_t,
                     const isdf_jastrow&, const double*, const double*, double, double*, double*,
                     void*, size_t, cudaStream_t);
int vmc_sample(const isdf_basis*, const double*, int, int, double*, int64_t, const double*,
               const double*, int, double, int64_t*, cudaStream_t);
size_t vmc_gn_step_ws(int64_t, int);
int vmc_objective(const double*, int64_t, double*, cudaStream_t);
int vmc_polyak(const double*, double*, int, int64_t, cudaStream_t);
int vmc_gn_step(const double*, const double*, int64_t, int, double, double, double*, double*,
                double*, void*, size_t, cudaStream_t);

static int check_jastrow(const isdf_jastrow* J) {
  ISDF_ARG(J, "null Jastrow");
  ISDF_ARG(J->n_nuc >= 0 && J->n_nuc <= ISDF_MAX_NUC, "n_nuc out of range");
  ISDF_ARG(J->n_types >= 1 && J->n_types <= ISDF_MAX_TYPES, "n_types out of range");
  ISDF_ARG(J->n_terms >= 0 && J->n_terms <= ISDF_MAX_TERMS, "n_terms out of range");
  ISDF_ARG(J->d > 0.0 && std::isfinite(J->d), "d must be positive");
  for (int I = 0; I < J->n_nuc; ++I) {
    ISDF_ARG(J->nuc_type[I] >= 0 && J->nuc_type[I] < J->n_types, "nucleus type out of range");
    for (int c = 0; c < 3; ++c)
      ISDF_ARG(std::isfinite(J->nuc_xyz[I][c]), "nucleus position not finite");
  }
  for (int k = 0; k < J->n_terms; ++k)
    for (int e = 0; e < 3; ++e)
      ISDF_ARG(J->mno[k][e] >= 0 && J->mno[k][e] <= 8, "exponent out of range");
  // b_I enters only through the free terms (Eq. bh-scaled needs b_I > 0)
  for (int t = 0; t < J->n_types && J->n_terms > 0; ++t) {
    ISDF_ARG(J->b[t] > 0.0 && std::isfinite(J->b[t]), "b must be positive");
    for (int k = 0; k < J->n_terms; ++k)
      ISDF_ARG(std::isfinite(J->coef[t][k]), "Jastrow coefficient not finite");
  }
  if (chi_on(*J)) {
    ISDF_ARG(J->n_elec >= 2, "the one-body term needs n_elec >= 2");
    ISDF_ARG(J->n_nuc >= 1, "the one-body term needs nuclei");
    for (int t = 0; t < J->n_types; ++t)
      ISDF_ARG(std::isfinite(J->chi_a[t]) && std::isfinite(J->chi_b[t]) && J->chi_b[t] > 0.0,
               "one-body term: chi_a finite and chi_b positive");
  }
  return ISDF_OK;
}

}  // namespace isdf

using namespace isdf;

extern "C" {

const char* isdf_last_error(void) { return g_err; }
int isdf_abi_version(void) { return 2; }
uint64_t isdf_kernel_launches(void) { return g_launches.load(); }

size_t isdf_eval_orbitals_workspace(int n_bf, int64_t n_g) {
  return eval_orbitals_ws(n_bf, n_g, 0, 1);
}

size_t isdf_eval_orbitals_workspace_mode(int n_bf, int64_t n_g, int n_orb, int mode) {
  if (mode != 0 && mode != 1) return 0;
  return eval_orbitals_ws(n_bf, n_g, mode, n_orb > 0 ? n_orb : 1);
}

int isdf_eval_orbitals_mode(const isdf_basis* basis, const double* mo_coef, int n_orb,
                            const double* grid_xyz, int64_t n_g, double* phi, double* dphi,
                            int mode, void* ws, size_t ws_bytes, isdf_stream_t stream) {
  return eval_orbitals(basis, mo_coef, n_orb, grid_xyz, n_g, phi, dphi, mode, ws, ws_bytes,
                       (cudaStream_t)stream);
}

int isdf_eval_orbitals(const isdf_basis* basis, const double* mo_coef, int n_orb,
                       const double* grid_xyz, int64_t n_g, double* phi, double* dphi, void* ws,
                       size_t ws_bytes, isdf_stream_t stream) {
  return eval_orbitals(basis, mo_coef, n_orb, grid_xyz, n_g, phi, dphi, 0, ws, ws_bytes,
                       (cudaStream_t)stream);
}

size_t isdf_points_workspace(int64_t n_g, int n_mu) { return points_ws(n_g, n_mu); }

int isdf_points(const double* phi, const double* dphi, const double* w, int64_t n_g, int n_orb,
                int n_mu, int mode, int32_t* pivots, int* n_mu_out, void* ws, size_t ws_bytes,
                isdf_stream_t stream) {
  return points(phi, dphi, w, n_g, n_orb, n_mu, mode, pivots, n_mu_out, ws, ws_bytes,
                (cudaStream_t)stream);
}

size_t isdf_points_fixed_rank_workspace(int64_t n_g, int n_ch_phi, int n_ch_grad) {
  return points_ranks_ws(n_g, n_ch_phi, n_ch_grad);
}

int isdf_points_fixed_rank(const double* phi, const double* dphi, const double* w, int64_t n_g,
                           int n_orb, int n_ch_phi, int n_ch_grad, int32_t* pivots,
                           int* n_mu_out, void* ws, size_t ws_bytes, isdf_stream_t stream) {
  return points_ranks(phi, dphi, w, n_g, n_orb, n_ch_phi, n_ch_grad, pivots, n_mu_out, ws,
                      ws_bytes, (cudaStream_t)stream);
}

size_t isdf_fit_workspace(int64_t n_g, int n_orb, int n_mu) {
  return fit_ws(n_g, n_orb, n_mu, 0);
}

size_t isdf_fit_workspace_mode(int64_t n_g, int n_orb, int n_mu, int fit_mode) {
  return (fit_mode == 0 || fit_mode == 1) ? fit_ws(n_g, n_orb, n_mu, fit_mode) : 0;
}

size_t isdf_dgemm_emulated_workspace(int64_t M, int64_t N, int64_t K) {
  return em_dgemm_ws(M > 0 ? M : 1, N > 0 ? N : 1, K > 0 ? K : 1);
}

int isdf_dgemm_emulated(int64_t M, int64_t N, int64_t K, const double* A, int64_t lda,
                        const double* B, int64_t ldb, double alpha, double beta, double* C,
                        int64_t ldc, void* ws, size_t ws_bytes, isdf_stream_t stream) {
  ISDF_ARG(M >= 0 && N >= 0 && K >= 0, "negative sizes");
  ISDF_ARG(beta == 0.0 || beta == 1.0, "beta must be 0 or 1");
  ISDF_ARG(std::isfinite(alpha), "alpha must be finite");
  if (M == 0 || N == 0) return ISDF_OK;
  ISDF_ARG(C && (K == 0 || (A && B)), "null pointer argument");
  ISDF_ARG(lda >= K && ldb >= N && ldc >= N, "leading dimensions too small");
  return em_dgemm(M, N, K, A, lda, 1, B, ldb, 1, alpha, beta == 0.0, C, ldc, ws, ws_bytes,
                  (cudaStream_t)stream);
}

int isdf_fit(const double* phi, const double* dphi, int64_t n_g, int n_orb, const int32_t* pivots,
             int n_mu, double* xi, double* xi_grad, double* jitter_used,
             const isdf_options* options, void* ws, size_t ws_bytes, isdf_stream_t stream) {
  double j0 = 1e-14, growth = 10.0;
  int tries = 8, mode = 0;
  if (options) {
    ISDF_ARG(options->jitter_init >= 0.0 && options->jitter_growth >= 0.0,
             "negative jitter policy");
    if (options->jitter_init > 0.0) j0 = options->jitter_init;
    if (options->jitter_growth > 0.0) growth = options->jitter_growth;
    if (options->max_jitter_tries != 0) tries = options->max_jitter_tries < 0 ? 0 : options->max_jitter_tries;
    ISDF_ARG(options->fit_mode == 0 || options->fit_mode == 1, "fit_mode must be 0 or 1");
    mode = options->fit_mode;
  }
  return fit(phi, dphi, n_g, n_orb, pivots, n_mu, xi, xi_grad, jitter_used, j0, growth, tries,
             mode, ws, ws_bytes, (cudaStream_t)stream);
}

int isdf_gather_pivots(const double* phi, const double* dphi, int64_t n_g, int n_orb,
                       const int32_t* pivots, int n_mu, double* phi_piv, double* dphi_piv,
                       isdf_stream_t stream) {
  return gather_pivots(phi, dphi, n_g, n_orb, pivots, n_mu, phi_piv, dphi_piv,
                       (cudaStream_t)stream);
}

size_t tc_kernel_build_workspace(int64_t n_g, int n_mu, int64_t g_begin, int64_t g_end,
                                 int precision, const isdf_jastrow* jas) {
  if (precision == ISDF_PREC_FP64) return wbuild_fp64_ws(n_g, jas);
  return wbuild_tc_ws(n_g, n_mu, g_begin, g_end, precision, jas);
}

int tc_kernel_build(const double* grid_xyz, const double* w, const double* xi,
                    const double* xi_grad, int64_t n_g, int n_mu, int64_t g_begin, int64_t g_end,
                    const isdf_jastrow* jas, const isdf_options* options, double* W, double* calG,
                    void* ws, size_t ws_bytes, isdf_stream_t stream) {
  ISDF_TRY(check_jastrow(jas));
  ISDF_ARG(grid_xyz && w && xi && xi_grad && W && calG, "null pointer argument");
  ISDF_ARG(n_g > 0 && n_mu > 0, "empty sizes");
  ISDF_ARG(g_begin >= 0 && g_begin < g_end && g_end <= n_g, "bad grid slice");
  ISDF_ARG(n_g < (1ll << 31) - 64, "n_g too large");
  isdf_options opt = {ISDF_PREC_BF16X3, 0, 0, 1, 0, nullptr, 0.0, 0.0, 0, 0};
  if (options) opt = *options;
  ISDF_ARG(opt.wait_limit_ms >= 0, "negative wait limit");
  const WaitLimitScope wait_scope(opt.wait_limit_ms);
  cudaStream_t s = (cudaStream_t)stream;
  if (opt.precision == ISDF_PREC_FP64) {
    return wbuild_fp64(grid_xyz, w, xi, xi_grad, n_g, n_mu, g_begin, g_end, *jas, W, calG,
                       opt.sync_check, ws, ws_bytes, s);
  }
  if (opt.precision != ISDF_PREC_BF16X3 && opt.precision != ISDF_PREC_BF16X6 &&
      opt.precision != ISDF_PREC_TF32X3) {
    set_error("unknown precision %d", opt.precision);
    return ISDF_E_ARG;
  }
  return wbuild_tc(grid_xyz, w, xi, xi_grad, n_g, n_mu, g_begin, g_end, *jas, opt, W, calG, ws,
                   ws_bytes, s);
}

size_t tc_kernel_build_streamed_workspace(int64_t n_g, int n_mu, int64_t bra, int64_t ket,
                                          int precision, const isdf_jastrow* jas) {
  if (precision == ISDF_PREC_FP64 || bra <= 0 || ket <= 0) return 0;
  return wbuild_streamed_ws(n_g, n_mu, bra, ket, precision, jas);
}

int tc_kernel_build_streamed(const double* grid_xyz, const double* w, const double* xi_host,
                             const double* xi_grad_host, int64_t n_g, int n_mu, int64_t bra,
                             int64_t ket, const isdf_jastrow* jas, const isdf_options* options,
                             double* W, void* ws, size_t ws_bytes, isdf_stream_t stream) {
  ISDF_TRY(check_jastrow(jas));
  ISDF_ARG(grid_xyz && w && xi_host && xi_grad_host && W, "null pointer argument");
  ISDF_ARG(n_g > 0 && n_mu > 0, "empty sizes");
  ISDF_ARG(n_g < (1ll << 31) - 64, "n_g too large");
  isdf_options opt = {ISDF_PREC_BF16X3, 0, 0, 1, 0, nullptr, 0.0, 0.0, 0, 0};
  if (options) opt = *options;
  ISDF_ARG(opt.precision == ISDF_PREC_BF16X3 || opt.precision == ISDF_PREC_BF16X6 ||
               opt.precision == ISDF_PREC_TF32X3,
           "the streamed build takes the tensor-core precisions");
  ISDF_ARG(opt.wait_limit_ms >= 0, "negative wait limit");
  const WaitLimitScope wait_scope(opt.wait_limit_ms);
  return wbuild_streamed(grid_xyz, w, xi_host, xi_grad_host, n_g, n_mu, bra, ket, *jas, opt, W, ws,
                         ws_bytes, (cudaStream_t)stream);
}

size_t xtc_density_contract_workspace(int64_t n_g, int n_mu, int n_orb, int n_occ, int n_orb_x,
                                      int precision) {
  return xtc_ws(n_g, n_mu, n_orb, n_occ, n_orb_x, precision);
}

int xtc_density_contract(const double* phi_piv, int n_orb, int n_occ, const double* xi,
                         const double* w, const double* calG, int64_t n_g, int n_mu, double* D,
                         double* X_packed, int n_orb_x, int precision, void* ws, size_t ws_bytes,
                         isdf_stream_t stream) {
  return xtc(phi_piv, n_orb, n_occ, xi, w, calG, n_g, n_mu, D, X_packed, n_orb_x, precision, ws,
             ws_bytes, (cudaStream_t)stream);
}

size_t tc_kernel_adjoint_workspace(int64_t n_g, int n_mu, int n_nuc, int precision) {
  return adjoint_ws(n_g, n_mu, n_nuc, precision);
}

int tc_kernel_adjoint(const double* grid_xyz, const double* w, const double* xi,
                      const double* xi_grad, int64_t n_g, int n_mu, const isdf_jastrow* jas,
                      const double* Wbar, int precision, double* dtheta, void* ws,
                      size_t ws_bytes, isdf_stream_t stream) {
  ISDF_TRY(check_jastrow(jas));
  ISDF_ARG(precision == ISDF_PREC_FP64 || precision == ISDF_PREC_FP32,
           "adjoint precision must be ISDF_PREC_FP64 or ISDF_PREC_FP32");
  return adjoint(grid_xyz, w, xi, xi_grad, n_g, 0, n_g, n_mu, *jas, Wbar, precision, dtheta, ws,
                 ws_bytes, (cudaStream_t)stream);
}

int tc_kernel_adjoint_range(const double* grid_xyz, const double* w, const double* xi,
                            const double* xi_grad, int64_t n_g, int n_mu, int64_t g_begin,
                            int64_t g_end, const isdf_jastrow* jas, const double* Wbar,
                            int precision, double* dtheta, void* ws, size_t ws_bytes,
                            isdf_stream_t stream) {
  ISDF_TRY(check_jastrow(jas));
  ISDF_ARG(precision == ISDF_PREC_FP64 || precision == ISDF_PREC_FP32,
           "adjoint precision must be ISDF_PREC_FP64 or ISDF_PREC_FP32");
  return adjoint(grid_xyz, w, xi, xi_grad, n_g, g_begin, g_end, n_mu, *jas, Wbar, precision,
                 dtheta, ws, ws_bytes, (cudaStream_t)stream);
}

int isdf_mlp_n_params(void) { return mlp_n_params(); }

int isdf_mlp_features(const double* phi, const double* dphi, const double* w,
                      const double* grid_xyz, int64_t n_g, int n_orb, const double* nuc_xyz,
                      int n_nuc, float* feat, isdf_stream_t stream) {
  return mlp_features(phi, dphi, w, grid_xyz, n_g, n_orb, nuc_xyz, n_nuc, feat,
                      (cudaStream_t)stream);
}

int isdf_mlp_forward(const float* params, const float* feat, int64_t n, float* scores,
                     isdf_stream_t stream) {
  return mlp_forward(params, feat, n, scores, (cudaStream_t)stream);
}

int isdf_mlp_backward(const float* params, const float* feat, const float* labels, int64_t n,
                      float pos_w, int64_t n_total, float* grad, double* loss,
                      isdf_stream_t stream) {
  return mlp_backward(params, feat, labels, n, pos_w, n_total, grad, loss, (cudaStream_t)stream);
}

int isdf_mlp_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
                  isdf_stream_t stream) {
  return mlp_adam(params, grad, m, v, step, lr, (cudaStream_t)stream);
}

int isdf_mlp_topk(const float* scores, int64_t n, int k, int32_t* out, isdf_stream_t stream) {
  return mlp_topk(scores, n, k, out, (cudaStream_t)stream);
}

size_t isdf_points_restricted_workspace(int n_cand, int n_orb, int n_mu) {
  return points_restricted_ws(n_cand, n_orb, n_mu);
}

int isdf_points_restricted(const double* phi, const double* dphi, const double* w, int64_t n_g,
                           int n_orb, const int32_t* cand, int n_cand, int n_mu, int32_t* pivots,
                           int* n_mu_out, void* ws, size_t ws_bytes, isdf_stream_t stream) {
  return points_restricted(phi, dphi, w, n_g, n_orb, cand, n_cand, n_mu, pivots, n_mu_out, ws,
                           ws_bytes, (cudaStream_t)stream);
}

size_t isdf_fit_error_workspace(int64_t n_g, int n_orb, int n_mu) {
  return fit_error_ws(n_g, n_orb, n_mu);
}

int isdf_fit_error(const double* phi, const double* w, int64_t n_g, int n_orb,
                   const int32_t* pivots, int n_mu, double* eps, void* ws, size_t ws_bytes,
                   isdf_stream_t stream) {
  return fit_error(phi, w, n_g, n_orb, pivots, n_mu, eps, ws, ws_bytes, (cudaStream_t)stream);
}

size_t tc_energies_workspace(int n_mu, int n_occ) { return energies_ws(n_mu, n_occ); }

int tc_energies(const double* W, const double* D, const double* X_packed, const double* phi_piv,
                const double* dphi_piv, int n_mu, int n_orb, int n_occ, double* out, void* ws,
                size_t ws_bytes, isdf_stream_t stream) {
  return energies(W, D, X_packed, phi_piv, dphi_piv, n_mu, n_orb, n_occ, out, ws, ws_bytes,
                  (cudaStream_t)stream);
}

int tc_energies_noalloc(const double* W, const double* D, const double* X_packed,
                        const double* phi_piv, const double* dphi_piv, int n_mu, int n_orb,
                        int n_occ, double* out, isdf_stream_t stream) {
  return energies_noalloc(W, D, X_packed, phi_piv, dphi_piv, n_mu, n_orb, n_occ, out,
                          (cudaStream_t)stream);
}

size_t tc_xtc_one_body_workspace(int n_mu, int n_orb) { return xtc_one_body_ws(n_mu, n_orb); }

int tc_xtc_one_body(const double* W, const double* D, const double* X_packed,
                    const double* phi_piv, const double* dphi_piv, int n_mu, int n_orb, int n_occ,
                    double* delta_h, double* fock, double* e0, void* ws, size_t ws_bytes,
                    isdf_stream_t stream) {
  return xtc_one_body(W, D, X_packed, phi_piv, dphi_piv, n_mu, n_orb, n_occ, delta_h, fock, e0,
                      ws, ws_bytes, (cudaStream_t)stream);
}

size_t tc_two_body_panel_workspace(int n_mu, int n_orb, int64_t rows, int precision) {
  return xtc_panel_ws(n_mu, n_orb, rows, precision);
}

int tc_two_body_panel(const double* W, const double* D, const double* X_packed,
                      const double* phi_piv, const double* dphi_piv, int n_mu, int n_orb,
                      int64_t pr_begin, int64_t pr_end, int precision, double* K_panel,
                      double* dU_panel, void* ws, size_t ws_bytes, isdf_stream_t stream) {
  return xtc_panel(W, D, X_packed, phi_piv, dphi_piv, n_mu, n_orb, pr_begin, pr_end, precision,
                   K_panel, dU_panel, ws, ws_bytes, (cudaStream_t)stream);
}


int isdf_vmc_n_params(const isdf_jastrow* jas) { return jas ? vmc_n_params(*jas) : 0; }

size_t isdf_vmc_local_energy_workspace(int n_bf, int n_occ, int64_t n_walkers,
                                       const isdf_jastrow* jas) {
  return jas ? vmc_local_energy_ws(n_bf, n_occ, n_walkers, *jas) : 0;
}

int isdf_vmc_local_energy(const isdf_basis* basis, const double* mo_coef, int n_orb, int n_occ,
                          const double* walkers, int64_t n_walkers, const isdf_jastrow* jas,
                          const double* charges, const double* theta, double fd_step, double* E,
                          double* dE, void* ws, size_t ws_bytes, isdf_stream_t stream) {
  ISDF_TRY(check_jastrow(jas));
  return vmc_local_energy(basis, mo_coef, n_orb, n_occ, walkers, n_walkers, *jas, charges, theta,
                          fd_step, E, dE, ws, ws_bytes, (cudaStream_t)stream);
}

int isdf_vmc_sample(const isdf_basis* basis, const double* mo_coef, int n_orb, int n_occ,
                    double* walkers, int64_t n_walkers, const double* normals,
                    const double* uniforms, int n_steps, double sigma, int64_t* accepted,
                    isdf_stream_t stream) {
  return vmc_sample(basis, mo_coef, n_orb, n_occ, walkers, n_walkers, normals, uniforms, n_steps,
                    sigma, accepted, (cudaStream_t)stream);
}

int isdf_vmc_objective(const double* E, int64_t n_walkers, double* stats, isdf_stream_t stream) {
  return vmc_objective(E, n_walkers, stats, (cudaStream_t)stream);
}

int isdf_vmc_polyak(const double* theta, double* avg, int n_par, int64_t k,
                    isdf_stream_t stream) {
  return vmc_polyak(theta, avg, n_par, k, (cudaStream_t)stream);
}

size_t isdf_vmc_gn_step_workspace(int64_t n_walkers, int n_par) {
  return vmc_gn_step_ws(n_walkers, n_par);
}

int isdf_vmc_gn_step(const double* E, const double* dE, int64_t n_walkers, int n_par,
                     double lambda, double eta, double* theta, double* step, double* stats,
                     void* ws, size_t ws_bytes, isdf_stream_t stream) {
  return vmc_gn_step(E, dE, n_walkers, n_par, lambda, eta, theta, step, stats, ws, ws_bytes,
                     (cudaStream_t)stream);
}
}  // extern "C"
