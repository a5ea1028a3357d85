// Least-squares ISDF fit of the auxiliary densities (Eq. isdf-rho and the
// normal equations of Sec. II.D), FP64 on CUDA cores.
//
//   G[mu][g] = sum_p phi_p(r_mu) phi_p(r_g)                        (GEMM)
//   scalar:     Gram = G_PP o G_PP,        RHS = G o G
//   gradient c: Gram = dG^c_PP o G_PP,     RHS = dG^c o G
//   Cholesky of each Gram with the adaptive Tikhonov retry of Sec. IV.B,
//   then two blocked triangular solves over all grid columns in place.
// fit_mode 1 takes the right-hand-side GEMMs and the triangular solves (98 %
// of the flops) as FP64 products emulated exactly on the tensor cores
// (emu64.cu); the Grams and their Cholesky factors stay FP64 on CUDA cores.
#include "linalg.cuh"

namespace isdf {

size_t em_dgemm_ws(int64_t Mmax, int64_t Nmax, int64_t Kmax);
int em_dgemm(int64_t M, int64_t N, int64_t K, const double* A, int64_t a_rs, int64_t a_cs,
             const double* B, int64_t b_rs, int64_t b_cs, double alpha, bool overwrite,
             double* C, int64_t ldc, void* ws, size_t ws_bytes, cudaStream_t s);
size_t em_potrs_ws(int n, int64_t nrhs);
int em_potrs_lower(const double* L, int n, double* B, int64_t nrhs, int64_t ldb, void* ws,
                   size_t ws_bytes, cudaStream_t s);

namespace {

__global__ void gather_pivots_kernel(const double* __restrict__ src, int64_t n_g, int n_orb,
                                     const int32_t* __restrict__ piv, int n_mu,
                                     double* __restrict__ dst, int nplanes, int* err) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t per = (int64_t)n_mu * n_orb;
  if (e >= per * nplanes) return;
  int c = (int)(e / per);
  int64_t r = e % per;
  int mu = (int)(r / n_orb), p = (int)(r % n_orb);
  const int64_t g = piv[mu];
  dst[e] = index_ok(g, n_g, err) ? src[((int64_t)c * n_orb + p) * n_g + g] : __longlong_as_double(0x7ff8000000000000ll);
}

// x[i] = a[i] * b[i]
__global__ void hadamard_kernel(double* __restrict__ x, const double* __restrict__ a,
                                const double* __restrict__ b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] = a[i] * b[i];
}

// rhs_grad[c][i] *= G[i] for c < 3, then G[i] = G[i]^2
__global__ void rhs_finish_kernel(double* __restrict__ G, double* __restrict__ dG, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double g = G[i];
  dG[i] *= g;
  dG[n + i] *= g;
  dG[2 * n + i] *= g;
  G[i] = g * g;
}

__global__ void add_diag_kernel(double* A, const double* S, int n, double lam) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  int i = (int)(e / n), j = (int)(e % n);
  A[e] = S[e] + (i == j ? lam : 0.0);
}

__global__ void max_diag_kernel(const double* A, int n, double* out) {
  __shared__ double sm[256];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += 256) m = fmax(m, A[(int64_t)i * n + i]);
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

inline unsigned nblocks(int64_t n, int t = 256) { return (unsigned)ceil_div(n, t); }

}  // namespace

static int gather_pivots_err(const double* phi, const double* dphi, int64_t n_g, int n_orb,
                             const int32_t* piv, int n_mu, double* phiP, double* dphiP, int* err,
                             cudaStream_t s) {
  ISDF_ARG(phi && piv && phiP, "null pointer argument");
  ISDF_ARG(n_orb > 0 && n_g > 0, "empty sizes");
  if (n_mu <= 0) return ISDF_OK;
  int64_t per = (int64_t)n_mu * n_orb;
  gather_pivots_kernel<<<nblocks(per), 256, 0, s>>>(phi, n_g, n_orb, piv, n_mu, phiP, 1, err);
  ISDF_LAUNCH_CHECK();
  if (dphi && dphiP) {
    gather_pivots_kernel<<<nblocks(3 * per), 256, 0, s>>>(dphi, n_g, n_orb, piv, n_mu, dphiP, 3,
                                                          err);
    ISDF_LAUNCH_CHECK();
  }
  return ISDF_OK;
}

int gather_pivots(const double* phi, const double* dphi, int64_t n_g, int n_orb,
                  const int32_t* piv, int n_mu, double* phiP, double* dphiP, cudaStream_t s) {
  return gather_pivots_err(phi, dphi, n_g, n_orb, piv, n_mu, phiP, dphiP, nullptr, s);
}

// Workspace of the fit, carved in this order by both the size query and the call.
struct FitWs {
  int* err;
  double *phiP, *dphiP, *GPP, *Gram, *Save, *scal;
  int* info;
  void* em = nullptr;  // emulated products (fit_mode 1)
  size_t em_bytes = 0;
  void carve(Carve& cv, int64_t n_g, int n_orb, int n_mu, int mode) {
    err = cv.take<int>(64);
    phiP = cv.take<double>((size_t)n_mu * n_orb);
    dphiP = cv.take<double>((size_t)3 * n_mu * n_orb);
    GPP = cv.take<double>((size_t)n_mu * n_mu);
    Gram = cv.take<double>((size_t)n_mu * n_mu);
    Save = cv.take<double>((size_t)n_mu * n_mu);
    scal = cv.take<double>(2);
    info = cv.take<int>(1);
    if (mode == 1) {
      const size_t a = em_dgemm_ws(n_mu, n_g, n_orb), b = em_potrs_ws(n_mu, n_g);
      em_bytes = a > b ? a : b;
      em = cv.take<char>(em_bytes);
    }
  }
};

size_t fit_ws(int64_t n_g, int n_orb, int n_mu, int mode) {
  Carve c(nullptr, 0);
  FitWs f;
  f.carve(c, n_g, n_orb, n_mu, mode);
  return c.off;
}

int fit(const double* phi, const double* dphi, int64_t n_g, int n_orb, const int32_t* piv,
        int n_mu, double* xi, double* xig, double* jitter_used, double jitter_init,
        double jitter_growth, int max_tries, int mode, void* ws, size_t ws_bytes,
        cudaStream_t s) {
  ISDF_ARG(phi && dphi && piv && xi && xig, "null pointer argument");
  ISDF_ARG(n_g > 0 && n_orb > 0 && n_mu > 0, "empty sizes");
  ISDF_ARG(mode == 0 || mode == 1, "fit_mode must be 0 or 1");
  Carve cv(ws, ws_bytes);
  FitWs f;
  f.carve(cv, n_g, n_orb, n_mu, mode);
  int* err = f.err;
  double *phiP = f.phiP, *dphiP = f.dphiP, *GPP = f.GPP, *Gram = f.Gram, *Save = f.Save;
  double* scal = f.scal;
  int* info = f.info;
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);

  ISDF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  ISDF_TRY(gather_pivots_err(phi, dphi, n_g, n_orb, piv, n_mu, phiP, dphiP, err, s));
  ISDF_TRY(scan_nonfinite(phi, (int64_t)n_orb * n_g, err, s));
  ISDF_TRY(scan_nonfinite(dphi, (int64_t)3 * n_orb * n_g, err, s));
  int h_err = 0;
  ISDF_TRY(read_error_word(err, &h_err, s));
  if (h_err & DEV_ERR_ARG) {
    set_error("a pivot index lies outside [0, n_g = %lld)", (long long)n_g);
    return ISDF_E_ARG;
  }
  if (h_err & DEV_ERR_NONFINITE) {
    set_error("non-finite phi or dphi (NaN or Inf)");
    return ISDF_E_NONFINITE;
  }
  const int64_t nn = (int64_t)n_mu * n_mu;
  const int64_t ng = (int64_t)n_mu * n_g;

  // G_PP
  Dgemm g;
  g.M = n_mu; g.N = n_mu; g.K = n_orb;
  g.A = phiP; g.a_rs = n_orb; g.a_cs = 1; g.a_bs = 0;
  g.B = phiP; g.b_rs = 1; g.b_cs = n_orb; g.b_bs = 0;
  g.C = GPP; g.ldc = n_mu; g.c_bs = 0;
  ISDF_TRY(dgemm(g, s));

  // right-hand sides: G into xi, dG^c into xig, then the Hadamard products
  if (mode == 1) {
    ISDF_TRY(em_dgemm(n_mu, n_g, n_orb, phiP, n_orb, 1, phi, n_g, 1, 1.0, true, xi, n_g, f.em,
                      f.em_bytes, s));
    for (int c = 0; c < 3; ++c)
      ISDF_TRY(em_dgemm(n_mu, n_g, n_orb, dphiP + (int64_t)c * n_mu * n_orb, n_orb, 1,
                        dphi + (int64_t)c * n_orb * n_g, n_g, 1, 1.0, true, xig + c * ng, n_g,
                        f.em, f.em_bytes, s));
  } else {
    Dgemm r;
    r.M = n_mu; r.N = n_g; r.K = n_orb;
    r.A = phiP; r.a_rs = n_orb; r.a_cs = 1; r.a_bs = 0;
    r.B = phi; r.b_rs = n_g; r.b_cs = 1; r.b_bs = 0;
    r.C = xi; r.ldc = n_g; r.c_bs = 0;
    ISDF_TRY(dgemm(r, s));
    r.A = dphiP; r.a_bs = (int64_t)n_mu * n_orb;
    r.B = dphi; r.b_bs = (int64_t)n_orb * n_g;
    r.C = xig; r.c_bs = ng; r.batch = 3;
    ISDF_TRY(dgemm(r, s));
  }
  rhs_finish_kernel<<<nblocks(ng), 256, 0, s>>>(xi, xig, ng);
  ISDF_LAUNCH_CHECK();

  for (int ch = 0; ch < 4; ++ch) {
    if (ch == 0) {
      hadamard_kernel<<<nblocks(nn), 256, 0, s>>>(Save, GPP, GPP, nn);
      ISDF_LAUNCH_CHECK();
    } else {
      Dgemm q = g;
      q.A = dphiP + (int64_t)(ch - 1) * n_mu * n_orb;
      q.B = q.A;
      q.C = Gram;
      ISDF_TRY(dgemm(q, s));
      hadamard_kernel<<<nblocks(nn), 256, 0, s>>>(Save, Gram, GPP, nn);
      ISDF_LAUNCH_CHECK();
    }
    double lam = 0.0;
    double maxd = 0.0;
    int tries = 0;
    for (;;) {
      add_diag_kernel<<<nblocks(nn), 256, 0, s>>>(Gram, Save, n_mu, lam);
      ISDF_LAUNCH_CHECK();
      ISDF_TRY(dpotrf_lower(Gram, n_mu, info, s));
      int h_info = 0;
      ISDF_CUDA(cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, s));
      ISDF_CUDA(cudaStreamSynchronize(s));
      if (h_info == 0) break;
      if (tries == 0) {
        max_diag_kernel<<<1, 256, 0, s>>>(Save, n_mu, scal);
        ISDF_LAUNCH_CHECK();
        ISDF_CUDA(cudaMemcpyAsync(&maxd, scal, sizeof(double), cudaMemcpyDeviceToHost, s));
        ISDF_CUDA(cudaStreamSynchronize(s));
        lam = jitter_init * maxd;
      } else {
        lam *= jitter_growth;
      }
      if (++tries > max_tries) {
        set_error("Gram matrix %d not positive definite after %d jitter retries", ch, max_tries);
        return ISDF_E_NOT_PD;
      }
    }
    if (jitter_used) jitter_used[ch] = lam;
    double* rhs = ch == 0 ? xi : xig + (int64_t)(ch - 1) * ng;
    if (mode == 1)
      ISDF_TRY(em_potrs_lower(Gram, n_mu, rhs, n_g, n_g, f.em, f.em_bytes, s));
    else
      ISDF_TRY(dpotrs_lower(Gram, n_mu, rhs, n_g, n_g, s));
  }
  // overflow in the solves
  ISDF_TRY(scan_nonfinite(xi, ng, err, s));
  ISDF_TRY(scan_nonfinite(xig, 3 * ng, err, s));
  ISDF_TRY(read_error_word(err, &h_err, s));
  if (h_err & DEV_ERR_NONFINITE) {
    set_error("non-finite values in the fitted xi (overflow in the solves)");
    return ISDF_E_NONFINITE;
  }
  return ISDF_OK;
}

}  // namespace isdf
