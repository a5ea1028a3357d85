// Learned interpolation-point proposer (not in the paper): per-point
// features, a small MLP (8 -> 128 -> 128 -> 1, BF16 weights; its forward and
// backward passes are in mlp_tc.cu) trained by weighted binary cross-entropy
// against the plain pivoted-Cholesky selection, Adam, top-k candidate
// selection, the pivoted Cholesky restricted to the candidates, and the
// scalar-channel ISDF fit error that decides between selections.
#include <cuda_bf16.h>

#include <cmath>

#include "linalg.cuh"
#include "mlp_layout.cuh"

namespace isdf {

size_t points_ws(int64_t n_g, int n_mu);
int points(const double*, const double*, const double*, int64_t, int, int, int, int32_t*, int*,
           void*, size_t, cudaStream_t);

namespace {

using namespace mlpl;

struct Nuclei {
  int n;
  double xyz[ISDF_MAX_NUC][3];
};

__global__ void features_kernel(const double* __restrict__ phi, const double* __restrict__ dphi,
                                const double* __restrict__ w, const double* __restrict__ grid,
                                int64_t n_g, int n_orb, const __grid_constant__ Nuclei nuc,
                                float* __restrict__ feat) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_g) return;
  double rho = 0.0, tau = 0.0;
  for (int p = 0; p < n_orb; ++p) {
    const double v = phi[(int64_t)p * n_g + g];
    rho = fma(v, v, rho);
  }
  for (int c = 0; c < 3; ++c)
    for (int p = 0; p < n_orb; ++p) {
      const double v = dphi[((int64_t)c * n_orb + p) * n_g + g];
      tau = fma(v, v, tau);
    }
  double r1 = 1e300, r2 = 1e300;
  for (int I = 0; I < nuc.n; ++I) {
    const double dx = grid[3 * g] - nuc.xyz[I][0], dy = grid[3 * g + 1] - nuc.xyz[I][1],
                 dz = grid[3 * g + 2] - nuc.xyz[I][2];
    const double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (r < r1) { r2 = r1; r1 = r; } else if (r < r2) { r2 = r; }
  }
  if (nuc.n < 2) r2 = r1;
  const double wg = w[g];
  float* f = feat + g * MF;
  f[0] = (float)(log10(wg * wg * rho * rho + 1e-300) / 10.0);
  f[1] = (float)(log10(wg * wg * rho * tau + 1e-300) / 10.0);
  f[2] = (float)(log10(wg + 1e-300) / 10.0);
  f[3] = (float)(log10(rho + 1e-300) / 10.0);
  f[4] = (float)(log10(tau + 1e-300) / 10.0);
  f[5] = (float)(r1 / 5.0);
  f[6] = (float)(r2 / 5.0);
  f[7] = (float)log10(r1 + 1e-3);
}

__global__ void adam_kernel(float* __restrict__ par, const float* __restrict__ grad,
                            float* __restrict__ m, float* __restrict__ v, int n, float lr,
                            float c1, float c2) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float g = grad[k];
  const float mk = 0.9f * m[k] + 0.1f * g;
  const float vk = 0.999f * v[k] + 0.001f * g * g;
  m[k] = mk;
  v[k] = vk;
  par[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + 1e-8f);
}

__device__ __forceinline__ uint32_t fkey(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}

// k highest scores, ties by lowest index, output in ascending index order.
// One block: radix select of the k-th largest key, then an ordered compaction.
__global__ void __launch_bounds__(1024) topk_kernel(const float* __restrict__ s, int64_t n, int k,
                                                    int32_t* __restrict__ out) {
  __shared__ unsigned int cnt;
  __shared__ uint32_t prefix_s;
  __shared__ int warp_tot[32];
  __shared__ int base_s;
  uint32_t prefix = 0;
  int need = k;  // how many of the remaining keys (those matching prefix) we still want
  for (int b = 31; b >= 0; --b) {
    if (threadIdx.x == 0) cnt = 0;
    __syncthreads();
    const uint32_t mask_hi = b == 31 ? 0u : ~((1u << (b + 1)) - 1u);
    const uint32_t want = prefix | (1u << b);
    unsigned int c = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const uint32_t key = fkey(s[i]);
      if ((key & mask_hi) == (prefix & mask_hi) && (key & (1u << b))) ++c;
    }
    atomicAdd(&cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) {
      if ((int)cnt >= need) prefix_s = want;
      else prefix_s = prefix;
    }
    __syncthreads();
    if (prefix_s == prefix) need -= (int)cnt;
    prefix = prefix_s;
    __syncthreads();
  }
  // keys > prefix are all taken; `need` keys equal to prefix are taken, lowest index first
  const uint32_t kth = prefix;
  if (threadIdx.x == 0) base_s = 0;
  __syncthreads();
  int eq_taken_before = 0;
  for (int64_t c0 = 0; c0 < n; c0 += blockDim.x) {
    const int64_t i = c0 + threadIdx.x;
    const uint32_t key = i < n ? fkey(s[i]) : 0u;
    const int gt = i < n && key > kth;
    const int eq = i < n && key == kth;
    // ordered prefix of eq within the chunk
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned int eq_mask = __ballot_sync(0xffffffffu, eq);
    int eq_before_in_warp = __popc(eq_mask & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[wid] = __popc(eq_mask);
    __syncthreads();
    int eq_before = eq_before_in_warp;
    for (int q = 0; q < wid; ++q) eq_before += warp_tot[q];
    int eq_chunk = 0;
    for (int q = 0; q < 32; ++q) eq_chunk += warp_tot[q];
    const int take = gt || (eq && eq_taken_before + eq_before < need);
    unsigned int tmask = __ballot_sync(0xffffffffu, take);
    int t_before_in_warp = __popc(tmask & ((1u << lane) - 1u));
    __syncthreads();
    if (lane == 0) warp_tot[wid] = __popc(tmask);
    __syncthreads();
    int t_before = t_before_in_warp;
    for (int q = 0; q < wid; ++q) t_before += warp_tot[q];
    int t_chunk = 0;
    for (int q = 0; q < 32; ++q) t_chunk += warp_tot[q];
    if (take) out[base_s + t_before] = (int32_t)i;
    __syncthreads();
    if (threadIdx.x == 0) base_s += t_chunk;
    eq_taken_before += eq_chunk;
    __syncthreads();
  }
}

__global__ void gather_cols_kernel(const double* __restrict__ src, int64_t n_g, int64_t rows,
                                   const int32_t* __restrict__ idx, int n_idx,
                                   double* __restrict__ dst, int* err) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * n_idx) return;
  const int64_t r = e / n_idx;
  const int c = (int)(e % n_idx);
  const int64_t g = idx[c];
  dst[e] = index_ok(g, n_g, err) ? src[r * n_g + g] : __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void map_idx_kernel(const int32_t* __restrict__ sub, const int32_t* __restrict__ cand,
                               int n, int32_t* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = cand[sub[i]];
}

// r-terms of the fit error: out[0] += sum_g w^2 ((sum_p phi^2)^2 - sum_mu xi B),
// out[1] += sum_g w^2 (sum_p phi^2)^2
__global__ void fit_error_kernel(const double* __restrict__ phi, const double* __restrict__ w,
                                 const double* __restrict__ xi, const double* __restrict__ B,
                                 int64_t n_g, int n_orb, int n_mu, double* __restrict__ out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double num = 0.0, den = 0.0;
  if (g < n_g) {
    double rho = 0.0;
    for (int p = 0; p < n_orb; ++p) rho = fma(phi[(int64_t)p * n_g + g], phi[(int64_t)p * n_g + g], rho);
    double fitv = 0.0;
    for (int mu = 0; mu < n_mu; ++mu)
      fitv = fma(xi[(int64_t)mu * n_g + g], B[(int64_t)mu * n_g + g], fitv);
    const double ww = w[g] * w[g];
    num = ww * (rho * rho - fitv);
    den = ww * rho * rho;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(out, num);
    atomicAdd(out + 1, den);
  }
}

// B and X may be the same buffer (the Gram's saved copy), so neither is restrict.
__global__ void square_copy_kernel(const double* __restrict__ G, double* B, double* X,
                                   int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double g = G[i];
    B[i] = g * g;
    X[i] = g * g;
  }
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

__global__ void add_diag_copy_kernel(double* A, const double* S, int n, double lam) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n * n) return;
  A[e] = S[e] + ((e / n) == (e % n) ? lam : 0.0);
}

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)ceil_div(n, t); }

int gather_pivot_rows(const double* phi, int64_t n_g, int n_orb, const int32_t* piv, int n_mu,
                      double* phiP, int* err, cudaStream_t s) {
  // phiP[p][mu] = phi[p][piv[mu]]
  gather_cols_kernel<<<nb((int64_t)n_orb * n_mu), 256, 0, s>>>(phi, n_g, n_orb, piv, n_mu, phiP,
                                                              err);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

}  // namespace

// ----------------------------------------------------------------------------- host entry points

int mlp_n_params() { return N_PAR; }

int mlp_features(const double* phi, const double* dphi, const double* w, const double* grid,
                 int64_t n_g, int n_orb, const double* nuc_xyz, int n_nuc, float* feat,
                 cudaStream_t s) {
  ISDF_ARG(phi && dphi && w && grid && feat && nuc_xyz, "null pointer argument");
  ISDF_ARG(n_g > 0 && n_orb > 0 && n_nuc >= 1 && n_nuc <= ISDF_MAX_NUC, "bad sizes");
  Nuclei nu;
  nu.n = n_nuc;
  for (int I = 0; I < n_nuc; ++I)
    for (int c = 0; c < 3; ++c) nu.xyz[I][c] = nuc_xyz[3 * I + c];
  features_kernel<<<nb(n_g), 256, 0, s>>>(phi, dphi, w, grid, n_g, n_orb, nu, feat);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}


int mlp_forward_tc(const float*, const float*, int64_t, float*, cudaStream_t);
int mlp_backward_tc(const float*, const float*, const float*, int64_t, float, int64_t, float*,
                    double*, cudaStream_t);

int mlp_forward(const float* par, const float* feat, int64_t n, float* scores, cudaStream_t s) {
  ISDF_ARG(par && feat && scores && n > 0, "bad arguments");
  return mlp_forward_tc(par, feat, n, scores, s);
}

int mlp_backward(const float* par, const float* feat, const float* y, int64_t n, float pos_w,
                 int64_t n_total, float* grad, double* loss, cudaStream_t s) {
  ISDF_ARG(par && feat && y && grad && loss && n > 0 && n_total >= n, "bad arguments");
  return mlp_backward_tc(par, feat, y, n, pos_w, n_total, grad, loss, s);
}

int mlp_adam(float* par, const float* grad, float* m, float* v, int t, float lr, cudaStream_t s) {
  ISDF_ARG(par && grad && m && v && t >= 1, "bad arguments");
  const float c1 = 1.0f - powf(0.9f, (float)t), c2 = 1.0f - powf(0.999f, (float)t);
  adam_kernel<<<nb(N_PAR), 256, 0, s>>>(par, grad, m, v, N_PAR, lr, c1, c2);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

int mlp_topk(const float* scores, int64_t n, int k, int32_t* out, cudaStream_t s) {
  ISDF_ARG(scores && out && n > 0 && k > 0 && k <= n, "bad arguments");
  topk_kernel<<<1, 1024, 0, s>>>(scores, n, k, out);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

size_t points_restricted_ws(int n_cand, int n_orb, int n_mu) {
  Carve c(nullptr, 0);
  c.take<int>(64);
  c.take<double>((size_t)4 * n_orb * n_cand + n_cand);
  c.take<int32_t>(n_mu);
  c.take<unsigned char>(points_ws(n_cand, n_mu));
  return c.off;
}

int points_restricted(const double* phi, const double* dphi, const double* w, int64_t n_g,
                      int n_orb, const int32_t* cand, int n_cand, int n_mu, int32_t* pivots,
                      int* n_mu_out, void* ws, size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(phi && dphi && w && cand && pivots && n_mu_out, "null pointer argument");
  ISDF_ARG(n_cand > 0 && n_mu > 0 && n_orb > 0, "bad sizes");
  Carve cv(ws, ws_bytes);
  int* err = cv.take<int>(64);
  double* sub = cv.take<double>((size_t)4 * n_orb * n_cand + n_cand);
  int32_t* spiv = cv.take<int32_t>(n_mu);
  const size_t pws = points_ws(n_cand, n_mu);
  unsigned char* pw = cv.take<unsigned char>(pws);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  double* sphi = sub;
  double* sdphi = sub + (int64_t)n_orb * n_cand;
  double* sw = sub + (int64_t)4 * n_orb * n_cand;
  ISDF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  gather_cols_kernel<<<nb((int64_t)n_orb * n_cand), 256, 0, s>>>(phi, n_g, n_orb, cand, n_cand, sphi,
                                                                 err);
  ISDF_LAUNCH_CHECK();
  gather_cols_kernel<<<nb((int64_t)3 * n_orb * n_cand), 256, 0, s>>>(dphi, n_g, 3 * n_orb, cand,
                                                                     n_cand, sdphi, err);
  ISDF_LAUNCH_CHECK();
  gather_cols_kernel<<<nb(n_cand), 256, 0, s>>>(w, n_g, 1, cand, n_cand, sw, err);
  ISDF_LAUNCH_CHECK();
  int h_err = 0;
  ISDF_TRY(read_error_word(err, &h_err, s));
  if (h_err & DEV_ERR_ARG) {
    set_error("a candidate index lies outside [0, n_g = %lld)", (long long)n_g);
    return ISDF_E_ARG;
  }
  const int rc = points(sphi, sdphi, sw, n_cand, n_orb, n_mu, 0, spiv, n_mu_out, pw, pws, s);
  if (rc != ISDF_OK && rc != ISDF_E_RANK) return rc;
  if (*n_mu_out > 0) {
    map_idx_kernel<<<nb(*n_mu_out), 256, 0, s>>>(spiv, cand, *n_mu_out, pivots);
    ISDF_LAUNCH_CHECK();
  }
  ISDF_CUDA(cudaStreamSynchronize(s));
  return rc;
}

size_t fit_error_ws(int64_t n_g, int n_orb, int n_mu) {
  Carve c(nullptr, 0);
  c.take<int>(64);
  c.take<double>((size_t)n_mu * n_orb);
  for (int i = 0; i < 2; ++i) c.take<double>((size_t)n_mu * n_mu);
  for (int i = 0; i < 3; ++i) c.take<double>((size_t)n_mu * n_g);
  c.take<double>(2);
  c.take<int>(1);
  return c.off;
}

int fit_error(const double* phi, const double* w, int64_t n_g, int n_orb, const int32_t* piv,
              int n_mu, double* eps, void* ws, size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(phi && w && piv && eps && n_g > 0 && n_orb > 0 && n_mu > 0, "bad arguments");
  Carve cv(ws, ws_bytes);
  int* err = cv.take<int>(64);
  double* phiP = cv.take<double>((size_t)n_mu * n_orb);  // [n_orb][n_mu]
  double* Gram = cv.take<double>((size_t)n_mu * n_mu);
  double* Save = cv.take<double>((size_t)n_mu * n_mu);
  double* G = cv.take<double>((size_t)n_mu * n_g);
  double* B = cv.take<double>((size_t)n_mu * n_g);
  double* X = cv.take<double>((size_t)n_mu * n_g);
  double* acc = cv.take<double>(2);
  int* info = cv.take<int>(1);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  ISDF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  ISDF_TRY(gather_pivot_rows(phi, n_g, n_orb, piv, n_mu, phiP, err, s));  // phiP [n_orb][n_mu]
  ISDF_TRY(scan_nonfinite(phi, (int64_t)n_orb * n_g, err, s));
  ISDF_TRY(scan_nonfinite(w, n_g, err, s));
  int h_err = 0;
  ISDF_TRY(read_error_word(err, &h_err, s));
  if (h_err & DEV_ERR_ARG) {
    set_error("a pivot index lies outside [0, n_g = %lld)", (long long)n_g);
    return ISDF_E_ARG;
  }
  if (h_err & DEV_ERR_NONFINITE) {
    set_error("non-finite phi or w (NaN or Inf)");
    return ISDF_E_NONFINITE;
  }
  // G_PP = phiP^T phiP, G = phiP^T phi
  Dgemm g;
  g.M = n_mu; g.N = n_mu; g.K = n_orb;
  g.A = phiP; g.a_rs = 1; g.a_cs = n_mu; g.a_bs = 0;
  g.B = phiP; g.b_rs = n_mu; g.b_cs = 1; g.b_bs = 0;
  g.C = Gram; g.ldc = n_mu; g.c_bs = 0;
  ISDF_TRY(dgemm(g, s));
  Dgemm r;
  r.M = n_mu; r.N = n_g; r.K = n_orb;
  r.A = phiP; r.a_rs = 1; r.a_cs = n_mu; r.a_bs = 0;
  r.B = phi; r.b_rs = n_g; r.b_cs = 1; r.b_bs = 0;
  r.C = G; r.ldc = n_g; r.c_bs = 0;
  ISDF_TRY(dgemm(r, s));
  square_copy_kernel<<<nb((int64_t)n_mu * n_mu), 256, 0, s>>>(Gram, Save, Save, (int64_t)n_mu * n_mu);
  ISDF_LAUNCH_CHECK();
  square_copy_kernel<<<nb((int64_t)n_mu * n_g), 256, 0, s>>>(G, B, X, (int64_t)n_mu * n_g);
  ISDF_LAUNCH_CHECK();
  double lam = 0.0;
  for (int tries = 0;; ++tries) {
    add_diag_copy_kernel<<<nb((int64_t)n_mu * n_mu), 256, 0, s>>>(Gram, Save, n_mu, lam);
    ISDF_LAUNCH_CHECK();
    ISDF_TRY(dpotrf_lower(Gram, n_mu, info, s));
    int h_info = 0;
    ISDF_CUDA(cudaMemcpyAsync(&h_info, info, sizeof(int), cudaMemcpyDeviceToHost, s));
    ISDF_CUDA(cudaStreamSynchronize(s));
    if (h_info == 0) break;
    if (tries >= 8) {
      set_error("fit-error Gram not positive definite after jitter");
      return ISDF_E_NOT_PD;
    }
    if (tries == 0) {
      double d0 = 0.0;
      max_diag_kernel<<<1, 256, 0, s>>>(Save, n_mu, acc);
      ISDF_LAUNCH_CHECK();
      ISDF_CUDA(cudaMemcpyAsync(&d0, acc, sizeof(double), cudaMemcpyDeviceToHost, s));
      ISDF_CUDA(cudaStreamSynchronize(s));
      lam = 1e-14 * d0;
    } else {
      lam *= 10.0;
    }
  }
  ISDF_TRY(dpotrs_lower(Gram, n_mu, X, n_g, n_g, s));
  ISDF_CUDA(cudaMemsetAsync(acc, 0, 2 * sizeof(double), s));
  fit_error_kernel<<<nb(n_g), 256, 0, s>>>(phi, w, X, B, n_g, n_orb, n_mu, acc);
  ISDF_LAUNCH_CHECK();
  double h[2];
  ISDF_CUDA(cudaMemcpyAsync(h, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ISDF_CUDA(cudaStreamSynchronize(s));
  *eps = h[0] / h[1];
  if (!std::isfinite(*eps)) {
    set_error("fit error is not finite");
    return ISDF_E_NONFINITE;
  }
  return ISDF_OK;
}

}  // namespace isdf
