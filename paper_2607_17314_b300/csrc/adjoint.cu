// Adjoint of the Jastrow kernels with respect to the correlator parameters
// (not in the paper).  For a seed Wbar = {Wbar^x, Wbar^y, Wbar^z, Wbar^sq} and
// L(theta) = sum_c <Wbar^c, W^c(theta)> (W from Eqs. K1-isdf / K3-isdf):
//
//   dL/dtheta_j = sum_{g,g'} sum_{c<3} (M^c + 2 M^sq K_c)(g,g') d K_c(g,g') / d theta_j
//   M^c(g,g')   = sum_mu (w xi~^c)[mu][g] Bhat^c[mu][g'],  Bhat^c = Wbar^c (w xi)
//   (M^sq uses w xi and Wbar^sq), with K_sq = sum_c K_c^2.
//
// Bhat is one FP64 GEMM; the pair kernel recomputes the M^c tile from the
// factors (nothing of size N_g^2 is stored), regenerates grad_1 u and its
// parameter derivatives for each pair (term loops unrolled over the supported
// exponents m, n <= 3, o <= 4, so powers come from register tables), and
// reduces the per-thread sums per block into FP64 atomics.  Parameters: theta = (d, b, c_0 .. c_{K-1}) for a
// correlator with one nucleus type.
#include "linalg.cuh"

namespace isdf {
namespace {

constexpr int AT = 32;       // tile edge (g and g')
template <class T>
struct AMu {
  static constexpr int v = sizeof(T) == 8 ? 16 : 32;  // mu chunk of the M tile (<= 32 KB)
};
constexpr int AMAXK = 30;    // free terms supported

template <class T>
struct AdjArgs {
  const T* Ah;     // [4][n_mu][n_g] (w xi~^c, w xi)
  const T* Bh;     // [4][n_mu][n_g] Bhat^c
  const double* grid;
  int64_t n_g;
  int n_mu;
  const T* tab;    // [n_g][n_nuc][8]: A, gA(3), A_b, gA_b(3)
  double* dtheta;  // [2 + K]
};

// Per-point nucleus table: A = b r/(1+br), grad A = b/(1+br)^2 e,
// dA/db = r/(1+br)^2, d(grad A)/db = (1-br)/(1+br)^3 e.
template <class T>
__global__ void adj_table_kernel(const double* grid, int64_t n_g, const __grid_constant__ isdf_jastrow J,
                                 T* tab) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_g * J.n_nuc) return;
  const int64_t g = e / J.n_nuc;
  const int I = (int)(e % J.n_nuc);
  const double b = J.b[J.nuc_type[I]];
  double v[3];
  for (int c = 0; c < 3; ++c) v[c] = grid[3 * g + c] - J.nuc_xyz[I][c];
  const double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  const double den = 1.0 + b * r;
  const double inv = r > 0.0 ? 1.0 / r : 0.0;
  T* o = tab + e * 8;
  o[0] = (T)(b * r / den);
  for (int c = 0; c < 3; ++c) o[1 + c] = (T)(b / (den * den) * v[c] * inv);
  o[4] = (T)(r / (den * den));
  for (int c = 0; c < 3; ++c) o[5 + c] = (T)((1.0 - b * r) / (den * den * den) * v[c] * inv);
}

// p[e] for a warp-uniform exponent e (register arrays stay in registers)
template <class T, int N>
__device__ __forceinline__ T sel(const T (&p)[N], int e) {
  T v = p[0];
#pragma unroll
  for (int i = 1; i < N; ++i) v = e == i ? p[i] : v;
  return v;
}

template <class T>
__global__ void __launch_bounds__(256) adj_pair_kernel(AdjArgs<T> a, const __grid_constant__ isdf_jastrow J) {
  constexpr int AMU = AMu<T>::v;
  __shared__ T As[4][AMU][AT];
  __shared__ T Bs[4][AMU][AT];
  __shared__ double red[8][AMAXK + 2];
  const int t = threadIdx.x;
  const int64_t g0 = (int64_t)blockIdx.y * AT, h0 = (int64_t)blockIdx.x * AT;
  // each thread: g row (t / 8), g' columns (t % 8) + 8 j, j < 4
  const int tg = t >> 3, th = t & 7;
  T M[4][4];
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int j = 0; j < 4; ++j) M[c][j] = (T)0;
  const int64_t plane = (int64_t)a.n_mu * a.n_g;
  for (int mu0 = 0; mu0 < a.n_mu; mu0 += AMU) {
    for (int e = t; e < 4 * AMU * AT; e += 256) {
      const int c = e / (AMU * AT), r = (e / AT) % AMU, col = e % AT;
      const int mu = mu0 + r;
      const int64_t ga = g0 + col, hb = h0 + col;
      As[c][r][col] = (mu < a.n_mu && ga < a.n_g) ? a.Ah[c * plane + (int64_t)mu * a.n_g + ga] : (T)0;
      Bs[c][r][col] = (mu < a.n_mu && hb < a.n_g) ? a.Bh[c * plane + (int64_t)mu * a.n_g + hb] : (T)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < AMU; ++r) {
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const T av = As[c][r][tg];
#pragma unroll
        for (int j = 0; j < 4; ++j) M[c][j] += av * Bs[c][r][th + 8 * j];
      }
    }
    __syncthreads();
  }

  const int K = J.n_terms;
  const T d = (T)J.d;
  // per-thread sums of the 4 pairs (term k at index 2 + k); the term loops are
  // unrolled so that the accumulators stay in registers
  T acc[AMAXK + 2];
#pragma unroll
  for (int p = 0; p < AMAXK + 2; ++p) acc[p] = (T)0;
  const int64_t g = g0 + tg;
  if (g < a.n_g) {
    const double* rg = a.grid + 3 * g;
    for (int j = 0; j < 4; ++j) {
      const int64_t h = h0 + th + 8 * j;
      if (h >= a.n_g || h == g) continue;
      const double* rh = a.grid + 3 * h;
      const T dx = (T)(rg[0] - rh[0]), dy = (T)(rg[1] - rh[1]), dz = (T)(rg[2] - rh[2]);
      const T r = sqrt(dx * dx + dy * dy + dz * dz);
      const T ex = dx / r, ey = dy / r, ez = dz / r;
      const T den = (T)1 + d * r;
      const T E = d * r / den;
      const T dEdr = d / (den * den);
      const T E_d = r / (den * den);
      const T dEdr_d = ((T)1 - d * r) / (den * den * den);
      T pE[5];
      pE[0] = (T)1;
#pragma unroll
      for (int i = 1; i < 5; ++i) pE[i] = pE[i - 1] * E;
      // pass 1: grad u
      T cE = J.cusp ? (T)0.5 / d : (T)0;
      T gx = 0, gy = 0, gz = 0;
      for (int I = 0; I < J.n_nuc; ++I) {
        const T* ti = a.tab + (g * J.n_nuc + I) * 8;
        const T* tj = a.tab + (h * J.n_nuc + I) * 8;
        const T Ai = ti[0], Aj = tj[0];
        const T pi[4] = {(T)1, Ai, Ai * Ai, Ai * Ai * Ai};
        const T pj[4] = {(T)1, Aj, Aj * Aj, Aj * Aj * Aj};
        T cA = 0;
#pragma unroll
        for (int k = 0; k < AMAXK; ++k) {
          if (k < K) {
            const int m = J.mno[k][0], n = J.mno[k][1], o = J.mno[k][2];
            const T c = (T)J.coef[0][k];
            T Da = 0;
            if (m > 0) Da += (T)m * sel(pi, m - 1) * sel(pj, n);
            if (n > 0) Da += (T)n * sel(pj, m) * sel(pi, n - 1);
            cA += c * Da * sel(pE, o);
            if (o > 0)
              cE += c * (sel(pi, m) * sel(pj, n) + sel(pj, m) * sel(pi, n)) * (T)o * sel(pE, o - 1);
          }
        }
        gx += cA * ti[1];
        gy += cA * ti[2];
        gz += cA * ti[3];
      }
      const T Kx = gx + cE * dEdr * ex, Ky = gy + cE * dEdr * ey, Kz = gz + cE * dEdr * ez;
      const T msq2 = (T)2 * M[3][j];
      const T cx = M[0][j] + msq2 * Kx, cy = M[1][j] + msq2 * Ky, cz = M[2][j] + msq2 * Kz;
      const T ce = cx * ex + cy * ey + cz * ez;  // coef . e_ij
      // pass 2: parameter derivatives contracted with coef
      T cE_d = J.cusp ? (T)-0.5 / (d * d) : (T)0;
      T cE_b = 0;
      T s_d = 0, s_b = 0;  // sum_I coef . (d(cA_I gA_I)/d{d,b})
      for (int I = 0; I < J.n_nuc; ++I) {
        const T* ti = a.tab + (g * J.n_nuc + I) * 8;
        const T* tj = a.tab + (h * J.n_nuc + I) * 8;
        const T Ai = ti[0], Aj = tj[0], Ai_b = ti[4], Aj_b = tj[4];
        const T pi[4] = {(T)1, Ai, Ai * Ai, Ai * Ai * Ai};
        const T pj[4] = {(T)1, Aj, Aj * Aj, Aj * Aj * Aj};
        const T cg = cx * ti[1] + cy * ti[2] + cz * ti[3];        // coef . gA
        const T cgb = cx * ti[5] + cy * ti[6] + cz * ti[7];       // coef . dgA/db
        T cA = 0, cA_d = 0, cA_b = 0;
#pragma unroll
        for (int k = 0; k < AMAXK; ++k) {
          if (k < K) {
            const int m = J.mno[k][0], n = J.mno[k][1], o = J.mno[k][2];
            const T c = (T)J.coef[0][k];
            const T S = sel(pi, m) * sel(pj, n) + sel(pj, m) * sel(pi, n);
            T S_b = 0, Da = 0, Da_b = 0;
            if (m > 0) {
              S_b += (T)m * sel(pi, m - 1) * sel(pj, n) * Ai_b +
                     (T)m * sel(pj, m - 1) * sel(pi, n) * Aj_b;
              Da += (T)m * sel(pi, m - 1) * sel(pj, n);
              if (m > 1) Da_b += (T)(m * (m - 1)) * sel(pi, m - 2) * sel(pj, n) * Ai_b;
              if (n > 0) Da_b += (T)(m * n) * sel(pi, m - 1) * sel(pj, n - 1) * Aj_b;
            }
            if (n > 0) {
              S_b += (T)n * sel(pi, m) * sel(pj, n - 1) * Aj_b +
                     (T)n * sel(pj, m) * sel(pi, n - 1) * Ai_b;
              Da += (T)n * sel(pj, m) * sel(pi, n - 1);
              if (m > 0) Da_b += (T)(n * m) * sel(pj, m - 1) * sel(pi, n - 1) * Aj_b;
              if (n > 1) Da_b += (T)(n * (n - 1)) * sel(pj, m) * sel(pi, n - 2) * Ai_b;
            }
            const T Eo = sel(pE, o);
            const T Eo_d = o > 0 ? (T)o * sel(pE, o - 1) * E_d : (T)0;
            T dc = Da * Eo * cg;  // d/dc_k of the cA_I gA_I part
            if (o > 0) {
              const T Eo1 = sel(pE, o - 1);
              const T Eo1_d = o > 1 ? (T)(o - 1) * sel(pE, o - 2) * E_d : (T)0;
              dc += S * (T)o * Eo1 * dEdr * ce;
              cE_d += c * S * (T)o * Eo1_d;
              cE_b += c * S_b * (T)o * Eo1;
            }
            acc[2 + k] += dc;
            cA += c * Da * Eo;
            cA_d += c * Da * Eo_d;
            cA_b += c * Da_b * Eo;
          }
        }
        s_d += cA_d * cg;
        s_b += cA_b * cg + cA * cgb;
      }
      acc[0] += (cE_d * dEdr + cE * dEdr_d) * ce + s_d;
      acc[1] += cE_b * dEdr * ce + s_b;
    }
  }
  // block reduction: warp shuffles, then one row per warp in shared memory
  const int P = 2 + K;
#pragma unroll
  for (int p = 0; p < AMAXK + 2; ++p) {
    if (p >= P) break;
    double v = (double)acc[p];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) red[t >> 5][p] = v;
  }
  __syncthreads();
  if (t < P) {
    double s = 0.0;
    for (int w8 = 0; w8 < 8; ++w8) s += red[w8][t];
    atomicAdd(a.dtheta + t, s);
  }
}

template <class T>
__global__ void to_type_kernel(const double* src, const double* scale, int64_t n, int64_t ld,
                               T* dst) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  double v = src[e];
  if (scale) v *= scale[e % ld];
  dst[e] = (T)v;
}

inline unsigned nb(int64_t n) { return (unsigned)ceil_div(n, 256); }

template <class T>
int run_adjoint(const double* grid, const double* w, const double* xi, const double* xig, int64_t n_g,
                int n_mu, const isdf_jastrow& J, const double* Wbar, double* dtheta, void* ws,
                size_t ws_bytes, cudaStream_t s) {
  const int64_t plane = (int64_t)n_mu * n_g;
  Carve cv(ws, ws_bytes);
  double* Bh64 = cv.take<double>(4 * plane);
  T* Ah = cv.take<T>(4 * plane);
  T* Bh = cv.take<T>(4 * plane);
  T* tab = cv.take<T>((size_t)n_g * J.n_nuc * 8);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  // Bhat^c = Wbar^c (w xi)
  Dgemm g;
  g.M = n_mu; g.N = n_g; g.K = n_mu;
  g.A = Wbar; g.a_rs = n_mu; g.a_cs = 1; g.a_bs = (int64_t)n_mu * n_mu;
  g.B = xi; g.b_rs = n_g; g.b_cs = 1; g.b_bs = 0;
  g.C = Bh64; g.ldc = n_g; g.c_bs = plane;
  g.batch = 4;
  // w scales the inner index of B: fold it in after the GEMM via the conversion
  ISDF_TRY(dgemm(g, s));
  to_type_kernel<T><<<nb(4 * plane), 256, 0, s>>>(Bh64, w, 4 * plane, n_g, Bh);
  ISDF_LAUNCH_CHECK();
  to_type_kernel<T><<<nb(3 * plane), 256, 0, s>>>(xig, w, 3 * plane, n_g, Ah);
  ISDF_LAUNCH_CHECK();
  to_type_kernel<T><<<nb(plane), 256, 0, s>>>(xi, w, plane, n_g, Ah + 3 * plane);
  ISDF_LAUNCH_CHECK();
  if (J.n_nuc > 0) {
    adj_table_kernel<T><<<nb(n_g * J.n_nuc), 256, 0, s>>>(grid, n_g, J, tab);
    ISDF_LAUNCH_CHECK();
  }
  ISDF_CUDA(cudaMemsetAsync(dtheta, 0, sizeof(double) * (2 + J.n_terms), s));
  AdjArgs<T> a;
  a.Ah = Ah; a.Bh = Bh; a.grid = grid; a.n_g = n_g; a.n_mu = n_mu; a.tab = tab; a.dtheta = dtheta;
  dim3 grd((unsigned)ceil_div(n_g, AT), (unsigned)ceil_div(n_g, AT));
  ISDF_ARG(grd.y < 65536u, "n_g too large for the adjoint grid");
  adj_pair_kernel<T><<<grd, 256, 0, s>>>(a, J);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

}  // namespace

size_t adjoint_ws(int64_t n_g, int n_mu, int n_nuc, int precision) {
  const size_t el = precision == ISDF_PREC_FP64 ? 8 : 4;
  Carve c(nullptr, 0);
  const size_t plane = (size_t)n_mu * n_g;
  c.take<double>(4 * plane);
  c.take<unsigned char>(4 * plane * el);
  c.take<unsigned char>(4 * plane * el);
  c.take<unsigned char>((size_t)n_g * n_nuc * 8 * el);
  return c.off;
}

int adjoint(const double* grid, const double* w, const double* xi, const double* xig, int64_t n_g,
            int n_mu, const isdf_jastrow& J, const double* Wbar, int precision, double* dtheta,
            void* ws, size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(grid && w && xi && xig && Wbar && dtheta, "null pointer argument");
  ISDF_ARG(n_g > 0 && n_mu > 0, "empty sizes");
  if (J.n_types != 1 || J.n_terms > AMAXK) {
    set_error("the adjoint takes one nucleus type and at most %d free terms", AMAXK);
    return ISDF_E_UNSUPPORTED;
  }
  for (int k = 0; k < J.n_terms; ++k)
    if (J.mno[k][0] > 3 || J.mno[k][1] > 3 || J.mno[k][2] > 4) {
      set_error("the adjoint takes exponents m, n <= 3 and o <= 4 (term %d)", k);
      return ISDF_E_UNSUPPORTED;
    }
  if (precision == ISDF_PREC_FP64)
    return run_adjoint<double>(grid, w, xi, xig, n_g, n_mu, J, Wbar, dtheta, ws, ws_bytes, s);
  return run_adjoint<float>(grid, w, xi, xig, n_g, n_mu, J, Wbar, dtheta, ws, ws_bytes, s);
}

}  // namespace isdf
