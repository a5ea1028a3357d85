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
// parameter derivatives for each pair, and reduces the per-thread sums per
// block into FP64 atomics.  The terms are folded by exponent group {m, n}
// (m, n <= 3; 10 groups fixed at compile time) and E power o <= 4: per pair,
// the nucleus sums of S, dS/dA, their b-derivatives and cg-weighted forms are
// taken once per group, and the derivative of term k is the (group, power)
// combination that it belongs to.  Parameters: theta = (d, b, c_0 .. c_{K-1}) for a
// correlator with one nucleus type.
#include <cuda_bf16.h>

#include "jastrow.cuh"
#include "linalg.cuh"

namespace isdf {

int splitgemm(int limbs, int batch, const void* const* A, const void* const* B, int64_t M,
              int64_t N, int64_t Kp, int64_t kchunk, int64_t fold, double* out, int64_t ldo,
              int64_t out_bs, double scale, int* err, cudaStream_t s);

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
  int64_t g_begin, g_end;  // outer points of this call (the sums are additive over slices)
  int n_mu;
  const T* tab;    // [n_g][n_nuc][8]: A, gA(3), A_b, gA_b(3)
  const double* chi;  // [n][3] grad chi / (N - 1) of the outer points chi0 .. (one-body term), or null
  int64_t chi0;
  double* sums;    // [2 + NGRP * 5]: d, b, then (group, E power) sums
  T gc[10][5];     // C_G[o] = sum of c_k over the terms of group G with E power o
};

// Terms grouped by the unordered exponent pair {m, n} (m <= n <= 3): group G
// holds (m, n) = (gm(G), gn(G)); S = A^m B^n + B^m A^n and its derivatives are
// the same for (m, n) and (n, m).
constexpr int NGRP = 10;
__host__ __device__ constexpr int gm(int G) { return G < 4 ? 0 : G < 7 ? 1 : G < 9 ? 2 : 3; }
__host__ __device__ constexpr int gn(int G) { return G < 4 ? G : G < 7 ? G - 3 : G < 9 ? G - 5 : 3; }
__host__ __device__ constexpr int grp_of(int m, int n) {
  return m > n ? grp_of(n, m) : m == 0 ? n : m == 1 ? 3 + n : m == 2 ? 5 + n : 9;
}

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

// Block reduction of the per-thread sums into a.sums: warp shuffles, then one
// row per warp in shared memory, then FP64 atomics.
template <class T>
__device__ __forceinline__ void adj_block_reduce(const T (&acc)[2 + NGRP * 5],
                                                 double (&red)[8][2 + NGRP * 5], double* sums) {
  constexpr int P = 2 + NGRP * 5;
  const int t = threadIdx.x;
#pragma unroll
  for (int q = 0; q < P; ++q) {
    double v = (double)acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) red[t >> 5][q] = v;
  }
  __syncthreads();
  if (t < P) {
    double sum = 0.0;
    for (int w8 = 0; w8 < 8; ++w8) sum += red[w8][t];
    atomicAdd(sums + t, sum);
  }
}

// Contribution of the ordered pair (g, h), h != g, to the per-thread sums:
// [0] d, [1] b, [2 + 5 G + o] group G and E power o, given the recomputed
// M^c(g, h) (m0 .. m2) and M^sq(g, h) (m3).
template <class T>
__device__ __forceinline__ void adj_pair_terms(const AdjArgs<T>& a, const isdf_jastrow& J, T d,
                                               int64_t g, int64_t h, const double* rg, T m0,
                                               T m1, T m2, T m3, T (&acc)[2 + NGRP * 5]) {
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
  // E weights of each group: P0 = sum_o C_G[o] E^o, P1 = its E-derivative, P2 the second
  T P0[NGRP], P1[NGRP], P2[NGRP];
#pragma unroll
  for (int G = 0; G < NGRP; ++G) {
    P0[G] = (T)0;
    P1[G] = (T)0;
    P2[G] = (T)0;
#pragma unroll
    for (int o = 0; o < 5; ++o) {
      P0[G] += a.gc[G][o] * pE[o];
      if (o > 0) P1[G] += a.gc[G][o] * (T)o * pE[o - 1];
      if (o > 1) P2[G] += a.gc[G][o] * (T)(o * (o - 1)) * pE[o - 2];
    }
  }
  // pass 1: grad u, and Y_G = sum_I S_G
  T cE = J.cusp ? (T)0.5 / d : (T)0;
  T gx = 0, gy = 0, gz = 0;
  T Y[NGRP];
#pragma unroll
  for (int G = 0; G < NGRP; ++G) Y[G] = (T)0;
  for (int I = 0; I < J.n_nuc; ++I) {
    const T* ti = a.tab + (g * J.n_nuc + I) * 8;
    const T* tj = a.tab + (h * J.n_nuc + I) * 8;
    const T Ai = ti[0], Aj = tj[0];
    const T pi[4] = {(T)1, Ai, Ai * Ai, Ai * Ai * Ai};
    const T pj[4] = {(T)1, Aj, Aj * Aj, Aj * Aj * Aj};
    T cA = 0;
#pragma unroll
    for (int G = 0; G < NGRP; ++G) {
      const int m = gm(G), n = gn(G);
      const T S = pi[m] * pj[n] + pj[m] * pi[n];
      T Da = 0;
      if (m > 0) Da += (T)m * pi[m > 0 ? m - 1 : 0] * pj[n];
      if (n > 0) Da += (T)n * pi[n > 0 ? n - 1 : 0] * pj[m];
      cA += P0[G] * Da;
      cE += P1[G] * S;
      Y[G] += S;
    }
    gx += cA * ti[1];
    gy += cA * ti[2];
    gz += cA * ti[3];
  }
  T Kx = gx + cE * dEdr * ex, Ky = gy + cE * dEdr * ey, Kz = gz + cE * dEdr * ez;
  if (a.chi) {  // parameter-free, so it enters only through K_c in the M^sq factor
    const double* hc = a.chi + 3 * (g - a.chi0);
    Kx += (T)hc[0];
    Ky += (T)hc[1];
    Kz += (T)hc[2];
  }
  const T msq2 = (T)2 * m3;
  const T cx = m0 + msq2 * Kx, cy = m1 + msq2 * Ky, cz = m2 + msq2 * Kz;
  const T ce = cx * ex + cy * ey + cz * ez;  // coef . e_ij
  // pass 2: X_G = sum_I Da cg, Z_G = sum_I dS/db, V_G = sum_I (dDa/db cg + Da cgb)
  T X[NGRP], Z[NGRP], V[NGRP];
#pragma unroll
  for (int G = 0; G < NGRP; ++G) X[G] = Z[G] = V[G] = (T)0;
  for (int I = 0; I < J.n_nuc; ++I) {
    const T* ti = a.tab + (g * J.n_nuc + I) * 8;
    const T* tj = a.tab + (h * J.n_nuc + I) * 8;
    const T Ai = ti[0], Aj = tj[0], Ai_b = ti[4], Aj_b = tj[4];
    const T pi[4] = {(T)1, Ai, Ai * Ai, Ai * Ai * Ai};
    const T pj[4] = {(T)1, Aj, Aj * Aj, Aj * Aj * Aj};
    const T cg = cx * ti[1] + cy * ti[2] + cz * ti[3];        // coef . gA
    const T cgb = cx * ti[5] + cy * ti[6] + cz * ti[7];       // coef . dgA/db
#pragma unroll
    for (int G = 0; G < NGRP; ++G) {
      const int m = gm(G), n = gn(G);
      T Da = 0, Db = 0, DaA = 0, DaB = 0;
      if (m > 0) {
        Da += (T)m * pi[m > 0 ? m - 1 : 0] * pj[n];
        Db += (T)m * pj[m > 0 ? m - 1 : 0] * pi[n];
      }
      if (n > 0) {
        Da += (T)n * pi[n > 0 ? n - 1 : 0] * pj[m];
        Db += (T)n * pj[n > 0 ? n - 1 : 0] * pi[m];
      }
      if (m > 1) DaA += (T)(m * (m - 1)) * pi[m > 1 ? m - 2 : 0] * pj[n];
      if (n > 1) DaA += (T)(n * (n - 1)) * pi[n > 1 ? n - 2 : 0] * pj[m];
      if (m > 0 && n > 0)
        DaB += (T)(m * n) * (pi[m > 0 ? m - 1 : 0] * pj[n > 0 ? n - 1 : 0] +
                             pi[n > 0 ? n - 1 : 0] * pj[m > 0 ? m - 1 : 0]);
      X[G] += Da * cg;
      Z[G] += Da * Ai_b + Db * Aj_b;
      V[G] += (DaA * Ai_b + DaB * Aj_b) * cg + Da * cgb;
    }
  }
  T sYd = 0, sXd = 0, sZb = 0, sVb = 0;
  const T ce_dEdr = ce * dEdr;
#pragma unroll
  for (int G = 0; G < NGRP; ++G) {
    sYd += P2[G] * Y[G];
    sXd += P1[G] * X[G];
    sZb += P1[G] * Z[G];
    sVb += P0[G] * V[G];
#pragma unroll
    for (int o = 0; o < 5; ++o)
      acc[2 + 5 * G + o] += pE[o] * X[G] + (o > 0 ? (T)o * pE[o > 0 ? o - 1 : 0] * ce_dEdr * Y[G] : (T)0);
  }
  const T cE_d = (J.cusp ? (T)-0.5 / (d * d) : (T)0) + E_d * sYd;
  acc[0] += (cE_d * dEdr + cE * dEdr_d) * ce + E_d * sXd;
  acc[1] += sZb * ce_dEdr + sVb;
}

template <class T>
__global__ void __launch_bounds__(256) adj_pair_kernel(AdjArgs<T> a, const __grid_constant__ isdf_jastrow J) {
  constexpr int AMU = AMu<T>::v;
  __shared__ T As[4][AMU][AT];
  __shared__ T Bs[4][AMU][AT];
  __shared__ double red[8][2 + NGRP * 5];
  const int t = threadIdx.x;
  const int64_t g0 = a.g_begin + (int64_t)blockIdx.y * AT, h0 = (int64_t)blockIdx.x * AT;
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
      As[c][r][col] = (mu < a.n_mu && ga < a.g_end) ? a.Ah[c * plane + (int64_t)mu * a.n_g + ga] : (T)0;
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

  const T d = (T)J.d;
  // per-thread sums over its pairs: [0] d, [1] b, [2 + 5 G + o] group G, E power o
  T acc[2 + NGRP * 5];
#pragma unroll
  for (int q = 0; q < 2 + NGRP * 5; ++q) acc[q] = (T)0;
  const int64_t g = g0 + tg;
  if (g < a.g_end) {
    const double* rg = a.grid + 3 * g;
    for (int j = 0; j < 4; ++j) {
      const int64_t h = h0 + th + 8 * j;
      if (h >= a.n_g || h == g) continue;
      adj_pair_terms<T>(a, J, d, g, h, rg, M[0][j], M[1][j], M[2][j], M[3][j], acc);
    }
  }
  adj_block_reduce<T>(acc, red, a.sums);
}

// Pair terms of the outer rows [a.g_begin, a.g_end) with M read from the slab
// the tensor-core GEMM wrote: slab[c][g - a.g_begin][h] (FP64, c = x, y, z, sq).
__global__ void __launch_bounds__(256, 2) adj_pair_slab_kernel(AdjArgs<float> a,
                                                            const double* __restrict__ slab,
                                                            const __grid_constant__ isdf_jastrow J) {
  __shared__ double red[8][2 + NGRP * 5];
  const int t = threadIdx.x;
  const int64_t g0 = a.g_begin + (int64_t)blockIdx.y * AT, h0 = (int64_t)blockIdx.x * AT;
  const int tg = t >> 3, th = t & 7;
  const float d = (float)J.d;
  float acc[2 + NGRP * 5];
#pragma unroll
  for (int q = 0; q < 2 + NGRP * 5; ++q) acc[q] = 0.f;
  const int64_t g = g0 + tg;
  if (g < a.g_end) {
    const double* rg = a.grid + 3 * g;
    const int64_t cstride = (a.g_end - a.g_begin) * a.n_g;
    const double* mrow = slab + (g - a.g_begin) * a.n_g;
    for (int j = 0; j < 4; ++j) {
      const int64_t h = h0 + th + 8 * j;
      if (h >= a.n_g || h == g) continue;
      const double* mp = mrow + h;
      adj_pair_terms<float>(a, J, d, g, h, rg, (float)mp[0], (float)mp[cstride],
                            (float)mp[2 * cstride], (float)mp[3 * cstride], acc);
    }
  }
  adj_block_reduce<float>(acc, red, a.sums);
}

// dst[l][r][c] = BF16 limb l of w[r0 + r] src[c * src_rs + r0 + r] (r < rows,
// c < cols; zero in the padding): the K-major (mu-contiguous) operands of the
// M-tile GEMM, transposed through 32 x 32 shared-memory tiles.
constexpr int kAdjLimbs = 3;
__global__ void adj_split_t_kernel(const double* __restrict__ src, int64_t src_rs, int64_t r0,
                                   const double* __restrict__ w, int64_t rows, int64_t cols,
                                   int64_t rows_pad, int64_t cols_pad,
                                   __nv_bfloat16* __restrict__ dst) {
  __shared__ double tl[32][33];
  const int64_t rb = (int64_t)blockIdx.x * 32, cb = (int64_t)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t c = cb + i, r = rb + threadIdx.x;
    tl[i][threadIdx.x] = (c < cols && r < rows) ? w[r0 + r] * src[c * src_rs + r0 + r] : 0.0;
  }
  __syncthreads();
  const int64_t plane = rows_pad * cols_pad;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = rb + i, c = cb + threadIdx.x;
    if (r >= rows_pad || c >= cols_pad) continue;
    float v = (float)tl[threadIdx.x][i];  // limbs of the FP32 rounding
#pragma unroll
    for (int l = 0; l < kAdjLimbs; ++l) {
      const __nv_bfloat16 hb = __float2bfloat16_rn(v);
      dst[l * plane + r * cols_pad + c] = hb;
      v -= __bfloat162float(hb);
    }
  }
}

// dtheta = (d, b, c_0 .. c_{K-1}) from the (group, E power) sums
__global__ void adj_scatter_kernel(const double* sums, const __grid_constant__ isdf_jastrow J,
                                   double* dtheta) {
  const int k = threadIdx.x;
  if (k >= 2 + J.n_terms) return;
  if (k < 2) {
    dtheta[k] = sums[k];
  } else {
    const int* t = J.mno[k - 2];
    dtheta[k] = sums[2 + 5 * grp_of(t[0], t[1]) + t[2]];
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
                int64_t g_begin, int64_t g_end, int n_mu, const isdf_jastrow& J, const double* Wbar,
                double* dtheta, void* ws, size_t ws_bytes, cudaStream_t s) {
  const int64_t plane = (int64_t)n_mu * n_g;
  Carve cv(ws, ws_bytes);
  double* Bh64 = cv.take<double>(4 * plane);
  T* Ah = cv.take<T>(4 * plane);
  T* Bh = cv.take<T>(4 * plane);
  T* tab = cv.take<T>((size_t)n_g * J.n_nuc * 8);
  double* sums = cv.take<double>(2 + NGRP * 5);
  double* chi = cv.take<double>((size_t)3 * n_g);
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
  ISDF_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * (2 + NGRP * 5), s));
  AdjArgs<T> a;
  a.Ah = Ah; a.Bh = Bh; a.grid = grid; a.n_g = n_g; a.n_mu = n_mu; a.tab = tab; a.sums = sums;
  a.g_begin = g_begin; a.g_end = g_end;
  a.chi = nullptr;
  a.chi0 = g_begin;
  if (chi_on(J)) {
    ISDF_TRY(chi_table(grid, g_begin, g_end - g_begin, J, chi, s));
    a.chi = chi;
  }
  double gc[NGRP][5] = {};
  for (int k = 0; k < J.n_terms; ++k)
    gc[grp_of(J.mno[k][0], J.mno[k][1])][J.mno[k][2]] += J.coef[0][k];
  for (int G = 0; G < NGRP; ++G)
    for (int o = 0; o < 5; ++o) a.gc[G][o] = (T)gc[G][o];
  dim3 grd((unsigned)ceil_div(n_g, AT), (unsigned)ceil_div(g_end - g_begin, AT));
  ISDF_ARG(grd.y < 65536u, "n_g too large for the adjoint grid");
  adj_pair_kernel<T><<<grd, 256, 0, s>>>(a, J);
  ISDF_LAUNCH_CHECK();
  adj_scatter_kernel<<<1, 64, 0, s>>>(sums, J, dtheta);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

// FP32 pair arithmetic with the M tiles on the tensor cores: per outer slice
// of S points, M^c = (w xi~^c)_slice^T Bhat^c as a split-BF16 tcgen05 GEMM
// (three limbs, FP32 accumulation folded every 256 mu into FP32 running sums,
// FP64 output) into an FP64 slab [4][S][n_g], then the pair terms from it.
struct AdjTcWs {
  double* Bh64;        // [4][n_mu][n_g] Wbar^c xi
  float* tab;          // [n_g][n_nuc][8]
  double* sums;        // [2 + NGRP * 5]
  double* chi;         // [n_g][3]
  int* err;            // [64] device wait-status word of the GEMMs
  __nv_bfloat16* Bt;   // [4][limbs][Np][Kp] (w Bhat^c)^T
  __nv_bfloat16* As;   // [4][limbs][Sp][Kp] (w xi~^c)^T of one slice
  double* slab;        // [4][S][n_g]
  void carve(Carve& cv, int64_t n_g, int n_mu, int n_nuc, int64_t S) {
    const int64_t Np = round_up(n_g, 128), Kp = round_up(n_mu, 32), Sp = round_up(S, 128);
    Bh64 = cv.take<double>((size_t)4 * n_mu * n_g);
    tab = cv.take<float>((size_t)n_g * n_nuc * 8);
    sums = cv.take<double>(2 + NGRP * 5);
    chi = cv.take<double>((size_t)3 * n_g);
    err = cv.take<int>(64);
    Bt = cv.take<__nv_bfloat16>((size_t)4 * kAdjLimbs * Np * Kp);
    As = cv.take<__nv_bfloat16>((size_t)4 * kAdjLimbs * Sp * Kp);
    slab = cv.take<double>((size_t)4 * S * n_g);
  }
};

// Outer points per slab: at most 2048, and the slab at most ~2 GB.
int64_t adj_slice(int64_t n_g) {
  int64_t S = ((int64_t)1 << 26) / n_g;
  S = S > 2048 ? 2048 : S;
  S = (S / 128) * 128;
  return S < 128 ? 128 : S;
}

int run_adjoint_tc(const double* grid, const double* w, const double* xi, const double* xig,
                   int64_t n_g, int64_t g_begin, int64_t g_end, int n_mu, const isdf_jastrow& J,
                   const double* Wbar, double* dtheta, void* ws, size_t ws_bytes, cudaStream_t s) {
  const int64_t plane = (int64_t)n_mu * n_g;
  const int64_t S = adj_slice(n_g);
  const int64_t Np = round_up(n_g, 128), Kp = round_up(n_mu, 32);
  Carve cv(ws, ws_bytes);
  AdjTcWs b;
  b.carve(cv, n_g, n_mu, J.n_nuc, S);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  ISDF_CUDA(cudaMemsetAsync(b.err, 0, 64 * sizeof(int), s));
  // Bhat^c = Wbar^c xi (FP64); w scales the inner index in the transposed split
  Dgemm g;
  g.M = n_mu; g.N = n_g; g.K = n_mu;
  g.A = Wbar; g.a_rs = n_mu; g.a_cs = 1; g.a_bs = (int64_t)n_mu * n_mu;
  g.B = xi; g.b_rs = n_g; g.b_cs = 1; g.b_bs = 0;
  g.C = b.Bh64; g.ldc = n_g; g.c_bs = plane;
  g.batch = 4;
  ISDF_TRY(dgemm(g, s));
  const dim3 tb(32, 8);
  for (int c = 0; c < 4; ++c) {
    adj_split_t_kernel<<<dim3((unsigned)(Np / 32), (unsigned)(Kp / 32)), tb, 0, s>>>(
        b.Bh64 + c * plane, n_g, 0, w, n_g, n_mu, Np, Kp, b.Bt + (size_t)c * kAdjLimbs * Np * Kp);
    ISDF_LAUNCH_CHECK();
  }
  if (J.n_nuc > 0) {
    adj_table_kernel<float><<<nb(n_g * J.n_nuc), 256, 0, s>>>(grid, n_g, J, b.tab);
    ISDF_LAUNCH_CHECK();
  }
  ISDF_CUDA(cudaMemsetAsync(b.sums, 0, sizeof(double) * (2 + NGRP * 5), s));
  AdjArgs<float> a;
  a.Ah = nullptr; a.Bh = nullptr; a.grid = grid; a.n_g = n_g; a.n_mu = n_mu; a.tab = b.tab;
  a.sums = b.sums;
  a.chi = nullptr;
  a.chi0 = g_begin;
  if (chi_on(J)) {
    ISDF_TRY(chi_table(grid, g_begin, g_end - g_begin, J, b.chi, s));
    a.chi = b.chi;
  }
  double gc[NGRP][5] = {};
  for (int k = 0; k < J.n_terms; ++k)
    gc[grp_of(J.mno[k][0], J.mno[k][1])][J.mno[k][2]] += J.coef[0][k];
  for (int G = 0; G < NGRP; ++G)
    for (int o = 0; o < 5; ++o) a.gc[G][o] = (float)gc[G][o];
  for (int64_t s0 = g_begin; s0 < g_end; s0 += S) {
    const int64_t Sr = g_end - s0 < S ? g_end - s0 : S;
    const int64_t Srp = round_up(Sr, 128);
    const void* A[4];
    const void* B[4];
    for (int c = 0; c < 4; ++c) {
      const double* src = c < 3 ? xig + c * plane : xi;
      __nv_bfloat16* dst = b.As + (size_t)c * kAdjLimbs * Srp * Kp;
      adj_split_t_kernel<<<dim3((unsigned)(Srp / 32), (unsigned)(Kp / 32)), tb, 0, s>>>(
          src, n_g, s0, w, Sr, n_mu, Srp, Kp, dst);
      ISDF_LAUNCH_CHECK();
      A[c] = dst;
      B[c] = b.Bt + (size_t)c * kAdjLimbs * Np * Kp;
    }
    ISDF_CUDA(cudaMemsetAsync(b.slab, 0, sizeof(double) * 4 * Sr * n_g, s));
    ISDF_TRY(splitgemm(kAdjLimbs, 4, A, B, Sr, n_g, Kp, Kp, 256, b.slab, n_g, Sr * n_g, 1.0,
                       b.err, s));
    a.g_begin = s0;
    a.g_end = s0 + Sr;
    const dim3 grd((unsigned)ceil_div(n_g, AT), (unsigned)ceil_div(Sr, AT));
    adj_pair_slab_kernel<<<grd, 256, 0, s>>>(a, b.slab, J);
    ISDF_LAUNCH_CHECK();
  }
  adj_scatter_kernel<<<1, 64, 0, s>>>(b.sums, J, dtheta);
  ISDF_LAUNCH_CHECK();
  int h_err = 0;
  ISDF_TRY(read_error_word(b.err, &h_err, s));
  if (h_err & DEV_ERR_TIMEOUT) {
    set_error("adjoint: a bounded wait of the M-tile GEMM expired");
    return ISDF_E_TIMEOUT;
  }
  return ISDF_OK;
}

}  // namespace

size_t adjoint_ws(int64_t n_g, int n_mu, int n_nuc, int precision) {
  if (precision != ISDF_PREC_FP64) {
    Carve c(nullptr, 0);
    AdjTcWs b;
    b.carve(c, n_g, n_mu, n_nuc, adj_slice(n_g));
    return c.off;
  }
  const size_t el = 8;
  Carve c(nullptr, 0);
  const size_t plane = (size_t)n_mu * n_g;
  c.take<double>(4 * plane);
  c.take<unsigned char>(4 * plane * el);
  c.take<unsigned char>(4 * plane * el);
  c.take<unsigned char>((size_t)n_g * n_nuc * 8 * el);
  c.take<double>(2 + NGRP * 5);
  c.take<double>((size_t)3 * n_g);
  return c.off;
}

int adjoint(const double* grid, const double* w, const double* xi, const double* xig, int64_t n_g,
            int64_t g_begin, int64_t g_end, int n_mu, const isdf_jastrow& J, const double* Wbar,
            int precision, double* dtheta, void* ws, size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(grid && w && xi && xig && Wbar && dtheta, "null pointer argument");
  ISDF_ARG(n_g > 0 && n_mu > 0, "empty sizes");
  ISDF_ARG(g_begin >= 0 && g_begin < g_end && g_end <= n_g, "bad grid slice");
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
    return run_adjoint<double>(grid, w, xi, xig, n_g, g_begin, g_end, n_mu, J, Wbar, dtheta, ws,
                               ws_bytes, s);
  return run_adjoint_tc(grid, w, xi, xig, n_g, g_begin, g_end, n_mu, J, Wbar, dtheta, ws,
                        ws_bytes, s);
}

}  // namespace isdf
