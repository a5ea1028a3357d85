// Jastrow kernels u^(1),c and u^(3) (Eqs. K1-isdf, K3-isdf) in FP64 on CUDA
// cores: the FP64 GPU path.  Stage 1 generates K_c(g,g') per (g', g) tile
// into shared memory and contracts it with (w xi); stage 2 is an FP64 GEMM.
#include "jastrow.cuh"
#include "linalg.cuh"

namespace isdf {
namespace {

constexpr int FBM = 64, FBG = 32, FBK = 16;

struct S1F64 {
  const double* grid;  // [n_g][3]
  const double* w;
  const double* xi;    // [n_mu][n_g]
  int64_t n_g;
  int n_mu;
  int64_t g_begin, g_end;
  double* calG;        // [4][n_mu][n_gs]
  BhTable tab;
  const double* chi;   // [n_gs][3] grad chi / (N - 1) of the outer points, or null
};

template <bool RADIAL>
__global__ void __launch_bounds__(256) s1_fp64_kernel(S1F64 a, const __grid_constant__ isdf_jastrow J) {
  __shared__ double As[FBK][FBM];
  __shared__ double Ks[4][FBK][FBG];
  const int t = threadIdx.x;
  const int ty = t >> 3, tx = t & 7;
  const int64_t n_gs = a.g_end - a.g_begin;
  const int64_t gl0 = (int64_t)blockIdx.x * FBG;  // local (slice) index
  const int nu0 = blockIdx.y * FBM;
  double acc[4][2][4] = {};
  for (int64_t k0 = 0; k0 < a.n_g; k0 += FBK) {
    for (int e = t; e < FBM * FBK; e += 256) {
      int nu = e / FBK, kk = e % FBK;
      int64_t k = k0 + kk;
      double v = 0.0;
      if (nu0 + nu < a.n_mu && k < a.n_g) v = a.w[k] * a.xi[(int64_t)(nu0 + nu) * a.n_g + k];
      As[kk][nu] = v;
    }
    for (int e = t; e < FBK * FBG; e += 256) {
      int kk = e / FBG, gg = e % FBG;
      int64_t gp = k0 + kk;
      int64_t gl = gl0 + gg;
      double K[3] = {0.0, 0.0, 0.0};
      if (gl < n_gs && gp < a.n_g) {
        int64_t g = a.g_begin + gl;
        if (g != gp) {
          if (RADIAL) {
            if (J.cusp) radial_grad(J.d, a.grid + 3 * g, a.grid + 3 * gp, K);
          }
          else bh_grad(J, a.tab, g, gp, a.grid + 3 * g, a.grid + 3 * gp, K);
          if (a.chi) {
            K[0] += a.chi[3 * gl];
            K[1] += a.chi[3 * gl + 1];
            K[2] += a.chi[3 * gl + 2];
          }
        }
      }
      Ks[0][kk][gg] = K[0];
      Ks[1][kk][gg] = K[1];
      Ks[2][kk][gg] = K[2];
      Ks[3][kk][gg] = K[0] * K[0] + K[1] * K[1] + K[2] * K[2];
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < FBK; ++kk) {
      double av[2] = {As[kk][ty], As[kk][ty + 32]};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        double bv[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Ks[c][kk][tx + 8 * j];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[c][i][j] = fma(av[i], bv[j], acc[c][i][j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      int nu = nu0 + ty + 32 * i;
      if (nu >= a.n_mu) continue;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int64_t gl = gl0 + tx + 8 * j;
        if (gl < n_gs) a.calG[((int64_t)c * a.n_mu + nu) * n_gs + gl] = acc[c][i][j];
      }
    }
}

// A[g][I] and grad A[g][I] for every point and nucleus.
__global__ void bh_table_kernel(const double* grid, int64_t n_g, const __grid_constant__ isdf_jastrow J,
                                double* A, double* dA) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_g * J.n_nuc) return;
  int64_t g = e / J.n_nuc;
  int I = (int)(e % J.n_nuc);
  const double b = J.b[J.nuc_type[I]];
  double v[3];
  for (int c = 0; c < 3; ++c) v[c] = grid[3 * g + c] - J.nuc_xyz[I][c];
  double r = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
  double den = 1.0 + b * r;
  A[e] = b * r / den;
  double s = r > 0.0 ? b / (den * den * r) : 0.0;
  for (int c = 0; c < 3; ++c) dA[3 * e + c] = s * v[c];
}

__global__ void chi_table_kernel(const double* grid, int64_t g0, int64_t n,
                                 const __grid_constant__ isdf_jastrow J, double* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const double* r = grid + 3 * (g0 + e);
  chi_grad_pair(J, r[0], r[1], r[2], out + 3 * e);
}

}  // namespace

int chi_table(const double* grid, int64_t g0, int64_t n, const isdf_jastrow& J, double* out,
              cudaStream_t s) {
  if (n <= 0) return ISDF_OK;
  chi_table_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(grid, g0, n, J, out);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

size_t wbuild_fp64_ws(int64_t n_g, const isdf_jastrow* J) {
  Carve c(nullptr, 0);
  c.take<int>(64);
  int nn = J ? (J->n_terms == 0 ? 0 : J->n_nuc) : ISDF_MAX_NUC;
  c.take<double>((size_t)n_g * nn);
  c.take<double>((size_t)3 * n_g * nn);
  if (!J || chi_on(*J)) c.take<double>((size_t)3 * n_g);
  return c.off;
}

int bh_table(const double* grid, int64_t n_g, const isdf_jastrow& J, double* A, double* dA,
             cudaStream_t s) {
  int64_t n = n_g * J.n_nuc;
  if (n == 0) return ISDF_OK;
  bh_table_kernel<<<(unsigned)ceil_div(n, 256), 256, 0, s>>>(grid, n_g, J, A, dA);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

int wbuild_fp64(const double* grid, const double* w, const double* xi, const double* xig,
                int64_t n_g, int n_mu, int64_t g_begin, int64_t g_end, const isdf_jastrow& J,
                double* W, double* calG, int sync_check, void* ws, size_t ws_bytes,
                cudaStream_t s) {
  const bool radial = J.n_terms == 0;
  S1F64 a;
  a.grid = grid; a.w = w; a.xi = xi; a.n_g = n_g; a.n_mu = n_mu;
  a.g_begin = g_begin; a.g_end = g_end; a.calG = calG;
  a.tab.A = nullptr; a.tab.dA = nullptr;
  Carve cv(ws, ws_bytes);
  int* err = cv.take<int>(64);
  double* A = radial ? nullptr : cv.take<double>((size_t)n_g * J.n_nuc);
  double* dA = radial ? nullptr : cv.take<double>((size_t)3 * n_g * J.n_nuc);
  const int64_t n_gs = g_end - g_begin;
  double* chi = chi_on(J) ? cv.take<double>((size_t)3 * n_g) : nullptr;
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  if (!radial) {
    ISDF_TRY(bh_table(grid, n_g, J, A, dA, s));
    a.tab.A = A; a.tab.dA = dA;
  }
  a.chi = chi;
  if (chi) ISDF_TRY(chi_table(grid, g_begin, n_gs, J, chi, s));
  dim3 grd((unsigned)ceil_div(n_gs, FBG), (unsigned)ceil_div(n_mu, FBM));
  if (radial) s1_fp64_kernel<true><<<grd, 256, 0, s>>>(a, J);
  else s1_fp64_kernel<false><<<grd, 256, 0, s>>>(a, J);
  ISDF_LAUNCH_CHECK();
  // stage 2: W[c] = (w xi~^c) calG[c]^T, W[3] = (w xi) calG[3]^T over the slice
  Dgemm g;
  g.M = n_mu; g.N = n_mu; g.K = n_gs;
  g.A = xig + g_begin; g.a_rs = n_g; g.a_cs = 1; g.a_bs = (int64_t)n_mu * n_g;
  g.B = calG; g.b_rs = 1; g.b_cs = n_gs; g.b_bs = (int64_t)n_mu * n_gs;
  g.C = W; g.ldc = n_mu; g.c_bs = (int64_t)n_mu * n_mu;
  g.kscale = w + g_begin;
  g.batch = 3;
  ISDF_TRY(dgemm(g, s));
  g.A = xi + g_begin;
  g.B = calG + 3 * (int64_t)n_mu * n_gs;
  g.C = W + 3 * (int64_t)n_mu * n_mu;
  g.batch = 1;
  ISDF_TRY(dgemm(g, s));
  if (sync_check) {
    // every input value reaches W: a NaN or Inf there leaves a non-finite W
    ISDF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    ISDF_TRY(scan_nonfinite(W, (int64_t)4 * n_mu * n_mu, err, s));
    int h_err = 0;
    ISDF_TRY(read_error_word(err, &h_err, s));
    if (h_err & DEV_ERR_NONFINITE) {
      set_error("W is not finite (NaN or Inf in the grid, weights or xi)");
      return ISDF_E_NONFINITE;
    }
  }
  return ISDF_OK;
}

}  // namespace isdf
