// FP64 dense linear algebra kernels (CUDA cores).
#include "linalg.cuh"

namespace isdf {

namespace {

constexpr int TM = 64, TN = 64, TK = 16;

__global__ void __launch_bounds__(256) dgemm_kernel(Dgemm g) {
  __shared__ double As[TK][TM + 1];
  __shared__ double Bs[TK][TN + 1];
  const int z = blockIdx.z;
  const double* A = g.A + (int64_t)z * g.a_bs;
  const double* B = g.B + (int64_t)z * g.b_bs;
  double* C = g.C + (int64_t)z * g.c_bs;
  const int64_t m0 = (int64_t)blockIdx.y * TM;
  const int64_t n0 = (int64_t)blockIdx.x * TN;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4] = {};
  const bool a_kfast = (g.a_cs == 1);
  const bool b_nfast = (g.b_cs == 1);
  for (int64_t k0 = 0; k0 < g.K; k0 += TK) {
    for (int e = threadIdx.x; e < TM * TK; e += 256) {
      int mm, kk;
      if (a_kfast) { mm = e / TK; kk = e % TK; } else { mm = e % TM; kk = e / TM; }
      int64_t m = m0 + mm, k = k0 + kk;
      double v = (m < g.M && k < g.K) ? A[m * g.a_rs + k * g.a_cs] : 0.0;
      if (g.kscale && k < g.K) v *= g.kscale[k];
      As[kk][mm] = v;
    }
    for (int e = threadIdx.x; e < TN * TK; e += 256) {
      int nn, kk;
      if (b_nfast) { nn = e % TN; kk = e / TN; } else { nn = e / TK; kk = e % TK; }
      int64_t n = n0 + nn, k = k0 + kk;
      Bs[kk][nn] = (n < g.N && k < g.K) ? B[k * g.b_rs + n * g.b_cs] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int64_t m = m0 + ty + 16 * i;
    if (m >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int64_t n = n0 + tx + 16 * j;
      if (n >= g.N) continue;
      double* c = C + m * g.ldc + n;
      double v = g.alpha * acc[i][j];
      *c = (g.beta == 0.0) ? v : fma(g.beta, *c, v);
    }
  }
}

constexpr int NB = 64;

// Unblocked Cholesky of the jb x jb diagonal block at A[j0][j0] (lda n).
__global__ void __launch_bounds__(256) potrf_diag_kernel(double* A, int n, int j0, int jb,
                                                         int* info) {
  __shared__ double T[NB][NB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e / jb, j = e % jb;
    T[i][j] = A[(int64_t)(j0 + i) * n + j0 + j];
  }
  __syncthreads();
  for (int k = 0; k < jb; ++k) {
    __shared__ double piv;
    if (threadIdx.x == 0) {
      double d = T[k][k];
      if (!(d > 0.0)) {
        if (*info == 0) *info = j0 + k + 1;
        d = 1.0;  // keep going with finite values; the caller retries
      }
      piv = sqrt(d);
      T[k][k] = piv;
    }
    __syncthreads();
    for (int i = k + 1 + threadIdx.x; i < jb; i += blockDim.x) T[i][k] = T[i][k] / piv;
    __syncthreads();
    for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
      int i = e / jb, j = e % jb;
      if (i > k && j > k && j <= i) T[i][j] = fma(-T[i][k], T[j][k], T[i][j]);
    }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e / jb, j = e % jb;
    if (j <= i) A[(int64_t)(j0 + i) * n + j0 + j] = T[i][j];
  }
}

// Panel: rows r >= j0+jb, columns [j0, j0+jb): x L11^T = a  (one row per thread).
__global__ void __launch_bounds__(128) potrf_panel_kernel(double* A, int n, int j0, int jb) {
  __shared__ double T[NB][NB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e / jb, j = e % jb;
    T[i][j] = (j <= i) ? A[(int64_t)(j0 + i) * n + j0 + j] : 0.0;
  }
  __syncthreads();
  int r = j0 + jb + blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double* row = A + (int64_t)r * n + j0;
  double x[NB];
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    if (k < jb) {
      double v = row[k];
      for (int l = 0; l < k; ++l) v = fma(-x[l], T[k][l], v);
      x[k] = v / T[k][k];
    }
  }
#pragma unroll
  for (int k = 0; k < NB; ++k)
    if (k < jb) row[k] = x[k];
}

constexpr int TB = 32;  // block size of the many-RHS triangular solves

// Forward block solve: Y = L11^{-1} B[j0:j0+jb, :] (one column per thread).
__global__ void __launch_bounds__(128) trsm_fwd_block(const double* L, int n, int j0, int jb,
                                                      double* B, int64_t nrhs, int64_t ldb) {
  __shared__ double T[TB][TB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e / jb, j = e % jb;
    T[i][j] = (j <= i) ? L[(int64_t)(j0 + i) * n + j0 + j] : 0.0;
  }
  __syncthreads();
  int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nrhs) return;
  double y[TB];
#pragma unroll
  for (int i = 0; i < TB; ++i) {
    if (i < jb) {
      double v = B[(int64_t)(j0 + i) * ldb + col];
      for (int l = 0; l < i; ++l) v = fma(-T[i][l], y[l], v);
      y[i] = v / T[i][i];
    }
  }
#pragma unroll
  for (int i = 0; i < TB; ++i)
    if (i < jb) B[(int64_t)(j0 + i) * ldb + col] = y[i];
}

// Backward block solve: X = L11^{-T} Y[j0:j0+jb, :].
__global__ void __launch_bounds__(128) trsm_bwd_block(const double* L, int n, int j0, int jb,
                                                      double* B, int64_t nrhs, int64_t ldb) {
  __shared__ double T[TB][TB + 1];
  for (int e = threadIdx.x; e < jb * jb; e += blockDim.x) {
    int i = e / jb, j = e % jb;
    T[i][j] = (j <= i) ? L[(int64_t)(j0 + i) * n + j0 + j] : 0.0;
  }
  __syncthreads();
  int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nrhs) return;
  double x[TB];
#pragma unroll
  for (int ii = TB - 1; ii >= 0; --ii) {
    if (ii < jb) {
      double v = B[(int64_t)(j0 + ii) * ldb + col];
#pragma unroll
      for (int l = ii + 1; l < TB; ++l)
        if (l < jb) v = fma(-T[l][ii], x[l], v);
      x[ii] = v / T[ii][ii];
    }
  }
#pragma unroll
  for (int i = 0; i < TB; ++i)
    if (i < jb) B[(int64_t)(j0 + i) * ldb + col] = x[i];
}

}  // namespace

int dgemm(const Dgemm& g, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return ISDF_OK;
  if (g.K <= 0) {
    // C = beta C
    if (g.beta == 0.0) {
      for (int z = 0; z < g.batch; ++z)
        for (int64_t m = 0; m < g.M; ++m)
          ISDF_CUDA(cudaMemsetAsync(g.C + z * g.c_bs + m * g.ldc, 0, g.N * sizeof(double), s));
    }
    return ISDF_OK;
  }
  dim3 grid((unsigned)ceil_div(g.N, TN), (unsigned)ceil_div(g.M, TM), (unsigned)g.batch);
  ISDF_ARG(grid.y < 65536u && grid.z < 65536u, "dgemm grid too large");
  dgemm_kernel<<<grid, 256, 0, s>>>(g);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

int dpotrf_lower(double* A, int n, int* info_dev, cudaStream_t s) {
  ISDF_CUDA(cudaMemsetAsync(info_dev, 0, sizeof(int), s));
  for (int j0 = 0; j0 < n; j0 += NB) {
    int jb = n - j0 < NB ? n - j0 : NB;
    potrf_diag_kernel<<<1, 256, 0, s>>>(A, n, j0, jb, info_dev);
    ISDF_LAUNCH_CHECK();
    int rest = n - j0 - jb;
    if (rest <= 0) break;
    potrf_panel_kernel<<<(unsigned)ceil_div(rest, 128), 128, 0, s>>>(A, n, j0, jb);
    ISDF_LAUNCH_CHECK();
    Dgemm g;
    g.M = rest; g.N = rest; g.K = jb;
    g.A = A + (int64_t)(j0 + jb) * n + j0; g.a_rs = n; g.a_cs = 1; g.a_bs = 0;
    g.B = A + (int64_t)(j0 + jb) * n + j0; g.b_rs = 1; g.b_cs = n; g.b_bs = 0;
    g.C = A + (int64_t)(j0 + jb) * n + (j0 + jb); g.ldc = n; g.c_bs = 0;
    g.alpha = -1.0; g.beta = 1.0;
    ISDF_TRY(dgemm(g, s));
  }
  return ISDF_OK;
}

int dpotrs_lower(const double* L, int n, double* B, int64_t nrhs, int64_t ldb, cudaStream_t s) {
  unsigned nb = (unsigned)ceil_div(nrhs, 128);
  for (int j0 = 0; j0 < n; j0 += TB) {
    int jb = n - j0 < TB ? n - j0 : TB;
    trsm_fwd_block<<<nb, 128, 0, s>>>(L, n, j0, jb, B, nrhs, ldb);
    ISDF_LAUNCH_CHECK();
    int rest = n - j0 - jb;
    if (rest <= 0) break;
    Dgemm g;
    g.M = rest; g.N = nrhs; g.K = jb;
    g.A = L + (int64_t)(j0 + jb) * n + j0; g.a_rs = n; g.a_cs = 1; g.a_bs = 0;
    g.B = B + (int64_t)j0 * ldb; g.b_rs = ldb; g.b_cs = 1; g.b_bs = 0;
    g.C = B + (int64_t)(j0 + jb) * ldb; g.ldc = ldb; g.c_bs = 0;
    g.alpha = -1.0; g.beta = 1.0;
    ISDF_TRY(dgemm(g, s));
  }
  int last = ((n - 1) / TB) * TB;
  for (int j0 = last; j0 >= 0; j0 -= TB) {
    int jb = n - j0 < TB ? n - j0 : TB;
    trsm_bwd_block<<<nb, 128, 0, s>>>(L, n, j0, jb, B, nrhs, ldb);
    ISDF_LAUNCH_CHECK();
    if (j0 == 0) break;
    // B[0:j0] -= L[j0:j0+jb, 0:j0]^T X[j0:j0+jb]
    Dgemm g;
    g.M = j0; g.N = nrhs; g.K = jb;
    g.A = L + (int64_t)j0 * n; g.a_rs = 1; g.a_cs = n; g.a_bs = 0;
    g.B = B + (int64_t)j0 * ldb; g.b_rs = ldb; g.b_cs = 1; g.b_bs = 0;
    g.C = B; g.ldc = ldb; g.c_bs = 0;
    g.alpha = -1.0; g.beta = 1.0;
    ISDF_TRY(dgemm(g, s));
  }
  return ISDF_OK;
}

// ---------------------------------------------------------------- input checks

namespace {

__global__ void scan_nonfinite_kernel(const double* __restrict__ x, int64_t n, int* err) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(err, DEV_ERR_NONFINITE);
}

}  // namespace

int scan_nonfinite(const double* x, int64_t n, int* err, cudaStream_t s) {
  if (n <= 0) return ISDF_OK;
  int dev = 0, nsm = 148;
  ISDF_CUDA(cudaGetDevice(&dev));
  ISDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t want = ceil_div(n, 256);
  const unsigned blocks = (unsigned)(want < 8 * nsm ? want : 8 * nsm);
  scan_nonfinite_kernel<<<blocks, 256, 0, s>>>(x, n, err);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

int read_error_word(const int* err, int* h_err, cudaStream_t s) {
  ISDF_CUDA(cudaMemcpyAsync(h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  ISDF_CUDA(cudaStreamSynchronize(s));
  return ISDF_OK;
}

}  // namespace isdf
