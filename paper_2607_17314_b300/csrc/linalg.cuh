// FP64 dense linear algebra on CUDA cores (sm_103a): strided GEMM, blocked
// Cholesky, blocked triangular solves with many right-hand sides.
#pragma once

#include "common.cuh"

namespace isdf {

// C(m,n) = alpha * sum_k A(m,k) B(k,n) + beta * C(m,n)   (beta == 0: overwrite)
// A(m,k) = A[m*a_rs + k*a_cs], B(k,n) = B[k*b_rs + n*b_cs], C(m,n) = C[m*ldc + n].
// Batch index z offsets A, B, C by z*a_bs, z*b_bs, z*c_bs.
struct Dgemm {
  int64_t M, N, K;
  const double* A;
  int64_t a_rs, a_cs, a_bs;
  const double* B;
  int64_t b_rs, b_cs, b_bs;
  double* C;
  int64_t ldc, c_bs;
  double alpha = 1.0, beta = 0.0;
  int batch = 1;
  const double* kscale = nullptr;  // optional: A(m,k) is multiplied by kscale[k]
};
int dgemm(const Dgemm& g, cudaStream_t s);

// In-place lower Cholesky of the n x n matrix A (lda = n); only the lower
// triangle of the result is meaningful.  *info_dev (device int) is set to
// j+1 at the first non-positive pivot j (0 = success).  ws: n doubles.
int dpotrf_lower(double* A, int n, int* info_dev, cudaStream_t s);

// Solve (L L^T) X = B in place for B [n][nrhs] (row stride ldb), L lower
// triangular from dpotrf_lower (lda = n).
int dpotrs_lower(const double* L, int n, double* B, int64_t nrhs, int64_t ldb,
                 cudaStream_t s);

// OR DEV_ERR_NONFINITE into the device word *err when any of x[0..n) is NaN
// or Inf.  Asynchronous.
int scan_nonfinite(const double* x, int64_t n, int* err, cudaStream_t s);

// Copy the device error word to *h_err and synchronise `s`.
int read_error_word(const int* err, int* h_err, cudaStream_t s);

// A device index that a kernel finds outside [0, n) is never dereferenced: the
// gathered value becomes a quiet NaN and DEV_ERR_ARG is OR-ed into the error
// word when the call has one.
__device__ __forceinline__ bool index_ok(int64_t i, int64_t n, int* err) {
  if (i >= 0 && i < n) return true;
  if (err) atomicOr(err, DEV_ERR_ARG);
  return false;
}

}  // namespace isdf
