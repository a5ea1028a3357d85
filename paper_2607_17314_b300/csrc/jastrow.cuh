// Electron-1 gradient of the Boys-Handy correlator (Eqs. bh-scaled, bh-u),
// evaluated per grid pair on the device.
//
//   A_iI = b_I r_iI / (1 + b_I r_iI),  grad_i A_iI = b_I / (1 + b_I r_iI)^2 e_iI
//   E_ij = d r_ij / (1 + d r_ij),      grad_i E_ij = d / (1 + d r_ij)^2 e_ij
//   grad_i u = sum_I cA_I grad_i A_iI + cE grad_i E_ij, with
//   cA_I = sum_k c_k [m A_i^(m-1) A_j^n + n A_j^m A_i^(n-1)] E^o
//   cE   = cusp/(2d) + sum_I sum_k c_k [A_i^m A_j^n + A_j^m A_i^n] o E^(o-1)
#pragma once

#include "common.cuh"

namespace isdf {

// Per-point nucleus table: A[g][I] and grad A[g][I][0..2] (FP64).
struct BhTable {
  const double* A;   // [n_g][n_nuc]
  const double* dA;  // [n_g][n_nuc][3]
};

__device__ __forceinline__ double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

// Gradient for the point pair (gi, gj) with coordinates ri, rj.
__device__ __forceinline__ void bh_grad(const isdf_jastrow& J, const BhTable& T, int64_t gi,
                                        int64_t gj, const double* ri, const double* rj,
                                        double out[3]) {
  const double dx = ri[0] - rj[0], dy = ri[1] - rj[1], dz = ri[2] - rj[2];
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  const double d = J.d;
  const double den = 1.0 + d * r;
  const double E = d * r / den;
  const double dEdr = d / (den * den);
  double cE = J.cusp ? 0.5 / d : 0.0;
  double gx = 0.0, gy = 0.0, gz = 0.0;
  for (int I = 0; I < J.n_nuc; ++I) {
    const int t = J.nuc_type[I];
    const double Ai = T.A[gi * J.n_nuc + I];
    const double Aj = T.A[gj * J.n_nuc + I];
    double cA = 0.0;
    for (int k = 0; k < J.n_terms; ++k) {
      const int m = J.mno[k][0], n = J.mno[k][1], o = J.mno[k][2];
      const double c = J.coef[t][k];
      const double Eo = ipow(E, o);
      double da = 0.0;
      if (m > 0) da += m * ipow(Ai, m - 1) * ipow(Aj, n);
      if (n > 0) da += n * ipow(Aj, m) * ipow(Ai, n - 1);
      cA += c * da * Eo;
      if (o > 0) cE += c * (ipow(Ai, m) * ipow(Aj, n) + ipow(Aj, m) * ipow(Ai, n)) * o * ipow(E, o - 1);
    }
    const double* dA = T.dA + (gi * J.n_nuc + I) * 3;
    gx += cA * dA[0];
    gy += cA * dA[1];
    gz += cA * dA[2];
  }
  const double s = r > 0.0 ? cE * dEdr / r : 0.0;
  out[0] = gx + s * dx;
  out[1] = gy + s * dy;
  out[2] = gz + s * dz;
}

// One-body term of Eq. tau-def: on when some type has chi_a != 0.
__host__ __device__ inline bool chi_on(const isdf_jastrow& J) {
  for (int t = 0; t < J.n_types && t < ISDF_MAX_TYPES; ++t)
    if (J.chi_a[t] != 0.0) return true;
  return false;
}

// grad chi(r) / (N - 1) at the point (x, y, z): the one-body part of every
// ordered pair's electron-1 gradient, chi(r) = sum_I a_t r_I / (1 + beta_t r_I)
// (zero direction on a nucleus).
__device__ __forceinline__ void chi_grad_pair(const isdf_jastrow& J, double x, double y, double z,
                                              double out[3]) {
  double gx = 0.0, gy = 0.0, gz = 0.0;
  for (int I = 0; I < J.n_nuc; ++I) {
    const int t = J.nuc_type[I];
    const double vx = x - J.nuc_xyz[I][0], vy = y - J.nuc_xyz[I][1], vz = z - J.nuc_xyz[I][2];
    const double r = sqrt(vx * vx + vy * vy + vz * vz);
    const double den = 1.0 + J.chi_b[t] * r;
    const double s = r > 0.0 ? J.chi_a[t] / (den * den * r) : 0.0;
    gx += s * vx;
    gy += s * vy;
    gz += s * vz;
  }
  const double inv = 1.0 / (double)(J.n_elec - 1);
  out[0] = gx * inv;
  out[1] = gy * inv;
  out[2] = gz * inv;
}

// grad chi / (N - 1) of the points g0 .. g0 + n - 1 into out [n][3] (FP64).
int chi_table(const double* grid, int64_t g0, int64_t n, const isdf_jastrow& J, double* out,
              cudaStream_t s);

// Radial correlator u = r / (2 (1 + d r)): grad u = 1 / (2 (1 + d r)^2) e_ij.
__device__ __forceinline__ void radial_grad(double d, const double* ri, const double* rj,
                                            double out[3]) {
  const double dx = ri[0] - rj[0], dy = ri[1] - rj[1], dz = ri[2] - rj[2];
  const double r = sqrt(dx * dx + dy * dy + dz * dz);
  const double den = 1.0 + d * r;
  const double s = r > 0.0 ? 0.5 / (den * den * r) : 0.0;
  out[0] = s * dx;
  out[1] = s * dy;
  out[2] = s * dz;
}

}  // namespace isdf
