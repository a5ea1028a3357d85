// Reference-variance VMC optimisation of the correlator (Sec. II.C: Eqs. Eloc,
// var-loss and gn), FP64 on the CUDA cores.
//
// Trial function Psi_T = exp(tau) Phi_0 with Phi_0 the closed-shell reference
// determinant (electrons 0 .. n_occ-1 spin up, the rest spin down) and tau the
// Boys-Handy correlator summed over electron pairs.  Four pieces:
//
//   1. Orbitals at the walkers' electrons: every contracted Gaussian's value,
//      gradient and Laplacian at every electron (one thread per electron),
//      then phi = C_occ^T chi as one batched FP64 GEMM.
//   2. Per walker (one CTA): the two spin determinants inverted by
//      Gauss-Jordan elimination with partial pivoting in shared memory, the
//      determinant's drift grad_i Phi_0/Phi_0 and lap_i Phi_0/Phi_0 from the
//      row-expansion identities, and the Coulomb potential.
//   3. Per (walker, parameter set) CTA: grad_i tau and lap_i tau.  tau is
//      linear in the coefficients c, so the CTA writes, for each electron, the
//      part that no coefficient multiplies and one part per coefficient
//      (no atomics: each (electron, coefficient) slot has one owner thread),
//      then E_loc of Eq. Eloc and, for the unshifted set, the exact dE/dc
//      (E_loc is quadratic in c).  d and b_t enter nonlinearly: their
//      derivatives are central differences over shifted parameter sets.
//   4. The Gauss-Newton step of Eq. gn on the clipped objective of Eq.
//      var-loss: one CTA for the clipping statistics and the residual
//      Jacobian, a GEMM for C, an FP64 Cholesky solve.
//
// The Metropolis sampler of |Phi_0|^2 keeps each walker's inverse
// determinants in shared memory and moves one electron at a time: the
// acceptance ratio is the row-expansion of the new orbital row against the
// inverse, and an accepted move updates the inverse by Sherman-Morrison.
#include <algorithm>

#include "jastrow.cuh"
#include "linalg.cuh"

namespace isdf {
namespace {

constexpr int kVmcThreads = 256;
constexpr int kMaxOcc = 64;
constexpr size_t kVmcSmemMax = 227 * 1024;

struct VmcNuc {
  int n;
  double xyz[ISDF_MAX_NUC][3];
  double Z[ISDF_MAX_NUC];
};

// Deterministic block sum (fixed thread-to-term assignment and tree order).
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    red[32] = s;
  }
  __syncthreads();
  return red[32];
}

// x^p with p x^(p-1) and p (p-1) x^(p-2).
__device__ __forceinline__ void pow3(double x, int p, double& v, double& d1, double& d2) {
  double xp = 1.0, xm = 0.0, xmm = 0.0;
  for (int i = 0; i < p; ++i) {
    xmm = xm;
    xm = xp;
    xp *= x;
  }
  v = xp;
  d1 = p * xm;
  d2 = p * (p - 1) * xmm;
}

// Value of contracted Gaussian f at (px, py, pz).
__device__ __forceinline__ double ao_value(const isdf_basis& b, int f, double px, double py,
                                           double pz) {
  const double x = px - b.center[3 * f], y = py - b.center[3 * f + 1],
               z = pz - b.center[3 * f + 2];
  const double r2 = x * x + y * y + z * z;
  double e = 0.0;
  for (int k = 0; k < b.n_prim; ++k) {
    const double t = b.exps[f * b.n_prim + k] * r2;
    if (t < 746.0) e += b.coefs[f * b.n_prim + k] * exp(-t);
  }
  double v = e;
  for (int i = 0; i < b.powers[3 * f]; ++i) v *= x;
  for (int i = 0; i < b.powers[3 * f + 1]; ++i) v *= y;
  for (int i = 0; i < b.powers[3 * f + 2]; ++i) v *= z;
  return v;
}

// chi, grad chi and lap chi of every function at every point -> out [5][n_bf][n]:
//   d^2/dx^2 [x^p e^(-a r^2)] = [p(p-1) x^(p-2) - 2a(2p+1) x^p + 4a^2 x^(p+2)] e^(-a r^2),
// summed over the primitives through e0 = sum c e, e1 = sum a c e, e2 = sum a^2 c e.
__global__ void __launch_bounds__(128) ao_lap_kernel(isdf_basis b, const double* __restrict__ pts,
                                                     int64_t n, double* __restrict__ out) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n) return;
  const int64_t plane = (int64_t)b.n_bf * n;
  for (int f = 0; f < b.n_bf; ++f) {
    const double x = pts[3 * g] - b.center[3 * f], y = pts[3 * g + 1] - b.center[3 * f + 1],
                 z = pts[3 * g + 2] - b.center[3 * f + 2];
    const double r2 = x * x + y * y + z * z;
    double e0 = 0.0, e1 = 0.0, e2 = 0.0;
    for (int k = 0; k < b.n_prim; ++k) {
      const double a = b.exps[f * b.n_prim + k];
      const double t = a * r2;
      if (t < 746.0) {
        const double v = b.coefs[f * b.n_prim + k] * exp(-t);
        e0 += v;
        e1 += a * v;
        e2 += a * a * v;
      }
    }
    const int px = b.powers[3 * f], py = b.powers[3 * f + 1], pz = b.powers[3 * f + 2];
    double X0, X1, X2, Y0, Y1, Y2, Z0, Z1, Z2;
    pow3(x, px, X0, X1, X2);
    pow3(y, py, Y0, Y1, Y2);
    pow3(z, pz, Z0, Z1, Z2);
    // second-derivative factor of one axis (without the other two axes' powers)
    const double sx = X2 * e0 - 2.0 * (2 * px + 1) * X0 * e1 + 4.0 * x * x * X0 * e2;
    const double sy = Y2 * e0 - 2.0 * (2 * py + 1) * Y0 * e1 + 4.0 * y * y * Y0 * e2;
    const double sz = Z2 * e0 - 2.0 * (2 * pz + 1) * Z0 * e1 + 4.0 * z * z * Z0 * e2;
    const int64_t o = (int64_t)f * n + g;
    out[o] = X0 * Y0 * Z0 * e0;
    out[plane + o] = (X1 * e0 - 2.0 * x * X0 * e1) * Y0 * Z0;
    out[2 * plane + o] = (Y1 * e0 - 2.0 * y * Y0 * e1) * X0 * Z0;
    out[3 * plane + o] = (Z1 * e0 - 2.0 * z * Z0 * e1) * X0 * Y0;
    out[4 * plane + o] = sx * Y0 * Z0 + sy * X0 * Z0 + sz * X0 * Y0;
  }
}

// In-place Gauss-Jordan inversion of the augmented [n][2n] matrix [A | I] in
// shared memory (partial pivoting, ties to the lowest row); the right half
// becomes A^-1.  A zero pivot propagates Inf/NaN (singular determinant).
__device__ void gj_invert(double* aug, int n, double* fac, int* sh_piv) {
  const int w2 = 2 * n;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + (int)threadIdx.x; r < n; r += 32) {
        const double v = fabs(aug[r * w2 + k]);
        if (v > best) {
          best = v;
          bi = r;
        }
      }
      for (int o = 16; o; o >>= 1) {
        const double ov = __shfl_down_sync(0xffffffffu, best, o);
        const int oi = __shfl_down_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (threadIdx.x == 0) *sh_piv = bi;
    }
    __syncthreads();
    const int p = *sh_piv;
    if (p != k)
      for (int c = threadIdx.x; c < w2; c += blockDim.x) {
        const double t = aug[k * w2 + c];
        aug[k * w2 + c] = aug[p * w2 + c];
        aug[p * w2 + c] = t;
      }
    __syncthreads();
    const double inv = 1.0 / aug[k * w2 + k];
    for (int r = threadIdx.x; r < n; r += blockDim.x) fac[r] = aug[r * w2 + k];
    __syncthreads();
    for (int c = threadIdx.x; c < w2; c += blockDim.x) aug[k * w2 + c] *= inv;
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * w2; idx += blockDim.x) {
      const int r = idx / w2, c = idx - r * w2;
      if (r != k) aug[r * w2 + c] -= fac[r] * aug[k * w2 + c];
    }
    __syncthreads();
  }
}

// Per walker: drift[w][i] = (grad_i Phi_0/Phi_0, lap_i Phi_0/Phi_0) and the
// potential V[w].  orb [5][n_occ][n_pts] with n_pts = n_walk * N.
__global__ void __launch_bounds__(kVmcThreads) slater_kernel(const double* __restrict__ orb,
                                                             int n_occ, int64_t n_walk,
                                                             const double* __restrict__ walkers,
                                                             VmcNuc nuc, double* __restrict__ drift,
                                                             double* __restrict__ V) {
  extern __shared__ double sm[];
  const int n = n_occ, N = 2 * n_occ;
  double* aug = sm;             // [n][2n]
  double* fac = aug + 2 * n * n;  // [n]
  double* red = fac + n;        // [33]
  int* piv = (int*)(red + 40);
  const int64_t w = blockIdx.x;
  const int64_t n_pts = n_walk * N;
  const int64_t plane = (int64_t)n * n_pts;
  for (int s = 0; s < 2; ++s) {
    const int64_t e0 = w * N + s * n;  // first electron of this spin
    for (int idx = threadIdx.x; idx < 2 * n * n; idx += blockDim.x) {
      const int r = idx / (2 * n), c = idx - r * 2 * n;
      aug[idx] = c < n ? orb[(int64_t)c * n_pts + e0 + r] : (c - n == r ? 1.0 : 0.0);
    }
    __syncthreads();
    gj_invert(aug, n, fac, piv);
    // drift of electron a: sum_j d phi_j(r_a) (D^-1)[j][a]
    for (int idx = threadIdx.x; idx < 4 * n; idx += blockDim.x) {
      const int comp = idx / n, a = idx - comp * n;
      const double* P = orb + (1 + comp) * plane + e0 + a;
      double acc = 0.0;
      for (int j = 0; j < n; ++j) acc += P[(int64_t)j * n_pts] * aug[j * 2 * n + n + a];
      drift[(e0 + a) * 4 + comp] = acc;
    }
    __syncthreads();
  }
  // V = sum_{i<j} 1/r_ij - sum_{i,I} Z_I / r_iI + sum_{I<J} Z_I Z_J / R_IJ
  const double* R = walkers + w * N * 3;
  const int n_ee = N * (N - 1) / 2;
  double v = 0.0;
  for (int idx = threadIdx.x; idx < n_ee + N * nuc.n; idx += blockDim.x) {
    if (idx < n_ee) {
      int i = 0, rem = idx;
      while (rem >= N - 1 - i) {
        rem -= N - 1 - i;
        ++i;
      }
      const int j = i + 1 + rem;
      const double dx = R[3 * i] - R[3 * j], dy = R[3 * i + 1] - R[3 * j + 1],
                   dz = R[3 * i + 2] - R[3 * j + 2];
      v += 1.0 / sqrt(dx * dx + dy * dy + dz * dz);
    } else {
      const int q = idx - n_ee, i = q / nuc.n, I = q - i * nuc.n;
      const double dx = R[3 * i] - nuc.xyz[I][0], dy = R[3 * i + 1] - nuc.xyz[I][1],
                   dz = R[3 * i + 2] - nuc.xyz[I][2];
      v -= nuc.Z[I] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  }
  v = block_sum(v, red);
  if (threadIdx.x == 0) {
    double vnn = 0.0;
    for (int I = 0; I < nuc.n; ++I)
      for (int K = I + 1; K < nuc.n; ++K) {
        const double dx = nuc.xyz[I][0] - nuc.xyz[K][0], dy = nuc.xyz[I][1] - nuc.xyz[K][1],
                     dz = nuc.xyz[I][2] - nuc.xyz[K][2];
        vnn += nuc.Z[I] * nuc.Z[K] / sqrt(dx * dx + dy * dy + dz * dz);
      }
    V[w] = v + vnn;
  }
}

// Shared-memory layout of eloc_kernel (in doubles).
struct ElocLayout {
  int pos, drift, gt, coef, nt, acc, red, snuc, pair, total;
  __host__ __device__ ElocLayout(int N, int n_nuc, int n_pc, bool terms, bool table) {
    pos = 0;
    drift = pos + 3 * N;
    gt = drift + 4 * N;
    coef = gt + 3 * N;
    nt = coef + (n_pc > 0 ? n_pc : 1);
    acc = nt + (terms ? 6 * N * n_nuc : 0);
    red = acc + 4 * N * (n_pc + 1);
    snuc = red + 40;
    pair = snuc + (terms ? 9 * n_nuc : 0);
    total = pair + (terms && table ? 5 * N * N : 0);
  }
};

// Local energy of walker blockIdx.x for parameter set blockIdx.y (MAXA: the
// largest exponent m, n of the free terms is at most MAXA):
//   set 0 = theta, 1/2 = d +- h, 3+2t / 4+2t = b_t +- h.
// E_set [n_sets][n_walk]; dEc [n_pc][n_walk] (set 0 only, may be null).
template <int MAXA, bool TABLE>
__global__ void __launch_bounds__(kVmcThreads) eloc_kernel(
    isdf_jastrow J, const double* __restrict__ theta, double h, int64_t n_walk, int N,
    const double* __restrict__ walkers, const double* __restrict__ drift_g,
    const double* __restrict__ V, double* __restrict__ E_set, double* __restrict__ dEc) {
  extern __shared__ double sm[];
  const int T = J.n_types, K = J.n_terms, n_nuc = J.n_nuc;
  const int n_pc = T * K;
  const bool terms = K > 0 && n_nuc > 0;
  const ElocLayout L(N, n_nuc, n_pc, terms, TABLE);
  double* pos = sm + L.pos;
  double* drift = sm + L.drift;
  double* gt = sm + L.gt;
  double* coef = sm + L.coef;
  double* nt = sm + L.nt;
  double* acc = sm + L.acc;
  double* red = sm + L.red;
  double* pair = sm + L.pair;  // TABLE: [N][N][5] = F0, F1 (dx, dy, dz), F2 of one o
  double* snuc = sm + L.snuc;  // [n_nuc][9]: sum over all electrons j of A_jI^a
  const int64_t w = blockIdx.x;
  const int set = blockIdx.y;
  // parameters of this set
  double d = theta ? theta[0] : J.d;
  double b[ISDF_MAX_TYPES];
  for (int t = 0; t < T; ++t) b[t] = theta ? theta[1 + t] : J.b[t];
  if (set == 1) d += h;
  if (set == 2) d -= h;
  if (set >= 3) {
    const int t = (set - 3) >> 1;
    b[t] += ((set - 3) & 1) ? -h : h;
  }
  for (int p = threadIdx.x; p < n_pc; p += blockDim.x)
    coef[p] = theta ? theta[1 + T + p] : J.coef[p / K][p % K];
  for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) pos[q] = walkers[w * N * 3 + q];
  for (int q = threadIdx.x; q < 4 * N; q += blockDim.x) drift[q] = drift_g[w * N * 4 + q];
  __syncthreads();
  // nucleus table: A, A', lap A and the unit vector e_iI for every (i, I)
  if (terms)
    for (int q = threadIdx.x; q < N * n_nuc; q += blockDim.x) {
      const int i = q / n_nuc, I = q - i * n_nuc;
      const double bb = b[J.nuc_type[I]];
      const double vx = pos[3 * i] - J.nuc_xyz[I][0], vy = pos[3 * i + 1] - J.nuc_xyz[I][1],
                   vz = pos[3 * i + 2] - J.nuc_xyz[I][2];
      const double r = sqrt(vx * vx + vy * vy + vz * vz);
      const double rinv = r > 0.0 ? 1.0 / r : 0.0;
      const double dn = 1.0 + bb * r;
      const double A1 = bb / (dn * dn);
      double* o = nt + 6 * q;
      o[0] = bb * r / dn;
      o[1] = A1;
      o[2] = -2.0 * bb * bb / (dn * dn * dn) + 2.0 * A1 * rinv;
      o[3] = vx * rinv;
      o[4] = vy * rinv;
      o[5] = vz * rinv;
    }
  __syncthreads();
  const bool chi = chi_on(J);
  const double chi_scale = chi ? (double)(N - 1) / (double)(J.n_elec - 1) : 0.0;
  // Coefficient-free part (cusp and one-body terms), one thread per electron.
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double gx = 0.0, gy = 0.0, gz = 0.0, l = 0.0;
    if (J.cusp) {
      const double s = 0.5 / d;
      for (int j = 0; j < N; ++j) {
        if (j == i) continue;
        const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                     dz = pos[3 * i + 2] - pos[3 * j + 2];
        const double r = sqrt(dx * dx + dy * dy + dz * dz);
        const double rinv = r > 0.0 ? 1.0 / r : 0.0;
        const double den = 1.0 + d * r;
        const double E1 = d / (den * den);
        gx += s * E1 * dx * rinv;
        gy += s * E1 * dy * rinv;
        gz += s * E1 * dz * rinv;
        l += s * (-2.0 * d * d / (den * den * den) + 2.0 * E1 * rinv);
      }
    }
    if (chi) {
      // (N - 1) partners each add grad chi(r_i) / (n_elec - 1) and its Laplacian
      double cg[3];
      chi_grad_pair(J, pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], cg);
      double lc = 0.0;
      for (int I = 0; I < n_nuc; ++I) {
        const int tt = J.nuc_type[I];
        const double vx = pos[3 * i] - J.nuc_xyz[I][0], vy = pos[3 * i + 1] - J.nuc_xyz[I][1],
                     vz = pos[3 * i + 2] - J.nuc_xyz[I][2];
        const double rI = sqrt(vx * vx + vy * vy + vz * vz);
        const double den = 1.0 + J.chi_b[tt] * rI;
        lc += -2.0 * J.chi_a[tt] * J.chi_b[tt] / (den * den * den) +
              (rI > 0.0 ? 2.0 * J.chi_a[tt] / (den * den * rI) : 0.0);
      }
      gx += (double)(N - 1) * cg[0];
      gy += (double)(N - 1) * cg[1];
      gz += (double)(N - 1) * cg[2];
      l += chi_scale * lc;
    }
    acc[4 * i] = gx;
    acc[4 * i + 1] = gy;
    acc[4 * i + 2] = gz;
    acc[4 * i + 3] = l;
  }
  for (int q = threadIdx.x; q < 4 * N * n_pc; q += blockDim.x) acc[4 * N + q] = 0.0;
  __syncthreads();
  // Free terms.  For electron i, nucleus I and the exponent o of E_ij, the
  // partner sums are moments of A_jI:
  //   T0[a] = sum_j A_jI^a E^o,  T1[a] = sum_j A_jI^a (E^o)' e_ij,
  //   T2[a] = sum_j A_jI^a [(E^o)'' + (E^o)' 2/r_ij]   (lap of E^o = this bracket),
  // and term (m, n, o) with S = A_i^m A_j^n + A_j^m A_i^n sums to
  //   grad = A'(m A_i^(m-1) T0[n] + n A_i^(n-1) T0[m]) e_iI + A_i^m T1[n] + A_i^n T1[m]
  //   lap  = A'^2 (m(m-1) A_i^(m-2) T0[n] + n(n-1) A_i^(n-2) T0[m])
  //          + lap A (m A_i^(m-1) T0[n] + n A_i^(n-1) T0[m])
  //          + 2 A' (m A_i^(m-1) e_iI.T1[n] + n A_i^(n-1) e_iI.T1[m])
  //          + A_i^m T2[n] + A_i^n T2[m].
  // One warp per electron; lane = (nucleus, slice of partners); the terms are
  // linear in the moments, so each lane's partial moments give partial terms
  // and one warp reduction per (term, type) sums nuclei and slices.
  if (terms) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, n_warps = blockDim.x >> 5;
    const int nl = n_nuc < 32 ? n_nuc : 32;
    const int nsl = 32 / nl;
    const int Il = lane % nl, js = lane / nl;
    const int n_chunks = (n_nuc + nl - 1) / nl;
    unsigned omask = 0;
    for (int k = 0; k < K; ++k) omask |= 1u << J.mno[k][2];
    if (omask & 1u) {
      // o = 0: E^0 = 1 has no derivative, so T1 = T2 = 0 and T0[a] is the sum
      // over all electrons of A_jI^a minus electron i's own term
      for (int I = threadIdx.x; I < n_nuc; I += blockDim.x) {
        double S[MAXA + 1];
#pragma unroll
        for (int a = 0; a <= MAXA; ++a) S[a] = 0.0;
        for (int j = 0; j < N; ++j) {
          const double Aj = nt[6 * (j * n_nuc + I)];
          double pw = 1.0;
#pragma unroll
          for (int a = 0; a <= MAXA; ++a) {
            S[a] += pw;
            pw *= Aj;
          }
        }
#pragma unroll
        for (int a = 0; a <= MAXA; ++a) snuc[9 * I + a] = S[a];
      }
      __syncthreads();
    }
    for (int o = 0; o <= 8; ++o) {
      if (!((omask >> o) & 1u)) continue;
      if (TABLE && o > 0) {
        // pair factors of this o, once per pair instead of once per lane
        __syncthreads();
        for (int q = threadIdx.x; q < N * N; q += blockDim.x) {
          const int i = q / N, j = q - i * N;
          const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                       dz = pos[3 * i + 2] - pos[3 * j + 2];
          const double r = sqrt(dx * dx + dy * dy + dz * dz);
          const double rinv = r > 0.0 ? 1.0 / r : 0.0;
          const double den = 1.0 + d * r;
          const double E = d * r / den;
          const double E1 = d / (den * den);
          const double lapE = -2.0 * d * d / (den * den * den) + 2.0 * E1 * rinv;
          const double Eo1 = o > 0 ? o * ipow(E, o - 1) : 0.0;
          const double F1 = Eo1 * E1 * rinv;
          double* f = pair + 5 * q;
          f[0] = ipow(E, o);
          f[1] = F1 * dx;
          f[2] = F1 * dy;
          f[3] = F1 * dz;
          f[4] = (o > 1 ? o * (o - 1) * ipow(E, o - 2) * E1 * E1 : 0.0) + Eo1 * lapE;
        }
        __syncthreads();
      }
      for (int i = warp; i < N; i += n_warps)
        for (int ch = 0; ch < n_chunks; ++ch) {
          const int I = ch * nl + Il;
          const bool on = js < nsl && I < n_nuc;
          double T0[MAXA + 1], T1x[MAXA + 1], T1y[MAXA + 1], T1z[MAXA + 1], T2[MAXA + 1];
#pragma unroll
          for (int a = 0; a <= MAXA; ++a) T0[a] = T1x[a] = T1y[a] = T1z[a] = T2[a] = 0.0;
          if (on && o == 0 && js == 0) {
            const double Ai = nt[6 * (i * n_nuc + I)];
            double pw = 1.0;
#pragma unroll
            for (int a = 0; a <= MAXA; ++a) {
              T0[a] = snuc[9 * I + a] - pw;
              pw *= Ai;
            }
          }
          if (on && TABLE && o > 0)
            for (int j = js; j < N; j += nsl) {
              if (j == i) continue;
              const double* f = pair + 5 * (i * N + j);
              const double F0 = f[0], F1x = f[1], F1y = f[2], F1z = f[3], F2 = f[4];
              const double Aj = nt[6 * (j * n_nuc + I)];
              double pw = 1.0;
#pragma unroll
              for (int a = 0; a <= MAXA; ++a) {
                T0[a] += F0 * pw;
                T1x[a] += F1x * pw;
                T1y[a] += F1y * pw;
                T1z[a] += F1z * pw;
                T2[a] += F2 * pw;
                pw *= Aj;
              }
            }
          if (on && !TABLE && o > 0)
            for (int j = js; j < N; j += nsl) {
              if (j == i) continue;
              const double dx = pos[3 * i] - pos[3 * j], dy = pos[3 * i + 1] - pos[3 * j + 1],
                           dz = pos[3 * i + 2] - pos[3 * j + 2];
              const double r = sqrt(dx * dx + dy * dy + dz * dz);
              const double rinv = r > 0.0 ? 1.0 / r : 0.0;
              const double den = 1.0 + d * r;
              const double E = d * r / den;
              const double E1 = d / (den * den);
              const double lapE = -2.0 * d * d / (den * den * den) + 2.0 * E1 * rinv;
              const double F0 = ipow(E, o);
              const double Eo1 = o > 0 ? o * ipow(E, o - 1) : 0.0;
              const double F1 = Eo1 * E1 * rinv;  // times (dx, dy, dz) = times r e_ij
              const double F2 = (o > 1 ? o * (o - 1) * ipow(E, o - 2) * E1 * E1 : 0.0) + Eo1 * lapE;
              const double Aj = nt[6 * (j * n_nuc + I)];
              double pw = 1.0;
#pragma unroll
              for (int a = 0; a <= MAXA; ++a) {
                T0[a] += F0 * pw;
                const double f1 = F1 * pw;
                T1x[a] += f1 * dx;
                T1y[a] += f1 * dy;
                T1z[a] += f1 * dz;
                T2[a] += F2 * pw;
                pw *= Aj;
              }
            }
          const double* ni = nt + 6 * (i * n_nuc + (on ? I : 0));
          const double Ai = on ? ni[0] : 0.0, A1 = on ? ni[1] : 0.0, lapA = on ? ni[2] : 0.0;
          const double ex = on ? ni[3] : 0.0, ey = on ? ni[4] : 0.0, ez = on ? ni[5] : 0.0;
          const int ti = on ? J.nuc_type[I] : -1;
          for (int k = 0; k < K; ++k) {
            if (J.mno[k][2] != o) continue;
            const int m = J.mno[k][0], n = J.mno[k][1];
            double t0m = 0, t0n = 0, t1mx = 0, t1my = 0, t1mz = 0, t1nx = 0, t1ny = 0, t1nz = 0,
                   t2m = 0, t2n = 0;
#pragma unroll
            for (int a = 0; a <= MAXA; ++a) {
              if (a == m) {
                t0m = T0[a]; t1mx = T1x[a]; t1my = T1y[a]; t1mz = T1z[a]; t2m = T2[a];
              }
              if (a == n) {
                t0n = T0[a]; t1nx = T1x[a]; t1ny = T1y[a]; t1nz = T1z[a]; t2n = T2[a];
              }
            }
            const double am = ipow(Ai, m), an = ipow(Ai, n);
            const double dm = m > 0 ? m * ipow(Ai, m - 1) : 0.0;
            const double dn = n > 0 ? n * ipow(Ai, n - 1) : 0.0;
            const double sm2 = m > 1 ? m * (m - 1) * ipow(Ai, m - 2) : 0.0;
            const double sn2 = n > 1 ? n * (n - 1) * ipow(Ai, n - 2) : 0.0;
            const double s1 = dm * t0n + dn * t0m;
            const double ga = s1 * A1;
            double v[4];
            v[0] = ga * ex + am * t1nx + an * t1mx;
            v[1] = ga * ey + am * t1ny + an * t1my;
            v[2] = ga * ez + am * t1nz + an * t1mz;
            const double ct = dm * (ex * t1nx + ey * t1ny + ez * t1nz) +
                              dn * (ex * t1mx + ey * t1my + ez * t1mz);
            v[3] = A1 * A1 * (sm2 * t0n + sn2 * t0m) + lapA * s1 + 2.0 * A1 * ct + am * t2n +
                   an * t2m;
            for (int t = 0; t < T; ++t) {
              double u[4];
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                u[c] = ti == t ? v[c] : 0.0;
                for (int off = 16; off; off >>= 1) u[c] += __shfl_down_sync(0xffffffffu, u[c], off);
              }
              if (lane == 0) {
                double* a = acc + 4 * ((1 + t * K + k) * N + i);
#pragma unroll
                for (int c = 0; c < 4; ++c) a[c] += u[c];
              }
            }
          }
        }
      }
  }
  __syncthreads();
  // E_loc = -1/2 sum_i [lap Phi/Phi + 2 grad tau . grad Phi/Phi + lap tau + |grad tau|^2] + V
  double kin = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    double g0 = acc[4 * i], g1 = acc[4 * i + 1], g2 = acc[4 * i + 2], lt = acc[4 * i + 3];
    for (int p = 0; p < n_pc; ++p) {
      const double* a = acc + 4 * ((p + 1) * N + i);
      const double c = coef[p];
      g0 += c * a[0];
      g1 += c * a[1];
      g2 += c * a[2];
      lt += c * a[3];
    }
    gt[3 * i] = g0;
    gt[3 * i + 1] = g1;
    gt[3 * i + 2] = g2;
    const double* dr = drift + 4 * i;
    kin += dr[3] + 2.0 * (g0 * dr[0] + g1 * dr[1] + g2 * dr[2]) + lt + g0 * g0 + g1 * g1 + g2 * g2;
  }
  kin = block_sum(kin, red);  // synchronises, so gt is visible below
  if (threadIdx.x == 0) E_set[(int64_t)set * n_walk + w] = -0.5 * kin + V[w];
  // dE/dc_p = -1/2 sum_i [2 G_p,i . (grad Phi/Phi + grad tau)_i + L_p,i]
  if (set == 0 && dEc)
    for (int p = threadIdx.x; p < n_pc; p += blockDim.x) {
      double s = 0.0;
      for (int i = 0; i < N; ++i) {
        const double* a = acc + 4 * ((p + 1) * N + i);
        const double* dr = drift + 4 * i;
        s += 2.0 * (a[0] * (dr[0] + gt[3 * i]) + a[1] * (dr[1] + gt[3 * i + 1]) +
                    a[2] * (dr[2] + gt[3 * i + 2])) +
             a[3];
      }
      dEc[(int64_t)p * n_walk + w] = -0.5 * s;
    }
}

// E[w] = E_set[0][w]; dE[0] and dE[1+t] by central differences of the shifted sets.
__global__ void eloc_finish_kernel(const double* __restrict__ E_set, int64_t n_walk, int T,
                                   bool b_sets, double h, double* __restrict__ E,
                                   double* __restrict__ dE) {
  const int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n_walk) return;
  E[w] = E_set[w];
  if (!dE) return;
  const double inv = 0.5 / h;
  dE[w] = (E_set[n_walk + w] - E_set[2 * n_walk + w]) * inv;
  for (int t = 0; t < T; ++t)
    dE[(1 + t) * n_walk + w] =
        b_sets ? (E_set[(3 + 2 * t) * n_walk + w] - E_set[(4 + 2 * t) * n_walk + w]) * inv : 0.0;
}

// ------------------------------------------------------------------ sampler

// Shared-memory layout of sample_kernel (in doubles).
struct SampLayout {
  int pos, dinv, aug, chi, part, phi, v, col, misc, total;
  __host__ __device__ SampLayout(int n_occ, int n_bf) {
    const int N = 2 * n_occ;
    pos = 0;
    dinv = pos + 3 * N;
    aug = dinv + 2 * n_occ * n_occ;
    chi = aug + 2 * n_occ * n_occ;
    part = chi + n_bf;
    phi = part + kVmcThreads;
    v = phi + n_occ;
    col = v + n_occ;
    misc = col + n_occ;
    total = misc + 48;
  }
};

// phi[j] = sum_f C[f][j] chi_f(x) for j < n (block-wide, deterministic order).
__device__ void orbitals_at(const isdf_basis& b, const double* __restrict__ C, int n_orb, int n,
                            const double* x, double* chi, double* part, double* phi) {
  for (int f = threadIdx.x; f < b.n_bf; f += blockDim.x) chi[f] = ao_value(b, f, x[0], x[1], x[2]);
  __syncthreads();
  const int nsl = blockDim.x / n;
  const int j = threadIdx.x % n, sl = threadIdx.x / n;
  if (sl < nsl) {
    double s = 0.0;
    for (int f = sl; f < b.n_bf; f += nsl) s += C[(int64_t)f * n_orb + j] * chi[f];
    part[sl * n + j] = s;
  }
  __syncthreads();
  if (threadIdx.x < n) {
    double s = 0.0;
    for (int q = 0; q < nsl; ++q) s += part[q * n + threadIdx.x];
    phi[threadIdx.x] = s;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kVmcThreads) sample_kernel(
    isdf_basis b, const double* __restrict__ C, int n_orb, int n_occ,
    double* __restrict__ walkers, int64_t n_walk, const double* __restrict__ normals,
    const double* __restrict__ uniforms, int n_steps, double sigma,
    unsigned long long* __restrict__ accepted) {
  extern __shared__ double sm[];
  const int n = n_occ, N = 2 * n_occ;
  const SampLayout L(n_occ, b.n_bf);
  double* pos = sm + L.pos;
  double* dinv = sm + L.dinv;  // [2][n][n]: (D_s^-1)[j][a]
  double* aug = sm + L.aug;
  double* chi = sm + L.chi;
  double* part = sm + L.part;
  double* phi = sm + L.phi;
  double* v = sm + L.v;
  double* col = sm + L.col;
  double* misc = sm + L.misc;  // [0..2] proposal, [3..] pivot scratch
  int* piv = (int*)(misc + 40);
  const int64_t w = blockIdx.x;
  for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) pos[q] = walkers[w * N * 3 + q];
  __syncthreads();
  // initial inverses
  for (int s = 0; s < 2; ++s) {
    for (int a = 0; a < n; ++a) {
      orbitals_at(b, C, n_orb, n, pos + 3 * (s * n + a), chi, part, phi);
      for (int c = threadIdx.x; c < 2 * n; c += blockDim.x)
        aug[a * 2 * n + c] = c < n ? phi[c] : (c - n == a ? 1.0 : 0.0);
      __syncthreads();
    }
    gj_invert(aug, n, col, piv);
    for (int q = threadIdx.x; q < n * n; q += blockDim.x) {
      const int j = q / n, a = q - j * n;
      dinv[s * n * n + q] = aug[j * 2 * n + n + a];
    }
    __syncthreads();
  }
  unsigned long long count = 0;
  for (int st = 0; st < n_steps; ++st)
    for (int i = 0; i < N; ++i) {
      const int s = i / n, a = i - s * n;
      double* Di = dinv + s * n * n;
      const int64_t ix = ((int64_t)st * N + i) * n_walk + w;
      if (threadIdx.x < 3) misc[threadIdx.x] = pos[3 * i + threadIdx.x] + sigma * normals[3 * ix + threadIdx.x];
      __syncthreads();
      orbitals_at(b, C, n_orb, n, misc, chi, part, phi);
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double s2 = 0.0;
        for (int j = 0; j < n; ++j) s2 += phi[j] * Di[j * n + c];
        v[c] = s2;
      }
      __syncthreads();
      const double q = v[a];
      if (uniforms[ix] < q * q) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) col[j] = Di[j * n + a];
        __syncthreads();
        const double qi = 1.0 / q;
        for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
          const int j = idx / n, c = idx - j * n;
          Di[idx] = c == a ? col[j] * qi : Di[idx] - col[j] * v[c] * qi;
        }
        if (threadIdx.x < 3) pos[3 * i + threadIdx.x] = misc[threadIdx.x];
        ++count;
      }
      __syncthreads();
    }
  for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) walkers[w * N * 3 + q] = pos[q];
  if (threadIdx.x == 0) atomicAdd(accepted, count);
}

// ------------------------------------------------------------------ Gauss-Newton

// One CTA: clipping statistics (Eq. var-loss), residuals r, residual Jacobian
// (P = 0 with r = NULL: the statistics alone)
// dr [P][n_w] (clipped energies follow their bound), grad = 2/(n_w-1) dr r,
// C = lam I (the GEMM adds dr dr^T / n_w), stats = (clipped mean, variance,
// raw mean, mean absolute deviation).
__global__ void __launch_bounds__(1024) gn_stats_kernel(const double* __restrict__ E,
                                                        const double* __restrict__ dE,
                                                        int64_t n_w, int P, double lam,
                                                        double* __restrict__ dr,
                                                        double* __restrict__ r,
                                                        double* __restrict__ grad,
                                                        double* __restrict__ C,
                                                        double* __restrict__ stats) {
  __shared__ double red[40];
  const double inv_n = 1.0 / (double)n_w;
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < n_w; k += blockDim.x) s += E[k];
  const double m = block_sum(s, red) * inv_n;
  s = 0.0;
  for (int64_t k = threadIdx.x; k < n_w; k += blockDim.x) s += fabs(E[k] - m);
  const double dev = block_sum(s, red) * inv_n;
  const double lo = m - 5.0 * dev, hi = m + 5.0 * dev;
  s = 0.0;
  for (int64_t k = threadIdx.x; k < n_w; k += blockDim.x) s += fmin(fmax(E[k], lo), hi);
  const double mean = block_sum(s, red) * inv_n;
  s = 0.0;
  for (int64_t k = threadIdx.x; k < n_w; k += blockDim.x) {
    const double x = fmin(fmax(E[k], lo), hi) - mean;
    if (r) r[k] = x;
    s += x * x;
  }
  const double var = block_sum(s, red) / (double)(n_w - 1);
  for (int p = 0; p < P; ++p) {
    const double* dp = dE + (int64_t)p * n_w;
    double* rp = dr + (int64_t)p * n_w;
    s = 0.0;
    for (int64_t k = threadIdx.x; k < n_w; k += blockDim.x) s += dp[k];
    const double dm = block_sum(s, red) * inv_n;
    s = 0.0;
    for (int64_t k = threadIdx.x; k < n_w; k += blockDim.x) {
      const double x = E[k] - m;
      const double sg = (double)((x > 0.0) - (x < 0.0));
      s += sg * (dp[k] - dm);
    }
    const double ddev = block_sum(s, red) * inv_n;
    s = 0.0;
    for (int64_t k = threadIdx.x; k < n_w; k += blockDim.x) {
      const double e = E[k];
      const double x = e < lo ? dm - 5.0 * ddev : (e > hi ? dm + 5.0 * ddev : dp[k]);
      rp[k] = x;
      s += x;
    }
    const double cm = block_sum(s, red) * inv_n;
    s = 0.0;
    for (int64_t k = threadIdx.x; k < n_w; k += blockDim.x) {
      const double x = rp[k] - cm;
      rp[k] = x;
      s += x * r[k];
    }
    const double gp = block_sum(s, red) * (2.0 / (double)(n_w - 1));
    if (threadIdx.x == 0) grad[p] = gp;
  }
  for (int q = threadIdx.x; q < P * P; q += blockDim.x) C[q] = (q / P == q % P) ? lam : 0.0;
  if (threadIdx.x == 0) {
    stats[0] = mean;
    stats[1] = var;
    stats[2] = m;
    stats[3] = dev;
  }
}

// step = -eta x; theta += step when theta is given and the factorisation succeeded.
__global__ void gn_finish_kernel(const double* __restrict__ x, int P, double eta,
                                 const int* __restrict__ info, double* __restrict__ step,
                                 double* __restrict__ theta) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double st = -eta * x[p];
  step[p] = st;
  if (theta && *info == 0) theta[p] += st;
}

// Polyak-Ruppert running mean: avg += (theta - avg) / k (k = 1, 2, ...).
// The first averaged iterate is theta itself: avg is not read then, so it may hold
// anything (an uninitialised buffer, NaN) before the first call.
__global__ void polyak_kernel(const double* __restrict__ theta, double* __restrict__ avg, int P,
                              double inv_k, int first) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P) avg[p] = first ? theta[p] : avg[p] + (theta[p] - avg[p]) * inv_k;
}

struct ElocWs {
  double *ao, *orb, *drift, *V, *E_set;
  size_t off;
  ElocWs(void* ws, size_t bytes, int n_bf, int n_occ, int64_t n_walk, int n_sets) {
    Carve c(ws, bytes);
    const int64_t n_pts = n_walk * 2 * n_occ;
    ao = c.take<double>((size_t)5 * n_bf * n_pts);
    orb = c.take<double>((size_t)5 * n_occ * n_pts);
    drift = c.take<double>((size_t)4 * n_pts);
    V = c.take<double>((size_t)n_walk);
    E_set = c.take<double>((size_t)n_sets * n_walk);
    off = c.off;
  }
};

struct GnWs {
  double *dr, *r, *grad, *C;
  int* info;
  size_t off;
  GnWs(void* ws, size_t bytes, int64_t n_w, int P) {
    Carve c(ws, bytes);
    dr = c.take<double>((size_t)P * n_w);
    r = c.take<double>((size_t)n_w);
    grad = c.take<double>((size_t)P);
    C = c.take<double>((size_t)P * P);
    info = c.take<int>(1);
    off = c.off;
  }
};

int n_sets_of(const isdf_jastrow& J, bool want_grad) {
  if (!want_grad) return 1;
  return 3 + ((J.n_terms > 0 && J.n_nuc > 0) ? 2 * J.n_types : 0);
}

size_t eloc_smem(const isdf_jastrow& J, int N, bool table) {
  const ElocLayout L(N, J.n_nuc, J.n_types * J.n_terms, J.n_terms > 0 && J.n_nuc > 0, table);
  return (size_t)L.total * sizeof(double);
}

}  // namespace

int vmc_n_params(const isdf_jastrow& J) { return 1 + J.n_types + J.n_types * J.n_terms; }

size_t vmc_local_energy_ws(int n_bf, int n_occ, int64_t n_walk, const isdf_jastrow& J) {
  return ElocWs(nullptr, 0, n_bf, n_occ, n_walk, n_sets_of(J, true)).off;
}

int vmc_local_energy(const isdf_basis* basis, const double* C, int n_orb, int n_occ,
                     const double* walkers, int64_t n_walk, const isdf_jastrow& J,
                     const double* charges, const double* theta, double h, double* E, double* dE,
                     void* ws, size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(basis && C && walkers && E && charges, "null pointer argument");
  ISDF_ARG(n_occ >= 1 && n_occ <= kMaxOcc && n_occ <= n_orb, "n_occ must be in [1, min(64, n_orb)]");
  ISDF_ARG(n_walk >= 1 && basis->n_bf > 0 && basis->n_prim > 0, "empty sizes");
  ISDF_ARG(!dE || (h > 0.0 && std::isfinite(h)), "fd_step must be positive");
  const int N = 2 * n_occ;
  const size_t smem = eloc_smem(J, N, false);
  ISDF_ARG(smem <= kVmcSmemMax, "electrons x nuclei x coefficients exceed shared memory (%zu B)",
           smem);
  const int n_sets = n_sets_of(J, dE != nullptr);
  ElocWs W(ws, ws_bytes, basis->n_bf, n_occ, n_walk, n_sets);
  const size_t need = vmc_local_energy_ws(basis->n_bf, n_occ, n_walk, J);
  ISDF_ARG(ws && ws_bytes >= need, "workspace too small: need %zu bytes", need);
  VmcNuc nuc;
  nuc.n = J.n_nuc;
  for (int I = 0; I < J.n_nuc; ++I) {
    for (int c = 0; c < 3; ++c) nuc.xyz[I][c] = J.nuc_xyz[I][c];
    nuc.Z[I] = charges[I];
    ISDF_ARG(std::isfinite(charges[I]), "charge not finite");
  }
  const int64_t n_pts = n_walk * N;
  ao_lap_kernel<<<(unsigned)ceil_div(n_pts, 128), 128, 0, s>>>(*basis, walkers, n_pts, W.ao);
  ISDF_LAUNCH_CHECK();
  Dgemm g;
  g.M = n_occ; g.N = n_pts; g.K = basis->n_bf;
  g.A = C; g.a_rs = 1; g.a_cs = n_orb; g.a_bs = 0;
  g.B = W.ao; g.b_rs = n_pts; g.b_cs = 1; g.b_bs = (int64_t)basis->n_bf * n_pts;
  g.C = W.orb; g.ldc = n_pts; g.c_bs = (int64_t)n_occ * n_pts;
  g.batch = 5;
  ISDF_TRY(dgemm(g, s));
  const size_t smem_sl = (size_t)(2 * n_occ * n_occ + n_occ + 40 + 8) * sizeof(double);
  ISDF_CUDA(cudaFuncSetAttribute(slater_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_sl));
  slater_kernel<<<(unsigned)n_walk, kVmcThreads, smem_sl, s>>>(W.orb, n_occ, n_walk, walkers, nuc,
                                                               W.drift, W.V);
  ISDF_LAUNCH_CHECK();
  const int T = J.n_types;
  double* dEc = dE ? dE + (int64_t)(1 + T) * n_walk : nullptr;
  int max_a = 0;
  for (int k = 0; k < J.n_terms; ++k)
    max_a = std::max(max_a, std::max(J.mno[k][0], J.mno[k][1]));
  const bool table = eloc_smem(J, N, true) <= kVmcSmemMax;
  auto kern = max_a <= 3 ? (table ? eloc_kernel<3, true> : eloc_kernel<3, false>)
                         : (table ? eloc_kernel<8, true> : eloc_kernel<8, false>);
  const size_t smem_run = eloc_smem(J, N, table);
  ISDF_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem_run));
  kern<<<dim3((unsigned)n_walk, (unsigned)n_sets), kVmcThreads, smem_run, s>>>(
      J, theta, h, n_walk, N, walkers, W.drift, W.V, W.E_set, J.n_terms > 0 ? dEc : nullptr);
  ISDF_LAUNCH_CHECK();
  eloc_finish_kernel<<<(unsigned)ceil_div(n_walk, 256), 256, 0, s>>>(W.E_set, n_walk, T,
                                                                     n_sets > 3, h, E, dE);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

int vmc_sample(const isdf_basis* basis, const double* C, int n_orb, int n_occ, double* walkers,
               int64_t n_walk, const double* normals, const double* uniforms, int n_steps,
               double sigma, int64_t* accepted, cudaStream_t s) {
  ISDF_ARG(basis && C && walkers && accepted, "null pointer argument");
  ISDF_ARG(n_steps >= 0 && (n_steps == 0 || (normals && uniforms)), "random inputs missing");
  ISDF_ARG(n_occ >= 1 && n_occ <= kMaxOcc && n_occ <= n_orb, "n_occ must be in [1, min(64, n_orb)]");
  ISDF_ARG(n_walk >= 1 && basis->n_bf > 0 && basis->n_prim > 0, "empty sizes");
  ISDF_ARG(std::isfinite(sigma) && sigma > 0.0, "sigma must be positive");
  const SampLayout L(n_occ, basis->n_bf);
  const size_t smem = (size_t)L.total * sizeof(double);
  ISDF_ARG(smem <= kVmcSmemMax, "n_bf and n_occ exceed shared memory (%zu B)", smem);
  ISDF_CUDA(cudaMemsetAsync(accepted, 0, sizeof(int64_t), s));
  ISDF_CUDA(cudaFuncSetAttribute(sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  sample_kernel<<<(unsigned)n_walk, kVmcThreads, smem, s>>>(
      *basis, C, n_orb, n_occ, walkers, n_walk, normals, uniforms, n_steps, sigma,
      (unsigned long long*)accepted);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

int vmc_objective(const double* E, int64_t n_w, double* stats, cudaStream_t s) {
  ISDF_ARG(E && stats, "null pointer argument");
  ISDF_ARG(n_w >= 2, "need n_walkers >= 2");
  gn_stats_kernel<<<1, 1024, 0, s>>>(E, nullptr, n_w, 0, 0.0, nullptr, nullptr, nullptr, nullptr,
                                     stats);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

int vmc_polyak(const double* theta, double* avg, int P, int64_t k, cudaStream_t s) {
  ISDF_ARG(theta && avg, "null pointer argument");
  ISDF_ARG(P >= 1 && k >= 1, "need n_par >= 1 and k >= 1");
  polyak_kernel<<<(unsigned)ceil_div(P, 128), 128, 0, s>>>(theta, avg, P, 1.0 / (double)k,
                                                            k == 1 ? 1 : 0);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

size_t vmc_gn_step_ws(int64_t n_w, int P) { return GnWs(nullptr, 0, n_w, P).off; }

int vmc_gn_step(const double* E, const double* dE, int64_t n_w, int P, double lam, double eta,
                double* theta, double* step, double* stats, void* ws, size_t ws_bytes,
                cudaStream_t s) {
  ISDF_ARG(E && dE && step && stats, "null pointer argument");
  ISDF_ARG(n_w >= 2 && P >= 1 && P <= 4096, "need n_walkers >= 2 and 1 <= n_par <= 4096");
  ISDF_ARG(lam >= 0.0 && std::isfinite(lam) && std::isfinite(eta), "lambda >= 0 and finite eta");
  GnWs W(ws, ws_bytes, n_w, P);
  ISDF_ARG(ws && ws_bytes >= W.off, "workspace too small: need %zu bytes", W.off);
  gn_stats_kernel<<<1, 1024, 0, s>>>(E, dE, n_w, P, lam, W.dr, W.r, W.grad, W.C, stats);
  ISDF_LAUNCH_CHECK();
  Dgemm g;
  g.M = P; g.N = P; g.K = n_w;
  g.A = W.dr; g.a_rs = n_w; g.a_cs = 1; g.a_bs = 0;
  g.B = W.dr; g.b_rs = 1; g.b_cs = n_w; g.b_bs = 0;
  g.C = W.C; g.ldc = P; g.c_bs = 0;
  g.alpha = 1.0 / (double)n_w;
  g.beta = 1.0;
  ISDF_TRY(dgemm(g, s));
  ISDF_TRY(dpotrf_lower(W.C, P, W.info, s));
  ISDF_TRY(dpotrs_lower(W.C, P, W.grad, 1, 1, s));
  gn_finish_kernel<<<(unsigned)ceil_div(P, 128), 128, 0, s>>>(W.grad, P, eta, W.info, step,
                                                             theta);
  ISDF_LAUNCH_CHECK();
  int info = 0;
  ISDF_CUDA(cudaMemcpyAsync(&info, W.info, sizeof(int), cudaMemcpyDeviceToHost, s));
  ISDF_CUDA(cudaStreamSynchronize(s));
  if (info != 0) {
    set_error("Gauss-Newton matrix not positive definite at pivot %d", info - 1);
    return ISDF_E_NOT_PD;
  }
  return ISDF_OK;
}

}  // namespace isdf
