// Assembly of the effective xTC Hamiltonian's corrections from the ISDF
// factors (Sec. III.B final assembly and the assembly subsection that
// follows it; Eqs. K-recombine-final, deltaU-four, xtc-deltah, xtc-fock,
// xtc-const), for every orbital index, not only the occupied block.
//
// With phi_p(mu) = phi_piv, d^c_p(mu) = dphi_piv[c], the pivot tensors
//   Cs[mu][(q,s)] = phi_q(mu) phi_s(mu),
//   Dl^c[mu][(p,r)] = phi_p(mu) d^c_r(mu) - phi_r(mu) d^c_p(mu),
// and X read as Xm[mu][(q,s)] = X_{qs mu} (symmetric in q, s), the four-index
// corrections in the composite-index matrix form M[(p,r)][(q,s)] = M^{pq}_{rs} are
//   T   = sum_c Dl^c^T W^c Cs + Cs^T W^3 Cs          (K1 - K1swap + K3)
//   K   = (T + T^T) / 2                              (Eq. K-recombine-final)
//   U   = Cs^T D Cs - Cs^T Xm
//   dU  = -(U + U^T)                                 (final assembly of Sec. III.B)
// A panel of rows R of K and dU is therefore
//   K_R  = 1/2 [ (sum_c Dl^c_R^T W^c + Cs_R^T (W^3 + W^3^T)) Cs + sum_c (Cs_R^T W^c^T) Dl^c ]
//   dU_R = -[ (Cs_R^T (D + D^T) - Xm_R^T) Cs - Cs_R^T Xm ]
// i.e. one GEMM with inner dimension 4 N_mu and one with 2 N_mu per panel.
//
// The one-body increment, the xTC Fock correction and the constant contract
// these over the occupied orbitals; with P(mu,nu) = sum_o phi_o(mu) phi_o(nu),
// G = diag(P), Q^c(mu,nu) = sum_o d^c_o(mu) phi_o(nu) and S(v) = phi^T diag(v) phi
// the contractions reduce to O(N_mu^2 N_orb) work:
//   Coul  = S(D G + D^T G - Xo) - XG,   Xo_mu = sum_o X_{oo mu},  XG_pq = sum_mu X_{pq mu} G_mu
//   Exch  = phi^T [(D o P) phi - Y^T],  Y_{q mu} = sum_o phi_o(mu) X_{oq mu}
//   Delta h = Coul - (Exch + Exch^T) / 2                               (Eq. xtc-deltah)
//   A     = sum_c phi^T diag(W^c G) d^c,   S3 = S(W^3 G + W^3^T G)
//   Ma    = phi^T (sum_c W^c o Q^c) phi - sum_c d^c^T (W^c o P) phi
//   M3    = phi^T (W^3 o P) phi
//   J     = (A - A^T) + S3 - (Ma - Ma^T) / 2 - (M3 + M3^T) / 2
//           = sum_i (2 K^{pi}_{qi} - K^{pi}_{iq})
//   f^xTC = Delta h + sum_i (2 W^{pi}_{qi} - W^{pi}_{iq}) = -Delta h - J   (Eq. xtc-fock,
//           W = -K + dU, and sum_o (2 dU^{po}_{qo} - dU^{po}_{oq}) = -2 Delta h)
//   E0    = -2/3 sum_i Delta h_ii                                      (Eq. xtc-const)
#include <cuda_bf16.h>

#include <cmath>

#include "linalg.cuh"

namespace isdf {

int split_operand(const double* src, int64_t src_rs, int64_t c0, const double* colw, int64_t rows,
                  int64_t cols, int64_t rows_pad, int64_t cols_pad, int limbs, void* dst,
                  cudaStream_t s);
int splitgemm(int limbs, int batch, const void* const* A, const void* const* B, int64_t M,
              int64_t N, int64_t Kp, int64_t kchunk, int64_t fold, double* out, int64_t ldo,
              int64_t out_bs, double scale, int* err, cudaStream_t s);

namespace {

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)ceil_div(n, t); }

__device__ __forceinline__ int64_t pair_row(int a, int b) {
  const int hi = a > b ? a : b, lo = a > b ? b : a;
  return (int64_t)hi * (hi + 1) / 2 + lo;
}

// out = a o b (first) or out += a o b
__global__ void hadamard_acc_kernel(double* out, const double* a, const double* b, int64_t n,
                                    int first) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = a[i] * b[i];
  out[i] = first ? v : out[i] + v;
}

__global__ void diag_kernel(const double* A, int n, double* d) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = A[(int64_t)i * n + i];
}

// Xo[mu] = sum_{o < n_occ} X_{oo mu};  Y[q][mu] = sum_{o < n_occ} phi_o(mu) X_{oq mu}
__global__ void x_occ_kernel(const double* __restrict__ Xp, const double* __restrict__ phiP,
                             int n_mu, int n_orb, int n_occ, double* Xo, double* Y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)(n_orb + 1) * n_mu) return;
  const int q = (int)(e / n_mu), mu = (int)(e % n_mu);
  double s = 0.0;
  if (q == n_orb) {
    for (int o = 0; o < n_occ; ++o) s += Xp[pair_row(o, o) * n_mu + mu];
    Xo[mu] = s;
  } else {
    for (int o = 0; o < n_occ; ++o) s = fma(phiP[(int64_t)mu * n_orb + o], Xp[pair_row(o, q) * n_mu + mu], s);
    Y[(int64_t)q * n_mu + mu] = s;
  }
}

// Z[mu][q] -= Y[q][mu]
__global__ void sub_transpose_kernel(double* Z, const double* Y, int n_mu, int n_orb) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n_mu * n_orb) return;
  const int mu = (int)(e / n_orb), q = (int)(e % n_orb);
  Z[e] -= Y[(int64_t)q * n_mu + mu];
}

// v = a + b - c (c may be null)
__global__ void vec_combine_kernel(double* v, const double* a, const double* b, const double* c,
                                   int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = a[i] + b[i] - (c ? c[i] : 0.0);
}

struct OneBody {
  const double* Cm;   // S(D G + D^T G - Xo)
  const double* XG;   // packed [npair]
  const double* Ex;   // Exch
  const double* Am;   // A
  const double* S3;   // S(W^3 G + W^3^T G)
  const double* Ma;
  const double* M3;
  int n;
  double* dh;
  double* f;
};

__global__ void one_body_kernel(OneBody a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int n = a.n;
  if (e >= (int64_t)n * n) return;
  const int p = (int)(e / n), q = (int)(e % n);
  const int64_t t = (int64_t)q * n + p;
  const double dh = a.Cm[e] - a.XG[pair_row(p, q)] - 0.5 * (a.Ex[e] + a.Ex[t]);
  const double J = (a.Am[e] - a.Am[t]) + a.S3[e] - 0.5 * (a.Ma[e] - a.Ma[t]) -
                   0.5 * (a.M3[e] + a.M3[t]);
  a.dh[e] = dh;
  a.f[e] = -dh - J;
}

__global__ void trace_kernel(const double* dh, int n, int n_occ, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n_occ; ++i) s += dh[(int64_t)i * n + i];
    *out = s;
  }
}

// Right operands of the panel GEMMs, K-major: out[l][(q,s)][mu] limb l of
//   kind 0: phi_q(mu) phi_s(mu)  (Cs^T)
//   kind 1..3: phi_q(mu) d^c_s(mu) - phi_s(mu) d^c_q(mu), c = kind - 1  (Dl^c^T)
//   kind 4: X_{qs mu}  (Xm^T)
// rows (q,s) padded to rows_pad, mu padded to kp; padding is zero.
__global__ void right_operand_kernel(const double* __restrict__ phiP,
                                     const double* __restrict__ dphiP,
                                     const double* __restrict__ Xp, int n_mu, int n_orb, int kind,
                                     int64_t rows_pad, int64_t kp, int limbs,
                                     __nv_bfloat16* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t plane = rows_pad * kp;
  if (e >= plane) return;
  const int64_t row = e / kp;
  const int mu = (int)(e % kp);
  double v = 0.0;
  if (row < (int64_t)n_orb * n_orb && mu < n_mu) {
    const int q = (int)(row / n_orb), s = (int)(row % n_orb);
    const double* ph = phiP + (int64_t)mu * n_orb;
    if (kind == 0) {
      v = ph[q] * ph[s];
    } else if (kind <= 3) {
      const double* d = dphiP + ((int64_t)(kind - 1) * n_mu + mu) * n_orb;
      v = ph[q] * d[s] - ph[s] * d[q];
    } else {
      v = Xp[pair_row(q, s) * n_mu + mu];
    }
  }
  for (int l = 0; l < limbs; ++l) {  // three limbs: split in FP64
    const __nv_bfloat16 h = __double2bfloat16(v);
    out[l * plane + e] = h;
    v -= (double)__bfloat162float(h);
  }
}

// FP64 right operands [(q,s)][mu] (same kinds) for the CUDA-core path.
__global__ void right_operand64_kernel(const double* __restrict__ phiP,
                                       const double* __restrict__ dphiP,
                                       const double* __restrict__ Xp, int n_mu, int n_orb, int kind,
                                       double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n_orb * n_orb * n_mu) return;
  const int64_t row = e / n_mu;
  const int mu = (int)(e % n_mu);
  const int q = (int)(row / n_orb), s = (int)(row % n_orb);
  const double* ph = phiP + (int64_t)mu * n_orb;
  double v;
  if (kind == 0) {
    v = ph[q] * ph[s];
  } else if (kind <= 3) {
    const double* d = dphiP + ((int64_t)(kind - 1) * n_mu + mu) * n_orb;
    v = ph[q] * d[s] - ph[s] * d[q];
  } else {
    v = Xp[pair_row(q, s) * n_mu + mu];
  }
  out[e] = v;
}

// Pivot tensors of the panel rows (p,r) = r0 + i, i < B, as [mu][i] columns:
// F[0][mu][i] = Cs(mu, (p,r)) and F[1+c][mu][i] = Dl^c(mu, (p,r)); and the
// two row-local parts of the DeltaU left factors: L4 -= Xm_R^T, L5 = -Cs_R^T.
__global__ void panel_factor_kernel(const double* __restrict__ phiP,
                                    const double* __restrict__ dphiP, int n_mu, int n_orb,
                                    int64_t r0, int B, double* __restrict__ F) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)n_mu * B) return;
  const int mu = (int)(e / B), i = (int)(e % B);
  const int64_t row = r0 + i;
  const int p = (int)(row / n_orb), r = (int)(row % n_orb);
  const double* ph = phiP + (int64_t)mu * n_orb;
  const int64_t plane = (int64_t)n_mu * B;
  F[e] = ph[p] * ph[r];
  for (int c = 0; c < 3; ++c) {
    const double* d = dphiP + ((int64_t)c * n_mu + mu) * n_orb;
    F[(1 + c) * plane + e] = ph[p] * d[r] - ph[r] * d[p];
  }
}

__global__ void du_left_kernel(const double* __restrict__ Xp, const double* __restrict__ F,
                               int n_mu, int n_orb, int64_t r0, int B, double* __restrict__ L4,
                               double* __restrict__ L5) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)B * n_mu) return;
  const int i = (int)(e / n_mu), nu = (int)(e % n_mu);
  const int64_t row = r0 + i;
  const int p = (int)(row / n_orb), r = (int)(row % n_orb);
  L4[e] -= Xp[pair_row(p, r) * n_mu + nu];
  L5[e] = -F[(int64_t)nu * B + i];
}

}  // namespace

// ---------------------------------------------------------------- one-body part

size_t xtc_one_body_ws(int n_mu, int n_orb) {
  Carve c(nullptr, 0);
  for (int i = 0; i < 3; ++i) c.take<double>((size_t)n_mu * n_mu);  // P, T, HQ
  c.take<double>(3 * (size_t)n_mu * n_orb);           // Z (3 planes)
  c.take<double>((size_t)n_orb * n_mu);               // Y
  c.take<double>(8 * (size_t)n_mu);                   // G, Xo, v1 (3), vab, v3s, tmp
  c.take<double>(2 * (size_t)n_mu);                   // DG, DtG
  c.take<double>((size_t)n_orb * (n_orb + 1) / 2);    // XG
  c.take<double>(6 * (size_t)n_orb * n_orb);          // Cm, Ex, Am, S3, Ma, M3
  c.take<double>(1);
  return c.off;
}

int xtc_one_body(const double* W, const double* D, const double* Xp, const double* phiP,
                 const double* dphiP, int n_mu, int n_orb, int n_occ, double* dh, double* f,
                 double* e0_host, void* ws, size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(W && D && Xp && phiP && dphiP && dh && f, "null pointer argument");
  ISDF_ARG(n_mu > 0 && n_orb > 0 && n_occ >= 1 && n_occ <= n_orb,
           "bad sizes (n_occ must be in [1, n_orb])");
  Carve cv(ws, ws_bytes);
  const int64_t nn = (int64_t)n_mu * n_mu, no = (int64_t)n_orb * n_orb;
  double* P = cv.take<double>(nn);
  double* T = cv.take<double>(nn);
  double* HQ = cv.take<double>(nn);
  double* Z = cv.take<double>(3 * (size_t)n_mu * n_orb);
  double* Y = cv.take<double>((size_t)n_orb * n_mu);
  double* vec = cv.take<double>(8 * (size_t)n_mu);
  double* DG = cv.take<double>(2 * (size_t)n_mu);
  double* XG = cv.take<double>((size_t)n_orb * (n_orb + 1) / 2);
  double* mats = cv.take<double>(6 * (size_t)no);
  double* tr = cv.take<double>(1);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  double* G = vec;
  double* Xo = vec + n_mu;
  double* v1 = vec + 2 * n_mu;   // [3][n_mu]
  double* vab = vec + 5 * n_mu;
  double* v3s = vec + 6 * n_mu;
  double* DtG = DG + n_mu;
  double *Cm = mats, *Ex = mats + no, *Am = mats + 2 * no, *S3 = mats + 3 * no,
         *Ma = mats + 4 * no, *M3 = mats + 5 * no;
  const int64_t npair = (int64_t)n_orb * (n_orb + 1) / 2;

  // P = Phi_o Phi_o^T and G = diag(P)
  Dgemm g;
  g.M = n_mu; g.N = n_mu; g.K = n_occ;
  g.A = phiP; g.a_rs = n_orb; g.a_cs = 1; g.a_bs = 0;
  g.B = phiP; g.b_rs = 1; g.b_cs = n_orb; g.b_bs = 0;
  g.C = P; g.ldc = n_mu; g.c_bs = 0;
  ISDF_TRY(dgemm(g, s));
  diag_kernel<<<nb(n_mu), 256, 0, s>>>(P, n_mu, G);
  ISDF_LAUNCH_CHECK();
  // HQ = sum_c W^c o Q^c with Q^c = d^c_o Phi_o^T
  for (int c = 0; c < 3; ++c) {
    Dgemm q = g;
    q.A = dphiP + (int64_t)c * n_mu * n_orb;
    q.C = T;
    ISDF_TRY(dgemm(q, s));
    hadamard_acc_kernel<<<nb(nn), 256, 0, s>>>(HQ, W + c * nn, T, nn, c == 0);
    ISDF_LAUNCH_CHECK();
  }
  // Z^c = (W^c o P) phi, then Ma = -sum_c d^c^T Z^c (inner dimension 3 n_mu)
  Dgemm zg;
  zg.M = n_mu; zg.N = n_orb; zg.K = n_mu;
  zg.A = T; zg.a_rs = n_mu; zg.a_cs = 1; zg.a_bs = 0;
  zg.B = phiP; zg.b_rs = n_orb; zg.b_cs = 1; zg.b_bs = 0;
  zg.ldc = n_orb; zg.c_bs = 0;
  for (int c = 0; c < 3; ++c) {
    hadamard_acc_kernel<<<nb(nn), 256, 0, s>>>(T, W + c * nn, P, nn, 1);
    ISDF_LAUNCH_CHECK();
    zg.C = Z + (int64_t)c * n_mu * n_orb;
    ISDF_TRY(dgemm(zg, s));
  }
  // phi^T M phi style products: A(p,k) = X[k][p], B(k,q) = Y[k][q]
  auto tgemm = [&](const double* Aop, const double* Bop, int64_t K, double* C, double alpha,
                   double beta, const double* kscale) -> int {
    Dgemm t;
    t.M = n_orb; t.N = n_orb; t.K = K;
    t.A = Aop; t.a_rs = 1; t.a_cs = n_orb; t.a_bs = 0;
    t.B = Bop; t.b_rs = n_orb; t.b_cs = 1; t.b_bs = 0;
    t.C = C; t.ldc = n_orb; t.c_bs = 0;
    t.alpha = alpha; t.beta = beta;
    t.kscale = kscale;
    return dgemm(t, s);
  };
  ISDF_TRY(tgemm(dphiP, Z, 3 * (int64_t)n_mu, Ma, -1.0, 0.0, nullptr));
  // Ma += phi^T (HQ phi)
  zg.A = HQ; zg.C = Z;
  ISDF_TRY(dgemm(zg, s));
  ISDF_TRY(tgemm(phiP, Z, n_mu, Ma, 1.0, 1.0, nullptr));
  // M3 = phi^T ((W^3 o P) phi)
  hadamard_acc_kernel<<<nb(nn), 256, 0, s>>>(T, W + 3 * nn, P, nn, 1);
  ISDF_LAUNCH_CHECK();
  zg.A = T; zg.C = Z;
  ISDF_TRY(dgemm(zg, s));
  ISDF_TRY(tgemm(phiP, Z, n_mu, M3, 1.0, 0.0, nullptr));
  // Exch = phi^T ((D o P) phi - Y^T)
  x_occ_kernel<<<nb((int64_t)(n_orb + 1) * n_mu), 256, 0, s>>>(Xp, phiP, n_mu, n_orb, n_occ, Xo,
                                                               Y);
  ISDF_LAUNCH_CHECK();
  hadamard_acc_kernel<<<nb(nn), 256, 0, s>>>(T, D, P, nn, 1);
  ISDF_LAUNCH_CHECK();
  ISDF_TRY(dgemm(zg, s));
  sub_transpose_kernel<<<nb((int64_t)n_mu * n_orb), 256, 0, s>>>(Z, Y, n_mu, n_orb);
  ISDF_LAUNCH_CHECK();
  ISDF_TRY(tgemm(phiP, Z, n_mu, Ex, 1.0, 0.0, nullptr));
  // vectors: v1^c = W^c G, W^3 G + W^3^T G, D G, D^T G
  Dgemm mv;
  mv.N = 1; mv.K = n_mu; mv.M = n_mu;
  mv.B = G; mv.b_rs = 1; mv.b_cs = 1; mv.b_bs = 0;
  mv.ldc = 1; mv.c_bs = 0;
  mv.a_rs = n_mu; mv.a_cs = 1; mv.a_bs = nn;
  mv.A = W; mv.C = v1; mv.c_bs = n_mu; mv.batch = 3;
  ISDF_TRY(dgemm(mv, s));
  mv.batch = 1; mv.c_bs = 0;
  mv.A = W + 3 * nn; mv.C = v3s;
  ISDF_TRY(dgemm(mv, s));
  mv.a_rs = 1; mv.a_cs = n_mu; mv.beta = 1.0;   // + W^3^T G
  ISDF_TRY(dgemm(mv, s));
  mv.beta = 0.0;
  mv.A = D; mv.a_rs = 1; mv.a_cs = n_mu; mv.C = DtG;
  ISDF_TRY(dgemm(mv, s));
  mv.A = D; mv.a_rs = n_mu; mv.a_cs = 1; mv.C = DG;
  ISDF_TRY(dgemm(mv, s));
  vec_combine_kernel<<<nb(n_mu), 256, 0, s>>>(vab, DG, DtG, Xo, n_mu);
  ISDF_LAUNCH_CHECK();
  // Coul part S(vab), S3 = S(v3s), A = sum_c phi^T diag(v1^c) d^c
  ISDF_TRY(tgemm(phiP, phiP, n_mu, Cm, 1.0, 0.0, vab));
  ISDF_TRY(tgemm(phiP, phiP, n_mu, S3, 1.0, 0.0, v3s));
  for (int c = 0; c < 3; ++c)
    ISDF_TRY(tgemm(phiP, dphiP + (int64_t)c * n_mu * n_orb, n_mu, Am, 1.0, c ? 1.0 : 0.0,
                   v1 + (int64_t)c * n_mu));
  // XG = Xp G (packed pairs)
  Dgemm xg;
  xg.M = npair; xg.N = 1; xg.K = n_mu;
  xg.A = Xp; xg.a_rs = n_mu; xg.a_cs = 1; xg.a_bs = 0;
  xg.B = G; xg.b_rs = 1; xg.b_cs = 1; xg.b_bs = 0;
  xg.C = XG; xg.ldc = 1; xg.c_bs = 0;
  ISDF_TRY(dgemm(xg, s));
  OneBody ob{Cm, XG, Ex, Am, S3, Ma, M3, n_orb, dh, f};
  one_body_kernel<<<nb(no), 256, 0, s>>>(ob);
  ISDF_LAUNCH_CHECK();
  if (e0_host) {
    trace_kernel<<<1, 32, 0, s>>>(dh, n_orb, n_occ, tr);
    ISDF_LAUNCH_CHECK();
    double h = 0.0;
    ISDF_CUDA(cudaMemcpyAsync(&h, tr, sizeof(double), cudaMemcpyDeviceToHost, s));
    ISDF_CUDA(cudaStreamSynchronize(s));
    *e0_host = -2.0 / 3.0 * h;
    if (!std::isfinite(*e0_host)) {
      set_error("E0 is not finite (NaN or Inf in W, D, X or the pivot factors)");
      return ISDF_E_NONFINITE;
    }
  }
  return ISDF_OK;
}

// ---------------------------------------------------------------- two-body panels

// Left factors of a panel of rows (p,r) in [r0, r0 + B), [B][n_mu] each:
//   L0 = sum_c Dl^c_R^T W^c + Cs_R^T (W^3 + W^3^T)      (K, times Cs)
//   L(1+c) = Cs_R^T W^c^T                               (K, times Dl^c)
//   L4 = Cs_R^T (D + D^T) - Xm_R^T                      (DeltaU, times Cs)
//   L5 = -Cs_R^T                                         (DeltaU, times Xm)
static int panel_left(const double* W, const double* D, const double* Xp, const double* phiP,
                      const double* dphiP, int n_mu, int n_orb, int64_t r0, int B, bool want_k,
                      bool want_u, double* F, double* L, cudaStream_t s) {
  const int64_t stride = (int64_t)B * n_mu, nn = (int64_t)n_mu * n_mu;
  panel_factor_kernel<<<nb(stride), 256, 0, s>>>(phiP, dphiP, n_mu, n_orb, r0, B, F);
  ISDF_LAUNCH_CHECK();
  // out[i][nu] (+)= sum_mu F_f[mu][i] M(mu, nu), M = Mat or Mat^T
  auto lg = [&](int f, const double* Mat, bool trans, double* out, double beta) -> int {
    Dgemm t;
    t.M = B; t.N = n_mu; t.K = n_mu;
    t.A = F + f * stride; t.a_rs = 1; t.a_cs = B; t.a_bs = 0;
    t.B = Mat;
    t.b_rs = trans ? 1 : n_mu;
    t.b_cs = trans ? n_mu : 1;
    t.b_bs = 0;
    t.C = out; t.ldc = n_mu; t.c_bs = 0;
    t.beta = beta;
    return dgemm(t, s);
  };
  if (want_k) {
    ISDF_TRY(lg(0, W + 3 * nn, false, L, 0.0));
    ISDF_TRY(lg(0, W + 3 * nn, true, L, 1.0));
    for (int c = 0; c < 3; ++c) ISDF_TRY(lg(1 + c, W + c * nn, false, L, 1.0));
    for (int c = 0; c < 3; ++c) ISDF_TRY(lg(0, W + c * nn, true, L + (1 + c) * stride, 0.0));
  }
  if (want_u) {
    ISDF_TRY(lg(0, D, false, L + 4 * stride, 0.0));
    ISDF_TRY(lg(0, D, true, L + 4 * stride, 1.0));
    du_left_kernel<<<nb(stride), 256, 0, s>>>(Xp, F, n_mu, n_orb, r0, B, L + 4 * stride,
                                              L + 5 * stride);
    ISDF_LAUNCH_CHECK();
  }
  return ISDF_OK;
}

struct PanelLayout {
  int limbs;
  int64_t rows_pad, kp;
};

// The panel GEMMs cancel strongly (the antisymmetric Dl^c and the P12
// symmetrisation): two limbs leave ~3e-5 relative error in K and DeltaU, so
// the tensor-core precisions both use three limbs (six products).
static PanelLayout panel_layout(int n_mu, int n_orb, int precision) {
  (void)precision;
  PanelLayout L;
  L.limbs = 3;
  L.rows_pad = round_up((int64_t)n_orb * n_orb, 128);
  L.kp = round_up(n_mu, 32);
  return L;
}

size_t xtc_panel_ws(int n_mu, int n_orb, int64_t rows, int precision) {
  Carve c(nullptr, 0);
  c.take<int>(64);
  c.take<double>(6 * (size_t)rows * n_mu);                 // left factors
  c.take<double>(4 * (size_t)rows * n_mu);                 // panel pivot tensors
  const int64_t no2 = (int64_t)n_orb * n_orb;
  if (precision == ISDF_PREC_FP64) {
    c.take<double>(5 * (size_t)no2 * n_mu);               // right operands
  } else {
    PanelLayout L = panel_layout(n_mu, n_orb, precision);
    const int64_t lp = round_up(rows, 128);
    c.take<uint16_t>(5 * (size_t)L.limbs * L.rows_pad * L.kp);   // right operands
    c.take<uint16_t>(6 * (size_t)L.limbs * lp * L.kp);           // left operands
  }
  return c.off;
}

int xtc_panel(const double* W, const double* D, const double* Xp, const double* phiP,
              const double* dphiP, int n_mu, int n_orb, int64_t r0, int64_t r1, int precision,
              double* Kp, double* Up, void* ws, size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(phiP && dphiP && (Kp || Up), "null pointer argument");
  ISDF_ARG(!Kp || W, "K panel needs W");
  ISDF_ARG(!Up || (D && Xp), "DeltaU panel needs D and X");
  ISDF_ARG(n_mu > 0 && n_orb > 0, "empty sizes");
  const int64_t no2 = (int64_t)n_orb * n_orb;
  ISDF_ARG(r0 >= 0 && r0 < r1 && r1 <= no2, "panel rows must satisfy 0 <= begin < end <= n_orb^2");
  ISDF_ARG(precision == ISDF_PREC_FP64 || precision == ISDF_PREC_BF16X3 ||
               precision == ISDF_PREC_BF16X6,
           "precision must be FP64, BF16X3 or BF16X6");
  const int B = (int)(r1 - r0);
  ISDF_ARG(r1 - r0 < (1 << 30), "panel too tall");
  Carve cv(ws, ws_bytes);
  int* err = cv.take<int>(64);
  double* L = cv.take<double>(6 * (size_t)B * n_mu);
  double* F = cv.take<double>(4 * (size_t)B * n_mu);
  const int64_t stride = (int64_t)B * n_mu;
  if (precision == ISDF_PREC_FP64) {
    double* R = cv.take<double>(5 * (size_t)no2 * n_mu);
    ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
    ISDF_TRY(panel_left(W, D, Xp, phiP, dphiP, n_mu, n_orb, r0, B, Kp != nullptr, Up != nullptr,
                        F, L, s));
    for (int kind = 0; kind < 5; ++kind) {
      if ((kind >= 1 && kind <= 3 && !Kp) || (kind == 4 && !Up)) continue;
      right_operand64_kernel<<<nb(no2 * n_mu), 256, 0, s>>>(phiP, dphiP, Xp, n_mu, n_orb, kind,
                                                             R + kind * no2 * n_mu);
      ISDF_LAUNCH_CHECK();
    }
    // out[i][(q,s)] = sum_mu Lf[i][mu] R_kind[(q,s)][mu]
    auto pg = [&](const double* Lf, int kind, double* out, double alpha, double beta) -> int {
      Dgemm t;
      t.M = B; t.N = no2; t.K = n_mu;
      t.A = Lf; t.a_rs = n_mu; t.a_cs = 1; t.a_bs = 0;
      t.B = R + kind * no2 * n_mu; t.b_rs = 1; t.b_cs = n_mu; t.b_bs = 0;
      t.C = out; t.ldc = no2; t.c_bs = 0;
      t.alpha = alpha; t.beta = beta;
      return dgemm(t, s);
    };
    if (Kp) {
      ISDF_TRY(pg(L, 0, Kp, 0.5, 0.0));
      for (int c = 0; c < 3; ++c) ISDF_TRY(pg(L + (1 + c) * stride, 1 + c, Kp, 0.5, 1.0));
    }
    if (Up) {
      ISDF_TRY(pg(L + 4 * stride, 0, Up, -1.0, 0.0));
      ISDF_TRY(pg(L + 5 * stride, 4, Up, -1.0, 1.0));
    }
    return ISDF_OK;
  }
  const PanelLayout PL = panel_layout(n_mu, n_orb, precision);
  const int64_t lp = round_up(B, 128);
  uint16_t* R = cv.take<uint16_t>(5 * (size_t)PL.limbs * PL.rows_pad * PL.kp);
  uint16_t* Ll = cv.take<uint16_t>(6 * (size_t)PL.limbs * lp * PL.kp);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  ISDF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  ISDF_TRY(panel_left(W, D, Xp, phiP, dphiP, n_mu, n_orb, r0, B, Kp != nullptr, Up != nullptr, F,
                      L, s));
  const size_t rplane = (size_t)PL.limbs * PL.rows_pad * PL.kp;
  const size_t lplane = (size_t)PL.limbs * lp * PL.kp;
  for (int kind = 0; kind < 5; ++kind) {
    if ((kind >= 1 && kind <= 3 && !Kp) || (kind == 4 && !Up)) continue;
    right_operand_kernel<<<nb(PL.rows_pad * PL.kp), 256, 0, s>>>(
        phiP, dphiP, Xp, n_mu, n_orb, kind, PL.rows_pad, PL.kp, PL.limbs,
        (__nv_bfloat16*)(R + kind * rplane));
    ISDF_LAUNCH_CHECK();
  }
  for (int j = 0; j < 6; ++j) {
    if ((j <= 3 && !Kp) || (j >= 4 && !Up)) continue;
    ISDF_TRY(split_operand(L + j * stride, n_mu, 0, nullptr, B, n_mu, lp, PL.kp, PL.limbs,
                           Ll + j * lplane, s));
  }
  if (Kp) {
    ISDF_CUDA(cudaMemsetAsync(Kp, 0, sizeof(double) * (size_t)B * no2, s));
    const void* A[4] = {Ll, Ll + lplane, Ll + 2 * lplane, Ll + 3 * lplane};
    const void* Bo[4] = {R, R + rplane, R + 2 * rplane, R + 3 * rplane};
    ISDF_TRY(splitgemm(PL.limbs, 4, A, Bo, B, no2, PL.kp, PL.kp, 256, Kp, no2, 0, 0.5, err, s));
  }
  if (Up) {
    ISDF_CUDA(cudaMemsetAsync(Up, 0, sizeof(double) * (size_t)B * no2, s));
    const void* A[2] = {Ll + 4 * lplane, Ll + 5 * lplane};
    const void* Bo[2] = {R, R + 4 * rplane};
    ISDF_TRY(splitgemm(PL.limbs, 2, A, Bo, B, no2, PL.kp, PL.kp, 256, Up, no2, 0, -1.0, err, s));
  }
  int h_err = 0;
  ISDF_TRY(read_error_word(err, &h_err, s));
  if (h_err & DEV_ERR_TIMEOUT) {
    set_error("tensor-core pipeline wait expired in the panel GEMM (device error word 0x%x)",
              h_err);
    return ISDF_E_TIMEOUT;
  }
  return ISDF_OK;
}

}  // namespace isdf
