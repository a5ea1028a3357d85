// xTC density contraction of the three-body term (Sec. III.B): an FP64 path
// and the split-BF16 tensor-core path described at the end of this comment.
//
// Terms 1 and 4 (factorisable):
//   G_nu = sum_{i<n_occ} phi_i(r_nu)^2,  w~_g = w_g sum_l G_l xi_l(g)
//   D4 = sum_c (calG^c o w~) calG^c^T,   H_gc = sum_l G_l calG^c_{l g}
//   V_{nu g} = sum_c H_gc calG^c_{nu g}, D1 = (w xi) V^T,  D = D4 + 2 D1
// Terms 2 and 3 in the low-rank projector form (occupied columns of the HF
// projector), streamed over grid batches:
//   A^s_{a,c}(g) = sum_nu C^a_s(nu) calG^c_{nu g},  rho~^s_a(g) = sum_nu C^a_s(nu) xi_nu(g)
//   Q1_{qs}(g)   = sum_{a,c} A^s_{a,c} A^q_{a,c}
//   Q2^c_{qs}(g) = sum_a (rho~^s_a A^q_{a,c} + A^s_{a,c} rho~^q_a)
//   X_{qs mu}    = sum_g w_g [ xi_mu(g) Q1_{qs}(g) + sum_c calG^c_{mu g} Q2^c_{qs}(g) ]
// for q <= s < n_orb_x, packed row s(s+1)/2 + q (the X_{qs} = X_{sq}
// symmetry of Sec. IV.C).
// With the split-BF16 precisions, D4, D1 and the two GEMM families of X run on
// the tcgen05 split GEMM (FP32 accumulation folded every 256 inner points,
// FP64 partial sums; X always with three limbs); the element-wise parts stay
// in FP64.
#include <cuda_bf16.h>

#include "linalg.cuh"

namespace isdf {

int split_operand(const double* src, int64_t src_rs, int64_t c0, const double* colw, int64_t rows,
                  int64_t cols, int64_t rows_pad, int64_t cols_pad, int limbs, void* dst,
                  cudaStream_t s);
int splitgemm(int limbs, int batch, const void* const* A, const void* const* B, int64_t M,
              int64_t N, int64_t Kp, int64_t kchunk, int64_t fold, double* out, int64_t ldo,
              int64_t out_bs, double scale, int* err, cudaStream_t s);

namespace {

// grid points per tensor-core chunk of the D contraction
constexpr int64_t DCHUNK = 32768;

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)ceil_div(n, t); }

__global__ void gnu_kernel(const double* phiP, int n_mu, int n_orb, int n_occ, double* G) {
  int nu = blockIdx.x * blockDim.x + threadIdx.x;
  if (nu >= n_mu) return;
  double s = 0.0;
  for (int i = 0; i < n_occ; ++i) {
    double v = phiP[(int64_t)nu * n_orb + i];
    s = fma(v, v, s);
  }
  G[nu] = s;
}

// out[q][g] = scale_g * sum_l G_l M[q][l][g]  for q < nplanes (M plane stride n_mu*n_g)
__global__ void gemv_cols_kernel(const double* G, const double* M, int n_mu, int64_t n_g,
                                 int nplanes, const double* scale, double* out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nplanes * n_g) return;
  int q = (int)(e / n_g);
  int64_t g = e % n_g;
  const double* m = M + (int64_t)q * n_mu * n_g + g;
  double s = 0.0;
  for (int l = 0; l < n_mu; ++l) s = fma(G[l], m[(int64_t)l * n_g], s);
  out[e] = scale ? scale[g] * s : s;
}

// V[nu][g] = sum_c H[c][g] calG[c][nu][g]
__global__ void v_kernel(const double* H, const double* calG, int n_mu, int64_t n_g, double* V) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t plane = (int64_t)n_mu * n_g;
  if (e >= plane) return;
  int64_t g = e % n_g;
  V[e] = H[g] * calG[e] + H[n_g + g] * calG[plane + e] + H[2 * n_g + g] * calG[2 * plane + e];
}

// P[(a*n_s + s)][nu] = phi_piv[nu][a] phi_piv[nu][s]   (a < n_occ, s < n_s)
__global__ void pair_factor_kernel(const double* phiP, int n_mu, int n_orb, int n_occ, int n_s,
                                   double* P) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t tot = (int64_t)n_occ * n_s * n_mu;
  if (e >= tot) return;
  int nu = (int)(e % n_mu);
  int64_t as = e / n_mu;
  int a = (int)(as / n_s), s = (int)(as % n_s);
  P[e] = phiP[(int64_t)nu * n_orb + a] * phiP[(int64_t)nu * n_orb + s];
}

// Q[0][pair][g] = w_g Q1, Q[1+c][pair][g] = w_g Q2^c for the batch columns.
// F layout: F[f][(a, s)][g] with f = 0 (rho~) and 1..3 (A^c), batch width nbg.
__global__ void q_kernel(const double* F, int n_occ, int n_s, int64_t nbg, int64_t bw,
                         const double* w, int64_t g0, double* Q) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t npair = (int64_t)n_s * (n_s + 1) / 2;
  if (e >= npair * bw) return;
  int64_t pr = e / bw, g = e % bw;
  int s = (int)((sqrt(8.0 * (double)pr + 1.0) - 1.0) / 2.0);
  while ((int64_t)(s + 1) * (s + 2) / 2 <= pr) ++s;
  while ((int64_t)s * (s + 1) / 2 > pr) --s;
  int q = (int)(pr - (int64_t)s * (s + 1) / 2);
  const int64_t fpl = (int64_t)n_occ * n_s * nbg;
  double q1 = 0.0, q2[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < n_occ; ++a) {
    const int64_t is = ((int64_t)a * n_s + s) * nbg + g;
    const int64_t iq = ((int64_t)a * n_s + q) * nbg + g;
    const double rs = F[is], rq = F[iq];
    for (int c = 0; c < 3; ++c) {
      const double As = F[(1 + c) * fpl + is], Aq = F[(1 + c) * fpl + iq];
      q1 = fma(As, Aq, q1);
      q2[c] = fma(rs, Aq, fma(As, rq, q2[c]));
    }
  }
  const double wg = w[g0 + g];
  Q[pr * nbg + g] = wg * q1;
  for (int c = 0; c < 3; ++c) Q[((1 + c) * npair + pr) * nbg + g] = wg * q2[c];
}

// The same products for the tensor-core precisions, in FP32 arithmetic (the
// X GEMMs that consume them carry ~3e-6 relative error, the FP32 sums of
// 3 n_occ terms ~1e-7): one block per (q tile, s tile) pair of QT x QT orbital
// indices (q tile <= s tile) and QG batch points, the F values of both tiles
// staged through shared memory QA occupied orbitals at a time; thread: one
// point (lane) and one q (warp), all QT values of s.  Writes along g coalesce.
constexpr int QT = 8, QG = 32, QA = 5;
__global__ void __launch_bounds__(256) q_tile_kernel(const double* __restrict__ F, int n_occ,
                                                     int n_s, int64_t nbg, int64_t bw,
                                                     const double* __restrict__ w, int64_t g0,
                                                     double* __restrict__ Q) {
  __shared__ float sA[4][QA][QT][QG];
  __shared__ float qA[4][QA][QT][QG];
  const int64_t tp = blockIdx.y;
  int st = (int)((sqrt(8.0 * (double)tp + 1.0) - 1.0) / 2.0);
  while ((int64_t)(st + 1) * (st + 2) / 2 <= tp) ++st;
  while ((int64_t)st * (st + 1) / 2 > tp) --st;
  const int qt = (int)(tp - (int64_t)st * (st + 1) / 2);
  const int64_t gb = (int64_t)blockIdx.x * QG;
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t fpl = (int64_t)n_occ * n_s * nbg;
  float acc[4][QT];
#pragma unroll
  for (int f = 0; f < 4; ++f)
#pragma unroll
    for (int j = 0; j < QT; ++j) acc[f][j] = 0.f;
  for (int a0 = 0; a0 < n_occ; a0 += QA) {
    for (int e = threadIdx.x; e < 4 * QA * QT * QG; e += 256) {
      const int gg = e % QG;
      int r = e / QG;
      const int ss = r % QT;
      r /= QT;
      const int aa = r % QA, f = r / QA;
      const int a = a0 + aa;
      const int64_t gi = gb + gg;
      const bool ok = a < n_occ && gi < bw;
      const int si = st * QT + ss, qi = qt * QT + ss;
      const int64_t base = f * fpl + (int64_t)a * n_s * nbg + gi;
      sA[f][aa][ss][gg] = (ok && si < n_s) ? (float)F[base + (int64_t)si * nbg] : 0.f;
      qA[f][aa][ss][gg] = (ok && qi < n_s) ? (float)F[base + (int64_t)qi * nbg] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int aa = 0; aa < QA; ++aa) {
      const float rq = qA[0][aa][wq][lane];
      const float ax = qA[1][aa][wq][lane], ay = qA[2][aa][wq][lane], az = qA[3][aa][wq][lane];
#pragma unroll
      for (int j = 0; j < QT; ++j) {
        const float rs = sA[0][aa][j][lane];
        const float bx = sA[1][aa][j][lane], by = sA[2][aa][j][lane], bz = sA[3][aa][j][lane];
        acc[0][j] = fmaf(bx, ax, fmaf(by, ay, fmaf(bz, az, acc[0][j])));
        acc[1][j] = fmaf(rs, ax, fmaf(bx, rq, acc[1][j]));
        acc[2][j] = fmaf(rs, ay, fmaf(by, rq, acc[2][j]));
        acc[3][j] = fmaf(rs, az, fmaf(bz, rq, acc[3][j]));
      }
    }
    __syncthreads();
  }
  const int q = qt * QT + wq;
  const int64_t g = gb + lane;
  if (g >= bw || q >= n_s) return;
  const int64_t npair = (int64_t)n_s * (n_s + 1) / 2;
  const double wg = w[g0 + g];
#pragma unroll
  for (int j = 0; j < QT; ++j) {
    const int sj = st * QT + j;
    if (sj >= n_s || q > sj) continue;
    const int64_t pr = (int64_t)sj * (sj + 1) / 2 + q;
#pragma unroll
    for (int f = 0; f < 4; ++f) Q[((int64_t)f * npair + pr) * nbg + g] = wg * (double)acc[f][j];
  }
}

constexpr int64_t XBATCH = 4096;
// X's GEMMs always split into three limbs: its products cancel strongly (two
// limbs leave ~2e-5 relative error in X, three ~3e-6) and they are small.
constexpr int kXLimbs = 3;

// Transposed limb split: dst[l][r][c] = limb l of src[c * src_rs + c0 + r]
// (r < rows, c < cols; zero in the padding), through 32 x 32 shared-memory
// tiles so that both the reads (along r) and the writes (along c) coalesce.
__global__ void split_t_kernel(const double* __restrict__ src, int64_t src_rs, int64_t c0,
                               int64_t rows, int64_t cols, int64_t rows_pad, int64_t cols_pad,
                               int limbs, __nv_bfloat16* __restrict__ dst) {
  __shared__ double t[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, cb = (int64_t)blockIdx.y * 32;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t c = cb + i, r = r0 + threadIdx.x;
    t[i][threadIdx.x] = (c < cols && r < rows) ? src[c * src_rs + c0 + r] : 0.0;
  }
  __syncthreads();
  const int64_t plane = rows_pad * cols_pad;
  for (int i = threadIdx.y; i < 32; i += 8) {
    const int64_t r = r0 + i, c = cb + threadIdx.x;
    if (r >= rows_pad || c >= cols_pad) continue;
    double v = t[threadIdx.x][i];
    if (limbs == 3) {  // three limbs reach below the FP32 rounding: split in FP64
      for (int l = 0; l < 3; ++l) {
        const __nv_bfloat16 h = __double2bfloat16(v);
        dst[l * plane + r * cols_pad + c] = h;
        v -= (double)__bfloat162float(h);
      }
      continue;
    }
    float f = (float)v;  // limbs of the FP32 rounding
    for (int l = 0; l < limbs; ++l) {
      const __nv_bfloat16 h = __float2bfloat16_rn(f);
      dst[l * plane + r * cols_pad + c] = h;
      f -= __bfloat162float(h);
    }
  }
}

}  // namespace

size_t xtc_ws(int64_t n_g, int n_mu, int n_orb, int n_occ, int n_orb_x, int precision) {
  (void)n_orb;
  if (precision == ISDF_PREC_TF32X3) precision = ISDF_PREC_BF16X3;
  Carve c(nullptr, 0);
  c.take<double>(n_mu);
  c.take<double>(n_g);
  c.take<double>(3 * n_g);
  c.take<double>((size_t)n_mu * n_g);
  if (precision != ISDF_PREC_FP64) {
    const int limbs = precision == ISDF_PREC_BF16X6 ? 3 : 2;
    const int64_t mp = round_up(n_mu, 128), kc = DCHUNK < round_up(n_g, 32) ? DCHUNK : round_up(n_g, 32);
    c.take<uint16_t>((size_t)8 * limbs * mp * kc);
    c.take<int>(64);
  }
  if (n_orb_x > 0) {
    const int64_t nbg = XBATCH < n_g ? XBATCH : n_g;
    const int64_t npair = (int64_t)n_orb_x * (n_orb_x + 1) / 2;
    const int64_t nas = (int64_t)n_occ * n_orb_x;
    c.take<double>((size_t)nas * n_mu);
    c.take<double>((size_t)4 * nas * nbg);
    c.take<double>((size_t)4 * npair * nbg);
    if (precision != ISDF_PREC_FP64) {
      const int64_t kmu = round_up(n_mu, 32), kg = round_up(nbg, 32);
      c.take<uint16_t>((size_t)kXLimbs * round_up(nas, 128) * kmu);
      c.take<uint16_t>((size_t)4 * kXLimbs * round_up(nbg, 128) * kmu);
      c.take<uint16_t>((size_t)4 * kXLimbs * round_up(npair, 128) * kg);
      c.take<uint16_t>((size_t)4 * kXLimbs * round_up(n_mu, 128) * kg);
    }
  }
  return c.off;
}

int xtc(const double* phiP, int n_orb, int n_occ, const double* xi, const double* w,
        const double* calG, int64_t n_g, int n_mu, double* D, double* Xp, int n_orb_x,
        int precision, void* ws, size_t ws_bytes, cudaStream_t s) {
  // the split GEMMs of this contraction have BF16 limbs only: TF32X3 runs as BF16X3
  if (precision == ISDF_PREC_TF32X3) precision = ISDF_PREC_BF16X3;
  ISDF_ARG(precision == ISDF_PREC_FP64 || precision == ISDF_PREC_BF16X3 ||
               precision == ISDF_PREC_BF16X6,
           "xtc precision must be FP64, BF16X3, BF16X6 or TF32X3");
  ISDF_ARG(phiP && xi && w && calG && D, "null pointer argument");
  ISDF_ARG(n_occ >= 1 && n_occ <= n_orb && n_mu > 0 && n_g > 0,
           "bad sizes (n_occ must be in [1, n_orb], n_mu and n_g positive)");
  ISDF_ARG(!Xp || (n_orb_x >= 1 && n_orb_x <= n_orb), "n_orb_x out of range");
  if (!Xp) n_orb_x = 0;
  Carve cv(ws, ws_bytes);
  double* G = cv.take<double>(n_mu);
  double* wt = cv.take<double>(n_g);
  double* H = cv.take<double>(3 * n_g);
  double* V = cv.take<double>((size_t)n_mu * n_g);
  const int limbs = precision == ISDF_PREC_BF16X6 ? 3 : 2;
  const int64_t mp = round_up(n_mu, 128);
  const int64_t kc = DCHUNK < round_up(n_g, 32) ? DCHUNK : round_up(n_g, 32);
  uint16_t* ops = nullptr;
  int* err = nullptr;
  if (precision != ISDF_PREC_FP64) {
    ops = cv.take<uint16_t>((size_t)8 * limbs * mp * kc);
    err = cv.take<int>(64);
  }
  double *P = nullptr, *F = nullptr, *Q = nullptr;
  const int64_t nbg = XBATCH < n_g ? XBATCH : n_g;
  const int64_t npair = (int64_t)n_orb_x * (n_orb_x + 1) / 2;
  uint16_t *Pl = nullptr, *Bt = nullptr, *Ql = nullptr, *Bb = nullptr;
  const int64_t kmu = round_up(n_mu, 32), kgx = round_up(nbg, 32);
  const int64_t nas_pad = round_up((int64_t)n_occ * n_orb_x, 128), np_pad = round_up(npair, 128);
  if (n_orb_x > 0) {
    P = cv.take<double>((size_t)n_occ * n_orb_x * n_mu);
    F = cv.take<double>((size_t)4 * n_occ * n_orb_x * nbg);
    Q = cv.take<double>((size_t)4 * npair * nbg);
    if (precision != ISDF_PREC_FP64) {
      Pl = cv.take<uint16_t>((size_t)kXLimbs * nas_pad * kmu);
      Bt = cv.take<uint16_t>((size_t)4 * kXLimbs * round_up(nbg, 128) * kmu);
      Ql = cv.take<uint16_t>((size_t)4 * kXLimbs * np_pad * kgx);
      Bb = cv.take<uint16_t>((size_t)4 * kXLimbs * mp * kgx);
    }
  }
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  const int64_t plane = (int64_t)n_mu * n_g;

  gnu_kernel<<<nb(n_mu), 256, 0, s>>>(phiP, n_mu, n_orb, n_occ, G);
  ISDF_LAUNCH_CHECK();
  gemv_cols_kernel<<<nb(n_g), 256, 0, s>>>(G, xi, n_mu, n_g, 1, w, wt);
  ISDF_LAUNCH_CHECK();
  gemv_cols_kernel<<<nb(3 * n_g), 256, 0, s>>>(G, calG, n_mu, n_g, 3, nullptr, H);
  ISDF_LAUNCH_CHECK();
  v_kernel<<<nb(plane), 256, 0, s>>>(H, calG, n_mu, n_g, V);
  ISDF_LAUNCH_CHECK();
  if (precision == ISDF_PREC_FP64) {
    // D4 = sum_c (calG^c o w~) calG^c^T
    for (int c = 0; c < 3; ++c) {
      Dgemm g;
      g.M = n_mu; g.N = n_mu; g.K = n_g;
      g.A = calG + c * plane; g.a_rs = n_g; g.a_cs = 1; g.a_bs = 0;
      g.B = calG + c * plane; g.b_rs = 1; g.b_cs = n_g; g.b_bs = 0;
      g.C = D; g.ldc = n_mu; g.c_bs = 0;
      g.kscale = wt;
      g.beta = c == 0 ? 0.0 : 1.0;
      ISDF_TRY(dgemm(g, s));
    }
    // D += 2 (w xi) V^T
    Dgemm g;
    g.M = n_mu; g.N = n_mu; g.K = n_g;
    g.A = xi; g.a_rs = n_g; g.a_cs = 1; g.a_bs = 0;
    g.B = V; g.b_rs = 1; g.b_cs = n_g; g.b_bs = 0;
    g.C = D; g.ldc = n_mu; g.c_bs = 0;
    g.kscale = w;
    g.alpha = 2.0; g.beta = 1.0;
    ISDF_TRY(dgemm(g, s));
  } else {
    // the same contractions as split-BF16 tcgen05 GEMMs over grid chunks
    ISDF_CUDA(cudaMemsetAsync(D, 0, sizeof(double) * (size_t)n_mu * n_mu, s));
    ISDF_CUDA(cudaMemsetAsync(err, 0, 64 * sizeof(int), s));
    const size_t opl = (size_t)limbs * mp * kc;
    for (int64_t g0 = 0; g0 < n_g; g0 += kc) {
      const int64_t cols = g0 + kc <= n_g ? kc : n_g - g0;
      const int64_t kp = round_up(cols, 32);
      const void* A[4];
      const void* B[4];
      for (int c = 0; c < 3; ++c) {
        uint16_t* a = ops + (2 * c) * opl;
        uint16_t* b = ops + (2 * c + 1) * opl;
        ISDF_TRY(split_operand(calG + c * plane, n_g, g0, wt, n_mu, cols, mp, kp, limbs, a, s));
        ISDF_TRY(split_operand(calG + c * plane, n_g, g0, nullptr, n_mu, cols, mp, kp, limbs, b, s));
        A[c] = a;
        B[c] = b;
      }
      ISDF_TRY(splitgemm(limbs, 3, A, B, n_mu, n_mu, kp, kp, 256, D, n_mu, 0, 1.0, err, s));
      uint16_t* a = ops + 6 * opl;
      uint16_t* b = ops + 7 * opl;
      ISDF_TRY(split_operand(xi, n_g, g0, w, n_mu, cols, mp, kp, limbs, a, s));
      ISDF_TRY(split_operand(V, n_g, g0, nullptr, n_mu, cols, mp, kp, limbs, b, s));
      const void* A1[1] = {a};
      const void* B1[1] = {b};
      ISDF_TRY(splitgemm(limbs, 1, A1, B1, n_mu, n_mu, kp, kp, 256, D, n_mu, 0, 2.0, err, s));
    }
    // every input value reaches D: a NaN or Inf there leaves a non-finite D
    ISDF_TRY(scan_nonfinite(D, (int64_t)n_mu * n_mu, err, s));
    int h_err = 0;
    ISDF_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    ISDF_CUDA(cudaStreamSynchronize(s));
    if (h_err & DEV_ERR_TIMEOUT) {
      set_error("tensor-core pipeline wait expired in the D contraction (device error word 0x%x)",
                h_err);
      return ISDF_E_TIMEOUT;
    }
    if (h_err & DEV_ERR_NONFINITE) {
      set_error("D is not finite (NaN or Inf in phi_piv, xi, w or calG)");
      return ISDF_E_NONFINITE;
    }
  }
  if (n_orb_x == 0) return ISDF_OK;

  const int64_t nas = (int64_t)n_occ * n_orb_x;
  pair_factor_kernel<<<nb(nas * n_mu), 256, 0, s>>>(phiP, n_mu, n_orb, n_occ, n_orb_x, P);
  ISDF_LAUNCH_CHECK();
  if (precision != ISDF_PREC_FP64) {
    // F = P [xi | calG^c](:, batch) and X += sum_f Q_f [xi | calG^c](:, batch)^T on the
    // split-BF16 GEMM; the batch operands are split per batch (the F family transposed)
    ISDF_TRY(split_operand(P, n_mu, 0, nullptr, nas, n_mu, nas_pad, kmu, kXLimbs, Pl, s));
    ISDF_CUDA(cudaMemsetAsync(Xp, 0, sizeof(double) * (size_t)npair * n_mu, s));
    const int64_t nq = npair * nbg;
    for (int64_t g0 = 0; g0 < n_g; g0 += nbg) {
      const int64_t bw = g0 + nbg <= n_g ? nbg : n_g - g0;
      const int64_t bw_pad = round_up(bw, 128), kg = round_up(bw, 32);
      const size_t tpl = (size_t)kXLimbs * bw_pad * kmu;
      const void* A4[4];
      const void* B4[4];
      for (int f = 0; f < 4; ++f) {
        const double* src = f == 0 ? xi : calG + (int64_t)(f - 1) * plane;
        uint16_t* dst = Bt + f * tpl;
        const dim3 grd((unsigned)ceil_div(bw_pad, 32), (unsigned)ceil_div(kmu, 32));
        split_t_kernel<<<grd, dim3(32, 8), 0, s>>>(src, n_g, g0, bw, n_mu, bw_pad, kmu, kXLimbs,
                                                  (__nv_bfloat16*)dst);
        ISDF_LAUNCH_CHECK();
        A4[f] = Pl;
        B4[f] = dst;
      }
      ISDF_CUDA(cudaMemsetAsync(F, 0, sizeof(double) * 4 * (size_t)nas * nbg, s));
      ISDF_TRY(splitgemm(kXLimbs, 4, A4, B4, nas, bw, kmu, kmu, 256, F, nbg, nas * nbg, 1.0, err, s));
      {
        const int64_t nt = ceil_div(n_orb_x, QT);
        const dim3 grd((unsigned)ceil_div(bw, QG), (unsigned)(nt * (nt + 1) / 2));
        q_tile_kernel<<<grd, 256, 0, s>>>(F, n_occ, n_orb_x, nbg, bw, w, g0, Q);
        ISDF_LAUNCH_CHECK();
      }
      const size_t qpl = (size_t)kXLimbs * np_pad * kg, bpl = (size_t)kXLimbs * mp * kg;
      for (int f = 0; f < 4; ++f) {
        const double* src = f == 0 ? xi : calG + (int64_t)(f - 1) * plane;
        ISDF_TRY(split_operand(Q + f * nq, nbg, 0, nullptr, npair, bw, np_pad, kg, kXLimbs,
                               Ql + f * qpl, s));
        ISDF_TRY(split_operand(src, n_g, g0, nullptr, n_mu, bw, mp, kg, kXLimbs, Bb + f * bpl, s));
        A4[f] = Ql + f * qpl;
        B4[f] = Bb + f * bpl;
      }
      const int64_t kr = kg < 1024 ? kg : 1024;
      ISDF_TRY(splitgemm(kXLimbs, 4, A4, B4, npair, n_mu, kg, kr, 256, Xp, n_mu, 0, 1.0, err, s));
    }
    ISDF_TRY(scan_nonfinite(Xp, npair * n_mu, err, s));
    int h_err = 0;
    ISDF_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    ISDF_CUDA(cudaStreamSynchronize(s));
    if (h_err & DEV_ERR_TIMEOUT) {
      set_error("tensor-core pipeline wait expired in the X contraction (device error word 0x%x)",
                h_err);
      return ISDF_E_TIMEOUT;
    }
    if (h_err & DEV_ERR_NONFINITE) {
      set_error("X is not finite (NaN or Inf in phi_piv, xi, w or calG)");
      return ISDF_E_NONFINITE;
    }
    return ISDF_OK;
  }
  for (int64_t g0 = 0; g0 < n_g; g0 += nbg) {
    const int64_t bw = g0 + nbg <= n_g ? nbg : n_g - g0;
    // F[0] = P xi[:, batch], F[1+c] = P calG^c[:, batch]   (row stride nbg)
    for (int f = 0; f < 4; ++f) {
      Dgemm g;
      g.M = nas; g.N = bw; g.K = n_mu;
      g.A = P; g.a_rs = n_mu; g.a_cs = 1; g.a_bs = 0;
      g.B = (f == 0 ? xi : calG + (int64_t)(f - 1) * plane) + g0;
      g.b_rs = n_g; g.b_cs = 1; g.b_bs = 0;
      g.C = F + (int64_t)f * nas * nbg; g.ldc = nbg; g.c_bs = 0;
      ISDF_TRY(dgemm(g, s));
    }
    const int64_t nq = npair * nbg;
    q_kernel<<<nb(npair * bw), 256, 0, s>>>(F, n_occ, n_orb_x, nbg, bw, w, g0, Q);
    ISDF_LAUNCH_CHECK();
    // X[pair][mu] += sum_f sum_g Q[f][pair][g] M_f[mu][g0 + g]
    for (int f = 0; f < 4; ++f) {
      Dgemm g;
      g.M = npair; g.N = n_mu; g.K = bw;
      g.A = Q + f * nq; g.a_rs = nbg; g.a_cs = 1; g.a_bs = 0;
      g.B = (f == 0 ? xi : calG + (int64_t)(f - 1) * plane) + g0;
      g.b_rs = 1; g.b_cs = n_g; g.b_bs = 0;
      g.C = Xp; g.ldc = n_mu; g.c_bs = 0;
      g.beta = (g0 == 0 && f == 0) ? 0.0 : 1.0;
      ISDF_TRY(dgemm(g, s));
    }
  }
  return ISDF_OK;
}

}  // namespace isdf
