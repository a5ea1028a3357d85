// Learned interpolation-point proposer (not in the paper): per-point
// features, a small MLP (8 -> 128 -> 128 -> 1, BF16 weights,
// FP32 arithmetic) trained by weighted binary cross-entropy against the plain
// pivoted-Cholesky selection, Adam, top-k candidate selection, the pivoted
// Cholesky restricted to the candidates, and the scalar-channel ISDF fit error
// that decides between selections.
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
constexpr int MP = 64;  // points per block
constexpr int WS = MH + 1;  // padded row stride in shared memory

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

__device__ __forceinline__ float bf(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Shared-memory image of the network with BF16-rounded weights.
struct Net {
  float* W1;  // [MH][MF]
  float* b1;
  float* W2;  // [MH][WS]
  float* b2;
  float* W3;
  float* X;   // [MP][MF]
  float* H1;  // [MP][WS]  relu(z1)
  float* Z2;  // [MP][WS]  z2, later d2
  float* S;   // [MP] scores, later ds
  float* R;   // [4][MP] reduction scratch
};

__device__ void load_net(const float* __restrict__ par, float* sm, Net& n) {
  n.W1 = sm;
  n.b1 = n.W1 + MH * MF;
  n.W2 = n.b1 + MH;
  n.b2 = n.W2 + MH * WS;
  n.W3 = n.b2 + MH;
  n.X = n.W3 + MH;
  n.H1 = n.X + MP * MF;
  n.Z2 = n.H1 + MP * WS;
  n.S = n.Z2 + MP * WS;
  n.R = n.S + MP;
  for (int e = threadIdx.x; e < MH * MF; e += blockDim.x) n.W1[e] = bf(par[O_W1 + e]);
  for (int e = threadIdx.x; e < MH * MH; e += blockDim.x)
    n.W2[(e / MH) * WS + e % MH] = bf(par[O_W2 + e]);
  for (int e = threadIdx.x; e < MH; e += blockDim.x) {
    n.b1[e] = bf(par[O_B1 + e]);
    n.b2[e] = bf(par[O_B2 + e]);
    n.W3[e] = bf(par[O_W3 + e]);
  }
}

constexpr size_t NET_FLOATS = MH * MF + MH + MH * WS + MH + MH + MP * MF + 2 * MP * WS + MP + 4 * MP;

// Forward for the block's points: fills H1, Z2 and S (scores).
__device__ void forward_block(Net& n, const float* __restrict__ feat, int64_t p0, int64_t n_pts,
                              float b3) {
  const int t = threadIdx.x;
  for (int e = t; e < MP * MF; e += blockDim.x) {
    const int64_t p = p0 + e / MF;
    n.X[e] = p < n_pts ? feat[p0 * MF + e] : 0.f;
  }
  __syncthreads();
  for (int e = t; e < MP * MH; e += blockDim.x) {
    const int p = e / MH, j = e % MH;
    float z = n.b1[j];
#pragma unroll
    for (int f = 0; f < MF; ++f) z = fmaf(n.W1[j * MF + f], n.X[p * MF + f], z);
    n.H1[p * WS + j] = fmaxf(z, 0.f);
  }
  __syncthreads();
  {
    const int j = t % MH, ph = t / MH;  // 256 threads: two halves of the points
    float z[MP / 2];
#pragma unroll
    for (int q = 0; q < MP / 2; ++q) z[q] = n.b2[j];
    for (int i = 0; i < MH; ++i) {
      const float wv = n.W2[j * WS + i];
#pragma unroll
      for (int q = 0; q < MP / 2; ++q) z[q] = fmaf(wv, n.H1[(ph * (MP / 2) + q) * WS + i], z[q]);
    }
#pragma unroll
    for (int q = 0; q < MP / 2; ++q) n.Z2[(ph * (MP / 2) + q) * WS + j] = z[q];
  }
  __syncthreads();
  // s[p] = sum_j W3[j] relu(z2[p][j]) + b3: one warp per 8 points
  for (int p = t / 32; p < MP; p += blockDim.x / 32) {
    float acc = 0.f;
    for (int j = t % 32; j < MH; j += 32) acc = fmaf(n.W3[j], fmaxf(n.Z2[p * WS + j], 0.f), acc);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (t % 32 == 0) n.S[p] = acc + b3;
  }
  __syncthreads();
}

__global__ void __launch_bounds__(256) forward_kernel(const float* __restrict__ par,
                                                      const float* __restrict__ feat, int64_t n_pts,
                                                      float* __restrict__ scores) {
  extern __shared__ float sm[];
  Net n;
  load_net(par, sm, n);
  __syncthreads();
  const int64_t p0 = (int64_t)blockIdx.x * MP;
  forward_block(n, feat, p0, n_pts, bf(par[O_B3]));
  for (int p = threadIdx.x; p < MP; p += blockDim.x)
    if (p0 + p < n_pts) scores[p0 + p] = n.S[p];
}

__device__ __forceinline__ float softplusf(float t) {
  return fmaxf(t, 0.f) + log1pf(expf(-fabsf(t)));
}

// Gradient of the mean weighted BCE over n_total points (this call covers
// n_pts of them), accumulated into grad; the loss sum into *loss.  Each block
// loops over point tiles blockIdx.x, blockIdx.x + gridDim.x, ... and keeps its
// gradient sums in registers, so that grad receives one set of atomic adds per
// block instead of one per tile.
__global__ void __launch_bounds__(256) backward_kernel(const float* __restrict__ par,
                                                       const float* __restrict__ feat,
                                                       const float* __restrict__ y, int64_t n_pts,
                                                       float pos_w, float inv_n,
                                                       float* __restrict__ grad,
                                                       double* __restrict__ loss) {
  extern __shared__ float sm[];
  Net n;
  load_net(par, sm, n);
  __syncthreads();
  const int t = threadIdx.x;
  const float b3 = bf(par[O_B3]);
  // block-persistent gradient sums
  const int j2 = t % MH, ih = t / MH;  // gW2 row j2, columns ih * 64 ..
  float gw2[MH / 2];
#pragma unroll
  for (int q = 0; q < MH / 2; ++q) gw2[q] = 0.f;
  float gb2 = 0.f, gw3 = 0.f, gb3 = 0.f;
  float gw1[MF];
#pragma unroll
  for (int f = 0; f < MF; ++f) gw1[f] = 0.f;
  float gb1 = 0.f;
  double lsum = 0.0;
  for (int64_t p0 = (int64_t)blockIdx.x * MP; p0 < n_pts; p0 += (int64_t)gridDim.x * MP) {
    forward_block(n, feat, p0, n_pts, b3);
    // ds and the loss
    if (t < MP) {
      const int64_t p = p0 + t;
      float ds = 0.f, l = 0.f;
      if (p < n_pts) {
        const float s = n.S[t], yy = y[p];
        const float sig = 1.f / (1.f + expf(-s));
        ds = (pos_w * yy * (sig - 1.f) + (1.f - yy) * sig) * inv_n;
        l = pos_w * yy * softplusf(-s) + (1.f - yy) * softplusf(s);
      }
      n.S[t] = ds;
      n.R[t] = l;
    }
    __syncthreads();
    if (t == 0)
      for (int p = 0; p < MP; ++p) lsum += n.R[p];
    // gW3, gb3 and d2 = ds W3 (z2 > 0), stored over Z2
    if (t < MH) {
      for (int p = 0; p < MP; ++p) gw3 = fmaf(n.S[p], fmaxf(n.Z2[p * WS + t], 0.f), gw3);
    }
    if (t == MH) {
      for (int p = 0; p < MP; ++p) gb3 += n.S[p];
    }
    __syncthreads();
    for (int e = t; e < MP * MH; e += blockDim.x) {
      const int p = e / MH, j = e % MH;
      const float z = n.Z2[p * WS + j];
      n.Z2[p * WS + j] = z > 0.f ? n.S[p] * n.W3[j] : 0.f;
    }
    __syncthreads();
    // gW2[j][i] += sum_p d2[p][j] h1[p][i], gb2[j] += sum_p d2[p][j]
    for (int p = 0; p < MP; ++p) {
      const float d = n.Z2[p * WS + j2];
      gb2 += d;
#pragma unroll
      for (int q = 0; q < MH / 2; ++q) gw2[q] = fmaf(d, n.H1[p * WS + ih * (MH / 2) + q], gw2[q]);
    }
    // d1[p][i] = (sum_j d2[p][j] W2[j][i]) (z1 > 0)  (h1 > 0 <=> z1 > 0)
    {
      const int i = t % MH, ph = t / MH;
      float d1[MP / 2];
#pragma unroll
      for (int q = 0; q < MP / 2; ++q) d1[q] = 0.f;
      for (int j = 0; j < MH; ++j) {
        const float wv = n.W2[j * WS + i];
#pragma unroll
        for (int q = 0; q < MP / 2; ++q) d1[q] = fmaf(n.Z2[(ph * (MP / 2) + q) * WS + j], wv, d1[q]);
      }
#pragma unroll
      for (int q = 0; q < MP / 2; ++q) {
        const int p = ph * (MP / 2) + q;
        const float d = n.H1[p * WS + i] > 0.f ? d1[q] : 0.f;
        gb1 += d;
#pragma unroll
        for (int f = 0; f < MF; ++f) gw1[f] = fmaf(d, n.X[p * MF + f], gw1[f]);
      }
    }
    __syncthreads();  // the next tile's forward overwrites X, H1, Z2 and S
  }
  if (t == 0) atomicAdd(loss, lsum);
  if (t < MH) atomicAdd(grad + O_W3 + t, gw3);
  if (t == MH) atomicAdd(grad + O_B3, gb3);
#pragma unroll
  for (int q = 0; q < MH / 2; ++q) atomicAdd(grad + O_W2 + j2 * MH + ih * (MH / 2) + q, gw2[q]);
  if (ih == 0) atomicAdd(grad + O_B2 + j2, gb2);
  {
    const int i = t % MH;
#pragma unroll
    for (int f = 0; f < MF; ++f) atomicAdd(grad + O_W1 + i * MF + f, gw1[f]);
    atomicAdd(grad + O_B1 + i, gb1);
  }
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

static int set_smem(const void* fn) {
  ISDF_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(NET_FLOATS * sizeof(float))));
  return ISDF_OK;
}

int mlp_forward_tc(const float*, const float*, int64_t, float*, cudaStream_t);
int mlp_backward_tc(const float*, const float*, const float*, int64_t, float, int64_t, float*,
                    double*, cudaStream_t);

int mlp_forward(const float* par, const float* feat, int64_t n, float* scores, cudaStream_t s) {
  ISDF_ARG(par && feat && scores && n > 0, "bad arguments");
  return mlp_forward_tc(par, feat, n, scores, s);
  ISDF_TRY(set_smem((const void*)forward_kernel));
  forward_kernel<<<nb(n, MP), 256, NET_FLOATS * sizeof(float), s>>>(par, feat, n, scores);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

int mlp_backward(const float* par, const float* feat, const float* y, int64_t n, float pos_w,
                 int64_t n_total, float* grad, double* loss, cudaStream_t s) {
  ISDF_ARG(par && feat && y && grad && loss && n > 0 && n_total >= n, "bad arguments");
  return mlp_backward_tc(par, feat, y, n, pos_w, n_total, grad, loss, s);
  ISDF_TRY(set_smem((const void*)backward_kernel));
  int dev = 0, nsm = 148;
  ISDF_CUDA(cudaGetDevice(&dev));
  ISDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // one block per SM (the network image takes ~141 KB of shared memory)
  const int64_t tiles = ceil_div(n, MP);
  const unsigned blocks = (unsigned)(tiles < nsm ? tiles : nsm);
  backward_kernel<<<blocks, 256, NET_FLOATS * sizeof(float), s>>>(
      par, feat, y, n, pos_w, 1.0f / (float)n_total, grad, loss);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
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
