// The proposer network's forward and backward passes with its 128 x 128 layer
// products on the tcgen05 tensor cores (not in the paper; the network is the
// learned interpolation-point proposer).  Network: x (8 features) -> z1 = W1 x +
// b1 -> h1 = relu(z1) -> z2 = W2 h1 + b2 -> h2 = relu(z2) -> s = W3 h2 + b3, with
// BF16-rounded weights and FP32 values.
//
// Per persistent CTA (128 threads, thread p owns point p of a 128-point tile):
//   z2 [p][j]   = sum_i h1[p][i] W2[j][i]            A = h1 (two BF16 limbs), B = W2
//   d1 [p][i]   = sum_j d2[p][j] W2[j][i]            A = d2 (two limbs),      B = W2^T
//   gW2[j][i]  += sum_p d2[p][j] h1[p][i] (+ gb2)    A = d2^T, B = [h1^T; 1]  (two limbs each,
//   gW1[i][f]  += sum_p d1[p][i] x[p][f]  (+ gb1)    A = d1^T, B = [x^T; 1]    three products)
// The transposed operands are written in two rounds of 64 points (K = 64);
// gW2 and gW1 accumulate in tensor memory over all the CTA's tiles and reach
// global memory once.  z1 and h1 are recomputed from x where needed (8 FMAs per
// unit).  Layer 1 (K = 8) and layer 3 (N = 1) stay on the CUDA cores.
#include <cuda_bf16.h>

#include <cmath>

#include "linalg.cuh"
#include "mlp_layout.cuh"
#include "tc_ptx.cuh"

namespace isdf {
namespace {

using namespace mlpl;

constexpr int TP = 128;    // points per tile (MMA M of the layer products)
constexpr int HP = 64;     // points per transposed round (MMA K)
constexpr int NB2 = 144;   // rows of [h1^T; 1; 0]: 128 + ones row + padding to 16
constexpr int NB1 = 16;    // rows of [x^T; 1; 0]

// K-major operand tiles in 32-element (64-byte) sub-tiles, 64-byte swizzle.
__host__ __device__ constexpr uint32_t sub_bytes(int rows) { return (uint32_t)rows * 64u; }

// shared-memory layout (bytes from a 1024-aligned base)
constexpr uint32_t OFF_W2B = 0;                                  // [128 j][128 i]
constexpr uint32_t OFF_W2T = OFF_W2B + 4 * sub_bytes(128);       // [128 i][128 j]
constexpr uint32_t OFF_OPA = OFF_W2T + 4 * sub_bytes(128);       // 2 limbs x [128 p][128 k]
constexpr uint32_t LIMB_A = 4 * sub_bytes(128);
constexpr uint32_t OFF_TD = OFF_OPA + 2 * LIMB_A;                // 2 limbs x [128][64 p]
constexpr uint32_t LIMB_TD = 2 * sub_bytes(128);
constexpr uint32_t OFF_TB = OFF_TD + 2 * LIMB_TD;                // 2 limbs x [144][64 p]
constexpr uint32_t LIMB_TB = 2 * sub_bytes(NB2);
constexpr uint32_t OFF_F = OFF_TB + 2 * LIMB_TB;                 // floats
constexpr uint32_t F_W1 = 0, F_B1 = F_W1 + MH * MF, F_B2 = F_B1 + MH, F_W3 = F_B2 + MH,
                   F_GW3 = F_W3 + MH, F_GB3 = F_GW3 + MH, F_N = F_GB3 + 4;
constexpr uint32_t OFF_BAR = OFF_F + 4 * F_N;
constexpr uint32_t SMEM_TC = OFF_BAR + 64 + 1024;  // + alignment slack
static_assert(OFF_TD % 1024 == 0 && OFF_TB % 1024 == 0 && OFF_F % 1024 == 0, "alignment");
static_assert(SMEM_TC <= 232448, "shared memory budget");

__device__ __forceinline__ float bfr(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Byte offset of element (row, k) in a K-major operand of `rows` rows.
__device__ __forceinline__ uint32_t opnd_off(int rows, int row, int k) {
  return (uint32_t)(k >> 5) * sub_bytes(rows) + tc::sw64_offset((uint32_t)row, (uint32_t)(k & 31) >> 3) +
         (uint32_t)(k & 7) * 2u;
}

__device__ __forceinline__ void st_bf16(uint8_t* base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// Two BF16 limbs of v into operand limb planes base and base + limb_bytes.
__device__ __forceinline__ void st_limbs(uint8_t* base, uint32_t limb_bytes, uint32_t off, float v) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  *reinterpret_cast<__nv_bfloat16*>(base + off) = h;
  *reinterpret_cast<__nv_bfloat16*>(base + limb_bytes + off) =
      __float2bfloat16_rn(v - __bfloat162float(h));
}

__device__ __forceinline__ uint64_t opnd_desc(const uint8_t* base, int rows, int k16) {
  return tc::smem_desc(tc::smem_u32(base + (uint32_t)(k16 >> 1) * sub_bytes(rows) +
                                    (uint32_t)(k16 & 1) * 32u),
                       16, 512, 4);
}

struct MlpTcArgs {
  const float* par;
  const float* feat;
  const float* y;      // labels (backward)
  int64_t n;
  float pos_w, inv_n;
  float* scores;       // forward output
  float* grad;         // backward output (accumulated)
  double* loss;        // backward output (accumulated)
  uint64_t wait_ns;
};

template <bool BACKWARD>
__global__ void __launch_bounds__(128, 1) mlp_tc_kernel(const MlpTcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  float* fl = (float*)(sm + OFF_F);
  uint64_t* bar = (uint64_t*)(sm + OFF_BAR);
  uint32_t* tmem_slot = (uint32_t*)(bar + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  int* err = (int*)(tmem_slot + 2);
  const int t = threadIdx.x, warp = t >> 5;

  // weights: BF16 roundings; W2 as the B operand of z2 ([j][i]) and of d1 ([i][j])
  for (int e = t; e < MH * MF; e += 128) fl[F_W1 + e] = bfr(a.par[O_W1 + e]);
  for (int e = t; e < MH; e += 128) {
    fl[F_B1 + e] = bfr(a.par[O_B1 + e]);
    fl[F_B2 + e] = bfr(a.par[O_B2 + e]);
    fl[F_W3 + e] = bfr(a.par[O_W3 + e]);
    fl[F_GW3 + e] = 0.f;
  }
  if (t < 4) fl[F_GB3 + t] = 0.f;
  for (int e = t; e < MH * MH; e += 128) {
    const int j = e / MH, i = e % MH;
    const float wv = a.par[O_W2 + e];
    st_bf16(sm + OFF_W2B, opnd_off(128, j, i), wv);
    st_bf16(sm + OFF_W2T, opnd_off(128, i, j), wv);
  }
  if (BACKWARD) {
    // constant rows of [h1^T; 1; 0]: row 128 = 1 (first limb), rows 129 .. 143 = 0
    for (int e = t; e < (NB2 - MH) * HP; e += 128) {
      const int r = MH + e / HP, c = e % HP;
      const uint32_t off = opnd_off(NB2, r, c);
      st_bf16(sm + OFF_TB, off, r == MH ? 1.f : 0.f);
      st_bf16(sm + OFF_TB + LIMB_TB, off, 0.f);
    }
  }
  if (t == 0) {
    tc::mbar_init(bar, 1);
    *abort_flag = 0;
    *err = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, 512);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async_smem();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
  const float b3 = bfr(a.par[O_B3]);
  uint32_t phase = 0;
  bool g_started = false;
  double lsum = 0.0;
  bool ok = true;

  // issue-and-wait of one batch of MMAs (thread 0 issues; every thread waits)
  auto mma_wait = [&]() -> bool {
    const bool w = tc::mbar_wait(bar, phase, abort_flag, err, a.wait_ns);
    phase ^= 1u;
    tc::tc_fence_after();
    return __syncthreads_and(w) != 0;
  };

  const int64_t n_tiles = (a.n + TP - 1) / TP;
  for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
    const int64_t p = tile * TP + t;
    const bool valid = p < a.n;
    float x[MF];
#pragma unroll
    for (int f = 0; f < MF; ++f) x[f] = valid ? a.feat[p * MF + f] : 0.f;
    // layer 1 and the h1 operand (two limbs, row p)
    for (int i = 0; i < MH; ++i) {
      float z = fl[F_B1 + i];
#pragma unroll
      for (int f = 0; f < MF; ++f) z = fmaf(fl[F_W1 + i * MF + f], x[f], z);
      st_limbs(sm + OFF_OPA, LIMB_A, opnd_off(128, t, i), fmaxf(z, 0.f));
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc::tc_fence_after();
      constexpr uint32_t id = tc::idesc_f16(128, 128, 1);
      for (int l = 0; l < 2; ++l)
        for (int k = 0; k < 8; ++k)
          tc::umma_f16(tmem, opnd_desc(sm + OFF_OPA + l * LIMB_A, 128, k),
                       opnd_desc(sm + OFF_W2B, 128, k), id, (l | k) ? 1u : 0u);
      tc::umma_commit(bar);
    }
    if (!(ok = mma_wait())) break;
    // z2 row p: the score (layer 3)
    float s = b3;
    for (int c0 = 0; c0 < MH; c0 += 32) {
      uint32_t r[32];
      __syncwarp();
      tc::tmem_ld_32x32b_x32(tmem + lane_base + c0, r);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 32; ++q)
        s = fmaf(fl[F_W3 + c0 + q], fmaxf(__uint_as_float(r[q]) + fl[F_B2 + c0 + q], 0.f), s);
    }
    if (!BACKWARD) {
      if (valid) a.scores[p] = s;
      tc::tc_fence_before();
      __syncthreads();  // the next tile's MMAs overwrite z2 and read the h1 operand
      continue;
    }
    // ds and the loss; gW3 and gb3 (warp sums, then shared-memory atomics)
    float ds = 0.f;
    if (valid) {
      const float yy = a.y[p];
      const float sig = 1.f / (1.f + expf(-s));
      ds = (a.pos_w * yy * (sig - 1.f) + (1.f - yy) * sig) * a.inv_n;
      const float sp_m = fmaxf(-s, 0.f) + log1pf(expf(-fabsf(s)));
      const float sp_p = fmaxf(s, 0.f) + log1pf(expf(-fabsf(s)));
      lsum += (double)(a.pos_w * yy * sp_m + (1.f - yy) * sp_p);
    }
    {
      float v = ds;
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if ((t & 31) == 0) atomicAdd(&fl[F_GB3], v);
    }
    // d2 row p = ds W3 (z2 > 0) as the A operand of d1 (over the h1 operand,
    // whose MMA has completed); gW3 from relu(z2)
    for (int c0 = 0; c0 < MH; c0 += 32) {
      uint32_t r[32];
      __syncwarp();
      tc::tmem_ld_32x32b_x32(tmem + lane_base + c0, r);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        const int j = c0 + q;
        const float z = __uint_as_float(r[q]) + fl[F_B2 + j];
        const float d2 = z > 0.f ? ds * fl[F_W3 + j] : 0.f;
        st_limbs(sm + OFF_OPA, LIMB_A, opnd_off(128, t, j), d2);
        float g = ds * fmaxf(z, 0.f);
        for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
        if ((t & 31) == 0) atomicAdd(&fl[F_GW3 + j], g);
      }
    }
    tc::fence_proxy_async_smem();
    tc::tc_fence_before();
    __syncthreads();
    if (t == 0) {
      tc::tc_fence_after();
      constexpr uint32_t id = tc::idesc_f16(128, 128, 1);
      for (int l = 0; l < 2; ++l)
        for (int k = 0; k < 8; ++k)
          tc::umma_f16(tmem + 128, opnd_desc(sm + OFF_OPA + l * LIMB_A, 128, k),
                       opnd_desc(sm + OFF_W2T, 128, k), id, (l | k) ? 1u : 0u);
      tc::umma_commit(bar);
    }
    if (!(ok = mma_wait())) break;
    // gW2 (+ gb2): two rounds of 64 points, d2^T and [h1^T; 1] written by the
    // round's two warps (d2 recomputed from z2, h1 from x)
    for (int h = 0; h < 2 && ok; ++h) {
      if ((t >> 6) == h) {
        const int pl = t & 63;
        for (int c0 = 0; c0 < MH; c0 += 32) {
          uint32_t r[32];
          __syncwarp();
          tc::tmem_ld_32x32b_x32(tmem + lane_base + c0, r);
          tc::tmem_ld_wait();
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int j = c0 + q;
            const float z = __uint_as_float(r[q]) + fl[F_B2 + j];
            st_limbs(sm + OFF_TD, LIMB_TD, opnd_off(128, j, pl), z > 0.f ? ds * fl[F_W3 + j] : 0.f);
          }
        }
        for (int i = 0; i < MH; ++i) {
          float z = fl[F_B1 + i];
#pragma unroll
          for (int f = 0; f < MF; ++f) z = fmaf(fl[F_W1 + i * MF + f], x[f], z);
          st_limbs(sm + OFF_TB, LIMB_TB, opnd_off(NB2, i, pl), fmaxf(z, 0.f));
        }
      }
      tc::fence_proxy_async_smem();
      tc::tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc::tc_fence_after();
        constexpr uint32_t id = tc::idesc_f16(128, NB2, 1);
        const int la[3] = {0, 0, 1}, lb[3] = {0, 1, 0};
        for (int pr = 0; pr < 3; ++pr)
          for (int k = 0; k < 4; ++k) {
            const uint32_t acc = (g_started || pr || k) ? 1u : 0u;
            tc::umma_f16(tmem + 256, opnd_desc(sm + OFF_TD + la[pr] * LIMB_TD, 128, k),
                         opnd_desc(sm + OFF_TB + lb[pr] * LIMB_TB, NB2, k), id, acc);
          }
        tc::umma_commit(bar);
      }
      ok = mma_wait();
      g_started = true;
    }
    if (!ok) break;
    // d1 row p with the layer-1 mask; gW1 (+ gb1): d1^T and [x^T; 1] in two rounds
    for (int h = 0; h < 2 && ok; ++h) {
      if ((t >> 6) == h) {
        const int pl = t & 63;
        for (int c0 = 0; c0 < MH; c0 += 32) {
          uint32_t r[32];
          __syncwarp();
          tc::tmem_ld_32x32b_x32(tmem + lane_base + 128 + c0, r);
          tc::tmem_ld_wait();
#pragma unroll
          for (int q = 0; q < 32; ++q) {
            const int i = c0 + q;
            float z = fl[F_B1 + i];
#pragma unroll
            for (int f = 0; f < MF; ++f) z = fmaf(fl[F_W1 + i * MF + f], x[f], z);
            st_limbs(sm + OFF_TD, LIMB_TD, opnd_off(128, i, pl),
                     z > 0.f ? __uint_as_float(r[q]) : 0.f);
          }
        }
#pragma unroll
        for (int f = 0; f < NB1; ++f)
          st_limbs(sm + OFF_TB, LIMB_TB, opnd_off(NB2, f, pl),
                   f < MF ? x[f] : (f == MF && valid ? 1.f : 0.f));
      }
      tc::fence_proxy_async_smem();
      tc::tc_fence_before();
      __syncthreads();
      if (t == 0) {
        tc::tc_fence_after();
        constexpr uint32_t id = tc::idesc_f16(128, NB1, 1);
        const int la[3] = {0, 0, 1}, lb[3] = {0, 1, 0};
        for (int pr = 0; pr < 3; ++pr)
          for (int k = 0; k < 4; ++k) {
            const uint32_t acc = (tile != blockIdx.x || h || pr || k) ? 1u : 0u;
            tc::umma_f16(tmem + 400, opnd_desc(sm + OFF_TD + la[pr] * LIMB_TD, 128, k),
                         opnd_desc(sm + OFF_TB + lb[pr] * LIMB_TB, NB2, k), id, acc);
          }
        tc::umma_commit(bar);
      }
      ok = mma_wait();
    }
  }

  if (BACKWARD && ok && blockIdx.x < n_tiles) {
    // gW2 rows j (+ gb2 in column 128) and gW1 rows i (+ gb1 in column 8) from
    // tensor memory, once per CTA
    const int row = t;
    for (int c0 = 0; c0 < NB2; c0 += 16) {
      uint32_t r[16];
      __syncwarp();
      tc::tmem_ld_32x32b_x16(tmem + lane_base + 256 + c0, r);
      tc::tmem_ld_wait();
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int i = c0 + q;
        const float v = __uint_as_float(r[q]);
        if (i < MH) atomicAdd(a.grad + O_W2 + row * MH + i, v);
        else if (i == MH) atomicAdd(a.grad + O_B2 + row, v);
      }
    }
    {
      uint32_t r[16];
      __syncwarp();
      tc::tmem_ld_32x32b_x16(tmem + lane_base + 400, r);
      tc::tmem_ld_wait();
#pragma unroll
      for (int f = 0; f < MF; ++f) atomicAdd(a.grad + O_W1 + row * MF + f, __uint_as_float(r[f]));
      atomicAdd(a.grad + O_B1 + row, __uint_as_float(r[MF]));
    }
    atomicAdd(a.grad + O_W3 + t, fl[F_GW3 + t]);
    if (t == 0) atomicAdd(a.grad + O_B3, fl[F_GB3]);
    double v = lsum;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((t & 31) == 0) atomicAdd(a.loss, v);
  }
  if (!ok) {
    // a bounded wait expired: mark the output, give issued MMAs time to land
    if (t == 0) {
      if (BACKWARD) atomicAdd(a.loss, (double)NAN);
      else if (blockIdx.x * (int64_t)TP < a.n) a.scores[blockIdx.x * (int64_t)TP] = NAN;
    }
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 200000ull) {
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 512);
  }
}

template <bool BACKWARD>
int launch_mlp_tc(const MlpTcArgs& args, cudaStream_t s) {
  int dev = 0, nsm = 148;
  ISDF_CUDA(cudaGetDevice(&dev));
  ISDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t tiles = (args.n + TP - 1) / TP;
  const unsigned blocks = (unsigned)(tiles < nsm ? tiles : nsm);
  ISDF_CUDA(cudaFuncSetAttribute(mlp_tc_kernel<BACKWARD>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM_TC));
  mlp_tc_kernel<BACKWARD><<<blocks, 128, SMEM_TC, s>>>(args);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

}  // namespace

int mlp_forward_tc(const float* par, const float* feat, int64_t n, float* scores, cudaStream_t s) {
  MlpTcArgs a;
  memset(&a, 0, sizeof(a));
  a.par = par; a.feat = feat; a.n = n; a.scores = scores;
  a.wait_ns = wait_limit_ns();
  return launch_mlp_tc<false>(a, s);
}

int mlp_backward_tc(const float* par, const float* feat, const float* y, int64_t n, float pos_w,
                    int64_t n_total, float* grad, double* loss, cudaStream_t s) {
  MlpTcArgs a;
  memset(&a, 0, sizeof(a));
  a.par = par; a.feat = feat; a.y = y; a.n = n; a.pos_w = pos_w;
  a.inv_n = 1.0f / (float)n_total;
  a.grad = grad; a.loss = loss;
  a.wait_ns = wait_limit_ns();
  return launch_mlp_tc<true>(a, s);
}

}  // namespace isdf
