// Jastrow kernels u^(1),c and u^(3) (Eqs. K1-isdf, K3-isdf) on the
// 5th-generation tensor cores (tcgen05) of sm_103a, with split-BF16 operands
// and FP32 accumulation in tensor memory, folded into an FP32 running sum
// every kchunk inner-grid points and written to FP64 once per tile.
//
// Stage 1 (the O(N_mu N_g^2) contraction, Sec. IV.C doubly-blocked grid sum):
//   calG^c[nu][g] = sum_g' (w xi)[nu][g'] K_c(g, g'),  c = x, y, z, sq
// as a GEMM D[nu][g] = A[nu][g'] B[g][g'] whose B operand is never stored:
// eight generator warps evaluate K_c(g, g') for a 64 x 32 (g x g') block in
// FP32 registers (radial or multi-centre correlator), split each value into
// BF16 limbs and write them straight into the 64B-swizzled K-major
// shared-memory layout that the tensor core reads.  A TMA warp streams the
// (w xi) limbs, a bulk-copy warp the inner-point data, one thread issues one
// N = 256 tcgen05.mma per limb product and k-step (the four channels' B tiles
// back to back), and four epilogue warps fold each chunk accumulator into the
// running sum held in the other half of tensor memory.
//
// Stage 2: W^c = (w xi~^c) calG^c^T as a split-BF16 tcgen05 GEMM with both
// operands streamed by TMA, split-K over the grid with FP64 atomic reduction.
//
// A value v is carried as limbs v = l0 + l1 (+ l2), each l_i = bf16(v - sum_{j<i} l_j);
// a product uses every limb pair (i, j) with i + j < LIMBS (3 products for 2
// limbs, 6 for 3 limbs).
#include <cuda.h>
#include <cuda_bf16.h>

#include "jastrow.cuh"
#include "linalg.cuh"
#include "tc_ptx.cuh"

namespace isdf {

// ------------------------------------------------------------------ host: TMA maps

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

// Tensor map over a bf16 matrix [rows][cols] (cols contiguous) with a box of
// 32 columns x box_rows rows and the 64-byte swizzle.
static int make_map(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return ISDF_E_CUDA;
  }
  ISDF_ARG(((uintptr_t)base & 15) == 0 && (cols * 2) % 16 == 0, "TMA base/stride alignment");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ISDF_E_CUDA;
  }
  return ISDF_OK;
}

// The same map for other translation units (BF16 [rows][cols], 64-byte swizzle).
int tma_map_bf16(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int box_rows) {
  return make_map(m, base, rows, cols, box_rows);
}

// Tensor map over an FP32 (TF32 limbs) matrix [rows][cols] with a box of 32
// columns x box_rows rows and the 128-byte swizzle.
static int make_map_f32(CUtensorMap* m, const void* base, int64_t rows, int64_t cols,
                        int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled unavailable");
    return ISDF_E_CUDA;
  }
  ISDF_ARG(((uintptr_t)base & 15) == 0 && (cols * 4) % 16 == 0, "TMA base/stride alignment");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)cols * 4};
  cuuint32_t box[2] = {32, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return ISDF_E_CUDA;
  }
  return ISDF_OK;
}

namespace {

// ------------------------------------------------------------------ prep kernels

// As split_kernel with TF32 limbs in 32-bit words: each limb is the TF32
// rounding (to nearest, ties away) of the FP32 rounding of the remainder.
__global__ void split_tf32_kernel(const double* __restrict__ src, int64_t src_rs, int64_t c0,
                                  const double* __restrict__ colw, int64_t rows, int64_t cols,
                                  int64_t rows_pad, int64_t cols_pad, int limbs,
                                  uint32_t* __restrict__ dst) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t plane = rows_pad * cols_pad;
  if (e >= plane) return;
  int64_t r = e / cols_pad, c = e % cols_pad;
  double v = 0.0;
  if (r < rows && c < cols) {
    v = src[r * src_rs + c0 + c];
    if (colw) v *= colw[c0 + c];
  }
  float f = (float)v;  // limbs of the FP32 rounding; each remainder is exact in FP32
  for (int l = 0; l < limbs; ++l) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(f));
    dst[l * plane + e] = h;
    f -= __uint_as_float(h);
  }
}

// dst[l][r][c] (rows_pad x cols_pad per limb) = limb l of
// src[r * src_rs + c0 + c] * colw[c0 + c]; zero outside rows x cols.
__global__ void split_kernel(const double* __restrict__ src, int64_t src_rs, int64_t c0,
                             const double* __restrict__ colw, int64_t rows, int64_t cols,
                             int64_t rows_pad, int64_t cols_pad, int limbs,
                             __nv_bfloat16* __restrict__ dst) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t plane = rows_pad * cols_pad;
  if (e >= plane) return;
  int64_t r = e / cols_pad, c = e % cols_pad;
  double v = 0.0;
  if (r < rows && c < cols) {
    v = src[r * src_rs + c0 + c];
    if (colw) v *= colw[c0 + c];
  }
  if (limbs == 3) {  // three limbs reach below the FP32 rounding: split in FP64
    for (int l = 0; l < 3; ++l) {
      const __nv_bfloat16 h = __double2bfloat16(v);
      dst[l * plane + e] = h;
      v -= (double)__bfloat162float(h);
    }
    return;
  }
  float f = (float)v;  // limbs of the FP32 rounding; each remainder is exact in FP32
  for (int l = 0; l < limbs; ++l) {
    const __nv_bfloat16 h = __float2bfloat16_rn(f);
    dst[l * plane + e] = h;
    f -= __bfloat162float(h);
  }
}

// The same split over a 2-D grid (blockIdx.y = row), four columns per thread
// written as one 8-byte word per limb; cols_pad must be a multiple of 4.
__global__ void split_rows_kernel(const double* __restrict__ src, int64_t src_rs, int64_t c0,
                                  const double* __restrict__ colw, int64_t rows, int64_t cols,
                                  int64_t cols_pad, int64_t plane, int limbs,
                                  __nv_bfloat16* __restrict__ dst) {
  const int64_t r = blockIdx.y;
  const int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4;
  if (c >= cols_pad) return;
  // with two limbs (16 significant bits) the limbs split the FP32 rounding of
  // the value, so that the only FP64 arithmetic per element is the weight
  // product and one conversion (B300's FP64 pipe is narrow; each remainder is
  // exact in FP32); three limbs reach below it and split in FP64
  double x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int64_t cc = c + q;
    x[q] = 0.0;
    if (r < rows && cc < cols) {
      x[q] = src[r * src_rs + c0 + cc];
      if (colw) x[q] *= colw[c0 + cc];
    }
  }
  __nv_bfloat16* out = dst + r * cols_pad + c;
  if (limbs == 3) {
    for (int l = 0; l < 3; ++l) {
      uint32_t bits[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat16 h = __double2bfloat16(x[q]);
        bits[q] = (uint32_t)__bfloat16_as_ushort(h);
        x[q] -= (double)__bfloat162float(h);
      }
      *reinterpret_cast<uint2*>(out + l * plane) =
          make_uint2(bits[0] | (bits[1] << 16), bits[2] | (bits[3] << 16));
    }
    return;
  }
  float v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = (float)x[q];
  for (int l = 0; l < limbs; ++l) {
    uint32_t bits[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const __nv_bfloat16 h = __float2bfloat16_rn(v[q]);
      bits[q] = (uint32_t)__bfloat16_as_ushort(h);
      v[q] -= __bfloat162float(h);
    }
    *reinterpret_cast<uint2*>(out + l * plane) =
        make_uint2(bits[0] | (bits[1] << 16), bits[2] | (bits[3] << 16));
  }
}

// hi/lo: FP32 pair of every point (hi = FP32 rounding, lo = FP32 of the
// remainder).  Padding points sit at the origin.
__global__ void coords_kernel(const double* __restrict__ grid, int64_t n_g, int64_t n_pad,
                              float4* __restrict__ hi, float4* __restrict__ lo) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_pad) return;
  double x = 0, y = 0, z = 0;
  if (g < n_g) { x = grid[3 * g]; y = grid[3 * g + 1]; z = grid[3 * g + 2]; }
  float xh = (float)x, yh = (float)y, zh = (float)z;
  hi[g] = make_float4(xh, yh, zh, 0.f);
  lo[g] = make_float4((float)(x - xh), (float)(y - yh), (float)(z - zh), 0.f);
}

// ------------------------------------------------------------------ stage 1

// Tile: 128 nu (M) x 64 g (N) per CTA, 32 inner points g' per stage; the B
// tiles of one limb for the four channels are stored back to back (limb-major)
// and consumed by one N = 256 MMA per limb product.  Tensor
// memory holds one FP32 chunk accumulator (4 channels x 64 columns) that the
// MMAs fill over kchunk inner points, and an FP32 running sum of the same
// shape into which the epilogue warps fold each chunk with IEEE-rounded adds.
// Short tensor-core accumulation runs keep the accumulation error small;
// the tile is written to FP64 calG once, after its last chunk.
//
// BH selects the multi-centre generator, which needs shared memory for a
// per-row nucleus table (sized at launch) and so keeps one operand stage less.
template <int LIMBS, bool BH>
struct S1C {
  static constexpr int BM = 128, BN = 64, BK = 32;
  static constexpr int STAGES = BH ? (LIMBS == 2 ? 3 : 2) : (LIMBS == 2 ? 4 : 3);
  static constexpr int CSTAGES = 8;  // coordinate ring
  static constexpr uint32_t A_LIMB = BM * BK * 2;
  static constexpr uint32_t B_TILE = BN * BK * 2;
  static constexpr uint32_t A_BYTES = LIMBS * A_LIMB;
  static constexpr uint32_t B_BYTES = 4 * LIMBS * B_TILE;
  static constexpr uint32_t C_BASE = BK * 32;  // inner-point coordinates, FP32 hi then lo
  static constexpr uint32_t STAGE = A_BYTES + B_BYTES;
  static constexpr uint32_t ACC_COLS = 4 * BN;
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
  static constexpr int NGW = 8;  // generator warps: 2 .. 9
  static constexpr int NEW = 4;  // epilogue warps: 10 .. 13
  static constexpr int CW = 2 + NGW + NEW;  // coordinate producer warp
  static constexpr int THREADS = 32 * (CW + 1);
  static constexpr int COLS = BN * BK / (32 * NGW);  // inner points per generator thread
  // operand stages + alignment slack + barriers; the coordinate ring and the
  // nucleus table are added at launch
  static constexpr uint32_t FIXED = STAGES * STAGE + 1024 + 512;
  static_assert(COLS == 8, "one 16-byte chunk per generator thread and operand");
  static_assert(STAGE % 1024 == 0 && A_BYTES % 1024 == 0 && B_TILE % 1024 == 0, "alignment");
  static_assert(TMEM_COLS == 512, "tensor memory budget");
  static_assert(FIXED + CSTAGES * C_BASE <= 232448, "shared memory budget");
};

constexpr uint32_t kSmemLimit = 232448;

struct S1Params {
  const float4* xyz_hi;  // [n_k] points as FP32 hi/lo pairs (padded)
  const float4* xyz_lo;
  int64_t n_g;           // real points
  int64_t n_k;           // padded inner extent (multiple of 32)
  int n_mu;
  int n_mu_tiles;
  int64_t g_begin, g_end;
  int64_t n_g_tiles;
  int64_t kchunk;        // fold interval, multiple of 32
  float d;
  uint32_t cbytes;       // bytes per coordinate-ring stage
  uint32_t tab_bytes;    // bytes of the per-row nucleus table
  double* calG;          // [4][n_mu][g_end - g_begin]
  int* err;
  uint64_t wait_ns;      // bound of every mbarrier wait
  int64_t k_begin;       // first inner point of this launch (multiple of 32): the inner
                         // coordinates and A_{g'I} blocks are read from k_begin on, the
                         // (w xi) operand map covers the n_k inner points from there
  int accumulate;        // 1: add the tile into calG instead of writing it
  int debug;
  // multi-centre correlator (BH kernels only)
  int n_nuc;
  int oexp[2];           // E exponents o of the pair-term groups
  float rho[4];          // radial factor sum_e rho_e E^e of the E-gradient
  const float4* rowslots;  // [n_k][n_nuc][ns4] per (point, nucleus) slots
  const float4* fvec;      // [n_k] gradient part independent of the inner point
  const float* ajtab;      // [n_k / 32][n_nuc][32] A_{g'I}
};

__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc::smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(src)), "r"(bytes), "r"(tc::smem_u32(bar))
      : "memory");
}

// Limbs of two values packed as bf16x2 words; each limb is the
// round-to-nearest bf16 of the remainder left by the previous ones.
template <int LIMBS>
__device__ __forceinline__ void split_pack(float a, float b, uint32_t (&out)[LIMBS]) {
#pragma unroll
  for (int l = 0; l < LIMBS; ++l) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    uint32_t w = *reinterpret_cast<uint32_t*>(&h);
    out[l] = w;
    if (l + 1 < LIMBS) {
      a -= __uint_as_float(w << 16);
      b -= __uint_as_float(w & 0xffff0000u);
    }
  }
}

// Difference vector r_g - r_g' from FP32 hi/lo pairs: the hi parts of close
// points cancel exactly, so every pair keeps relative accuracy ~1e-7 whatever
// the order of the grid points.
__device__ __forceinline__ void pair_diff(const float4& gh, const float4& gl, const float4& h,
                                          const float4& l, float& dx, float& dy, float& dz) {
  dx = (gh.x - h.x) + (gl.x - l.x);
  dy = (gh.y - h.y) + (gl.y - l.y);
  dz = (gh.z - h.z) + (gl.z - l.z);
}

// Radial correlator u = r / (2 (1 + d r)):  K_c = f (r_g - r_g')_c with
// f = u'(r)/r, u' = 1/(2 (1 + d r)^2), and K_sq = |K|^2 = f (f r^2).  The self
// pair is the one pair whose hi/lo difference is exactly zero (distinct grid
// points never coincide), and these forms give it zero without an index test:
// r^2 is clamped only inside the square root, so f stays finite.
__device__ __forceinline__ void radial_pair(float dx, float dy, float dz, float d, float& kx,
                                            float& ky, float& kz, float& ksq) {
  const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
  const float rinv = rsqrtf(fmaxf(r2, 1e-30f));
  const float r = r2 * rinv;
  const float iden = rcp_approx(fmaf(d, r, 1.0f));
  const float f = 0.5f * iden * iden * rinv;
  kx = f * dx;
  ky = f * dy;
  kz = f * dz;
  ksq = f * (f * r2);
}

// Shared-memory carve-up and barriers common to the stage-1 roles.
struct S1Smem {
  uint8_t* stages;
  uint8_t* ring;
  uint8_t* tab;
  uint64_t* full;
  uint64_t* empty;
  uint64_t* cfull;
  uint64_t* cempty;
  uint64_t* acc_full;
  uint64_t* acc_empty;
  volatile int* abort_flag;
};

// (w xi) limbs by TMA, one 128 x 32 box per limb and stage.
template <class C, int LIMBS>
__device__ __forceinline__ void s1_load_a(const CUtensorMap* mA0, const CUtensorMap* mA1,
                                          const CUtensorMap* mA2, const S1Params& p,
                                          const S1Smem& sm, int64_t n_tiles) {
  tc::tma_prefetch_desc(mA0);
  if (LIMBS > 1) tc::tma_prefetch_desc(mA1);
  if (LIMBS > 2) tc::tma_prefetch_desc(mA2);
  uint32_t it = 0;
  bool skip = (p.debug & 1) != 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int mu0 = (int)(tile / p.n_g_tiles) * C::BM;
    for (int64_t k0 = 0; k0 < p.n_k; k0 += C::BK, ++it) {
      const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
      if (!tc::mbar_wait(&sm.empty[s], ph ^ 1, sm.abort_flag, p.err, p.wait_ns)) return;
      if (skip) {  // fault-path test: this stage's operand never arrives
        skip = false;
        continue;
      }
      uint8_t* st = sm.stages + s * C::STAGE;
      tc::mbar_arrive_expect_tx(&sm.full[s], C::A_BYTES);
      tc::tma_load_2d(st, mA0, &sm.full[s], (int32_t)k0, mu0);
      if (LIMBS > 1) tc::tma_load_2d(st + C::A_LIMB, mA1, &sm.full[s], (int32_t)k0, mu0);
      if (LIMBS > 2) tc::tma_load_2d(st + 2 * C::A_LIMB, mA2, &sm.full[s], (int32_t)k0, mu0);
    }
  }
}

// Inner-point data by bulk copy, running ahead of the generators: FP32 hi and
// lo coordinates, plus A_{g'I} for the multi-centre generator.
template <class C, bool BH>
__device__ __forceinline__ void s1_load_coords(const S1Params& p, const S1Smem& sm,
                                               int64_t n_tiles) {
  uint32_t cit = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    for (int64_t k0 = 0; k0 < p.n_k; k0 += C::BK, ++cit) {
      const uint32_t cs = cit % C::CSTAGES, ph = (cit / C::CSTAGES) & 1;
      if (!tc::mbar_wait(&sm.cempty[cs], ph ^ 1, sm.abort_flag, p.err, p.wait_ns)) return;
      uint8_t* dst = sm.ring + cs * p.cbytes;
      tc::mbar_arrive_expect_tx(&sm.cfull[cs], p.cbytes);
      bulk_copy_g2s(dst, p.xyz_hi + p.k_begin + k0, C::BK * 16, &sm.cfull[cs]);
      bulk_copy_g2s(dst + C::BK * 16, p.xyz_lo + p.k_begin + k0, C::BK * 16, &sm.cfull[cs]);
      if (BH && p.n_nuc > 0)
        bulk_copy_g2s(dst + C::C_BASE, p.ajtab + ((p.k_begin + k0) / C::BK) * p.n_nuc * C::BK,
                      (uint32_t)p.n_nuc * C::BK * 4, &sm.cfull[cs]);
    }
  }
}

// MMA issuer (one thread): one N = 256 MMA per limb product and k-step covers
// the four channels, since the limb-j tiles of channels 0..3 are contiguous.
template <class C, int LIMBS>
__device__ __forceinline__ void s1_issue_mma(const S1Params& p, const S1Smem& sm, uint32_t tmem,
                                             int64_t n_tiles, int64_t n_chunks) {
  constexpr uint32_t idesc = tc::idesc_f16(128, 4 * C::BN, 1);
  uint32_t it = 0, u = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    for (int64_t ch = 0; ch < n_chunks; ++ch, ++u) {
      const int64_t kb = ch * p.kchunk;
      const int64_t ke = kb + p.kchunk < p.n_k ? kb + p.kchunk : p.n_k;
      if (!tc::mbar_wait(sm.acc_empty, (u & 1) ^ 1, sm.abort_flag, p.err, p.wait_ns)) return;
      tc::tc_fence_after();
      for (int64_t k0 = kb; k0 < ke; k0 += C::BK, ++it) {
        const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
        if (!tc::mbar_wait(&sm.full[s], ph, sm.abort_flag, p.err, p.wait_ns)) return;
        tc::tc_fence_after();
        const uint32_t a_base = tc::smem_u32(sm.stages + s * C::STAGE);
        const uint32_t b_base = a_base + C::A_BYTES;
        const bool first = (k0 == kb);
#pragma unroll
        for (int i = 0; i < LIMBS; ++i)
#pragma unroll
          for (int j = 0; j < LIMBS - i; ++j)
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
              const uint64_t ad = tc::smem_desc(a_base + i * C::A_LIMB + kk * 32, 16, 512, 4);
              const uint64_t bd = tc::smem_desc(b_base + j * 4 * C::B_TILE + kk * 32, 16, 512, 4);
              const uint32_t acc = (first && i == 0 && j == 0 && kk == 0) ? 0u : 1u;
              tc::umma_f16(tmem, ad, bd, idesc, acc);
            }
        tc::umma_commit(&sm.empty[s]);
      }
      tc::umma_commit(sm.acc_full);
    }
  }
}

// Store one thread's 8 generated pairs (4 channels, LIMBS limbs) into the
// 64B-swizzled K-major B tiles of stage s and signal the MMA issuer.
template <class C, int LIMBS>
__device__ __forceinline__ void s1_store_b(const S1Smem& sm, uint32_t s, int row, int kc,
                                           const uint32_t (&pk)[4][LIMBS][4]) {
  const uint32_t bsm =
      tc::smem_u32(sm.stages + s * C::STAGE + C::A_BYTES) + tc::sw64_offset(row, kc >> 3);
#pragma unroll
  for (int c = 0; c < 4; ++c)
#pragma unroll
    for (int l = 0; l < LIMBS; ++l)
      tc::sts_u4(bsm + (l * 4 + c) * C::B_TILE, pk[c][l][0], pk[c][l][1], pk[c][l][2],
                 pk[c][l][3]);
  tc::fence_proxy_async_smem();
  tc::mbar_arrive(&sm.full[s]);
}

// Radial generator: K_c(g, g') for a 64 x 32 block, split into BF16 limbs.
// Thread gt owns row gt % 64 and inner points 8 (gt / 64) .. + 7.
template <class C, int LIMBS>
__device__ __forceinline__ void s1_gen_radial(const S1Params& p, const S1Smem& sm, int gt,
                                              int64_t n_tiles) {
  const int row = gt % C::BN;
  const int kc = (gt / C::BN) * C::COLS;
  const int64_t n_gs = p.g_end - p.g_begin;
  const float d = p.d;
  uint32_t it = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t g_tile = tile % p.n_g_tiles;
    const int64_t gl = g_tile * C::BN + row;
    const bool gvalid = gl < n_gs;
    const int64_t g = p.g_begin + (gvalid ? gl : 0);
    const float4 gh = gvalid ? p.xyz_hi[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 glo = gvalid ? p.xyz_lo[g] : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t k0 = 0; k0 < p.n_k; k0 += C::BK, ++it) {
      const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
      const uint32_t cs = it % C::CSTAGES, cph = (it / C::CSTAGES) & 1;
      if (!tc::mbar_wait(&sm.cfull[cs], cph, sm.abort_flag, p.err, p.wait_ns)) return;
      const uint32_t cbase = tc::smem_u32(sm.ring + cs * p.cbytes);
      float dx[8], dy[8], dz[8];
#pragma unroll
      for (int e = 0; e < 8; ++e)
        pair_diff(gh, glo, tc::lds_f4(cbase + (kc + e) * 16),
                  tc::lds_f4(cbase + (C::BK + kc + e) * 16), dx[e], dy[e], dz[e]);
      tc::mbar_arrive(&sm.cempty[cs]);  // this thread's reads precede the next bulk copy
      uint32_t pk[4][LIMBS][4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        float kv[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h)
          radial_pair(dx[e + h], dy[e + h], dz[e + h], d, kv[h][0], kv[h][1], kv[h][2],
                      kv[h][3]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t w[LIMBS];
          split_pack<LIMBS>(kv[0][c], kv[1][c], w);
#pragma unroll
          for (int l = 0; l < LIMBS; ++l) pk[c][l][e >> 1] = w[l];
        }
      }
      if (!tc::mbar_wait(&sm.empty[s], ph ^ 1, sm.abort_flag, p.err, p.wait_ns)) return;
      s1_store_b<C, LIMBS>(sm, s, row, kc, pk);
    }
  }
}

// Multi-centre (Boys-Handy) generator.  With A = A_{gI}, y = A_{g'I} and the
// terms grouped by their E exponent (group 0: o = 0; groups j = 1..NG: o_j),
//   grad_g u = f(g) + sum_I [sum_d P0_d y^d + sum_j E^{o_j} P_j(y)] grad A_{gI}
//              + [rho(E) + sum_j o_j E^{o_j - 1} sum_I Q_j(y)] dE/dr e_{gg'}
// where the polynomial coefficients P_j,d and Q_j,d are functions of A_{gI}
// and the nucleus type, tabulated per (row point, nucleus) in FP64 and held in
// shared memory as [I][slot / 4][row] float4 for the tile's 64 rows:
//   slots 0..2 grad A_{gI}; 3 .. 2 + DEG  P0_1 .. P0_DEG;
//   then per group j: P_j,0 .. P_j,DEG, Q_j,0 .. Q_j,DEG.
// f(g) collects the y-independent part P0_0 grad A_{gI}; rho(E) the cusp and
// the pure electron-electron terms.  Lane l of generator warp w owns row
// 8 w + l / 4 and inner points 8 (l % 4) .. + 7, so the four lanes sharing a
// row fill its table entries together (warp-level synchronisation only); all
// exits are warp-uniform.
template <class C, int LIMBS, int NG, int DEG>
__device__ __forceinline__ void s1_gen_bh(const S1Params& p, const S1Smem& sm, int gw, int lane,
                                          int64_t n_tiles) {
  constexpr int NS = 3 + DEG + 2 * NG * (DEG + 1);
  constexpr int NS4 = (NS + 3) / 4;
  const int row = gw * 8 + (lane >> 2);
  const int kc = (lane & 3) * C::COLS;
  const int64_t n_gs = p.g_end - p.g_begin;
  const float d = p.d;
  const int n_nuc = p.n_nuc;
  const uint32_t tab = tc::smem_u32(sm.tab);
  float4* tabp = reinterpret_cast<float4*>(sm.tab);
  uint32_t it = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t g_tile = tile % p.n_g_tiles;
    const int64_t gl = g_tile * C::BN + row;
    const bool gvalid = gl < n_gs;
    const int64_t g = p.g_begin + (gvalid ? gl : 0);
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 gh = gvalid ? p.xyz_hi[g] : zero;
    const float4 glo = gvalid ? p.xyz_lo[g] : zero;
    const float4 fg = gvalid ? p.fvec[g] : zero;
    const int64_t gself = gvalid ? g - p.k_begin : -1;  // in this launch's inner range
    // this warp's rows of the nucleus table (the previous tile's reads are done)
    __syncwarp();
    for (int idx = lane & 3; idx < n_nuc * NS4; idx += 4)
      tabp[idx * C::BN + row] = gvalid ? p.rowslots[g * n_nuc * NS4 + idx] : zero;
    __syncwarp();
    for (int64_t k0 = 0; k0 < p.n_k; k0 += C::BK, ++it) {
      const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
      const uint32_t cs = it % C::CSTAGES, cph = (it / C::CSTAGES) & 1;
      const bool okc = tc::mbar_wait(&sm.cfull[cs], cph, sm.abort_flag, p.err, p.wait_ns);
      if (!__all_sync(0xffffffffu, okc)) return;
      const uint32_t cbase = tc::smem_u32(sm.ring + cs * p.cbytes);
      float dx[8], dy[8], dz[8], fr[8], ce[8], gx[8], gy[8], gz[8];
      float eo[NG][8], wq[NG][8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        pair_diff(gh, glo, tc::lds_f4(cbase + (kc + e) * 16),
                  tc::lds_f4(cbase + (C::BK + kc + e) * 16), dx[e], dy[e], dz[e]);
        const float r2 = fmaxf(fmaf(dx[e], dx[e], fmaf(dy[e], dy[e], dz[e] * dz[e])), 1e-30f);
        const float rinv = rsqrtf(r2);
        const float r = r2 * rinv;
        const float iden = rcp_approx(fmaf(d, r, 1.0f));
        const float E = d * r * iden;
        fr[e] = d * iden * iden * rinv;
        ce[e] = fmaf(E, fmaf(E, fmaf(E, p.rho[3], p.rho[2]), p.rho[1]), p.rho[0]);
#pragma unroll
        for (int j = 0; j < NG; ++j) {
          float pw = 1.0f;
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (t < p.oexp[j] - 1) pw *= E;
          wq[j][e] = (float)p.oexp[j] * pw;
          eo[j][e] = pw * E;
        }
        gx[e] = fg.x;
        gy[e] = fg.y;
        gz[e] = fg.z;
      }
      const uint32_t abase = cbase + C::C_BASE + kc * 4;
#pragma unroll 1
      for (int I = 0; I < n_nuc; ++I) {
        float sl[NS4 * 4];
#pragma unroll
        for (int k4 = 0; k4 < NS4; ++k4) {
          const float4 v = tc::lds_f4(tab + ((I * NS4 + k4) * C::BN + row) * 16);
          sl[4 * k4] = v.x;
          sl[4 * k4 + 1] = v.y;
          sl[4 * k4 + 2] = v.z;
          sl[4 * k4 + 3] = v.w;
        }
        const float4 y0 = tc::lds_f4(abase + I * C::BK * 4);
        const float4 y1 = tc::lds_f4(abase + I * C::BK * 4 + 16);
        const float y[8] = {y0.x, y0.y, y0.z, y0.w, y1.x, y1.y, y1.z, y1.w};
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          float s0 = sl[2 + DEG];
#pragma unroll
          for (int dd = DEG - 1; dd >= 1; --dd) s0 = fmaf(s0, y[e], sl[2 + dd]);
          float ca = s0 * y[e];
#pragma unroll
          for (int j = 0; j < NG; ++j) {
            const int pb = 3 + DEG + j * 2 * (DEG + 1);
            const int qb = pb + DEG + 1;
            float pj = sl[pb + DEG], qj = sl[qb + DEG];
#pragma unroll
            for (int dd = DEG - 1; dd >= 0; --dd) {
              pj = fmaf(pj, y[e], sl[pb + dd]);
              qj = fmaf(qj, y[e], sl[qb + dd]);
            }
            ca = fmaf(eo[j][e], pj, ca);
            ce[e] = fmaf(wq[j][e], qj, ce[e]);
          }
          gx[e] = fmaf(ca, sl[0], gx[e]);
          gy[e] = fmaf(ca, sl[1], gy[e]);
          gz[e] = fmaf(ca, sl[2], gz[e]);
        }
      }
      tc::mbar_arrive(&sm.cempty[cs]);  // ring reads of this stage are done
      const bool may_self = gself >= k0 && gself < k0 + C::BK;
      uint32_t pk[4][LIMBS][4];
#pragma unroll
      for (int e = 0; e < 8; e += 2) {
        float kv[2][4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int q = e + h;
          const bool self = may_self && (k0 + kc + q) == gself;
          const float fac = ce[q] * fr[q];
          const float kx = fmaf(fac, dx[q], gx[q]);
          const float ky = fmaf(fac, dy[q], gy[q]);
          const float kz = fmaf(fac, dz[q], gz[q]);
          kv[h][0] = self ? 0.f : kx;
          kv[h][1] = self ? 0.f : ky;
          kv[h][2] = self ? 0.f : kz;
          kv[h][3] = self ? 0.f : fmaf(kx, kx, fmaf(ky, ky, kz * kz));
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          uint32_t w[LIMBS];
          split_pack<LIMBS>(kv[0][c], kv[1][c], w);
#pragma unroll
          for (int l = 0; l < LIMBS; ++l) pk[c][l][e >> 1] = w[l];
        }
      }
      const bool oke = tc::mbar_wait(&sm.empty[s], ph ^ 1, sm.abort_flag, p.err, p.wait_ns);
      if (!__all_sync(0xffffffffu, oke)) return;
      s1_store_b<C, LIMBS>(sm, s, row, kc, pk);
    }
  }
}

// Epilogue: fold each chunk into the running sum; write the tile at the end.
template <class C>
__device__ __forceinline__ void s1_epilogue(const S1Params& p, const S1Smem& sm, uint32_t tmem,
                                            int warp, int lane, int64_t n_tiles,
                                            int64_t n_chunks) {
  const int quad = warp & 3;
  const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
  const int64_t n_gs = p.g_end - p.g_begin;
  uint32_t u = 0;
  for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const int64_t g_tile = tile % p.n_g_tiles;
    const int mu = (int)(tile / p.n_g_tiles) * C::BM + 32 * quad + lane;
    for (int64_t ch = 0; ch < n_chunks; ++ch, ++u) {
      // tcgen05.ld/st/wait are warp-collective (.sync.aligned): every lane
      // leaves the spin-wait and the divergent stores before reaching them
      const bool ok = tc::mbar_wait(sm.acc_full, u & 1, sm.abort_flag, p.err, p.wait_ns);
      if (!__all_sync(0xffffffffu, ok)) return;
      tc::tc_fence_after();
      const bool first = (ch == 0), last = (ch + 1 == n_chunks);
#pragma unroll 1
      for (int blk = 0; blk < (int)C::ACC_COLS / 32; ++blk) {
        uint32_t r[32];
        __syncwarp();
        tc::tmem_fold_block(tmem + lane_base + blk * 32, tmem + lane_base + C::ACC_COLS + blk * 32,
                            first, r);
        if (!last) {
          tc::tmem_st_32x32b_x32(tmem + lane_base + C::ACC_COLS + blk * 32, r);
        } else if (mu < p.n_mu) {
          const int c = blk / (C::BN / 32);
          double* dst = p.calG + ((int64_t)c * p.n_mu + mu) * n_gs;
          const int64_t gbase = g_tile * C::BN + (blk % (C::BN / 32)) * 32;
#pragma unroll
          for (int j = 0; j < 32; ++j)
            if (gbase + j < n_gs) {
              const double v = (double)__uint_as_float(r[j]);
              dst[gbase + j] = p.accumulate ? dst[gbase + j] + v : v;
            }
        }
      }
      __syncwarp();
      if (!last) tc::tmem_st_wait();
      tc::tc_fence_before();
      tc::mbar_arrive(sm.acc_empty);
    }
  }
}

// Stage-1 kernel.  NG < 0: radial correlator; NG >= 1: multi-centre
// correlator with NG pair-term groups and polynomial degree DEG in A_{g'I}.
template <int LIMBS, int NG, int DEG>
__global__ void __launch_bounds__(S1C<LIMBS, (NG >= 0)>::THREADS, 1)
    s1_tc_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                 const __grid_constant__ CUtensorMap mA2, const __grid_constant__ S1Params p) {
  constexpr bool BH = NG >= 0;
  using C = S1C<LIMBS, BH>;
  extern __shared__ uint8_t smem_raw[];
  S1Smem sm;
  sm.stages = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  sm.ring = sm.stages + C::STAGES * C::STAGE;
  sm.tab = sm.ring + C::CSTAGES * p.cbytes;
  sm.full = (uint64_t*)(sm.tab + p.tab_bytes);
  sm.empty = sm.full + C::STAGES;
  sm.cfull = sm.empty + C::STAGES;
  sm.cempty = sm.cfull + C::CSTAGES;
  sm.acc_full = sm.cempty + C::CSTAGES;
  sm.acc_empty = sm.acc_full + 1;
  uint32_t* tmem_slot = (uint32_t*)(sm.acc_empty + 1);
  sm.abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      // every generator thread arrives: its own shared-memory writes must be
      // ordered before the tensor core reads them (a warp-level sync followed
      // by one lane's arrive does not give that ordering)
      tc::mbar_init(&sm.full[s], C::NGW * 32 + 1);
      tc::mbar_init(&sm.empty[s], 1);
    }
    for (int s = 0; s < C::CSTAGES; ++s) {
      tc::mbar_init(&sm.cfull[s], 1);
      tc::mbar_init(&sm.cempty[s], C::NGW * 32);
    }
    tc::mbar_init(sm.acc_full, 1);
    tc::mbar_init(sm.acc_empty, C::NEW * 32);
    *sm.abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, C::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t n_tiles = (int64_t)p.n_mu_tiles * p.n_g_tiles;
  const int64_t n_chunks = (p.n_k + p.kchunk - 1) / p.kchunk;

  if (warp == 0) {
    if (lane == 0) s1_load_a<C, LIMBS>(&mA0, &mA1, &mA2, p, sm, n_tiles);
  } else if (warp == C::CW) {
    if (lane == 0) s1_load_coords<C, BH>(p, sm, n_tiles);
  } else if (warp == 1) {
    if (lane == 0) s1_issue_mma<C, LIMBS>(p, sm, tmem, n_tiles, n_chunks);
  } else if (warp < 2 + C::NGW) {
    if constexpr (BH)
      s1_gen_bh<C, LIMBS, (BH ? NG : 1), (BH ? DEG : 2)>(p, sm, warp - 2, lane, n_tiles);
    else
      s1_gen_radial<C, LIMBS>(p, sm, threadIdx.x - 64, n_tiles);
  } else {
    s1_epilogue<C>(p, sm, tmem, warp, lane, n_tiles, n_chunks);
  }
  __syncthreads();
  if (*sm.abort_flag) {
    // a bounded wait expired: give issued copies and MMAs time to land
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 200000ull) {
    }
  }
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, C::TMEM_COLS);
  }
}

// ------------------------------------------------------------------ stage 1 on CTA pairs
//
// Stage 1 of the radial correlator on a pair of CTAs (a cluster of two) that
// share one 256 (nu) x 64 (g) tile: each CTA holds 128 rows of the (w xi)
// operand and of the accumulator, and generates the B values of 32 of the 64
// outer points; one thread of the even CTA issues M = 256, N = 256
// tcgen05.mma.cta_group::2 instructions that read B from both CTAs.  Each
// generated pair therefore feeds 256 rows instead of 128, and each SM reads
// only its own half of B from shared memory.  B rows (the MMA's N) are laid
// out channel-major per CTA: [ch0 g0-31 | ch1 | ch2 | ch3] in the even CTA and
// the same for g32-63 in the odd CTA, so accumulator column j holds channel
// (j % 128) / 32 of outer point 32 (j / 128) + j % 32.
//
// Signals: the odd CTA's (w xi) copies complete on the even CTA's stage
// barrier (cta_group::2 bulk tensor copy); its generator warps arrive there
// remotely (one arrival per warp); the commits of the pair MMAs arrive on the
// stage-free and chunk-ready barriers of both CTAs (multicast); the odd CTA's
// epilogue warps arrive on the even CTA's chunk-free barrier.  Every wait is
// bounded as in the single-CTA kernel.
// TF32: operands are TF32 limbs in 32-bit words (128-byte rows of the 32
// inner points, 128-byte swizzle, kind::tf32 MMAs of K = 8); otherwise BF16
// limbs (64-byte rows, 64-byte swizzle, kind::f16 MMAs of K = 16).  Both
// advance 32 bytes of K per MMA.
template <int LIMBS, int NGRP = 1, bool TF32 = false, bool BH = false>
struct S1P {
  static constexpr int BM = 128, BN = 64, BNH = 32, BK = 32;
  static constexpr int EB = TF32 ? 4 : 2;               // operand bytes
  static constexpr uint32_t ROWB = BK * EB;             // bytes of one operand row
  static constexpr int KSUB = ROWB / 32;                // MMAs per limb product and k-step
  static constexpr uint32_t SBO = 8 * ROWB;             // 8-row core-matrix stride
  static constexpr uint32_t SWZ = TF32 ? 2 : 4;         // descriptor layout: 128B / 64B swizzle
  // the multi-centre generator's per-row nucleus table and A_{g'I} ring take
  // shared memory from the stages
  static constexpr int STAGES = TF32 ? 3 : (LIMBS == 2 ? (BH ? 5 : 6) : (BH ? 3 : 4));
  static constexpr int CSTAGES = 8;
  static constexpr uint32_t A_LIMB = BM * ROWB;         // 8 KB (BF16), 16 KB (TF32)
  static constexpr uint32_t B_LIMB = 4 * BNH * ROWB;    // 128 rows
  static constexpr uint32_t A_BYTES = LIMBS * A_LIMB;
  static constexpr uint32_t STAGE = LIMBS * (A_LIMB + B_LIMB);
  static constexpr uint32_t C_BYTES = BK * 32;          // FP32 hi then lo, per ring slot
  static constexpr uint32_t ACC_COLS = 4 * BN;
  static constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;
  static constexpr int GW = 8;              // warps of one generator group
  static constexpr int NGW = GW * NGRP;     // generator warps 2 .. 1 + NGW; group k takes
                                            // the k-steps it with it % NGRP == k
  // epilogue warps: with one generator group, two per tensor-memory lane
  // quarter (each folds half of the accumulator columns, halving the fold's
  // load latency while the MMAs wait for the chunk accumulator)
  static constexpr int NEW = NGRP == 1 ? 8 : 4;
  static constexpr int EPH = NEW / 4;       // column parts of one lane quarter
  static constexpr int CW = 2 + NGW + NEW;  // coordinate producer warp
  static constexpr int THREADS = 32 * (CW + 1);
  static constexpr int PTS = BNH * BK / (32 * GW);    // inner points per generator thread
  static constexpr int FOLD = NGRP >= 2 ? 16 : 32;    // epilogue fold width (registers)
  static constexpr uint32_t SMEM = STAGES * STAGE + CSTAGES * C_BYTES + 1024 + 512;
  static_assert(PTS == 4, "one 4-point chunk per generator thread, channel and limb");
  static_assert(STAGE % 1024 == 0 && A_LIMB % 1024 == 0 && B_LIMB % 1024 == 0, "alignment");
  static_assert(SMEM <= 232448, "shared memory budget");
};

__device__ __forceinline__ void sts_u2(uint32_t saddr, uint32_t a, uint32_t b) {
  asm volatile("st.shared.v2.b32 [%0], {%1,%2};" ::"r"(saddr), "r"(a), "r"(b) : "memory");
}

// TF32 limbs of a value: l0 = TF32 rounding (to nearest, ties away) of v,
// l1 = TF32 rounding of the remainder v - l0 (exact in FP32), ...
__device__ __forceinline__ uint32_t tf32_rna(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return r;
}
template <int LIMBS>
__device__ __forceinline__ void split_tf32(float v, uint32_t (&out)[LIMBS]) {
#pragma unroll
  for (int l = 0; l < LIMBS; ++l) {
    const uint32_t h = tf32_rna(v);
    out[l] = h;
    if (l + 1 < LIMBS) v -= __uint_as_float(h);
  }
}

// Byte offset of the 16-byte chunk `chunk16` of row `row` in a K-major tile
// with 128-byte rows in the 128-byte-swizzle layout (chunk index XOR row % 8).
__device__ __forceinline__ uint32_t sw128_offset(uint32_t row, uint32_t chunk16) {
  return row * 128u + ((chunk16 ^ (row & 7u)) << 4);
}

// NG >= 0: the multi-centre generator (NG E-exponent groups, degree DEG in
// A_{g'I}) in place of the radial one; its coordinate ring also carries the
// A_{g'I} block (p.cbytes per slot) and a per-row nucleus table (p.tab_bytes)
// follows the ring.
template <int LIMBS, int NGRP, bool TF32, int NG = -1, int DEG = 0>
__global__ void __cluster_dims__(2, 1, 1)
    __launch_bounds__(S1P<LIMBS, NGRP, TF32, (NG >= 0)>::THREADS, 1)
    s1_pair_kernel(const __grid_constant__ CUtensorMap mA0, const __grid_constant__ CUtensorMap mA1,
                   const __grid_constant__ CUtensorMap mA2, const __grid_constant__ S1Params p) {
  constexpr bool BH = NG >= 0;
  using C = S1P<LIMBS, NGRP, TF32, BH>;
  static_assert(!BH || (NGRP == 1 && !TF32), "the multi-centre pair generator: one group, BF16");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* stages = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* ring = stages + C::STAGES * C::STAGE;
  const uint32_t cstride = BH ? p.cbytes : C::C_BYTES;  // bytes per ring slot
  uint8_t* tab = ring + C::CSTAGES * cstride;            // multi-centre row table
  uint64_t* full = (uint64_t*)(tab + (BH ? p.tab_bytes : 0u));
  uint64_t* empty = full + C::STAGES;
  uint64_t* cfull = empty + C::STAGES;
  uint64_t* cempty = cfull + C::CSTAGES;
  uint64_t* acc_full = cempty + C::CSTAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const uint32_t rank = tc::cluster_ctarank();
  const bool lead = rank == 0;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      // even CTA: its expect-tx arrival + one arrival per generator warp of the
      // group that fills this phase, in both CTAs
      tc::mbar_init(&full[s], lead ? 1 + 2 * C::GW : 1);
      tc::mbar_init(&empty[s], 1);
    }
    for (int s = 0; s < C::CSTAGES; ++s) {
      tc::mbar_init(&cfull[s], 1);
      tc::mbar_init(&cempty[s], C::GW);
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(acc_empty, lead ? 2 * C::NEW : 1);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc_pair(tmem_slot, C::TMEM_COLS);
    tc::tmem_relinquish_pair();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::cluster_sync();  // both CTAs' barriers exist before any remote arrival
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int64_t n_tiles = (int64_t)p.n_mu_tiles * p.n_g_tiles;  // n_mu_tiles counts 256-row pairs
  const int64_t n_chunks = (p.n_k + p.kchunk - 1) / p.kchunk;
  const int64_t pair0 = blockIdx.x >> 1, pstride = gridDim.x >> 1;
  const uint32_t full_lead = tc::mapa_shared(tc::smem_u32(full), 0);      // + 8 s
  const uint32_t acce_lead = tc::mapa_shared(tc::smem_u32(acc_empty), 0);

  if (warp == 0) {
    if (lane == 0) {
      // (w xi) limbs of this CTA's 128 rows, completing on the even CTA's stage barrier
      tc::tma_prefetch_desc(&mA0);
      if (LIMBS > 1) tc::tma_prefetch_desc(&mA1);
      if (LIMBS > 2) tc::tma_prefetch_desc(&mA2);
      uint32_t it = 0;
      bool skip = lead && (p.debug & 1) != 0;
      for (int64_t tile = pair0; tile < n_tiles; tile += pstride) {
        const int mu0 = (int)(tile / p.n_g_tiles) * 2 * C::BM + (int)rank * C::BM;
        for (int64_t k0 = 0; k0 < p.n_k; k0 += C::BK, ++it) {
          const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
          if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag, p.err, p.wait_ns)) goto done;
          if (skip) {  // fault-path test: this stage's operand never arrives
            skip = false;
            continue;
          }
          uint8_t* st = stages + s * C::STAGE;
          if (lead) {
            tc::mbar_arrive_expect_tx(&full[s], 2 * C::A_BYTES);
            tc::tma_load_2d(st, &mA0, &full[s], (int32_t)k0, mu0);
            if (LIMBS > 1) tc::tma_load_2d(st + C::A_LIMB, &mA1, &full[s], (int32_t)k0, mu0);
            if (LIMBS > 2) tc::tma_load_2d(st + 2 * C::A_LIMB, &mA2, &full[s], (int32_t)k0, mu0);
          } else {
            const uint32_t fb = full_lead + 8u * s;
            tc::tma_load_2d_pair(st, &mA0, fb, (int32_t)k0, mu0);
            if (LIMBS > 1) tc::tma_load_2d_pair(st + C::A_LIMB, &mA1, fb, (int32_t)k0, mu0);
            if (LIMBS > 2) tc::tma_load_2d_pair(st + 2 * C::A_LIMB, &mA2, fb, (int32_t)k0, mu0);
          }
        }
      }
    }
  } else if (warp == C::CW) {
    if (lane == 0) {
      uint32_t cit = 0;
      for (int64_t tile = pair0; tile < n_tiles; tile += pstride) {
        for (int64_t k0 = 0; k0 < p.n_k; k0 += C::BK, ++cit) {
          const uint32_t cs = cit % C::CSTAGES, ph = (cit / C::CSTAGES) & 1;
          if (!tc::mbar_wait(&cempty[cs], ph ^ 1, abort_flag, p.err, p.wait_ns)) goto done;
          uint8_t* dst = ring + cs * cstride;
          tc::mbar_arrive_expect_tx(&cfull[cs], cstride);
          bulk_copy_g2s(dst, p.xyz_hi + p.k_begin + k0, C::BK * 16, &cfull[cs]);
          bulk_copy_g2s(dst + C::BK * 16, p.xyz_lo + p.k_begin + k0, C::BK * 16, &cfull[cs]);
          if (BH && p.n_nuc > 0)
            bulk_copy_g2s(dst + C::C_BYTES, p.ajtab + ((p.k_begin + k0) / C::BK) * p.n_nuc * C::BK,
                          (uint32_t)p.n_nuc * C::BK * 4, &cfull[cs]);
        }
      }
    }
  } else if (warp == 1) {
    if (lead && lane == 0) {
      // A and B formats: BF16 (1) for kind::f16, TF32 (2) for kind::tf32
      constexpr uint32_t idesc = tc::idesc_f16(2 * C::BM, 4 * C::BN, TF32 ? 2 : 1);
      uint32_t it = 0, u = 0;
      for (int64_t tile = pair0; tile < n_tiles; tile += pstride) {
        for (int64_t ch = 0; ch < n_chunks; ++ch, ++u) {
          const int64_t kb = ch * p.kchunk;
          const int64_t ke = kb + p.kchunk < p.n_k ? kb + p.kchunk : p.n_k;
          if (!tc::mbar_wait(acc_empty, (u & 1) ^ 1, abort_flag, p.err, p.wait_ns)) goto done;
          tc::tc_fence_after();
          for (int64_t k0 = kb; k0 < ke; k0 += C::BK, ++it) {
            const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
            if (!tc::mbar_wait(&full[s], ph, abort_flag, p.err, p.wait_ns)) goto done;
            tc::tc_fence_after();
            const uint32_t a_base = tc::smem_u32(stages + s * C::STAGE);
            const uint32_t b_base = a_base + C::A_BYTES;
            const bool first = (k0 == kb);
#pragma unroll
            for (int i = 0; i < LIMBS; ++i)
#pragma unroll
              for (int j = 0; j < LIMBS - i; ++j)
#pragma unroll
                for (int kk = 0; kk < C::KSUB; ++kk) {
                  const uint64_t ad =
                      tc::smem_desc(a_base + i * C::A_LIMB + kk * 32, 16, C::SBO, C::SWZ);
                  const uint64_t bd =
                      tc::smem_desc(b_base + j * C::B_LIMB + kk * 32, 16, C::SBO, C::SWZ);
                  const uint32_t acc = (first && i == 0 && j == 0 && kk == 0) ? 0u : 1u;
                  if constexpr (TF32) tc::umma_tf32_pair(tmem, ad, bd, idesc, acc);
                  else tc::umma_f16_pair(tmem, ad, bd, idesc, acc);
                }
            tc::umma_commit_pair_multicast(&empty[s], 3);
          }
          tc::umma_commit_pair_multicast(acc_full, 3);
        }
      }
    }
  } else if (warp < 2 + C::NGW) {
   if constexpr (BH) {
    // multi-centre generator (the single-CTA kernel's arithmetic): lane l of
    // generator warp w owns outer point 4 w + l / 8 of this CTA's half and inner
    // points 4 (l % 8) .. + 3; the eight lanes of a row fill its table entries
    constexpr int NGc = NG >= 0 ? NG : 0;
    constexpr int NS = 3 + DEG + 2 * NGc * (DEG + 1);
    constexpr int NS4 = (NS + 3) / 4;
    const int wg = warp - 2;
    const int row = wg * 4 + (lane >> 3);
    const int kc = (lane & 7) * 4;
    const int64_t n_gs = p.g_end - p.g_begin;
    const float d = p.d;
    const int n_nuc = p.n_nuc;
    const uint32_t tabs = tc::smem_u32(tab);
    float4* tabp = reinterpret_cast<float4*>(tab);
    uint32_t it = 0;
    for (int64_t tile = pair0; tile < n_tiles; tile += pstride) {
      const int64_t g_tile = tile % p.n_g_tiles;
      const int64_t gl = g_tile * C::BN + (int64_t)rank * C::BNH + row;
      const bool gvalid = gl < n_gs;
      const int64_t g = p.g_begin + (gvalid ? gl : 0);
      const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 gh = gvalid ? p.xyz_hi[g] : zero;
      const float4 glo = gvalid ? p.xyz_lo[g] : zero;
      const float4 fg = gvalid ? p.fvec[g] : zero;
      const int64_t gself = gvalid ? g - p.k_begin : -1;  // in this launch's inner range
      // this warp's rows of the nucleus table (its previous reads are done)
      __syncwarp();
      for (int idx = lane & 7; idx < n_nuc * NS4; idx += 8)
        tabp[idx * C::BNH + row] = gvalid ? p.rowslots[g * n_nuc * NS4 + idx] : zero;
      __syncwarp();
      for (int64_t k0 = 0; k0 < p.n_k; k0 += C::BK, ++it) {
        const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
        const uint32_t cs = it % C::CSTAGES, cph = (it / C::CSTAGES) & 1;
        const bool okc = tc::mbar_wait(&cfull[cs], cph, abort_flag, p.err, p.wait_ns);
        if (!__all_sync(0xffffffffu, okc)) goto done;
        const uint32_t cbase = tc::smem_u32(ring + cs * cstride);
        float dx[4], dy[4], dz[4], fr[4], ce[4], gx[4], gy[4], gz[4];
        float eo[NGc > 0 ? NGc : 1][4], wq[NGc > 0 ? NGc : 1][4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          pair_diff(gh, glo, tc::lds_f4(cbase + (kc + e) * 16),
                    tc::lds_f4(cbase + (C::BK + kc + e) * 16), dx[e], dy[e], dz[e]);
          const float r2 = fmaxf(fmaf(dx[e], dx[e], fmaf(dy[e], dy[e], dz[e] * dz[e])), 1e-30f);
          const float rinv = rsqrtf(r2);
          const float r = r2 * rinv;
          const float iden = rcp_approx(fmaf(d, r, 1.0f));
          const float E = d * r * iden;
          fr[e] = d * iden * iden * rinv;
          ce[e] = fmaf(E, fmaf(E, fmaf(E, p.rho[3], p.rho[2]), p.rho[1]), p.rho[0]);
#pragma unroll
          for (int j = 0; j < NGc; ++j) {
            float pw = 1.0f;
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (t < p.oexp[j] - 1) pw *= E;
            wq[j][e] = (float)p.oexp[j] * pw;
            eo[j][e] = pw * E;
          }
          gx[e] = fg.x;
          gy[e] = fg.y;
          gz[e] = fg.z;
        }
        const uint32_t abase = cbase + C::C_BYTES + kc * 4;
#pragma unroll 1
        for (int I = 0; I < n_nuc; ++I) {
          float sl[NS4 * 4];
#pragma unroll
          for (int k4 = 0; k4 < NS4; ++k4) {
            const float4 v = tc::lds_f4(tabs + ((I * NS4 + k4) * C::BNH + row) * 16);
            sl[4 * k4] = v.x;
            sl[4 * k4 + 1] = v.y;
            sl[4 * k4 + 2] = v.z;
            sl[4 * k4 + 3] = v.w;
          }
          const float4 yv = tc::lds_f4(abase + I * C::BK * 4);
          const float y[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            float s0 = sl[2 + DEG];
#pragma unroll
            for (int dd = DEG - 1; dd >= 1; --dd) s0 = fmaf(s0, y[e], sl[2 + dd]);
            float ca = s0 * y[e];
#pragma unroll
            for (int j = 0; j < NGc; ++j) {
              const int pb = 3 + DEG + j * 2 * (DEG + 1);
              const int qb = pb + DEG + 1;
              float pj = sl[pb + DEG], qj = sl[qb + DEG];
#pragma unroll
              for (int dd = DEG - 1; dd >= 0; --dd) {
                pj = fmaf(pj, y[e], sl[pb + dd]);
                qj = fmaf(qj, y[e], sl[qb + dd]);
              }
              ca = fmaf(eo[j][e], pj, ca);
              ce[e] = fmaf(wq[j][e], qj, ce[e]);
            }
            gx[e] = fmaf(ca, sl[0], gx[e]);
            gy[e] = fmaf(ca, sl[1], gy[e]);
            gz[e] = fmaf(ca, sl[2], gz[e]);
          }
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&cempty[cs]);  // the warp's ring reads are done
        const bool may_self = gself >= k0 && gself < k0 + C::BK;
        uint32_t pk[4][LIMBS][2];
#pragma unroll
        for (int e = 0; e < 4; e += 2) {
          float kv[2][4];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int q = e + h;
            const bool self = may_self && (k0 + kc + q) == gself;
            const float fac = ce[q] * fr[q];
            const float kx = fmaf(fac, dx[q], gx[q]);
            const float ky = fmaf(fac, dy[q], gy[q]);
            const float kz = fmaf(fac, dz[q], gz[q]);
            kv[h][0] = self ? 0.f : kx;
            kv[h][1] = self ? 0.f : ky;
            kv[h][2] = self ? 0.f : kz;
            kv[h][3] = self ? 0.f : fmaf(kx, kx, fmaf(ky, ky, kz * kz));
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            uint32_t w[LIMBS];
            split_pack<LIMBS>(kv[0][c], kv[1][c], w);
#pragma unroll
            for (int l = 0; l < LIMBS; ++l) pk[c][l][e >> 1] = w[l];
          }
        }
        const bool oke = tc::mbar_wait(&empty[s], ph ^ 1, abort_flag, p.err, p.wait_ns);
        if (!__all_sync(0xffffffffu, oke)) goto done;
        const uint32_t bsm = tc::smem_u32(stages + s * C::STAGE + C::A_BYTES);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t off = tc::sw64_offset(c * C::BNH + row, kc >> 3) + (kc & 7) * 2;
#pragma unroll
          for (int l = 0; l < LIMBS; ++l) sts_u2(bsm + l * C::B_LIMB + off, pk[c][l][0], pk[c][l][1]);
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          if (lead) tc::mbar_arrive(&full[s]);
          else tc::mbar_arrive_cluster(full_lead + 8u * s);
        }
      }
    }
   } else {
    // generator: lane = outer point of this CTA's half, warp = 4 inner points
    const int grp = (warp - 2) / C::GW;
    const int row = lane;
    const int kc = ((warp - 2) % C::GW) * C::PTS;
    const int64_t n_gs = p.g_end - p.g_begin;
    const float d = p.d;
    uint32_t it = 0;
    for (int64_t tile = pair0; tile < n_tiles; tile += pstride) {
      const int64_t g_tile = tile % p.n_g_tiles;
      const int64_t gl = g_tile * C::BN + (int64_t)rank * C::BNH + row;
      const bool gvalid = gl < n_gs;
      const int64_t g = p.g_begin + (gvalid ? gl : 0);
      const float4 gh = gvalid ? p.xyz_hi[g] : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 glo = gvalid ? p.xyz_lo[g] : make_float4(0.f, 0.f, 0.f, 0.f);
      for (int64_t k0 = 0; k0 < p.n_k; k0 += C::BK, ++it) {
        if (NGRP > 1 && (int)(it % NGRP) != grp) continue;
        const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
        const uint32_t cs = it % C::CSTAGES, cph = (it / C::CSTAGES) & 1;
        const bool okc = tc::mbar_wait(&cfull[cs], cph, abort_flag, p.err, p.wait_ns);
        if (!__all_sync(0xffffffffu, okc)) goto done;
        const uint32_t cbase = tc::smem_u32(ring + cs * C::C_BYTES);
        float dx[C::PTS], dy[C::PTS], dz[C::PTS];
#pragma unroll
        for (int e = 0; e < C::PTS; ++e)
          pair_diff(gh, glo, tc::lds_f4(cbase + (kc + e) * 16),
                    tc::lds_f4(cbase + (C::BK + kc + e) * 16), dx[e], dy[e], dz[e]);
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&cempty[cs]);  // the warp's ring reads are done
        // limbs of the 4 points per channel: BF16 pairs in 2 words, TF32 in 4
        constexpr int NW = TF32 ? 4 : 2;
        uint32_t pk[4][LIMBS][NW];
#pragma unroll
        for (int e = 0; e < C::PTS; e += 2) {
          float kv[2][4];
#pragma unroll
          for (int h = 0; h < 2; ++h)
            radial_pair(dx[e + h], dy[e + h], dz[e + h], d, kv[h][0], kv[h][1], kv[h][2],
                        kv[h][3]);
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            if constexpr (TF32) {
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                uint32_t w[LIMBS];
                split_tf32<LIMBS>(kv[h][c], w);
#pragma unroll
                for (int l = 0; l < LIMBS; ++l) pk[c][l][(e + h) % NW] = w[l];
              }
            } else {
              uint32_t w[LIMBS];
              split_pack<LIMBS>(kv[0][c], kv[1][c], w);
#pragma unroll
              for (int l = 0; l < LIMBS; ++l) pk[c][l][(e >> 1) % NW] = w[l];
            }
          }
        }
        const bool oke = tc::mbar_wait(&empty[s], ph ^ 1, abort_flag, p.err, p.wait_ns);
        if (!__all_sync(0xffffffffu, oke)) goto done;
        const uint32_t bsm = tc::smem_u32(stages + s * C::STAGE + C::A_BYTES);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const uint32_t r = c * C::BNH + row;
          if constexpr (TF32) {
            const uint32_t off = sw128_offset(r, kc >> 2);  // 4 points = one 16-byte chunk
#pragma unroll
            for (int l = 0; l < LIMBS; ++l)
              tc::sts_u4(bsm + l * C::B_LIMB + off, pk[c][l][0], pk[c][l][1], pk[c][l][2],
                         pk[c][l][3]);
          } else {
            const uint32_t off = tc::sw64_offset(r, kc >> 3) + (kc & 7) * 2;
#pragma unroll
            for (int l = 0; l < LIMBS; ++l)
              sts_u2(bsm + l * C::B_LIMB + off, pk[c][l][0], pk[c][l][1]);
          }
        }
        tc::fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) {
          if (lead) tc::mbar_arrive(&full[s]);
          else tc::mbar_arrive_cluster(full_lead + 8u * s);
        }
      }
    }
   }
  } else {
    // epilogue: this CTA's 128 accumulator rows (lane quarter warp % 4, column
    // part (warp - first epilogue warp) / 4 of EPH)
    const int quad = warp & 3;
    const int part = (warp - 2 - C::NGW) >> 2;
    constexpr int NBLK = (int)C::ACC_COLS / C::FOLD / C::EPH;  // fold blocks per part
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    const int64_t n_gs = p.g_end - p.g_begin;
    uint32_t u = 0;
    for (int64_t tile = pair0; tile < n_tiles; tile += pstride) {
      const int64_t g_tile = tile % p.n_g_tiles;
      const int mu = (int)(tile / p.n_g_tiles) * 2 * C::BM + (int)rank * C::BM + 32 * quad + lane;
      for (int64_t ch = 0; ch < n_chunks; ++ch, ++u) {
        const bool ok = tc::mbar_wait(acc_full, u & 1, abort_flag, p.err, p.wait_ns);
        if (!__all_sync(0xffffffffu, ok)) goto done;
        tc::tc_fence_after();
        const bool first = (ch == 0), last = (ch + 1 == n_chunks);
        constexpr int FW = C::FOLD;
#pragma unroll 1
        for (int blk = part * NBLK; blk < (part + 1) * NBLK; ++blk) {
          uint32_t r[FW];
          __syncwarp();
          tc::tmem_fold_block_n<FW>(tmem + lane_base + blk * FW,
                                    tmem + lane_base + C::ACC_COLS + blk * FW, first, r);
          if (!last) {
            tc::tmem_st_n<FW>(tmem + lane_base + C::ACC_COLS + blk * FW, r);
          } else if (mu < p.n_mu) {
            // column j = blk FW + i: half j / 128 (outer points 32 (j / 128) ..),
            // channel (j % 128) / 32, point j % 32 of that half
            const int col = blk * FW;
            const int c = (col & 127) >> 5;
            double* dst = p.calG + ((int64_t)c * p.n_mu + mu) * n_gs;
            const int64_t gbase = g_tile * C::BN + (col >> 7) * C::BNH + (col & 31);
#pragma unroll
            for (int j = 0; j < FW; ++j)
              if (gbase + j < n_gs) {
                const double v = (double)__uint_as_float(r[j]);
                dst[gbase + j] = p.accumulate ? dst[gbase + j] + v : v;
              }
          }
        }
        __syncwarp();
        if (!last) tc::tmem_st_wait();
        tc::tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          if (lead) tc::mbar_arrive(acc_empty);
          else tc::mbar_arrive_cluster(acce_lead);
        }
      }
    }
  }
done:
  __syncthreads();
  if (*abort_flag) {
    // a bounded wait expired: give issued copies and MMAs time to land
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 200000ull) {
    }
  }
  tc::tc_fence_before();
  tc::cluster_sync();  // the pair's MMAs read both CTAs' shared memory and tensor memory
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc_pair(tmem, C::TMEM_COLS);
  }
}

// ------------------------------------------------------------------ generic split GEMM

// out[z][m][n] += scale * sum_k A_z[m][k] B_z[n][k] over the K range of this
// CTA, A_z and B_z in BF16 limbs.  One CTA per (n tile, m tile, K range, z).
// The tensor core accumulates fold_tiles x 32 points at a time; the epilogue
// folds each chunk into an FP32 running sum in tensor memory and finally
// adds the tile into the FP64 output with atomics.
constexpr int GB_MAXB = 4;

struct GemmMaps {
  CUtensorMap a[GB_MAXB][3];
  CUtensorMap b[GB_MAXB][3];
};

struct GemmParams {
  int64_t M, N;           // real output extents
  int64_t k_tiles;        // padded K / 32
  int64_t kchunk_tiles;   // k tiles per CTA
  int64_t fold_tiles;     // k tiles per tensor-core accumulation run
  int m_tiles, n_tiles, kchunks, batch;
  double* out;            // [batch][M][ldo] (or a single [M][ldo] when out_bs = 0)
  int64_t ldo, out_bs;
  double scale;
  int* err;
  uint64_t wait_ns;       // bound of every mbarrier wait
};

template <int LIMBS>
struct GC {
  static constexpr int BM = 128, BN = 128, BK = 32, STAGES = 4;
  static constexpr uint32_t TILE = 128 * BK * 2;
  static constexpr uint32_t STAGE = 2 * LIMBS * TILE;
  static constexpr int THREADS = 192;
  static constexpr uint32_t SMEM = STAGES * STAGE + 1024 + 256;
};

template <int LIMBS>
__global__ void __launch_bounds__(GC<LIMBS>::THREADS, 1)
    splitgemm_kernel(const __grid_constant__ GemmMaps maps, const GemmParams p) {
  using C = GC<LIMBS>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  int64_t unit = blockIdx.x;
  const int nt = (int)(unit % p.n_tiles); unit /= p.n_tiles;
  const int mt = (int)(unit % p.m_tiles); unit /= p.m_tiles;
  const int kc = (int)(unit % p.kchunks); unit /= p.kchunks;
  const int z = (int)unit;
  const int64_t kt0 = (int64_t)kc * p.kchunk_tiles;
  const int64_t kt1 = kt0 + p.kchunk_tiles < p.k_tiles ? kt0 + p.kchunk_tiles : p.k_tiles;
  const int64_t n_folds = (kt1 - kt0 + p.fold_tiles - 1) / p.fold_tiles;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(acc_empty, 4 * 32);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, 256);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int m0 = mt * C::BM, n0 = nt * C::BN;

  if (kt1 > kt0) {
    if (warp == 0) {
      if (lane == 0) {
        uint32_t it = 0;
        for (int64_t kt = kt0; kt < kt1; ++kt, ++it) {
          const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
          if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag, p.err, p.wait_ns)) break;
          tc::mbar_arrive_expect_tx(&full[s], C::STAGE);
          uint8_t* base = smem + s * C::STAGE;
          const int32_t x = (int32_t)(kt * C::BK);
#pragma unroll
          for (int l = 0; l < LIMBS; ++l) {
            tc::tma_load_2d(base + l * C::TILE, &maps.a[z][l], &full[s], x, m0);
            tc::tma_load_2d(base + (LIMBS + l) * C::TILE, &maps.b[z][l], &full[s], x, n0);
          }
        }
      }
    } else if (warp == 1) {
      if (lane == 0) {
        constexpr uint32_t idesc = tc::idesc_f16(128, 128, 1);
        uint32_t it = 0;
        for (int64_t f = 0; f < n_folds; ++f) {
          const int64_t fb = kt0 + f * p.fold_tiles;
          const int64_t fe = fb + p.fold_tiles < kt1 ? fb + p.fold_tiles : kt1;
          if (!tc::mbar_wait(acc_empty, (f & 1) ^ 1, abort_flag, p.err, p.wait_ns)) break;
          tc::tc_fence_after();
          bool ok = true;
          for (int64_t kt = fb; kt < fe; ++kt, ++it) {
            const uint32_t s = it % C::STAGES, ph = (it / C::STAGES) & 1;
            if (!tc::mbar_wait(&full[s], ph, abort_flag, p.err, p.wait_ns)) { ok = false; break; }
            tc::tc_fence_after();
            const uint32_t base = tc::smem_u32(smem + s * C::STAGE);
#pragma unroll
            for (int i = 0; i < LIMBS; ++i)
#pragma unroll
              for (int j = 0; j < LIMBS - i; ++j)
#pragma unroll
                for (int kk = 0; kk < 2; ++kk) {
                  const uint64_t ad = tc::smem_desc(base + i * C::TILE + kk * 32, 16, 512, 4);
                  const uint64_t bd = tc::smem_desc(base + (LIMBS + j) * C::TILE + kk * 32, 16, 512, 4);
                  const uint32_t acc = (kt == fb && i == 0 && j == 0 && kk == 0) ? 0u : 1u;
                  tc::umma_f16(tmem, ad, bd, idesc, acc);
                }
            tc::umma_commit(&empty[s]);
          }
          if (!ok) break;
          tc::umma_commit(acc_full);
        }
      }
    } else {
      // epilogue warps 2..5: lanes 32*(warp%4) .. +31
      const int quad = warp & 3;
      const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
      const int64_t m = m0 + 32 * quad + lane;
      double* dst = p.out + (int64_t)z * p.out_bs + m * p.ldo;
      for (int64_t f = 0; f < n_folds; ++f) {
        // warp-collective tcgen05.ld/st/wait: reconverge after the spin-wait
        // and after the divergent stores
        const bool ok = tc::mbar_wait(acc_full, f & 1, abort_flag, p.err, p.wait_ns);
        if (!__all_sync(0xffffffffu, ok)) break;
        tc::tc_fence_after();
        const bool first = (f == 0), last = (f + 1 == n_folds);
#pragma unroll 1
        for (int blk = 0; blk < 4; ++blk) {
          uint32_t r[32];
          __syncwarp();
          tc::tmem_fold_block(tmem + lane_base + blk * 32, tmem + lane_base + 128 + blk * 32, first, r);
          if (!last) {
            tc::tmem_st_32x32b_x32(tmem + lane_base + 128 + blk * 32, r);
          } else if (m < p.M) {
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              const int64_t n = n0 + blk * 32 + j;
              if (n < p.N) atomicAdd(dst + n, p.scale * (double)__uint_as_float(r[j]));
            }
          }
        }
        __syncwarp();
        if (!last) tc::tmem_st_wait();
        tc::tc_fence_before();
        tc::mbar_arrive(acc_empty);
      }
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 200000ull) {
    }
  }
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, 256);
  }
}

inline unsigned nb256(int64_t n) { return (unsigned)ceil_div(n, 256); }

// Inner points per stage-1 tensor-core accumulation run before each fold into
// the running sum (stage 2 folds every 256), and grid points per stage-2 CTA.
// The error of the tensor core's FP32 accumulation grows with the number of
// MMAs per run: 384 BF16 points (72 accumulating MMAs with three products)
// keep the H50-chain energies within 8.4e-7 Ha of the FP64 path (512: 9.9e-7);
// the TF32 form takes K = 8 per MMA, so 128 points give it a comparable count.
constexpr int64_t kDefaultChunk = 384;
constexpr int64_t kDefaultChunkTf32 = 128;
constexpr int64_t kS2Range = 8192;

}  // namespace

// ------------------------------------------------------------------ host drivers

// Split an FP64 row-major block into BF16 limbs [limbs][rows_pad][cols_pad].
int split_operand(const double* src, int64_t src_rs, int64_t c0, const double* colw, int64_t rows,
                  int64_t cols, int64_t rows_pad, int64_t cols_pad, int limbs, void* dst,
                  cudaStream_t s) {
  if (cols_pad % 4 == 0 && rows_pad < 65536) {
    const dim3 grd((unsigned)ceil_div(cols_pad, 1024), (unsigned)rows_pad);
    split_rows_kernel<<<grd, 256, 0, s>>>(src, src_rs, c0, colw, rows, cols, cols_pad,
                                          rows_pad * cols_pad, limbs, (__nv_bfloat16*)dst);
  } else {
    split_kernel<<<nb256(rows_pad * cols_pad), 256, 0, s>>>(src, src_rs, c0, colw, rows, cols,
                                                          rows_pad, cols_pad, limbs,
                                                          (__nv_bfloat16*)dst);
  }
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

// Split GEMM over `batch` pairs of limb operands (A_z [Mp][Kp], B_z [Np][Kp]),
// accumulating scale * A_z B_z^T into out (+ z * out_bs).  out must be
// initialised by the caller.
int splitgemm(int limbs, int batch, const void* const* A, const void* const* B, int64_t M,
              int64_t N, int64_t Kp, int64_t kchunk, int64_t fold, double* out, int64_t ldo,
              int64_t out_bs, double scale, int* err, cudaStream_t s) {
  ISDF_ARG(batch >= 1 && batch <= GB_MAXB, "splitgemm batch out of range");
  ISDF_ARG(limbs == 2 || limbs == 3, "limbs must be 2 or 3");
  ISDF_ARG(Kp % 32 == 0 && kchunk % 32 == 0 && kchunk > 0 && fold % 32 == 0 && fold > 0,
           "K padding");
  const int64_t Mp = round_up(M, 128), Np = round_up(N, 128);
  GemmMaps maps;
  memset(&maps, 0, sizeof(maps));
  for (int z = 0; z < batch; ++z)
    for (int l = 0; l < limbs; ++l) {
      ISDF_TRY(make_map(&maps.a[z][l], (const char*)A[z] + (size_t)l * Mp * Kp * 2, Mp, Kp, 128));
      ISDF_TRY(make_map(&maps.b[z][l], (const char*)B[z] + (size_t)l * Np * Kp * 2, Np, Kp, 128));
    }
  GemmParams p;
  p.M = M; p.N = N;
  p.k_tiles = Kp / 32;
  p.kchunk_tiles = kchunk / 32;
  p.fold_tiles = fold / 32;
  p.m_tiles = (int)(Mp / 128);
  p.n_tiles = (int)(Np / 128);
  p.kchunks = (int)ceil_div(p.k_tiles, p.kchunk_tiles);
  p.batch = batch;
  p.out = out; p.ldo = ldo; p.out_bs = out_bs; p.scale = scale; p.err = err;
  p.wait_ns = wait_limit_ns();
  int64_t units = (int64_t)p.m_tiles * p.n_tiles * p.kchunks * batch;
  ISDF_ARG(units < (1ll << 31), "too many GEMM work units");
  if (limbs == 2) {
    ISDF_CUDA(cudaFuncSetAttribute(splitgemm_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, GC<2>::SMEM));
    splitgemm_kernel<2><<<(unsigned)units, GC<2>::THREADS, GC<2>::SMEM, s>>>(maps, p);
  } else {
    ISDF_CUDA(cudaFuncSetAttribute(splitgemm_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, GC<3>::SMEM));
    splitgemm_kernel<3><<<(unsigned)units, GC<3>::THREADS, GC<3>::SMEM, s>>>(maps, p);
  }
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

// Multi-centre correlator in the form the stage-1 generator evaluates: the
// terms with (m, n) != (0, 0) grouped by their E exponent (group 0: o = 0,
// groups 1..ng: o = oexp[j-1]); per type, the coefficients of
//   P_j,d(A) = sum_e kp[t][j][d][e] A^e      (d A_{gI} part, y^d)
//   Q_j,d(A) = sum_e kq[t][j-1][d][e] A^e    (d E part, y^d)
// from d/dr_g [A^m y^n + y^m A^n] = (m A^(m-1) y^n + n A^(n-1) y^m) grad A and
// the E-derivative factor o E^(o-1) [A^m y^n + y^m A^n]; and rho(E), the
// E-gradient factor of the cusp and of the pure electron-electron terms
// (sum_I 2 c o E^(o-1)).
struct BhTc {
  int ng;   // groups with o > 0 in the kernel (1 or 2; unused groups are zero)
  int deg;  // polynomial degree in A_{g'I} (2 or 3)
  int ns4;  // float4 slots per (point, nucleus)
  int oexp[2];
  double kp[ISDF_MAX_TYPES][3][4][3];
  double kq[ISDF_MAX_TYPES][2][4][4];
  double rho[4];
};

static int bh_tc_form(const isdf_jastrow& J, BhTc& K) {
  memset(&K, 0, sizeof(K));
  int ng = 0, deg = 0;
  if (J.cusp) K.rho[0] += 0.5 / J.d;
  for (int k = 0; k < J.n_terms; ++k) {
    const int m = J.mno[k][0], n = J.mno[k][1], o = J.mno[k][2];
    ISDF_ARG(m <= 3 && n <= 3 && o <= 4,
             "tensor-core generator takes exponents m, n <= 3 and o <= 4 (term %d)", k);
    if (m == 0 && n == 0) {
      if (o > 0)
        for (int I = 0; I < J.n_nuc; ++I) K.rho[o - 1] += 2.0 * o * J.coef[J.nuc_type[I]][k];
      continue;
    }
    int j = 0;
    if (o > 0) {
      for (j = 1; j <= ng; ++j)
        if (K.oexp[j - 1] == o) break;
      if (j > ng) {
        ISDF_ARG(ng < 2, "tensor-core generator takes at most two E exponents among the "
                         "electron-electron-nucleus terms");
        K.oexp[ng++] = o;
        j = ng;
      }
    }
    for (int t = 0; t < J.n_types; ++t) {
      const double c = J.coef[t][k];
      if (m > 0) K.kp[t][j][n][m - 1] += c * m;
      if (n > 0) K.kp[t][j][m][n - 1] += c * n;
      if (o > 0) {
        K.kq[t][j - 1][n][m] += c;
        K.kq[t][j - 1][m][n] += c;
      }
    }
    if (m > 0 && n > deg) deg = n;
    if (n > 0 && m > deg) deg = m;
    if (o > 0 && m > deg) deg = m;
    if (o > 0 && n > deg) deg = n;
  }
  for (int j = ng; j < 2; ++j) K.oexp[j] = 1;  // empty groups
  K.ng = ng < 1 ? 1 : ng;
  K.deg = (deg <= 2 && K.ng == 1) ? 2 : 3;
  const int ns = 3 + K.deg + 2 * K.ng * (K.deg + 1);
  K.ns4 = (ns + 3) / 4;
  return ISDF_OK;
}

namespace {

__device__ __forceinline__ double poly_a(const double* c, int n, const double* ap) {
  double v = 0.0;
  for (int e = 0; e < n; ++e) v += c[e] * ap[e];
  return v;
}

// Per point g (padded; padding points at the origin) and nucleus I, in FP64:
// A = b r/(1 + b r), grad A = b/(1 + b r)^2 e_gI (zero on the nucleus), the
// slots of the stage-1 multi-centre generator, f(g) = sum_I P0,0(A) grad A
// (plus grad chi(r_g)/(N-1) with the one-body term) and the A_{gI} block table
// that the coordinate ring streams.
__global__ void bh_tc_table_kernel(const double* __restrict__ grid, int64_t n_g, int64_t n_k,
                                   const __grid_constant__ isdf_jastrow J,
                                   const __grid_constant__ BhTc K, float* __restrict__ rowslots,
                                   float4* __restrict__ fvec, float* __restrict__ ajtab) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_k) return;
  double x = 0, y = 0, z = 0;
  if (g < n_g) { x = grid[3 * g]; y = grid[3 * g + 1]; z = grid[3 * g + 2]; }
  double fx = 0, fy = 0, fz = 0;
  const int nslot = 4 * K.ns4;
  for (int I = 0; I < J.n_nuc; ++I) {
    const int t = J.nuc_type[I];
    const double b = J.b[t];
    const double vx = x - J.nuc_xyz[I][0], vy = y - J.nuc_xyz[I][1], vz = z - J.nuc_xyz[I][2];
    const double r = sqrt(vx * vx + vy * vy + vz * vz);
    const double den = 1.0 + b * r;
    const double A = b * r / den;
    const double dc = r > 0.0 ? b / (den * den) / r : 0.0;
    const double ap[4] = {1.0, A, A * A, A * A * A};
    float* sl = rowslots + (g * J.n_nuc + I) * nslot;
    int q = 0;
    sl[q++] = (float)(dc * vx);
    sl[q++] = (float)(dc * vy);
    sl[q++] = (float)(dc * vz);
    for (int dd = 1; dd <= K.deg; ++dd) sl[q++] = (float)poly_a(K.kp[t][0][dd], 3, ap);
    for (int j = 1; j <= K.ng; ++j) {
      for (int dd = 0; dd <= K.deg; ++dd) sl[q++] = (float)poly_a(K.kp[t][j][dd], 3, ap);
      for (int dd = 0; dd <= K.deg; ++dd) sl[q++] = (float)poly_a(K.kq[t][j - 1][dd], 4, ap);
    }
    while (q < nslot) sl[q++] = 0.f;
    const double p00 = poly_a(K.kp[t][0][0], 3, ap);
    fx += p00 * dc * vx;
    fy += p00 * dc * vy;
    fz += p00 * dc * vz;
    ajtab[(g >> 5) * J.n_nuc * 32 + I * 32 + (g & 31)] = (float)A;
  }
  if (chi_on(J)) {  // the one-body term of Eq. tau-def joins the inner-point-free part
    double h[3];
    chi_grad_pair(J, x, y, z, h);
    fx += h[0];
    fy += h[1];
    fz += h[2];
  }
  fvec[g] = make_float4((float)fx, (float)fy, (float)fz, 0.f);
}

template <int LIMBS, int NG, int DEG>
int launch_s1(unsigned grid1, const CUtensorMap* mA, const S1Params& p, cudaStream_t s) {
  using C = S1C<LIMBS, (NG >= 0)>;
  const uint32_t smem = C::FIXED + C::CSTAGES * p.cbytes + p.tab_bytes;
  ISDF_ARG(smem <= kSmemLimit,
           "too many centres for the tensor-core generator: %d nuclei with this term set need "
           "%u bytes of shared memory",
           p.n_nuc, smem);
  ISDF_CUDA(cudaFuncSetAttribute(s1_tc_kernel<LIMBS, NG, DEG>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  s1_tc_kernel<LIMBS, NG, DEG><<<grid1, C::THREADS, smem, s>>>(mA[0], mA[1], mA[2], p);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

#ifndef ISDF_PAIR_GROUPS
#define ISDF_PAIR_GROUPS 1
#endif

template <int LIMBS, bool TF32 = false>
int launch_s1_pair(unsigned grid1, const CUtensorMap* mA, const S1Params& p, cudaStream_t s) {
  constexpr int G = ISDF_PAIR_GROUPS;
  using C = S1P<LIMBS, G, TF32>;
  ISDF_CUDA(cudaFuncSetAttribute(s1_pair_kernel<LIMBS, G, TF32>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
  s1_pair_kernel<LIMBS, G, TF32><<<grid1, C::THREADS, C::SMEM, s>>>(mA[0], mA[1], mA[2], p);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

// The multi-centre generator on CTA pairs: the ring slot carries the A_{g'I}
// block (p.cbytes) and the per-row table (p.tab_bytes, 32 rows per CTA).
template <int LIMBS, int NG, int DEG>
int launch_s1_pair_bh(unsigned grid1, const CUtensorMap* mA, const S1Params& p, cudaStream_t s) {
  using C = S1P<LIMBS, 1, false, true>;
  const uint32_t smem = C::STAGES * C::STAGE + C::CSTAGES * p.cbytes + p.tab_bytes + 1024 + 512;
  ISDF_ARG(smem <= kSmemLimit,
           "too many centres for the tensor-core generator: %d nuclei with this term set need "
           "%u bytes of shared memory",
           p.n_nuc, smem);
  ISDF_CUDA(cudaFuncSetAttribute(s1_pair_kernel<LIMBS, 1, false, NG, DEG>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  s1_pair_kernel<LIMBS, 1, false, NG, DEG><<<grid1, C::THREADS, smem, s>>>(mA[0], mA[1], mA[2], p);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

}  // namespace

struct TcLayout {
  int limbs;    // stage-2 limbs (and stage-1 limbs for the BF16 precisions)
  int limbs1;   // stage-1 limbs
  int eb1;      // stage-1 operand bytes (2: BF16, 4: TF32)
  int bn;
  int64_t n_k, mu_pad, mu_pad1, gs, gs_pad;  // mu_pad1: stage-1 rows (whole 256-row pairs)
};

static TcLayout tc_layout(int64_t n_g, int n_mu, int64_t g_begin, int64_t g_end, int precision) {
  TcLayout L;
  // TF32X3: stage 1 in two TF32 limbs, stage 2 in three BF16 limbs
  L.limbs = (precision == ISDF_PREC_BF16X6 || precision == ISDF_PREC_TF32X3) ? 3 : 2;
  L.limbs1 = precision == ISDF_PREC_BF16X6 ? 3 : 2;
  L.eb1 = precision == ISDF_PREC_TF32X3 ? 4 : 2;
  L.bn = 64;
  L.n_k = round_up(n_g, 32);
  L.mu_pad = round_up(n_mu, 128);
  L.mu_pad1 = round_up(n_mu, 256);
  L.gs = g_end - g_begin;
  L.gs_pad = round_up(L.gs, 32);
  return L;
}

static bool tc_radial(const isdf_jastrow& J) { return J.n_terms == 0 && J.cusp && !chi_on(J); }

// Multi-centre tables: nuclei x float4 slots per point (0 for the radial
// correlator; the largest accepted layout when J is unknown).
static void bh_tc_dims(const isdf_jastrow* J, int& nn, int& ns4) {
  nn = 0;
  ns4 = 0;
  if (!J) {
    nn = 32;
    ns4 = 6;
    return;
  }
  if (tc_radial(*J)) return;
  BhTc K;
  nn = J->n_nuc;
  ns4 = bh_tc_form(*J, K) == ISDF_OK ? K.ns4 : 6;
}

// Per-call state of stage 1 shared by the resident and the streamed builds:
// the correlator's form, the full-grid coordinate and nucleus tables (outer
// points are read at their grid index, inner points from k_begin on).
struct S1Setup {
  bool radial, tf32, pair;
  BhTc K;
  int limbs1, eb1;
  int64_t n_k;        // full-grid padded extent of the tables
  int64_t kchunk;
  float4 *hi, *lo, *rowslots, *fvec;
  float* ajtab;
};

static void s1_tables_carve(Carve& cv, const S1Setup& S, int n_nuc, float4*& hi, float4*& lo,
                            float4*& rowslots, float4*& fvec, float*& ajtab) {
  hi = cv.take<float4>(S.n_k);
  lo = cv.take<float4>(S.n_k);
  rowslots = nullptr;
  fvec = nullptr;
  ajtab = nullptr;
  if (!S.radial && n_nuc > 0) {
    rowslots = cv.take<float4>((size_t)S.n_k * n_nuc * S.K.ns4);
    fvec = cv.take<float4>(S.n_k);
    ajtab = cv.take<float>((size_t)S.n_k * n_nuc);
  } else if (!S.radial) {
    fvec = cv.take<float4>(S.n_k);
  }
}

static int s1_setup(const isdf_jastrow& J, const isdf_options& opt, int64_t n_g, S1Setup& S) {
  S.radial = tc_radial(J);
  S.tf32 = opt.precision == ISDF_PREC_TF32X3;
  ISDF_ARG(!S.tf32 || S.radial, "the TF32 stage 1 takes the radial correlator only");
  memset(&S.K, 0, sizeof(S.K));
  if (!S.radial) ISDF_TRY(bh_tc_form(J, S.K));
  S.limbs1 = opt.precision == ISDF_PREC_BF16X6 ? 3 : 2;
  S.eb1 = S.tf32 ? 4 : 2;
  // The radial correlator runs on CTA pairs (256-row tiles).  Debug bit 1 asks
  // for the single-CTA kernel with two limbs; its three-limb form gave
  // run-to-run wrong elements on multi-tile grids and is not offered.  The
  // multi-centre generator is single-CTA.
  // The multi-centre generator runs on CTA pairs too, unless debug bit 1 asks
  // for its single-CTA kernel.
  S.pair = S.radial ? ((opt.debug_flags & 2) == 0 || S.limbs1 == 3 || S.tf32)
                    : (opt.debug_flags & 2) == 0;
  S.n_k = round_up(n_g, 32);
  S.kchunk = opt.kchunk > 0 ? round_up(opt.kchunk, 32) : (S.tf32 ? kDefaultChunkTf32 : kDefaultChunk);
  return ISDF_OK;
}

// Coordinates (FP32 hi/lo) and, for the multi-centre correlator, the per-point
// nucleus tables over the whole grid.
static int s1_tables(const double* grid, int64_t n_g, const isdf_jastrow& J, const S1Setup& S,
                     cudaStream_t s) {
  coords_kernel<<<nb256(S.n_k), 256, 0, s>>>(grid, n_g, S.n_k, S.hi, S.lo);
  ISDF_LAUNCH_CHECK();
  if (!S.radial) {
    if (J.n_nuc > 0) {
      bh_tc_table_kernel<<<nb256(S.n_k), 256, 0, s>>>(grid, n_g, S.n_k, J, S.K, (float*)S.rowslots,
                                                       S.fvec, S.ajtab);
      ISDF_LAUNCH_CHECK();
    } else {
      ISDF_CUDA(cudaMemsetAsync(S.fvec, 0, sizeof(float4) * S.n_k, s));
    }
  }
  return ISDF_OK;
}

// Stage-1 operand: limbs of (w xi)[:, k0 .. k0 + n_in) into A1
// [limbs1][mu_pad1][n_kb] (zero padding), from a source with row stride src_rs
// whose column k0 - c0 holds inner point k0.
static int s1_operand(const S1Setup& S, const double* src, int64_t src_rs, int64_t c0,
                      const double* w_in, int n_mu, int64_t n_in, int64_t mu_pad1, int64_t n_kb,
                      uint8_t* A1, CUtensorMap* mA, cudaStream_t s) {
  memset(mA, 0, 3 * sizeof(CUtensorMap));
  const size_t plane = (size_t)S.eb1 * mu_pad1 * n_kb;
  if (S.tf32) {
    split_tf32_kernel<<<nb256(mu_pad1 * n_kb), 256, 0, s>>>(src, src_rs, c0, w_in, n_mu, n_in,
                                                           mu_pad1, n_kb, S.limbs1, (uint32_t*)A1);
    ISDF_LAUNCH_CHECK();
    for (int l = 0; l < S.limbs1; ++l)
      ISDF_TRY(make_map_f32(&mA[l], A1 + l * plane, mu_pad1, n_kb, 128));
  } else {
    ISDF_TRY(split_operand(src, src_rs, c0, w_in, n_mu, n_in, mu_pad1, n_kb, S.limbs1, A1, s));
    for (int l = 0; l < S.limbs1; ++l)
      ISDF_TRY(make_map(&mA[l], A1 + l * plane, mu_pad1, n_kb, 128));
  }
  return ISDF_OK;
}

// One stage-1 launch: calG[c][nu][g - g_begin] (=, or += with accumulate) of
// the inner points k_begin .. k_begin + n_kb (padded) for the outer slice.
static int s1_launch(const S1Setup& S, const isdf_jastrow& J, const CUtensorMap* mA, int n_mu,
                     int64_t n_g, int64_t mu_pad, int64_t mu_pad1, int64_t k_begin, int64_t n_kb,
                     int64_t g_begin, int64_t g_end, double* calG, int accumulate, int debug,
                     int* err, cudaStream_t s) {
  S1Params p;
  p.xyz_hi = S.hi; p.xyz_lo = S.lo;
  p.n_g = n_g; p.n_k = n_kb; p.n_mu = n_mu;
  p.n_mu_tiles = S.pair ? (int)(mu_pad1 / 256) : (int)(mu_pad / 128);
  p.g_begin = g_begin; p.g_end = g_end;
  p.n_g_tiles = ceil_div(g_end - g_begin, 64);
  p.kchunk = S.kchunk;
  p.d = (float)J.d;
  p.calG = calG;
  p.err = err;
  p.wait_ns = wait_limit_ns();
  p.k_begin = k_begin;
  p.accumulate = accumulate;
  p.debug = debug;
  p.n_nuc = S.radial ? 0 : J.n_nuc;
  p.cbytes = S1C<2, false>::C_BASE + 4u * S1C<2, false>::BK * (uint32_t)p.n_nuc;
  // per-row table of the tile's outer points: 32 per CTA of a pair, 64 for a single CTA
  p.tab_bytes = S.radial ? 0u
                         : (uint32_t)(p.n_nuc * S.K.ns4 * (S.pair ? 32 : S1C<2, false>::BN) * 16);
  p.oexp[0] = S.radial ? 1 : S.K.oexp[0];
  p.oexp[1] = S.radial ? 1 : S.K.oexp[1];
  for (int e = 0; e < 4; ++e) p.rho[e] = S.radial ? 0.f : (float)S.K.rho[e];
  p.rowslots = S.rowslots;
  p.fvec = S.fvec;
  p.ajtab = S.ajtab;
  int dev = 0, nsm = 148;
  ISDF_CUDA(cudaGetDevice(&dev));
  ISDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int64_t n_tiles = (int64_t)p.n_mu_tiles * p.n_g_tiles;
  unsigned grid1 = (unsigned)(n_tiles < nsm ? n_tiles : nsm);
  if (S.pair) grid1 = 2u * (unsigned)(n_tiles < nsm / 2 ? n_tiles : nsm / 2);
  const BhTc& K = S.K;
  if (S.tf32) return launch_s1_pair<2, true>(grid1, mA, p, s);
  if (S.pair && S.radial)
    return S.limbs1 == 2 ? launch_s1_pair<2>(grid1, mA, p, s) : launch_s1_pair<3>(grid1, mA, p, s);
  if (S.pair) {
    if (K.ng == 1 && K.deg == 2)
      return S.limbs1 == 2 ? launch_s1_pair_bh<2, 1, 2>(grid1, mA, p, s)
                           : launch_s1_pair_bh<3, 1, 2>(grid1, mA, p, s);
    if (K.ng == 1)
      return S.limbs1 == 2 ? launch_s1_pair_bh<2, 1, 3>(grid1, mA, p, s)
                           : launch_s1_pair_bh<3, 1, 3>(grid1, mA, p, s);
    return S.limbs1 == 2 ? launch_s1_pair_bh<2, 2, 3>(grid1, mA, p, s)
                         : launch_s1_pair_bh<3, 2, 3>(grid1, mA, p, s);
  }
  if (S.radial) return launch_s1<2, -1, 0>(grid1, mA, p, s);
  if (K.ng == 1 && K.deg == 2)
    return S.limbs1 == 2 ? launch_s1<2, 1, 2>(grid1, mA, p, s) : launch_s1<3, 1, 2>(grid1, mA, p, s);
  if (K.ng == 1)
    return S.limbs1 == 2 ? launch_s1<2, 1, 3>(grid1, mA, p, s) : launch_s1<3, 1, 3>(grid1, mA, p, s);
  return S.limbs1 == 2 ? launch_s1<2, 2, 3>(grid1, mA, p, s) : launch_s1<3, 2, 3>(grid1, mA, p, s);
}

// Stage 2 over an outer slice of gs points: W[c] += (w xi~^c)_slice calG[c]^T
// (c < 3) and W[3] += (w xi)_slice calG[3]^T, in split-BF16 limbs.  src_xi /
// src_xig hold the slice's columns at column offset c0 with row stride src_rs.
static int s2_accumulate(const double* src_xi, const double* src_xig, int64_t src_rs,
                         int64_t xig_plane, int64_t c0, const double* w_slice, const double* calG,
                         int n_mu, int64_t gs, int limbs, int64_t mu_pad, int64_t gs_pad,
                         int64_t kchunk2, uint16_t* A2, uint16_t* B2, double* W, int* err,
                         cudaStream_t s) {
  const size_t plane = (size_t)limbs * mu_pad * gs_pad;
  const void* Ap[4];
  const void* Bp[4];
  for (int c = 0; c < 4; ++c) {
    const double* src = c < 3 ? src_xig + (int64_t)c * xig_plane : src_xi;
    ISDF_TRY(split_operand(src, src_rs, c0, w_slice, n_mu, gs, mu_pad, gs_pad, limbs,
                           A2 + c * plane, s));
    ISDF_TRY(split_operand(calG + (int64_t)c * n_mu * gs, gs, 0, nullptr, n_mu, gs, mu_pad,
                           gs_pad, limbs, B2 + c * plane, s));
    Ap[c] = A2 + c * plane;
    Bp[c] = B2 + c * plane;
  }
  return splitgemm(limbs, 4, Ap, Bp, n_mu, n_mu, gs_pad, kS2Range, kchunk2, W, n_mu,
                   (int64_t)n_mu * n_mu, 1.0, err, s);
}

static int s2_limbs(int precision) {
  // TF32X3: stage 1 in two TF32 limbs, stage 2 in three BF16 limbs
  return (precision == ISDF_PREC_BF16X6 || precision == ISDF_PREC_TF32X3) ? 3 : 2;
}

static int finish_checks(const isdf_options& opt, double* W, int n_mu, int* err, cudaStream_t s) {
  // every input value reaches W: a NaN or Inf there leaves a non-finite W
  ISDF_TRY(scan_nonfinite(W, (int64_t)4 * n_mu * n_mu, err, s));
  int h_err = 0;
  ISDF_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  ISDF_CUDA(cudaStreamSynchronize(s));
  (void)opt;
  if (h_err & DEV_ERR_TIMEOUT) {
    set_error("tensor-core pipeline wait expired (device error word 0x%x)", h_err);
    return ISDF_E_TIMEOUT;
  }
  if (h_err & DEV_ERR_NONFINITE) {
    set_error("W is not finite (NaN or Inf in the grid, weights or xi)");
    return ISDF_E_NONFINITE;
  }
  return ISDF_OK;
}

size_t wbuild_tc_ws(int64_t n_g, int n_mu, int64_t g_begin, int64_t g_end, int precision,
                    const isdf_jastrow* J) {
  TcLayout L = tc_layout(n_g, n_mu, g_begin, g_end, precision);
  Carve c(nullptr, 0);
  c.take<int>(64);
  c.take<float4>(L.n_k);
  c.take<float4>(L.n_k);
  int nn, ns4;
  bh_tc_dims(J, nn, ns4);
  if (nn > 0) {
    c.take<float4>((size_t)L.n_k * nn * ns4);
    c.take<float4>(L.n_k);
    c.take<float>((size_t)L.n_k * nn);
  } else if (J && !tc_radial(*J)) {
    c.take<float4>(L.n_k);
  }
  c.take<uint8_t>((size_t)L.limbs1 * L.eb1 * L.mu_pad1 * L.n_k);  // S1 A
  c.take<uint16_t>((size_t)4 * L.limbs * L.mu_pad * L.gs_pad);     // S2 A (4 channels)
  c.take<uint16_t>((size_t)4 * L.limbs * L.mu_pad * L.gs_pad);     // S2 B (calG limbs)
  return c.off;
}

int wbuild_tc(const double* grid, const double* w, const double* xi, const double* xig,
              int64_t n_g, int n_mu, int64_t g_begin, int64_t g_end, const isdf_jastrow& J,
              const isdf_options& opt, double* W, double* calG, void* ws, size_t ws_bytes,
              cudaStream_t s) {
  S1Setup S;
  ISDF_TRY(s1_setup(J, opt, n_g, S));
  const TcLayout L = tc_layout(n_g, n_mu, g_begin, g_end, opt.precision);
  Carve cv(ws, ws_bytes);
  int* err = cv.take<int>(64);
  s1_tables_carve(cv, S, J.n_nuc, S.hi, S.lo, S.rowslots, S.fvec, S.ajtab);
  uint8_t* A1 = cv.take<uint8_t>((size_t)L.limbs1 * L.eb1 * L.mu_pad1 * L.n_k);
  uint16_t* A2 = cv.take<uint16_t>((size_t)4 * L.limbs * L.mu_pad * L.gs_pad);
  uint16_t* B2 = cv.take<uint16_t>((size_t)4 * L.limbs * L.mu_pad * L.gs_pad);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  ISDF_CUDA(cudaMemsetAsync(err, 0, 64 * sizeof(int), s));
  const int64_t kchunk2 = opt.s2_kchunk > 0 ? round_up(opt.s2_kchunk, 32) : 256;

  ISDF_TRY(s1_tables(grid, n_g, J, S, s));
  CUtensorMap mA[3];
  ISDF_TRY(s1_operand(S, xi, n_g, 0, w, n_mu, n_g, L.mu_pad1, L.n_k, A1, mA, s));
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
  const bool timed = opt.stage_ms != nullptr && opt.sync_check;
  if (timed) {
    for (int i = 0; i < 4; ++i) ISDF_CUDA(cudaEventCreate(&ev[i]));
    ISDF_CUDA(cudaEventRecord(ev[0], s));
  }
  ISDF_TRY(s1_launch(S, J, mA, n_mu, n_g, L.mu_pad, L.mu_pad1, 0, L.n_k, g_begin, g_end, calG, 0,
                     opt.debug_flags, err, s));
  if (timed) ISDF_CUDA(cudaEventRecord(ev[1], s));
  ISDF_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * 4 * (size_t)n_mu * n_mu, s));
  if (timed) ISDF_CUDA(cudaEventRecord(ev[2], s));
  // stage 2: (w xi~^c) and (w xi) over the slice, calG in limbs
  ISDF_TRY(s2_accumulate(xi, xig, n_g, (int64_t)n_mu * n_g, g_begin, w, calG, n_mu, L.gs, L.limbs,
                         L.mu_pad, L.gs_pad, kchunk2, A2, B2, W, err, s));
  if (timed) ISDF_CUDA(cudaEventRecord(ev[3], s));
  if (opt.sync_check) {
    const int rc = finish_checks(opt, W, n_mu, err, s);
    if (timed) {
      ISDF_CUDA(cudaEventElapsedTime(&opt.stage_ms[0], ev[0], ev[1]));
      ISDF_CUDA(cudaEventElapsedTime(&opt.stage_ms[1], ev[2], ev[3]));
      for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
    }
    return rc;
  }
  return ISDF_OK;
}

// ------------------------------------------------------------------ streamed build

// Layout of the streamed build (Sec. II.D grid-batched streaming, Sec. IV.C
// doubly-blocked grid loops): the device holds the full-grid coordinate and
// nucleus tables, two inner (ket) batches of xi in FP64 (the copy of the next
// one overlaps the current one's stage 1), one outer (bra) batch of xi and
// xi~ in FP64, the bra batch's calG, and the limb operands.
struct StreamWs {
  int* err;
  double* ket[2];     // [n_mu][ket]
  double* bra;        // [4][n_mu][bra]: xi~ (3 planes), then xi
  double* calG;       // [4][n_mu][bra]
  uint8_t* A1;        // [limbs1][mu_pad1][round_up(ket, 32)] (element bytes eb1)
  uint16_t *A2, *B2;  // [4][limbs][mu_pad][round_up(bra, 32)]
  void carve(Carve& cv, S1Setup& S, int n_mu, int n_nuc, int64_t bra_n, int64_t ket_n,
             int limbs) {
    err = cv.take<int>(64);
    s1_tables_carve(cv, S, n_nuc, S.hi, S.lo, S.rowslots, S.fvec, S.ajtab);
    for (int i = 0; i < 2; ++i) ket[i] = cv.take<double>((size_t)n_mu * ket_n);
    bra = cv.take<double>((size_t)4 * n_mu * bra_n);
    calG = cv.take<double>((size_t)4 * n_mu * bra_n);
    const int64_t mu_pad1 = round_up(n_mu, 256), mu_pad = round_up(n_mu, 128);
    A1 = cv.take<uint8_t>((size_t)S.limbs1 * S.eb1 * mu_pad1 * round_up(ket_n, 32));
    A2 = cv.take<uint16_t>((size_t)4 * limbs * mu_pad * round_up(bra_n, 32));
    B2 = cv.take<uint16_t>((size_t)4 * limbs * mu_pad * round_up(bra_n, 32));
  }
};

size_t wbuild_streamed_ws(int64_t n_g, int n_mu, int64_t bra_n, int64_t ket_n, int precision,
                          const isdf_jastrow* J) {
  isdf_jastrow Jr;
  memset(&Jr, 0, sizeof(Jr));
  isdf_options opt = {precision, 0, 0, 1, 0, nullptr, 0.0, 0.0, 0, 0};
  S1Setup S;
  memset(&S, 0, sizeof(S));
  if (J) {
    if (s1_setup(*J, opt, n_g, S) != ISDF_OK) return 0;
  } else {
    // the largest accepted layout: a multi-centre correlator with 32 nuclei
    S.radial = false;
    S.K.ns4 = 6;
    S.limbs1 = precision == ISDF_PREC_BF16X6 ? 3 : 2;
    S.eb1 = precision == ISDF_PREC_TF32X3 ? 4 : 2;
    S.n_k = round_up(n_g, 32);
  }
  Carve c(nullptr, 0);
  StreamWs b;
  b.carve(c, S, n_mu, J ? J->n_nuc : 32, bra_n, ket_n, s2_limbs(precision));
  return c.off;
}

int wbuild_streamed(const double* grid, const double* w, const double* xi_h, const double* xig_h,
                    int64_t n_g, int n_mu, int64_t bra_n, int64_t ket_n, const isdf_jastrow& J,
                    const isdf_options& opt, double* W, void* ws, size_t ws_bytes,
                    cudaStream_t s) {
  ISDF_ARG(xi_h && xig_h && W && grid && w, "null pointer argument");
  ISDF_ARG(bra_n > 0 && ket_n > 0 && ket_n % 32 == 0, "batch sizes: bra > 0, ket a positive "
           "multiple of 32");
  S1Setup S;
  ISDF_TRY(s1_setup(J, opt, n_g, S));
  const int limbs = s2_limbs(opt.precision);
  const int64_t mu_pad1 = round_up(n_mu, 256), mu_pad = round_up(n_mu, 128);
  Carve cv(ws, ws_bytes);
  StreamWs b;
  b.carve(cv, S, n_mu, J.n_nuc, bra_n, ket_n, limbs);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  const int64_t kchunk2 = opt.s2_kchunk > 0 ? round_up(opt.s2_kchunk, 32) : 256;

  // a copy stream for the host-to-device batches and events between the two
  cudaStream_t cs = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, freed[2] = {nullptr, nullptr};
  cudaEvent_t bra_copied = nullptr, bra_freed = nullptr;
  int rc = ISDF_OK;
  auto cleanup = [&]() {
    for (int i = 0; i < 2; ++i) {
      if (copied[i]) cudaEventDestroy(copied[i]);
      if (freed[i]) cudaEventDestroy(freed[i]);
    }
    if (bra_copied) cudaEventDestroy(bra_copied);
    if (bra_freed) cudaEventDestroy(bra_freed);
    if (cs) cudaStreamDestroy(cs);
  };
#define STREAM_TRY(x)                 \
  do {                                \
    rc = (x);                         \
    if (rc != ISDF_OK) {              \
      cleanup();                      \
      return rc;                      \
    }                                 \
  } while (0)
#define STREAM_CUDA(x) STREAM_TRY(cuda_status((x), #x))
  STREAM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) {
    STREAM_CUDA(cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming));
    STREAM_CUDA(cudaEventCreateWithFlags(&freed[i], cudaEventDisableTiming));
  }
  STREAM_CUDA(cudaEventCreateWithFlags(&bra_copied, cudaEventDisableTiming));
  STREAM_CUDA(cudaEventCreateWithFlags(&bra_freed, cudaEventDisableTiming));
  STREAM_CUDA(cudaMemsetAsync(b.err, 0, 64 * sizeof(int), s));
  STREAM_CUDA(cudaMemsetAsync(W, 0, sizeof(double) * 4 * (size_t)n_mu * n_mu, s));
  STREAM_TRY(s1_tables(grid, n_g, J, S, s));
  // the copy stream starts after the tables and buffers are set up on s
  STREAM_CUDA(cudaEventRecord(freed[0], s));
  STREAM_CUDA(cudaEventRecord(freed[1], s));
  STREAM_CUDA(cudaEventRecord(bra_freed, s));

  const int64_t n_ket = ceil_div(n_g, ket_n), n_bra = ceil_div(n_g, bra_n);
  const int64_t total = n_ket * n_bra;
  // copy of ket batch `it` (bra-major order) into slot it % 2
  auto copy_ket = [&](int64_t it) -> int {
    const int64_t k = it % n_ket;
    const int64_t h0 = k * ket_n, hn = n_g - h0 < ket_n ? n_g - h0 : ket_n;
    const int slot = (int)(it & 1);
    ISDF_CUDA(cudaStreamWaitEvent(cs, freed[slot], 0));
    ISDF_CUDA(cudaMemcpy2DAsync(b.ket[slot], (size_t)hn * 8, xi_h + h0, (size_t)n_g * 8,
                                (size_t)hn * 8, (size_t)n_mu, cudaMemcpyHostToDevice, cs));
    ISDF_CUDA(cudaEventRecord(copied[slot], cs));
    return ISDF_OK;
  };
  auto copy_bra = [&](int64_t bi) -> int {
    const int64_t g0 = bi * bra_n, gn = n_g - g0 < bra_n ? n_g - g0 : bra_n;
    ISDF_CUDA(cudaStreamWaitEvent(cs, bra_freed, 0));
    for (int c = 0; c < 4; ++c) {
      const double* src = c < 3 ? xig_h + (int64_t)c * n_mu * n_g : xi_h;
      ISDF_CUDA(cudaMemcpy2DAsync(b.bra + (size_t)c * n_mu * gn, (size_t)gn * 8, src + g0,
                                  (size_t)n_g * 8, (size_t)gn * 8, (size_t)n_mu,
                                  cudaMemcpyHostToDevice, cs));
    }
    ISDF_CUDA(cudaEventRecord(bra_copied, cs));
    return ISDF_OK;
  };
  STREAM_TRY(copy_ket(0));
  for (int64_t bi = 0; bi < n_bra; ++bi) {
    const int64_t g0 = bi * bra_n, gn = n_g - g0 < bra_n ? n_g - g0 : bra_n;
    STREAM_TRY(copy_bra(bi));
    for (int64_t k = 0; k < n_ket; ++k) {
      const int64_t it = bi * n_ket + k;
      const int slot = (int)(it & 1);
      if (it + 1 < total) STREAM_TRY(copy_ket(it + 1));  // depth-one prefetch
      const int64_t h0 = k * ket_n, hn = n_g - h0 < ket_n ? n_g - h0 : ket_n;
      const int64_t nkb = round_up(hn, 32);
      STREAM_CUDA(cudaStreamWaitEvent(s, copied[slot], 0));
      CUtensorMap mA[3];
      STREAM_TRY(s1_operand(S, b.ket[slot], hn, 0, w + h0, n_mu, hn, mu_pad1, nkb, b.A1, mA, s));
      STREAM_CUDA(cudaEventRecord(freed[slot], s));
      STREAM_TRY(s1_launch(S, J, mA, n_mu, n_g, mu_pad, mu_pad1, h0, nkb, g0, g0 + gn, b.calG,
                           k > 0 ? 1 : 0, opt.debug_flags, b.err, s));
    }
    STREAM_CUDA(cudaStreamWaitEvent(s, bra_copied, 0));
    STREAM_TRY(s2_accumulate(b.bra + (size_t)3 * n_mu * gn, b.bra, gn, (int64_t)n_mu * gn, 0,
                             w + g0, b.calG, n_mu, gn, limbs, mu_pad, round_up(gn, 32), kchunk2,
                             b.A2, b.B2, W, b.err, s));
    STREAM_CUDA(cudaEventRecord(bra_freed, s));
  }
  rc = opt.sync_check ? finish_checks(opt, W, n_mu, b.err, s) : ISDF_OK;
  if (!opt.sync_check) cudaStreamSynchronize(s);  // the events and copy stream end with the call
  cleanup();
  return rc;
#undef STREAM_CUDA
#undef STREAM_TRY
}

}  // namespace isdf
