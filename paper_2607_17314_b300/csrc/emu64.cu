// FP64 matrix products on the BF16 tensor cores by exact integer slices, and
// the blocked triangular solves of the ISDF fit (Sec. IV.B) built on them.
//
// A row of A (a column of B) is scaled by 2^-e, e the smallest integer with
// |x| < 2^e over the row, so each scaled element lies in (-1, 1).  Its
// magnitude, truncated to 56 fraction bits, is cut into S = 8 base-2^7 digits
// d_1 .. d_8 that carry the element's sign; each digit is an integer of at most
// 7 bits, which BF16 holds exactly.  Then
//   (A B)_mn ~= 2^(e_m + e_n) sum_{p + q <= 9} 2^(-7 (p + q)) sum_k d_p(A_mk) d_q(B_kn).
// Each inner sum over k of one level L = p + q is a sum of integers: with at
// most 8 digit pairs per level and at most 128 terms, its magnitude stays below
// 8 * 127^2 * 128 < 2^24, so the tensor core's FP32 accumulation of a level is
// exact.  The epilogue combines the 8 levels exactly in a 64-bit integer scaled
// by 2^52 (the lowest level pair keeps its bits down to 2^-52 of the scale),
// sums the runs of one output tile in that integer and converts once to FP64.  The dropped pairs (p + q > 9: at most ~2^-53.2 of
// 2^(e_m + e_n) per term), the truncation below 2^-56 and the lowest level
// pair's rounding (1 unit of 2^-52) bound the error by (K + 4) 2^-52 of
// 2^(e_m + e_n), the size of FP64 rounding over K terms of that magnitude.
#include <cuda.h>
#include <cuda_bf16.h>

#include "linalg.cuh"
#include "tc_ptx.cuh"

namespace isdf {

int tma_map_bf16(CUtensorMap* m, const void* base, int64_t rows, int64_t cols, int box_rows);

namespace {

constexpr int kS = 8;              // digits per value
constexpr int kBits = 7;           // bits per digit
constexpr int kFrac = kS * kBits;  // 56 fraction bits
constexpr int kZeroExp = -4000;    // exponent of an all-zero row or column
constexpr int kBadExp = 4000;      // a NaN or Inf in the row or column

constexpr int EM_BM = 128, EM_BN = 64, EM_BK = 32, EM_STAGES = 2;
constexpr int EM_EPI_WARPS = 16;  // four per tensor-memory lane quarter, 16 columns each
constexpr int EM_EPI_COLS = EM_BN * 4 / EM_EPI_WARPS;
constexpr int EM_THREADS = 64 + 32 * EM_EPI_WARPS;
constexpr int EM_KCHUNK = 128;  // exact FP32 accumulation bound per level
constexpr uint32_t EM_AT = EM_BM * EM_BK * 2;
constexpr uint32_t EM_BT = EM_BN * EM_BK * 2;
constexpr uint32_t EM_STAGE = kS * (EM_AT + EM_BT);
constexpr uint32_t EM_SMEM = EM_STAGES * EM_STAGE + 1024 + 256;
constexpr uint32_t EM_TMEM = kS * EM_BN;  // 8 levels x 64 columns
static_assert(EM_TMEM == 512, "tensor memory holds the eight level accumulators");

constexpr int TRSM_TB = 128;  // block size of the triangular solves (= EM_KCHUNK)

// Smallest e with |x| < 2^e (integer arithmetic on the bits).
__device__ __forceinline__ int exp_of(double x) {
  const uint64_t b = (uint64_t)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  if (b == 0) return kZeroExp;
  const int be = (int)(b >> 52);
  if (be == 0x7FF) return kBadExp;
  if (be) return be - 1022;
  return (64 - __clzll((long long)b)) - 1074;
}

// The 8 signed digits of x 2^-e (|x| < 2^e), truncated below 2^-56.
__device__ __forceinline__ void digits_of(double x, int e, int (&d)[kS]) {
  const uint64_t bits = (uint64_t)__double_as_longlong(x);
  const uint64_t b = bits & 0x7FFFFFFFFFFFFFFFull;
  uint64_t M = 0;
  const int be = (int)(b >> 52);
  if (b != 0 && be != 0x7FF && e != kBadExp) {
    const uint64_t mant = be ? ((b & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : b;
    const int sh = (be ? be - 1075 : -1074) + kFrac - e;  // M = mant 2^sh < 2^56
    if (sh >= 0) M = mant << sh;
    else if (sh > -64) M = mant >> (-sh);
  }
  const bool neg = (bits >> 63) != 0;
#pragma unroll
  for (int p = 0; p < kS; ++p) {
    const int v = (int)((M >> (kFrac - kBits * (p + 1))) & 127u);
    d[p] = neg ? -v : v;
  }
}

// e[m] over the row m of A (A(m, k) = src[m rs + k cs]), one warp per row.
__global__ void em_row_exp_kernel(const double* __restrict__ src, int64_t rs, int64_t cs,
                                  int64_t rows, int64_t cols, int* __restrict__ e,
                                  int* __restrict__ err) {
  const int64_t m = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (m >= rows) return;
  int mx = kZeroExp;
  for (int64_t k = lane; k < cols; k += 32) mx = max(mx, exp_of(src[m * rs + k * cs]));
  for (int o = 16; o; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if (lane == 0) {
    e[m] = mx;
    if (mx == kBadExp && err) atomicOr(err, DEV_ERR_NONFINITE);
  }
}

// e[n] over the column n of B (B(k, n) = src[k rs + n cs]), one thread per column.
__global__ void em_col_exp_kernel(const double* __restrict__ src, int64_t rs, int64_t cs,
                                  int64_t K, int64_t N, int* __restrict__ e,
                                  int* __restrict__ err) {
  const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  int mx = kZeroExp;
  for (int64_t k = 0; k < K; ++k) mx = max(mx, exp_of(src[k * rs + n * cs]));
  e[n] = mx;
  if (mx == kBadExp && err) atomicOr(err, DEV_ERR_NONFINITE);
}

// Digits of A into out [kS][rows_pad][k_pad] (k contiguous); padding is zero.
// One thread per (row, 8 consecutive k).
__global__ void em_split_rows_kernel(const double* __restrict__ src, int64_t rs, int64_t cs,
                                     int64_t rows, int64_t cols, const int* __restrict__ e,
                                     int64_t rows_pad, int64_t k_pad,
                                     __nv_bfloat16* __restrict__ out) {
  const int64_t groups = k_pad / 8;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows_pad * groups) return;
  const int64_t m = t / groups, k0 = (t - m * groups) * 8;
  const int em = m < rows ? e[m] : kZeroExp;
  __align__(16) __nv_bfloat16 v[kS][8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t k = k0 + j;
    const double x = (m < rows && k < cols) ? src[m * rs + k * cs] : 0.0;
    int d[kS];
    digits_of(x, em, d);
#pragma unroll
    for (int p = 0; p < kS; ++p) v[p][j] = __int2bfloat16_rn(d[p]);
  }
  const int64_t plane = rows_pad * k_pad;
#pragma unroll
  for (int p = 0; p < kS; ++p)
    *reinterpret_cast<uint4*>(out + p * plane + m * k_pad + k0) =
        *reinterpret_cast<const uint4*>(v[p]);
}

// Digits of B (K x N) into out [kS][n_pad][k_pad] (k contiguous, i.e. B^T),
// through a shared-memory tile of 64 columns x 64 k per block: the reads run
// along the rows of B (consecutive threads, consecutive columns) and the
// writes along the k rows of the output (128 contiguous bytes per digit plane
// and column).
constexpr int SC_N = 64, SC_K = 64, SC_LD = SC_K + 8;  // row stride in BF16 (16-byte rows)
constexpr size_t SC_SMEM = (size_t)kS * SC_N * SC_LD * sizeof(__nv_bfloat16);

__global__ void __launch_bounds__(256) em_split_cols_kernel(
    const double* __restrict__ src, int64_t rs, int64_t cs, int64_t K, int64_t N,
    const int* __restrict__ e, int64_t n_pad, int64_t k_pad, __nv_bfloat16* __restrict__ out) {
  extern __shared__ __align__(16) __nv_bfloat16 sc_tile[];  // [kS][SC_N][SC_LD]
  auto tile = reinterpret_cast<__nv_bfloat16(*)[SC_N][SC_LD]>(sc_tile);
  const int64_t n0 = (int64_t)blockIdx.x * SC_N, k0 = (int64_t)blockIdx.y * SC_K;
  const int nl = threadIdx.x % SC_N, kq = threadIdx.x / SC_N;  // 4 groups of 16 k
  const int64_t n = n0 + nl;
  const int en = n < N ? e[n] : kZeroExp;
#pragma unroll 4
  for (int j = 0; j < SC_K / 4; j += 2) {
    int d0[kS], d1[kS];
    const int kl = kq * (SC_K / 4) + j;
    const int64_t k = k0 + kl;
    const double x0 = (n < N && k < K) ? src[k * rs + n * cs] : 0.0;
    const double x1 = (n < N && k + 1 < K) ? src[(k + 1) * rs + n * cs] : 0.0;
    digits_of(x0, en, d0);
    digits_of(x1, en, d1);
#pragma unroll
    for (int p = 0; p < kS; ++p)
      *reinterpret_cast<__nv_bfloat162*>(&tile[p][nl][kl]) =
          __halves2bfloat162(__int2bfloat16_rn(d0[p]), __int2bfloat16_rn(d1[p]));
  }
  __syncthreads();
  // 8 planes x 64 columns x 8 chunks of 16 bytes
  const int64_t plane = n_pad * k_pad;
  for (int q = threadIdx.x; q < kS * SC_N * (SC_K / 8); q += blockDim.x) {
    const int c = q % (SC_K / 8), row = (q / (SC_K / 8)) % SC_N, p = q / (SC_N * (SC_K / 8));
    const int64_t nn = n0 + row, kk = k0 + c * 8;
    if (nn < n_pad && kk < k_pad)
      *reinterpret_cast<uint4*>(out + p * plane + nn * k_pad + kk) =
          *reinterpret_cast<const uint4*>(&tile[p][row][c * 8]);
  }
}

struct EmMaps {
  CUtensorMap a[kS];
  CUtensorMap b[kS];
};

struct EmParams {
  int64_t M, N, k_tiles;
  int m_tiles, n_tiles, kchunks;
  const int* ea;
  const int* eb;
  double* C;
  int64_t ldc;
  double alpha;
  int kin;   // K chunks of <= 128 that one work unit takes in turn (V summed in 64 bits)
  int mode;  // 0: C = alpha A B; 1: C += alpha A B; 2: the same with atomics (K split)
  int vec;   // C rows 16-byte aligned: 16-byte stores
  int* err;
  uint64_t wait_ns;
};

// sign * V * 2^E rounded to the nearest FP64 (ties to even), by integer
// arithmetic on the bits; ldexp covers results outside the normal range.
__device__ __forceinline__ double i64_scaled(long long V, int E, bool negate) {
  if (V == 0) return 0.0;
  uint64_t sign = V < 0 ? 1ull : 0ull;
  uint64_t u = V < 0 ? (uint64_t)(-V) : (uint64_t)V;
  if (negate) sign ^= 1ull;
  const int lz = __clzll((long long)u);
  u <<= lz;                           // bit 63 set: value = u 2^(E - lz)
  uint64_t mant = u >> 11;            // 53 bits
  const uint64_t rem = u & 0x7FFull;  // 11 rounding bits
  if (rem > 0x400ull || (rem == 0x400ull && (mant & 1ull))) ++mant;
  int ex = 63 - lz + E;               // value = mant 2^(ex - 52)
  if (mant >> 53) {
    mant >>= 1;
    ++ex;
  }
  const int be = ex + 1023;
  if (be > 0 && be < 0x7FF)
    return __longlong_as_double((long long)((sign << 63) | ((uint64_t)be << 52) |
                                            (mant & 0xFFFFFFFFFFFFFull)));
  const double v = ldexp((double)mant, ex - 52);
  return sign ? -v : v;
}

// One tile's level accumulators -> FP64 outputs: a warp takes 32 rows and the
// EM_EPI_COLS columns [c0, c0 + EM_EPI_COLS) of the tile.  Per output
//   V = 2^52 sum_L acc_L 2^(-7 L),  L = 2 .. 9,
// formed from the level pairs P = acc_L 2^7 + acc_(L+1), exact in 32 bits
// (|acc_L| <= (L - 1) 127^2 128, so |P| < 2^31), then four 64-bit terms
// (the lowest pair keeps its bits down to 2^-52).  em_drain adds V of one K
// chunk to the thread's running sums (every chunk has the same row and column
// scales, so the sum is exact; |V| < 2^59.1 per chunk keeps up to 8 chunks in
// 64 bits) and signals acc_empty, so that the next products run while the
// outputs are formed and stored; em_store applies the scale 2^(e_m + e_n - 52)
// and alpha.  mode 0 stores, 1 adds, 2 adds atomically; each thread writes 8
// consecutive columns of its row (64 bytes) per block.
constexpr int EM_NB = EM_EPI_COLS / 8;

__device__ __forceinline__ void em_drain(uint32_t taddr, int c0, bool first,
                                         long long (&Vs)[EM_NB][8], uint64_t* acc_empty) {
#pragma unroll
  for (int b = 0; b < EM_NB; ++b) {
    uint32_t r[kS][8];
#pragma unroll
    for (int l = 0; l < kS; ++l)
      tc::tmem_ld_32x32b_x8(taddr + (uint32_t)(l * EM_BN + c0 + b * 8), r[l]);
    tc::tmem_ld_wait();
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int P[kS / 2];
#pragma unroll
      for (int h = 0; h < kS / 2; ++h)
        P[h] = __float2int_rn(__uint_as_float(r[2 * h][j])) * (1 << kBits) +
               __float2int_rn(__uint_as_float(r[2 * h + 1][j]));
      // pair h holds levels 2h + 2, 2h + 3: weight 2^(52 - 7 (2h + 3))
      const long long V = (long long)P[0] * (1ll << 31) + (long long)P[1] * (1ll << 17) +
                          (long long)P[2] * (1ll << 3) + (long long)(P[3] >> 11);
      Vs[b][j] = first ? V : Vs[b][j] + V;
    }
  }
  // the accumulators are free for the next products
  __syncwarp();
  tc::tc_fence_before();
  tc::mbar_arrive(acc_empty);
}

__device__ __forceinline__ void em_store(const EmParams& p, int64_t m, int64_t n0, int c0,
                                         const long long (&Vs)[EM_NB][8]) {
  const int ea = m < p.M ? p.ea[m] : kZeroExp;
  const bool unit_alpha = p.alpha == 1.0 || p.alpha == -1.0;
  const bool neg = p.alpha < 0.0;
#pragma unroll
  for (int b = 0; b < EM_NB; ++b) {
    const int64_t nb = n0 + c0 + b * 8;
    if (m >= p.M || nb >= p.N) continue;
    int ebv[8];
    if (nb + 8 <= p.N) {
      const int4 e0 = __ldg(reinterpret_cast<const int4*>(p.eb + nb));
      const int4 e1 = __ldg(reinterpret_cast<const int4*>(p.eb + nb) + 1);
      ebv[0] = e0.x; ebv[1] = e0.y; ebv[2] = e0.z; ebv[3] = e0.w;
      ebv[4] = e1.x; ebv[5] = e1.y; ebv[6] = e1.z; ebv[7] = e1.w;
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) ebv[j] = nb + j < p.N ? p.eb[nb + j] : kZeroExp;
    }
    double v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      double x = 0.0;
      if (ea != kZeroExp && ebv[j] != kZeroExp) {
        x = i64_scaled(Vs[b][j], ea + ebv[j] - 52, unit_alpha && neg);
        if (!unit_alpha) x *= p.alpha;
      }
      v[j] = x;
    }
    double* c = p.C + m * p.ldc + nb;
    if (p.vec && nb + 8 <= p.N && p.mode != 2) {
      double2* c2 = reinterpret_cast<double2*>(c);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        double2 o = make_double2(v[2 * j], v[2 * j + 1]);
        if (p.mode == 1) {
          const double2 q = c2[j];
          o.x += q.x;
          o.y += q.y;
        }
        c2[j] = o;
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (nb + j >= p.N) break;
        if (p.mode == 0) c[j] = v[j];
        else if (p.mode == 1) c[j] += v[j];
        else atomicAdd(c + j, v[j]);
      }
    }
  }
}

// Persistent: CTA b takes the work units b, b + gridDim.x, ... (unit = K part
// fastest, then the 128-row tile, then the 64-column tile, so that the CTAs
// running together share B tiles).  A unit covers p.kin runs of <= 128 k of
// one output tile (all of K when K <= 1024, else one run, the runs of a tile
// then being separate units added with atomics).  Warp 0 loads the 8 digit
// planes of both operands by TMA into a two-stage ring that runs ahead across
// runs and tiles; warp 1 issues the 36 products of each 16-k step into the 8
// level accumulators in tensor memory (level p + q - 2 at columns
// 64 (p + q - 2)) once the epilogue has drained the previous run, and commits
// after each run; warps 2 .. 17 drain and combine the levels (warp w: the rows
// of lane quarter w % 4, columns 16 ((w - 2) / 4) ..) and store once per unit.
__global__ void __launch_bounds__(EM_THREADS, 1)
    emgemm_kernel(const __grid_constant__ EmMaps maps, const EmParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t* full = (uint64_t*)(smem + EM_STAGES * EM_STAGE);
  uint64_t* empty = full + EM_STAGES;
  uint64_t* acc_full = empty + EM_STAGES;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = (uint32_t*)(acc_empty + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  constexpr int64_t KT = EM_KCHUNK / EM_BK;
  const int64_t units = (int64_t)p.kchunks * p.m_tiles * p.n_tiles;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < EM_STAGES; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(acc_full, 1);
    tc::mbar_init(acc_empty, EM_EPI_WARPS * 32);
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    tc::tmem_alloc(tmem_slot, EM_TMEM);
    tc::tmem_relinquish();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int kc = (int)(u % p.kchunks);
        const int mt = (int)((u / p.kchunks) % p.m_tiles);
        const int nt = (int)(u / ((int64_t)p.kchunks * p.m_tiles));
        const int64_t kt0 = (int64_t)kc * p.kin * KT;
        const int64_t kt1 = kt0 + p.kin * KT < p.k_tiles ? kt0 + p.kin * KT : p.k_tiles;
        for (int64_t kt = kt0; kt < kt1; ++kt, ++it) {
          const uint32_t s = it % EM_STAGES, ph = (it / EM_STAGES) & 1;
          if (!tc::mbar_wait(&empty[s], ph ^ 1, abort_flag, p.err, p.wait_ns)) {
            ok = false;
            break;
          }
          tc::mbar_arrive_expect_tx(&full[s], EM_STAGE);
          uint8_t* base = smem + s * EM_STAGE;
          const int32_t x = (int32_t)(kt * EM_BK);
#pragma unroll
          for (int q = 0; q < kS; ++q) {
            tc::tma_load_2d(base + q * EM_AT, &maps.a[q], &full[s], x, mt * EM_BM);
            tc::tma_load_2d(base + kS * EM_AT + q * EM_BT, &maps.b[q], &full[s], x, nt * EM_BN);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = tc::idesc_f16(EM_BM, EM_BN, 1);
      uint32_t it = 0, lt = 0;
      bool ok = true;
      for (int64_t u = blockIdx.x; u < units && ok; u += gridDim.x) {
       const int kc = (int)(u % p.kchunks);
       const int64_t ku = (int64_t)kc * p.kin * KT;
       const int64_t ku1 = ku + p.kin * KT < p.k_tiles ? ku + p.kin * KT : p.k_tiles;
       for (int64_t kt0 = ku; kt0 < ku1 && ok; kt0 += KT, ++lt) {
        const int64_t kt1 = kt0 + KT < ku1 ? kt0 + KT : ku1;
        if (!tc::mbar_wait(acc_empty, (lt & 1) ^ 1, abort_flag, p.err, p.wait_ns)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        for (int64_t kt = kt0; kt < kt1; ++kt, ++it) {
          const uint32_t s = it % EM_STAGES, ph = (it / EM_STAGES) & 1;
          if (!tc::mbar_wait(&full[s], ph, abort_flag, p.err, p.wait_ns)) {
            ok = false;
            break;
          }
          tc::tc_fence_after();
          const uint32_t base = tc::smem_u32(smem + s * EM_STAGE);
#pragma unroll
          for (int kk = 0; kk < 2; ++kk)
#pragma unroll
            for (int pa = 0; pa < kS; ++pa) {
              const uint64_t ad = tc::smem_desc(base + pa * EM_AT + kk * 32, 16, 512, 4);
#pragma unroll
              for (int qb = 0; qb < kS - pa; ++qb) {
                const uint64_t bd =
                    tc::smem_desc(base + kS * EM_AT + qb * EM_BT + kk * 32, 16, 512, 4);
                // the first product of every level zeroes it (pa = 0 reaches all levels)
                const uint32_t acc = (kt == kt0 && kk == 0 && pa == 0) ? 0u : 1u;
                tc::umma_f16(tmem + (uint32_t)((pa + qb) * EM_BN), ad, bd, idesc, acc);
              }
            }
          tc::umma_commit(&empty[s]);
        }
        if (ok) tc::umma_commit(acc_full);
       }
      }
    }
  } else {
    const int quad = warp & 3;
    const uint32_t lane_base = (uint32_t)(32 * quad) << 16;
    const int c0 = EM_EPI_COLS * ((warp - 2) / 4);
    uint32_t lt = 0;
    bool ok = true;
    for (int64_t u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int kc = (int)(u % p.kchunks);
      const int mt = (int)((u / p.kchunks) % p.m_tiles);
      const int nt = (int)(u / ((int64_t)p.kchunks * p.m_tiles));
      const int64_t ku = (int64_t)kc * p.kin * KT;
      const int64_t ku1 = ku + p.kin * KT < p.k_tiles ? ku + p.kin * KT : p.k_tiles;
      long long Vs[EM_NB][8];
      for (int64_t kt0 = ku; kt0 < ku1; kt0 += KT, ++lt) {
        // warp-collective tensor-memory loads: reconverge after the spin-wait
        const bool got = tc::mbar_wait(acc_full, lt & 1, abort_flag, p.err, p.wait_ns);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        em_drain(tmem + lane_base, c0, kt0 == ku, Vs, acc_empty);
      }
      if (!ok) break;
      em_store(p, (int64_t)mt * EM_BM + 32 * quad + lane, (int64_t)nt * EM_BN, c0, Vs);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (*abort_flag) {
    // a bounded wait expired: give issued copies and products time to land
    const uint64_t t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < 200000ull) {
    }
  }
  if (warp == 0) {
    tc::tc_fence_after();
    tc::tmem_dealloc(tmem, EM_TMEM);
  }
}

// Inverse of every diagonal block of the lower-triangular L [n][n]:
// out[j] (TB x TB, zero above the diagonal and beyond the block's size) by
// forward substitution, thread c producing column c.
__global__ void __launch_bounds__(TRSM_TB) trtri_blocks_kernel(const double* __restrict__ L, int n,
                                                               double* __restrict__ out) {
  extern __shared__ double Ls[];  // [TB][TB]
  const int j0 = blockIdx.x * TRSM_TB;
  const int jb = n - j0 < TRSM_TB ? n - j0 : TRSM_TB;
  double* X = out + (int64_t)blockIdx.x * TRSM_TB * TRSM_TB;
  for (int q = threadIdx.x; q < TRSM_TB * TRSM_TB; q += blockDim.x) {
    const int i = q / TRSM_TB, k = q - i * TRSM_TB;
    Ls[q] = (i < jb && k <= i) ? L[(int64_t)(j0 + i) * n + j0 + k] : 0.0;
  }
  __syncthreads();
  const int c = threadIdx.x;
  for (int i = 0; i < TRSM_TB; ++i) {
    double v = 0.0;
    if (i < jb && c < jb && i >= c) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = c; k < i; ++k) s -= Ls[i * TRSM_TB + k] * X[k * TRSM_TB + c];
      v = s / Ls[i * TRSM_TB + i];
    }
    X[i * TRSM_TB + c] = v;
  }
}

inline unsigned nblk(int64_t n, int b) { return (unsigned)ceil_div(n, b); }

}  // namespace

// ------------------------------------------------------------------ host side

// Workspace of one emulated product with at most Mmax rows, Nmax columns and
// Kmax inner terms: the digit planes of both operands, the exponents and an
// error word.
struct EmWs {
  __nv_bfloat16 *a, *b;
  int *ea, *eb, *err;
  int64_t m_cap, n_cap, k_cap;
  void carve(Carve& cv, int64_t Mmax, int64_t Nmax, int64_t Kmax) {
    m_cap = round_up(Mmax, EM_BM);
    n_cap = round_up(Nmax, EM_BN);
    k_cap = round_up(Kmax, EM_BK);
    a = cv.take<__nv_bfloat16>((size_t)kS * m_cap * k_cap);
    b = cv.take<__nv_bfloat16>((size_t)kS * n_cap * k_cap);
    ea = cv.take<int>((size_t)m_cap);
    eb = cv.take<int>((size_t)n_cap);
    err = cv.take<int>(64);
  }
};

size_t em_dgemm_ws(int64_t Mmax, int64_t Nmax, int64_t Kmax) {
  Carve c(nullptr, 0);
  EmWs w;
  w.carve(c, Mmax, Nmax, Kmax);
  return c.off;
}

// C (M x N, row stride ldc) = alpha A B (overwrite) or C += alpha A B, with
// A(m, k) = A[m a_rs + k a_cs] and B(k, n) = B[k b_rs + n b_cs] in FP64; the
// products on the tensor cores as described at the top of this file.  C may
// alias B's storage (the digits are taken before C is written).
int em_dgemm(int64_t M, int64_t N, int64_t K, const double* A, int64_t a_rs, int64_t a_cs,
             const double* B, int64_t b_rs, int64_t b_cs, double alpha, bool overwrite,
             double* C, int64_t ldc, void* ws, size_t ws_bytes, cudaStream_t s) {
  if (M <= 0 || N <= 0) return ISDF_OK;
  Carve cv(ws, ws_bytes);
  EmWs w;
  w.carve(cv, M, N, K > 0 ? K : 1);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  if (K <= 0) {
    if (overwrite)
      ISDF_CUDA(cudaMemset2DAsync(C, ldc * sizeof(double), 0, N * sizeof(double), M, s));
    return ISDF_OK;
  }
  const int64_t Mp = round_up(M, EM_BM), Np = round_up(N, EM_BN), Kp = round_up(K, EM_BK);
  em_row_exp_kernel<<<nblk(M, 8), 256, 0, s>>>(A, a_rs, a_cs, M, K, w.ea, w.err);
  ISDF_LAUNCH_CHECK();
  em_col_exp_kernel<<<nblk(N, 256), 256, 0, s>>>(B, b_rs, b_cs, K, N, w.eb, w.err);
  ISDF_LAUNCH_CHECK();
  em_split_rows_kernel<<<nblk(Mp * (Kp / 8), 256), 256, 0, s>>>(A, a_rs, a_cs, M, K, w.ea, Mp,
                                                                 Kp, w.a);
  ISDF_LAUNCH_CHECK();
  ISDF_CUDA(cudaFuncSetAttribute(em_split_cols_kernel,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SC_SMEM));
  em_split_cols_kernel<<<dim3((unsigned)ceil_div(Np, SC_N), (unsigned)ceil_div(Kp, SC_K)), 256,
                         SC_SMEM, s>>>(B, b_rs, b_cs, K, N, w.eb, Np, Kp, w.b);
  ISDF_LAUNCH_CHECK();
  EmMaps maps;
  memset(&maps, 0, sizeof(maps));
  for (int q = 0; q < kS; ++q) {
    ISDF_TRY(tma_map_bf16(&maps.a[q], w.a + (size_t)q * Mp * Kp, Mp, Kp, EM_BM));
    ISDF_TRY(tma_map_bf16(&maps.b[q], w.b + (size_t)q * Np * Kp, Np, Kp, EM_BN));
  }
  EmParams p;
  p.M = M;
  p.N = N;
  p.k_tiles = Kp / EM_BK;
  p.m_tiles = (int)(Mp / EM_BM);
  p.n_tiles = (int)(Np / EM_BN);
  // K chunks of <= 128 run in turn in one work unit (exact 64-bit sums) up to 8
  // of them; longer K is split over work units added with FP64 atomics
  const int kch = (int)ceil_div(Kp, EM_KCHUNK);
  p.kin = kch <= 8 ? kch : 1;
  p.kchunks = kch <= 8 ? 1 : kch;
  p.ea = w.ea;
  p.eb = w.eb;
  p.C = C;
  p.ldc = ldc;
  p.alpha = alpha;
  p.err = w.err;
  p.wait_ns = wait_limit_ns();
  if (p.kchunks == 1) {
    p.mode = overwrite ? 0 : 1;
  } else {
    if (overwrite)
      ISDF_CUDA(cudaMemset2DAsync(C, ldc * sizeof(double), 0, N * sizeof(double), M, s));
    p.mode = 2;
  }
  p.vec = ((uintptr_t)C % 16 == 0 && ldc % 2 == 0) ? 1 : 0;
  const int64_t units = (int64_t)p.m_tiles * p.n_tiles * p.kchunks;
  int dev = 0, nsm = 148;
  ISDF_CUDA(cudaGetDevice(&dev));
  ISDF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)(units < nsm ? units : nsm);
  ISDF_CUDA(cudaFuncSetAttribute(emgemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)EM_SMEM));
  emgemm_kernel<<<grid, EM_THREADS, EM_SMEM, s>>>(maps, p);
  ISDF_LAUNCH_CHECK();
  return ISDF_OK;
}

// The error word of the last em_dgemm on this workspace (device int).
int* em_err_word(void* ws, int64_t Mmax, int64_t Nmax, int64_t Kmax) {
  Carve cv(ws, ~size_t(0));
  EmWs w;
  w.carve(cv, Mmax, Nmax, Kmax);
  return w.err;
}

// Workspace of em_potrs_lower: the inverted diagonal blocks and one product's
// digit planes (at most n rows, nrhs columns, 128 inner terms).
size_t em_potrs_ws(int n, int64_t nrhs) {
  Carve c(nullptr, 0);
  c.take<double>((size_t)ceil_div(n, TRSM_TB) * TRSM_TB * TRSM_TB);
  EmWs w;
  w.carve(c, n, nrhs, TRSM_TB);
  return c.off;
}

// Solve (L L^T) X = B in place (B [n][nrhs], row stride ldb; L lower triangular
// [n][n]) by blocks of 128: each diagonal block is inverted once in FP64, and
// every block step is two emulated products,
//   forward   X_j = inv(L_jj) B_j,      B_r -= L_rj X_j     (r > j),
//   backward  X_j = inv(L_jj)^T Y_j,    Y_r -= L_jr^T X_j   (r < j).
int em_potrs_lower(const double* L, int n, double* B, int64_t nrhs, int64_t ldb, void* ws,
                   size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(L && B && n > 0 && nrhs > 0, "em_potrs_lower: empty arguments");
  Carve cv(ws, ws_bytes);
  const int nb = (int)ceil_div(n, TRSM_TB);
  double* Linv = cv.take<double>((size_t)nb * TRSM_TB * TRSM_TB);
  void* gws = (char*)ws + cv.off;
  const size_t gbytes = ws_bytes > cv.off ? ws_bytes - cv.off : 0;
  EmWs w;
  w.carve(cv, n, nrhs, TRSM_TB);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  const size_t smem = (size_t)TRSM_TB * TRSM_TB * sizeof(double);
  ISDF_CUDA(cudaFuncSetAttribute(trtri_blocks_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
  trtri_blocks_kernel<<<nb, TRSM_TB, smem, s>>>(L, n, Linv);
  ISDF_LAUNCH_CHECK();
  for (int j = 0; j < nb; ++j) {
    const int j0 = j * TRSM_TB, jb = n - j0 < TRSM_TB ? n - j0 : TRSM_TB;
    const double* Li = Linv + (size_t)j * TRSM_TB * TRSM_TB;
    double* Bj = B + (int64_t)j0 * ldb;
    ISDF_TRY(em_dgemm(jb, nrhs, jb, Li, TRSM_TB, 1, Bj, ldb, 1, 1.0, true, Bj, ldb, gws, gbytes,
                      s));
    const int rest = n - j0 - jb;
    if (rest > 0)
      ISDF_TRY(em_dgemm(rest, nrhs, jb, L + (int64_t)(j0 + jb) * n + j0, n, 1, Bj, ldb, 1, -1.0,
                        false, B + (int64_t)(j0 + jb) * ldb, ldb, gws, gbytes, s));
  }
  for (int j = nb - 1; j >= 0; --j) {
    const int j0 = j * TRSM_TB, jb = n - j0 < TRSM_TB ? n - j0 : TRSM_TB;
    const double* Li = Linv + (size_t)j * TRSM_TB * TRSM_TB;
    double* Bj = B + (int64_t)j0 * ldb;
    ISDF_TRY(em_dgemm(jb, nrhs, jb, Li, 1, TRSM_TB, Bj, ldb, 1, 1.0, true, Bj, ldb, gws, gbytes,
                      s));
    if (j0 > 0)
      ISDF_TRY(em_dgemm(j0, nrhs, jb, L + (int64_t)j0 * n, 1, n, Bj, ldb, 1, -1.0, false, B, ldb,
                        gws, gbytes, s));
  }
  return ISDF_OK;
}

}  // namespace isdf
