// Closed-shell test energies from the ISDF factors, occupied block only
// (Eqs. K1-isdf, K3-isdf, K-recombine-final, delta-u-dx-kernels, xtc-deltah,
// xtc-const), FP64.
//
//   Cs[mu][(q,s)] = phi_q(r_mu) phi_s(r_mu),  Ct^c[mu][(p,r)] = phi_p(r_mu) d_c phi_r(r_mu)
//   K1[(p,r),(q,s)] = sum_c Ct^c^T W^c Cs,  K3 = Cs^T W^3 Cs
//   T = K1 - K1swap + K3,  K^{pq}_{rs} = (T^{pq}_{rs} + T^{qp}_{sr}) / 2
//   DeltaU^{pq}_{rs} = -(U^{pq}_{rs} + U^{qp}_{sr}),  U = Cs^T D Cs - Cs^T X
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "linalg.cuh"

namespace isdf {
namespace {

inline unsigned nb(int64_t n, int t = 256) { return (unsigned)ceil_div(n, t); }

// Cs[mu][q*n + s] and Ct[c][mu][p*n + r]
__global__ void factors_kernel(const double* phiP, const double* dphiP, int n_mu, int n_orb,
                               int n, double* Cs, double* Ct) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n2 = (int64_t)n * n;
  if (e >= (int64_t)n_mu * n2) return;
  int mu = (int)(e / n2);
  int ab = (int)(e % n2);
  int a = ab / n, b = ab % n;
  const double* row = phiP + (int64_t)mu * n_orb;
  Cs[e] = row[a] * row[b];
  for (int c = 0; c < 3; ++c)
    Ct[c * n_mu * n2 + e] = row[a] * dphiP[((int64_t)c * n_mu + mu) * n_orb + b];
}

// Xo[(q,s)][mu] from the packed rows s(s+1)/2 + q (q <= s), symmetric.
__global__ void unpack_x_kernel(const double* Xp, int n_mu, int n, double* Xo) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int64_t n2 = (int64_t)n * n;
  if (e >= n2 * n_mu) return;
  int mu = (int)(e % n_mu);
  int qs = (int)(e / n_mu);
  int q = qs / n, s = qs % n;
  int lo = q < s ? q : s, hi = q < s ? s : q;
  Xo[e] = Xp[((int64_t)hi * (hi + 1) / 2 + lo) * n_mu + mu];
}

__global__ void energy_kernel(const double* K1, const double* K3, const double* DCD,
                              const double* XC, int n, double* out) {
  const int n2 = n * n;
  auto at = [&](const double* M, int p, int q, int r, int s) {
    return M[(int64_t)(p * n + r) * n2 + (q * n + s)];
  };
  auto T = [&](int p, int q, int r, int s) {
    return at(K1, p, q, r, s) - at(K1, r, s, p, q) + at(K3, p, q, r, s);
  };
  auto Kt = [&](int p, int q, int r, int s) { return 0.5 * (T(p, q, r, s) + T(q, p, s, r)); };
  auto U = [&](int p, int q, int r, int s) { return at(DCD, p, q, r, s) - at(XC, p, q, r, s); };
  auto dU = [&](int p, int q, int r, int s) { return -(U(p, q, r, s) + U(q, p, s, r)); };
  __shared__ double sk[256], su[256];
  double ek = 0.0, eu = 0.0;
  for (int ij = threadIdx.x; ij < n2; ij += blockDim.x) {
    int i = ij / n, j = ij % n;
    ek += 2.0 * Kt(i, j, i, j) - Kt(i, j, j, i);
    eu += 2.0 * dU(i, j, i, j) - dU(i, j, j, i);
  }
  sk[threadIdx.x] = ek;
  su[threadIdx.x] = eu;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      sk[threadIdx.x] += sk[threadIdx.x + o];
      su[threadIdx.x] += su[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = sk[0];
    out[1] = su[0];
    // Delta h_ii = -1/2 sum_o (2 dU^{io}_{io} - dU^{io}_{oi});  E0 = -2/3 sum_i Delta h_ii
    out[2] = (-2.0 / 3.0) * (-0.5) * su[0];
  }
}

}  // namespace

size_t energies_ws(int n_mu, int n_occ) {
  Carve c(nullptr, 0);
  const size_t n2 = (size_t)n_occ * n_occ;
  c.take<double>(n_mu * n2);      // Cs
  c.take<double>(3 * n_mu * n2);  // Ct
  c.take<double>(n_mu * n2);      // Y
  c.take<double>(n2 * n_mu);      // Xo
  for (int i = 0; i < 4; ++i) c.take<double>(n2 * n2);  // K1, K3, DCD, XC
  c.take<double>(4);
  return c.off;
}

int energies(const double* W, const double* D, const double* Xp, const double* phiP,
             const double* dphiP, int n_mu, int n_orb, int n, double* out_host, void* ws,
             size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(W && D && Xp && phiP && dphiP && out_host, "null pointer argument");
  ISDF_ARG(n > 0 && n <= n_orb && n_mu > 0, "bad sizes");
  const int64_t n2 = (int64_t)n * n;
  Carve cv(ws, ws_bytes);
  double* Cs = cv.take<double>(n_mu * n2);
  double* Ct = cv.take<double>(3 * n_mu * n2);
  double* Y = cv.take<double>(n_mu * n2);
  double* Xo = cv.take<double>(n2 * n_mu);
  double* K1 = cv.take<double>(n2 * n2);
  double* K3 = cv.take<double>(n2 * n2);
  double* DCD = cv.take<double>(n2 * n2);
  double* XC = cv.take<double>(n2 * n2);
  double* out = cv.take<double>(4);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  factors_kernel<<<nb(n_mu * n2), 256, 0, s>>>(phiP, dphiP, n_mu, n_orb, n, Cs, Ct);
  ISDF_LAUNCH_CHECK();
  unpack_x_kernel<<<nb(n2 * n_mu), 256, 0, s>>>(Xp, n_mu, n, Xo);
  ISDF_LAUNCH_CHECK();
  const int64_t nn = (int64_t)n_mu * n_mu;
  // Y = M Cs ; then out = L^T Y with L = Ct^c or Cs
  auto mCs = [&](const double* M) {
    Dgemm g;
    g.M = n_mu; g.N = n2; g.K = n_mu;
    g.A = M; g.a_rs = n_mu; g.a_cs = 1; g.a_bs = 0;
    g.B = Cs; g.b_rs = n2; g.b_cs = 1; g.b_bs = 0;
    g.C = Y; g.ldc = n2; g.c_bs = 0;
    return dgemm(g, s);
  };
  auto lty = [&](const double* Lm, double* C, double beta) {
    Dgemm g;
    g.M = n2; g.N = n2; g.K = n_mu;
    g.A = Lm; g.a_rs = 1; g.a_cs = n2; g.a_bs = 0;
    g.B = Y; g.b_rs = n2; g.b_cs = 1; g.b_bs = 0;
    g.C = C; g.ldc = n2; g.c_bs = 0;
    g.beta = beta;
    return dgemm(g, s);
  };
  for (int c = 0; c < 3; ++c) {
    ISDF_TRY(mCs(W + c * nn));
    ISDF_TRY(lty(Ct + (int64_t)c * n_mu * n2, K1, c == 0 ? 0.0 : 1.0));
  }
  ISDF_TRY(mCs(W + 3 * nn));
  ISDF_TRY(lty(Cs, K3, 0.0));
  ISDF_TRY(mCs(D));
  ISDF_TRY(lty(Cs, DCD, 0.0));
  {
    // XC[(p,r),(q,s)] = sum_mu Cs[mu][(p,r)] Xo[(q,s)][mu]
    Dgemm g;
    g.M = n2; g.N = n2; g.K = n_mu;
    g.A = Cs; g.a_rs = 1; g.a_cs = n2; g.a_bs = 0;
    g.B = Xo; g.b_rs = 1; g.b_cs = n_mu; g.b_bs = 0;
    g.C = XC; g.ldc = n2; g.c_bs = 0;
    ISDF_TRY(dgemm(g, s));
  }
  energy_kernel<<<1, 256, 0, s>>>(K1, K3, DCD, XC, n, out);
  ISDF_LAUNCH_CHECK();
  ISDF_CUDA(cudaMemcpyAsync(out_host, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  ISDF_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(out_host[i])) {
      set_error("energy %d is not finite (NaN or Inf in W, D, X or the pivot factors)", i);
      return ISDF_E_NONFINITE;
    }
  return ISDF_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the energies call.
//
// Some callers cannot allocate device memory: code that runs inside another
// framework's memory pool (cudaMalloc may synchronise the device and
// fragments a pool it does not own) and latency-critical loops that must not
// block on an allocator.  For them the scratch of the energies call lives in
// one fixed device array of this library instead of a caller workspace.  The
// array is kEnergiesScratchBytes large and every GPU that loads the library
// holds it until the process exits.  Its device address is looked up with the
// device current on the first call in each CUDA context of that device: once
// per device, and once more after a cudaDeviceReset, which ends the context
// that held the array (the module is loaded again, possibly elsewhere); make
// that first call before any stream capture.  All calls share the array and
// it keeps the last call's contents: every region the energies path reads is
// written earlier in the same call, so nothing needs clearing, but calls that
// overlap on the GPU (other streams, other host threads) race on it.

namespace {

constexpr size_t kEnergiesScratchBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_energies_scratch[kEnergiesScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Unique id of the calling thread's current context (0 if unavailable).
unsigned long long current_context_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_cur = (CtxGetCurrentFn)p;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = (CtxGetIdFn)p;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur && get_id && get_cur(&ctx) == CUDA_SUCCESS && ctx) get_id(ctx, &id);
  return id;
}

int scratch_address(void** out) {
  int dev = 0;
  ISDF_CUDA(cudaGetDevice(&dev));
  ISDF_ARG(dev >= 0 && dev < kMaxDevices, "device ordinal %d beyond the scratch table", dev);
  const unsigned long long ctx = current_context_id();
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_energies_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cudaGetSymbolAddress of the energies scratch failed on device %d: %s", dev,
                cudaGetErrorString(e));
      return ISDF_E_CUDA;
    }
    g_scratch_addr[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_addr[dev];
  return ISDF_OK;
}

}  // namespace

int energies_noalloc(const double* W, const double* D, const double* Xp, const double* phiP,
                     const double* dphiP, int n_mu, int n_orb, int n, double* out_host,
                     cudaStream_t s) {
  ISDF_ARG(n > 0 && n <= n_orb && n_mu > 0, "bad sizes");
  const size_t need = energies_ws(n_mu, n);
  ISDF_ARG(need <= kEnergiesScratchBytes,
           "n_mu = %d with n_occ = %d needs %zu bytes of scratch; the allocation-free call "
           "holds %zu bytes (use tc_energies with a workspace)",
           n_mu, n, need, kEnergiesScratchBytes);
  void* scratch = nullptr;
  ISDF_TRY(scratch_address(&scratch));
  return energies(W, D, Xp, phiP, dphiP, n_mu, n_orb, n, out_host, scratch,
                  kEnergiesScratchBytes, s);
}

}  // namespace isdf
