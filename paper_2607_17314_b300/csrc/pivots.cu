// Interpolation-point selection by weighted pivoted Cholesky (Alg. 1, the
// gradient branch and the pivot fusion of Sec. II.D), matrix-free as in
// Sec. IV.B: each step generates one column S(., g*) from the orbitals at the
// pivot and all grid points, subtracts the previous Cholesky columns and
// updates the residual diagonal.
//
// One kernel launch per fused step; one thread per grid point.  Every sum is
// a chain of correctly rounded fused multiply-adds in a fixed order and the
// argmax takes the lowest index on ties, so the selected indices do not
// depend on the launch configuration.  The step state (union size, turn,
// per-channel counts and stop flags) and the argmax partials are double
// buffered so that no block reads what another block of the same launch
// writes.
#include "common.cuh"

namespace isdf {
namespace {

constexpr int PT = 256;

struct PivState {
  int nu;      // union size
  int turn;    // 0 = scalar next, 1 = gradient next
  int k[2];    // columns per channel
  int done[2]; // channel stopped
};

struct PivArgs {
  const double* phi;   // [n_orb][n_g]
  const double* dphi;  // [3][n_orb][n_g]
  const double* w;     // [n_g]
  int64_t n_g;
  int n_orb;
  int n_mu;
  int cap;             // columns per channel in L
  int rank[2];         // mode 3: steps per channel
  double* d;           // [2][n_g]
  double* L;           // [2][cap][n_g]
  double* part_v;      // [2 ch][2 buf][nblk]
  int* part_i;         // [2 ch][2 buf][nblk]
  int nblk;
  PivState* st;        // [2]
  double* tol;         // [2]
  unsigned char* in_union;  // [n_g]
  int* union_piv;      // [n_mu]
  int* err;            // device error word
};

__device__ __forceinline__ void better(double& bv, int& bi, double v, int i) {
  if (v > bv || (v == bv && i < bi)) { bv = v; bi = i; }
}

// Block-wide (max, lowest index) reduction; result valid in thread 0.
__device__ void block_argmax(double& v, int& i) {
  __shared__ double sv[PT / 32];
  __shared__ int si[PT / 32];
  for (int o = 16; o > 0; o >>= 1) {
    double ov = __shfl_down_sync(0xffffffffu, v, o);
    int oi = __shfl_down_sync(0xffffffffu, i, o);
    better(v, i, ov, oi);
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sv[w] = v; si[w] = i; }
  __syncthreads();
  if (w == 0) {
    v = l < PT / 32 ? sv[l] : -1.0;
    i = l < PT / 32 ? si[l] : 0x7fffffff;
    for (int o = 16; o > 0; o >>= 1) {
      double ov = __shfl_down_sync(0xffffffffu, v, o);
      int oi = __shfl_down_sync(0xffffffffu, i, o);
      better(v, i, ov, oi);
    }
  }
  __syncthreads();
}

__global__ void __launch_bounds__(PT) diag_init_kernel(PivArgs a) {
  const int64_t g = (int64_t)blockIdx.x * PT + threadIdx.x;
  double d0 = -1.0, d1 = -1.0;
  if (g < a.n_g) {
    double t1 = 0.0, t2 = 0.0;
    for (int p = 0; p < a.n_orb; ++p) {
      double v = a.phi[(int64_t)p * a.n_g + g];
      t1 = __fma_rn(v, v, t1);
    }
    for (int c = 0; c < 3; ++c)
      for (int p = 0; p < a.n_orb; ++p) {
        double v = a.dphi[((int64_t)c * a.n_orb + p) * a.n_g + g];
        t2 = __fma_rn(v, v, t2);
      }
    double ww = __dmul_rn(a.w[g], a.w[g]);
    d0 = __dmul_rn(ww, __dmul_rn(t1, t1));
    d1 = __dmul_rn(ww, __dmul_rn(t1, t2));
    a.d[g] = d0;
    a.d[a.n_g + g] = d1;
    // a NaN or Inf in phi, dphi or w reaches both diagonals
    if (!isfinite(d0) || !isfinite(d1)) atomicOr(a.err, DEV_ERR_NONFINITE);
  }
  int i0 = g < a.n_g ? (int)g : 0x7fffffff, i1 = i0;
  block_argmax(d0, i0);
  block_argmax(d1, i1);
  if (threadIdx.x == 0) {
    // channel c, buffer 0
    a.part_v[(0 * 2 + 0) * a.nblk + blockIdx.x] = d0;
    a.part_i[(0 * 2 + 0) * a.nblk + blockIdx.x] = i0;
    a.part_v[(1 * 2 + 0) * a.nblk + blockIdx.x] = d1;
    a.part_i[(1 * 2 + 0) * a.nblk + blockIdx.x] = i1;
  }
}

// Reduce the partials of channel c / buffer b to (max, argmax) in every thread.
__device__ void reduce_partials(const PivArgs& a, int c, int b, double& bv, int& bi) {
  bv = -1.0;
  bi = 0x7fffffff;
  const double* pv = a.part_v + (c * 2 + b) * a.nblk;
  const int* pi = a.part_i + (c * 2 + b) * a.nblk;
  for (int j = threadIdx.x; j < a.nblk; j += PT) better(bv, bi, pv[j], pi[j]);
  block_argmax(bv, bi);
  __shared__ double rv;
  __shared__ int ri;
  if (threadIdx.x == 0) { rv = bv; ri = bi; }
  __syncthreads();
  bv = rv;
  bi = ri;
}

__global__ void __launch_bounds__(PT) tol_init_kernel(PivArgs a) {
  for (int c = 0; c < 2; ++c) {
    double v;
    int i;
    reduce_partials(a, c, 0, v, i);
    if (threadIdx.x == 0) a.tol[c] = 64.0 * 2.220446049250313e-16 * v;
  }
  if (threadIdx.x == 0) {
    PivState s0 = {0, 0, {0, 0}, {0, 0}};
    a.st[0] = s0;
    a.st[1] = s0;
  }
}

__global__ void __launch_bounds__(PT) pivot_step_kernel(PivArgs a, int parity, int mode) {
  const PivState s = a.st[parity];
  PivState ns = s;
  bool active = s.nu < a.n_mu && !(s.done[0] && s.done[1]);
  int c = s.turn;
  if (active && s.done[c]) c = 1 - c;
  if (mode == 1) c = 0;
  if (mode == 2) c = 1;
  if (mode == 3) c = s.done[0] ? 1 : 0;  // the scalar channel to its rank, then the gradient one
  double dgs = 0.0;
  int gs = 0;
  if (active) {
    reduce_partials(a, c, s.k[c] & 1, dgs, gs);
    const int cap = mode == 3 ? a.rank[c] : a.cap;
    if (s.k[c] >= cap || !(dgs > a.tol[c])) {
      ns.done[c] = 1;
      if (mode == 1 || mode == 2) ns.done[1 - c] = 1;
      ns.turn = 1 - s.turn;
      active = false;
    }
  }
  if (!active) {
    if (blockIdx.x == 0 && threadIdx.x == 0) a.st[1 - parity] = ns;
    return;
  }
  const int k = s.k[c];
  const int64_t n_g = a.n_g;
  const int64_t g = (int64_t)blockIdx.x * PT + threadIdx.x;
  double* dc = a.d + c * n_g;
  const double* Lc = a.L + (int64_t)c * a.cap * n_g;
  double nd = -1.0;
  int ni = 0x7fffffff;
  if (g < n_g) {
    double t1 = 0.0;
    for (int p = 0; p < a.n_orb; ++p) {
      const double* row = a.phi + (int64_t)p * n_g;
      t1 = __fma_rn(row[g], row[gs], t1);
    }
    double sgh;
    const double wgw = __dmul_rn(a.w[g], a.w[gs]);
    if (c == 1) {
      double t2 = 0.0;
      for (int cc = 0; cc < 3; ++cc)
        for (int p = 0; p < a.n_orb; ++p) {
          const double* row = a.dphi + ((int64_t)cc * a.n_orb + p) * n_g;
          t2 = __fma_rn(row[g], row[gs], t2);
        }
      sgh = __dmul_rn(wgw, __dmul_rn(t1, t2));
    } else {
      sgh = __dmul_rn(wgw, __dmul_rn(t1, t1));
    }
    for (int l = 0; l < k; ++l) {
      const double* Ll = Lc + (int64_t)l * n_g;
      sgh = __fma_rn(-Ll[g], Ll[gs], sgh);
    }
    const double v = __ddiv_rn(sgh, __dsqrt_rn(dgs));
    a.L[((int64_t)c * a.cap + k) * n_g + g] = v;
    double x = __fma_rn(-v, v, dc[g]);
    x = x > 0.0 ? x : 0.0;
    if (g == gs) x = 0.0;
    dc[g] = x;
    nd = x;
    ni = (int)g;
  }
  block_argmax(nd, ni);
  if (threadIdx.x == 0) {
    const int b = (k + 1) & 1;
    a.part_v[(c * 2 + b) * a.nblk + blockIdx.x] = nd;
    a.part_i[(c * 2 + b) * a.nblk + blockIdx.x] = ni;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ns.k[c] = k + 1;
    if (!a.in_union[gs]) {
      a.in_union[gs] = 1;
      a.union_piv[s.nu] = gs;
      ns.nu = s.nu + 1;
    }
    ns.turn = 1 - s.turn;
    a.st[1 - parity] = ns;
  }
}

}  // namespace

// Workspace of a selection with `cap` Cholesky columns per channel and at most
// n_mu union points.
static size_t points_ws_cap(int64_t n_g, int n_mu, int cap) {
  Carve c(nullptr, 0);
  int nblk = (int)ceil_div(n_g, PT);
  c.take<int>(64);
  c.take<double>(2 * (size_t)n_g);
  c.take<double>(2 * (size_t)cap * n_g);
  c.take<double>(4 * (size_t)nblk);
  c.take<int>(4 * (size_t)nblk);
  c.take<PivState>(2);
  c.take<double>(2);
  c.take<unsigned char>(n_g);
  c.take<int>(n_mu);
  return c.off;
}

size_t points_ws(int64_t n_g, int n_mu) { return points_ws_cap(n_g, n_mu, n_mu); }

size_t points_ranks_ws(int64_t n_g, int n_phi, int n_grad) {
  return points_ws_cap(n_g, n_phi + n_grad, n_phi > n_grad ? n_phi : n_grad);
}

// Modes 0-2 (fused alternating, scalar, gradient) select n_mu points; mode 3
// (the paper's fusion) runs the scalar channel to rank n_phi and the gradient
// channel to rank n_grad, with n_mu = n_phi + n_grad bounding the union.
static int points_run(const double* phi, const double* dphi, const double* w, int64_t n_g,
                      int n_orb, int n_mu, int mode, int n_phi, int n_grad, int32_t* pivots,
                      int* n_mu_out, void* ws, size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(phi && dphi && w && pivots && n_mu_out, "null pointer argument");
  ISDF_ARG(n_g > 0 && n_orb > 0 && n_mu > 0, "empty sizes");
  ISDF_ARG(n_g < 0x7fffffff, "n_g must fit in int32");
  ISDF_ARG(mode >= 0 && mode <= 3, "mode must be 0, 1, 2 or 3");
  PivArgs a;
  a.phi = phi; a.dphi = dphi; a.w = w; a.n_g = n_g; a.n_orb = n_orb; a.n_mu = n_mu;
  a.cap = mode == 3 ? (n_phi > n_grad ? n_phi : n_grad) : n_mu;
  a.rank[0] = n_phi;
  a.rank[1] = n_grad;
  a.nblk = (int)ceil_div(n_g, PT);
  Carve cv(ws, ws_bytes);
  a.err = cv.take<int>(64);
  a.d = cv.take<double>(2 * (size_t)n_g);
  a.L = cv.take<double>(2 * (size_t)a.cap * n_g);
  a.part_v = cv.take<double>(4 * (size_t)a.nblk);
  a.part_i = cv.take<int>(4 * (size_t)a.nblk);
  a.st = cv.take<PivState>(2);
  a.tol = cv.take<double>(2);
  a.in_union = cv.take<unsigned char>(n_g);
  a.union_piv = cv.take<int>(n_mu);
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  ISDF_CUDA(cudaMemsetAsync(a.in_union, 0, n_g, s));
  ISDF_CUDA(cudaMemsetAsync(a.err, 0, sizeof(int), s));
  diag_init_kernel<<<a.nblk, PT, 0, s>>>(a);
  ISDF_LAUNCH_CHECK();
  tol_init_kernel<<<1, PT, 0, s>>>(a);
  ISDF_LAUNCH_CHECK();
  int h_err = 0;
  ISDF_CUDA(cudaMemcpyAsync(&h_err, a.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  ISDF_CUDA(cudaStreamSynchronize(s));
  if (h_err & DEV_ERR_NONFINITE) {
    set_error("non-finite phi, dphi or w: a pivot diagonal is NaN or Inf");
    return ISDF_E_NONFINITE;
  }
  const int max_iter = 2 * n_mu + 4;
  // Steps run in batches of 32 launches replayed from a CUDA graph on a private
  // stream (the launch cost dominates the short steps of small grids); the host
  // reads the step state between batches to stop.  Steps past the end are no-ops.
  constexpr int kBatch = 32;
  cudaStream_t ps = nullptr;
  ISDF_CUDA(cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool use_graph = false;
  if (cudaStreamBeginCapture(ps, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    for (int b = 0; b < kBatch; ++b) pivot_step_kernel<<<a.nblk, PT, 0, ps>>>(a, b & 1, mode);
    if (cudaStreamEndCapture(ps, &graph) == cudaSuccess &&
        cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess)
      use_graph = true;
  }
  (void)cudaGetLastError();
  PivState h;
  int it = 0;
  int rc = ISDF_OK;
  for (;;) {
    if (use_graph) {
      if (cudaGraphLaunch(exec, ps) != cudaSuccess) { rc = ISDF_E_CUDA; break; }
      for (int b = 0; b < kBatch; ++b) count_launch();
      it += kBatch;
    } else {
      for (int b = 0; b < kBatch && it < max_iter; ++b, ++it) {
        pivot_step_kernel<<<a.nblk, PT, 0, ps>>>(a, it & 1, mode);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) { rc = ISDF_E_CUDA; break; }
      }
      if (rc != ISDF_OK) break;
    }
    if (cudaMemcpyAsync(&h, a.st + (it & 1), sizeof(PivState), cudaMemcpyDeviceToHost, ps) !=
            cudaSuccess ||
        cudaStreamSynchronize(ps) != cudaSuccess) {
      rc = ISDF_E_CUDA;
      break;
    }
    if (h.nu >= n_mu || (h.done[0] && h.done[1]) || it >= max_iter) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(ps);
  if (rc != ISDF_OK) {
    set_error("pivot step launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    return rc;
  }
  *n_mu_out = h.nu;
  if (h.nu > 0)
    ISDF_CUDA(cudaMemcpyAsync(pivots, a.union_piv, sizeof(int) * h.nu, cudaMemcpyDeviceToDevice, s));
  ISDF_CUDA(cudaStreamSynchronize(s));
  if (mode == 3) {
    if (h.k[0] < n_phi || h.k[1] < n_grad) {
      set_error("rank exhausted: %d of %d scalar and %d of %d gradient steps", h.k[0], n_phi,
                h.k[1], n_grad);
      return ISDF_E_RANK;
    }
    return ISDF_OK;
  }
  if (h.nu < n_mu) {
    set_error("rank exhausted: %d of %d points", h.nu, n_mu);
    return ISDF_E_RANK;
  }
  return ISDF_OK;
}

int points(const double* phi, const double* dphi, const double* w, int64_t n_g, int n_orb,
           int n_mu, int mode, int32_t* pivots, int* n_mu_out, void* ws, size_t ws_bytes,
           cudaStream_t s) {
  ISDF_ARG(mode >= 0 && mode <= 2, "mode must be 0, 1 or 2");
  return points_run(phi, dphi, w, n_g, n_orb, n_mu, mode, 0, 0, pivots, n_mu_out, ws, ws_bytes,
                    s);
}

int points_ranks(const double* phi, const double* dphi, const double* w, int64_t n_g, int n_orb,
                 int n_phi, int n_grad, int32_t* pivots, int* n_mu_out, void* ws,
                 size_t ws_bytes, cudaStream_t s) {
  ISDF_ARG(n_phi >= 0 && n_grad >= 0 && n_phi + n_grad > 0, "channel ranks must be >= 0 with a "
           "positive sum");
  return points_run(phi, dphi, w, n_g, n_orb, n_phi + n_grad, 3, n_phi, n_grad, pivots, n_mu_out,
                    ws, ws_bytes, s);
}

}  // namespace isdf
