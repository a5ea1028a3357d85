// Orbitals and orbital gradients on the molecular grid (Alg. 2 step 2).
//
// Step 1 evaluates every contracted Cartesian Gaussian and its gradient at
// every grid point (one thread per point, consecutive threads on
// consecutive points so that the [f][g] stores are coalesced); step 2 is the
// AO -> MO contraction phi = C^T chi as an FP64 GEMM.
#include "linalg.cuh"

namespace isdf {
namespace {

__global__ void __launch_bounds__(128) ao_eval_kernel(isdf_basis b, const double* __restrict__ grid,
                                                      int64_t n_g, double* __restrict__ chi) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= n_g) return;
  const double gx = grid[3 * g], gy = grid[3 * g + 1], gz = grid[3 * g + 2];
  const int64_t plane = (int64_t)b.n_bf * n_g;
  for (int f = 0; f < b.n_bf; ++f) {
    const double x = gx - b.center[3 * f], y = gy - b.center[3 * f + 1],
                 z = gz - b.center[3 * f + 2];
    const double r2 = x * x + y * y + z * z;
    double e = 0.0, ae = 0.0;  // sum_k c_k exp(-a_k r2), sum_k a_k c_k exp(-a_k r2)
    for (int k = 0; k < b.n_prim; ++k) {
      const double a = b.exps[f * b.n_prim + k];
      const double t = a * r2;
      if (t < 746.0) {
        const double v = b.coefs[f * b.n_prim + k] * exp(-t);
        e += v;
        ae += a * v;
      }
    }
    const int px = b.powers[3 * f], py = b.powers[3 * f + 1], pz = b.powers[3 * f + 2];
    // x^p and p x^(p-1)
    double xp = 1.0, yp = 1.0, zp = 1.0, xm = 0.0, ym = 0.0, zm = 0.0;
    for (int i = 0; i < px; ++i) { xm = xp; xp *= x; }
    for (int i = 0; i < py; ++i) { ym = yp; yp *= y; }
    for (int i = 0; i < pz; ++i) { zm = zp; zp *= z; }
    xm *= px; ym *= py; zm *= pz;
    const double poly = xp * yp * zp;
    // d/dx [x^p exp(-a r^2)] = (p x^(p-1) - 2 a x^(p+1)) exp(-a r^2)
    const double gxv = (xm * e - 2.0 * x * xp * ae) * yp * zp;
    const double gyv = (ym * e - 2.0 * y * yp * ae) * xp * zp;
    const double gzv = (zm * e - 2.0 * z * zp * ae) * xp * yp;
    const int64_t o = (int64_t)f * n_g + g;
    chi[o] = poly * e;
    chi[plane + o] = gxv;
    chi[2 * plane + o] = gyv;
    chi[3 * plane + o] = gzv;
  }
}

}  // namespace

size_t em_dgemm_ws(int64_t Mmax, int64_t Nmax, int64_t Kmax);
int em_dgemm(int64_t M, int64_t N, int64_t K, const double* A, int64_t a_rs, int64_t a_cs,
             const double* B, int64_t b_rs, int64_t b_cs, double alpha, bool overwrite,
             double* C, int64_t ldc, void* ws, size_t ws_bytes, cudaStream_t s);

// mode 1 adds the workspace of the emulated products (n_orb <= the bound given).
size_t eval_orbitals_ws(int n_bf, int64_t n_g, int mode, int n_orb_max) {
  Carve c(nullptr, 0);
  c.take<double>((size_t)4 * n_bf * n_g);
  if (mode == 1) c.take<char>(em_dgemm_ws(n_orb_max, n_g, n_bf));
  return c.off;
}

int eval_orbitals(const isdf_basis* basis, const double* C, int n_orb, const double* grid,
                  int64_t n_g, double* phi, double* dphi, int mode, void* ws, size_t ws_bytes,
                  cudaStream_t s) {
  ISDF_ARG(basis && C && grid && phi && dphi, "null pointer argument");
  ISDF_ARG(n_orb > 0 && n_g > 0 && basis->n_bf > 0 && basis->n_prim > 0, "empty sizes");
  ISDF_ARG(mode == 0 || mode == 1, "mode must be 0 or 1");
  Carve cv(ws, ws_bytes);
  double* chi = cv.take<double>((size_t)4 * basis->n_bf * n_g);
  const size_t em_bytes = mode == 1 ? em_dgemm_ws(n_orb, n_g, basis->n_bf) : 0;
  char* em = mode == 1 ? cv.take<char>(em_bytes) : nullptr;
  ISDF_ARG(ws && cv.ok(), "workspace too small: need %zu bytes", cv.off);
  ao_eval_kernel<<<(unsigned)ceil_div(n_g, 128), 128, 0, s>>>(*basis, grid, n_g, chi);
  ISDF_LAUNCH_CHECK();
  const int64_t nbf = basis->n_bf;
  if (mode == 1) {
    // phi^c = C^T chi^c: A(m, k) = C[k][m]
    for (int c = 0; c < 4; ++c)
      ISDF_TRY(em_dgemm(n_orb, n_g, nbf, C, 1, n_orb, chi + c * nbf * n_g, n_g, 1, 1.0, true,
                        c == 0 ? phi : dphi + (int64_t)(c - 1) * n_orb * n_g, n_g, em, em_bytes,
                        s));
    return ISDF_OK;
  }
  Dgemm g;
  g.M = n_orb; g.N = n_g; g.K = nbf;
  g.A = C; g.a_rs = 1; g.a_cs = n_orb; g.a_bs = 0;
  g.B = chi; g.b_rs = n_g; g.b_cs = 1; g.b_bs = nbf * n_g;
  g.C = phi; g.ldc = n_g; g.c_bs = (int64_t)n_orb * n_g;
  ISDF_TRY(dgemm(g, s));
  g.B = chi + nbf * n_g; g.C = dphi; g.batch = 3;
  ISDF_TRY(dgemm(g, s));
  return ISDF_OK;
}

}  // namespace isdf
