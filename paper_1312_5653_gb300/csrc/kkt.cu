// Full-space method of Sec. 3.2 (arXiv 1312.5653): the KKT operator of Sec. 2, the block-diagonal
// preconditioner P_mgw = diag(M, beta M, S) of Eq. murphypreconditioner with its S block applied
// through the factored Schur solve, and preconditioned MINRES; plus the FP64 S apply of Sec. 3.1.
// M^{-1} is a fixed-degree Chebyshev iteration with Jacobi scaling: the eigenvalues of D^{-1} M for
// Q1 mass on uniform grids lie in (2^-d, (3/2)^d) (tensor products of the 1D range (1/2, 3/2)), so
// the degree fixes the accuracy and the operator is linear, as MINRES requires.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "api_internal.h"
#include "outer.h"

namespace schur {

#define KKT_CK(call)                                                                 \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return set_error(e_ == cudaErrorMemoryAllocation ? SCHUR_ENOMEM : SCHUR_ECUDA, \
                       std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

// x += d; r -= Ad; d = c1 d + c2 D^{-1} r   (one Chebyshev step, all columns)
__global__ void k_cheb_step(long long n, int R, double* x, double* r, double* d, const double* __restrict__ Ad, int ld,
                            double c1, double c2, double dinv, int first) {
  const int c = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    size_t k = (size_t)c * ld + i;
    if (first) {
      d[k] = c2 * dinv * r[k];
      x[k] = 0.0;
      continue;
    }
    x[k] += d[k];
    r[k] -= Ad[k];
    d[k] = c1 * d[k] + c2 * dinv * r[k];
  }
}

__global__ void k_copy_cols(long long n, int R, const double* __restrict__ src, int lds, double* dst, int ldd,
                            double scale) {
  const int c = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    dst[(size_t)c * ldd + i] = scale * src[(size_t)c * lds + i];
}

// y = a0 x0 + a1 x1 + a2 x2 (per-column coefficients coef[c*3 + k]; a null x_k is skipped)
__global__ void k_lin3(long long n, int R, double* y, int ldy, const double* __restrict__ coef, const double* x0,
                       const double* x1, const double* x2, int ldx) {
  const int c = blockIdx.y;
  const double a0 = coef[c * 3], a1 = coef[c * 3 + 1], a2 = coef[c * 3 + 2];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    size_t k = (size_t)c * ldx + i;
    double v = a0 * x0[k];
    if (x1) v += a1 * x1[k];
    if (x2) v += a2 * x2[k];
    y[(size_t)c * ldy + i] = v;
  }
}

// Full-grid node of interior node i (coordinates 1..nel-1 per axis) shifted by offset o (3^dim
// neighbourhood), as an index into a vector over all prod(nel[a] + 1) grid nodes, boundary included.
__device__ __forceinline__ long long full_index(const Geom& g, long long i, int o) {
  const long long m0 = g.nel[0] - 1, m1 = g.nel[1] - 1;
  long long G0 = i % m0 + 1, t = i / m0, G1, G2;
  if (g.dim == 2) {
    G1 = t + 1;
    G2 = 0;
  } else {
    G1 = t % m1 + 1;
    G2 = t / m1 + 1;
  }
  G0 += o % 3 - 1;
  G1 += (o / 3) % 3 - 1;
  if (g.dim == 3) G2 += o / 9 - 1;
  return G0 + (long long)(g.nel[0] + 1) * (G1 + (long long)(g.nel[1] + 1) * G2);
}

__device__ __forceinline__ bool full_on_boundary(const Geom& g, long long f) {
  const long long e0 = g.nel[0] + 1, e1 = g.nel[1] + 1;
  const long long c0 = f % e0, c1 = (f / e0) % e1, c2 = f / (e0 * e1);
  return c0 == 0 || c0 == g.nel[0] || c1 == 0 || c1 == g.nel[1] || (g.dim == 3 && (c2 == 0 || c2 == g.nel[2]));
}

// out = K ybar + K_c y_c on the interior nodes: the stiffness rows of the interior nodes applied to a
// vector over the whole grid whose boundary values are the Dirichlet data (Sec. 2: the constraint
// K y + K_c y_c = M u, and the right-hand side of Eq. schurcomplementsystem).
__global__ void k_full_stiffness(Geom g, Coef27 cf, const double* __restrict__ yfull, int ldf, double* out, int ld,
                                 int R) {
  const int r = blockIdx.y;
  const int noff = g.dim == 2 ? 9 : 27;
  const double* yf = yfull + (size_t)r * ldf;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.n; i += (long long)gridDim.x * blockDim.x) {
    double acc = 0;
    for (int o = 0; o < noff; ++o) acc += cf.c[o].re * yf[full_index(g, i, o)];
    out[(size_t)r * ld + i] = acc;
  }
}

// y = ybar - w and u = lambda / beta on the interior nodes (Eq. updateyandu, w = M^{-1} K lambda)
__global__ void k_control_update(Geom g, const double* __restrict__ yfull, int ldf, const double* __restrict__ w,
                                 const double* __restrict__ lam, int ldw, double inv_beta, double* y, double* u,
                                 int ld, int R) {
  const int r = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.n; i += (long long)gridDim.x * blockDim.x) {
    const double yb = yfull[(size_t)r * ldf + full_index(g, i, g.dim == 2 ? 4 : 13)];
    y[(size_t)r * ld + i] = yb - w[(size_t)r * ldw + i];
    u[(size_t)r * ld + i] = lam[(size_t)r * ldw + i] * inv_beta;
  }
}

// v = K y + K_c y_c - M u (the residual of the state equation, Eq. relativeconstraintviolation):
// interior neighbours take y, boundary neighbours the Dirichlet data of yfull
__global__ void k_constraint(Geom g, Coef27 cf, const double* __restrict__ y, const double* __restrict__ u, int ld,
                             const double* __restrict__ yfull, int ldf, double* v, int ldv, int R) {
  const int r = blockIdx.y;
  const int noff = g.dim == 2 ? 9 : 27;
  const long long s1 = g.nel[0] - 1, s2 = s1 * (g.nel[1] - 1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.n; i += (long long)gridDim.x * blockDim.x) {
    double acc = 0;
    for (int o = 0; o < noff; ++o) {
      const long long f = full_index(g, i, o);
      if (full_on_boundary(g, f)) {
        acc += cf.c[o].re * yfull[(size_t)r * ldf + f];
      } else {
        const int d0 = o % 3 - 1, d1 = (o / 3) % 3 - 1, d2 = g.dim == 3 ? o / 9 - 1 : 0;
        const long long q = i + d0 + s1 * d1 + s2 * d2;
        acc += cf.c[o].re * y[(size_t)r * ld + q] - cf.c[o].im * u[(size_t)r * ld + q];
      }
    }
    v[(size_t)r * ldv + i] = acc;
  }
}

static int grid_for(long long n) { return std::max(1, (int)std::min<long long>((n + 255) / 256, 8 * 152)); }

// w = M^{-1} t by `deg` Chebyshev steps (columns of length n, leading dimension ld); uses 3
// scratch columns blocks of n x R.
static int mass_inverse(schur_ctx* c, const double* t, int ldt, double* w, int ldw, int R, int deg, double* scr,
                        cudaStream_t st) {
  const Geom& g = c->mp->hm.g;
  const long long n = g.n;
  const double lo = std::pow(0.5, g.dim), hi = std::pow(1.5, g.dim);
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  const double dinv = 1.0 / stencil_diag(g, 0);
  double* r = scr;
  double* d = scr + (size_t)n * R;
  double* Ad = scr + 2 * (size_t)n * R;
  Coef27 sten = make_coef(g, 1.0);
  const int gs = grid_for(n);
  k_copy_cols<<<dim3(gs, R), 256, 0, st>>>(n, R, t, ldt, r, (int)n, 1.0);
  KKT_CK(cudaGetLastError());
  double rho = 1.0 / sigma;
  // d0 = D^{-1} r0 / theta; x0 = 0
  k_cheb_step<<<dim3(gs, R), 256, 0, st>>>(n, R, w, r, d, Ad, (int)n, 0.0, 1.0 / theta, dinv, 1);
  KKT_CK(cudaGetLastError());
  for (int k = 1; k <= deg; ++k) {
    k_apply_real<<<dim3(gs, R), 256, 0, st>>>(g, sten, 0, d, (int)n, Ad, (int)n, R, 1.0, 0.0);
    KKT_CK(cudaGetLastError());
    double rho_new = 1.0 / (2.0 * sigma - rho);
    double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
    if (k == deg) {
      // last step: x += d only (x_k = x_{k-1} + d_{k-1})
      c1 = 0.0;
      c2 = 0.0;
    }
    k_cheb_step<<<dim3(gs, R), 256, 0, st>>>(n, R, w, r, d, Ad, (int)n, c1, c2, dinv, 0);
    KKT_CK(cudaGetLastError());
    rho = rho_new;
  }
  if (ldw != (int)n) return set_error(SCHUR_EINVAL, "internal: mass_inverse expects ld == n");
  return SCHUR_OK;
}

static int cheb_degree(int dim, double tol) {
  double kappa = std::pow(3.0, dim);  // (3/2)^d / (1/2)^d
  double rho = (std::sqrt(kappa) - 1.0) / (std::sqrt(kappa) + 1.0);
  return (int)std::ceil(std::log(tol / 2.0) / std::log(rho)) + 1;
}

static int kkt_ws(schur_ctx* c, int R) {
  if (R <= c->kkt_R) return SCHUR_OK;
  kkt_free(c);
  const size_t n = (size_t)c->mp->hm.g.n;
  // 14 blocks of 3n x R (MINRES vectors) + 4 of n x R (Chebyshev scratch, contiguous column copies)
  KKT_CK(cudaMalloc(&c->kkt_buf, (14 * 3 * n + 4 * n) * R * sizeof(double)));
  KKT_CK(cudaMalloc(&c->kkt_part, (size_t)R * 1216 * sizeof(double)));
  KKT_CK(cudaMallocHost(&c->kkt_hpart, (size_t)R * 1216 * sizeof(double)));
  KKT_CK(cudaMalloc(&c->kkt_coef, (size_t)R * 3 * sizeof(double)));
  c->kkt_R = R;
  return SCHUR_OK;
}

void kkt_free(schur_ctx* c) {
  if (c->kkt_buf) cudaFree(c->kkt_buf);
  if (c->kkt_part) cudaFree(c->kkt_part);
  if (c->kkt_hpart) cudaFreeHost(c->kkt_hpart);
  if (c->kkt_coef) cudaFree(c->kkt_coef);
  c->kkt_buf = c->kkt_part = c->kkt_hpart = c->kkt_coef = nullptr;
  c->kkt_R = 0;
}

// column dots <x_c, y_c> over length len (synchronises)
static int dots(schur_ctx* c, long long len, const double* x, int ldx, const double* y, int ldy, int R, double* out,
                cudaStream_t st) {
  const int nblk = std::max(1, (int)std::min<long long>((len + 255) / 256, 1216 / std::max(1, 1)));
  int nb = std::min(nblk, 1216);
  k_dot_real<<<dim3(nb, R), 256, 0, st>>>(len, x, ldx, y, ldy, R, c->kkt_part, nb);
  KKT_CK(cudaGetLastError());
  KKT_CK(cudaMemcpyAsync(c->kkt_hpart, c->kkt_part, (size_t)R * nb * sizeof(double), cudaMemcpyDeviceToHost, st));
  KKT_CK(cudaStreamSynchronize(st));
  for (int r = 0; r < R; ++r) {
    double s = 0;
    for (int b = 0; b < nb; ++b) s += c->kkt_hpart[(size_t)r * nb + b];
    out[r] = s;
  }
  return SCHUR_OK;
}

static int kkt_apply_impl(schur_ctx* c, const double* v, double* r, int R, int ld, cudaStream_t st) {
  const Geom& g = c->mp->hm.g;
  const long long n = g.n;
  Coef27 sten = make_coef(g, 1.0);
  const int gs = grid_for(n);
  for (int col = 0; col < R; ++col) {
    const double* y = v + (size_t)col * ld;
    const double* u = y + n;
    const double* l = y + 2 * n;
    double* ry = r + (size_t)col * ld;
    double* ru = ry + n;
    double* rl = ry + 2 * n;
    // r_y = M y + K l ; r_u = beta M u - M l ; r_l = K y - M u
    k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, sten, 0, y, (int)n, ry, (int)n, 1, 1.0, 0.0);
    k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, sten, 1, l, (int)n, ry, (int)n, 1, 1.0, 1.0);
    k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, sten, 0, u, (int)n, ru, (int)n, 1, c->beta, 0.0);
    k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, sten, 0, l, (int)n, ru, (int)n, 1, -1.0, 1.0);
    k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, sten, 1, y, (int)n, rl, (int)n, 1, 1.0, 0.0);
    k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, sten, 0, u, (int)n, rl, (int)n, 1, -1.0, 1.0);
    KKT_CK(cudaGetLastError());
  }
  return SCHUR_OK;
}

// z = P_mgw^{-1} r for R columns (R <= kMaxR), leading dimension ld >= 3n
static int kkt_precond_impl(schur_ctx* c, const double* r, double* z, int R, int ld, cudaStream_t st) {
  const Geom& g = c->mp->hm.g;
  const long long n = g.n;
  int rc = kkt_ws(c, R);
  if (rc) return rc;
  double* base = c->kkt_buf + 14 * 3 * (size_t)n * R;
  double* tin = base;                      // n x R contiguous
  double* tout = base + (size_t)n * R;     // n x R
  double* scr = base + 2 * (size_t)n * R;  // needs 3 n R: reuse tail of MINRES area
  double* scr3 = c->kkt_buf + 11 * 3 * (size_t)n * R;  // blocks 11..13 are scratch
  const int gs = grid_for(n);
  const int deg = cheb_degree(g.dim, 1e-13);
  (void)scr;
  for (int blk = 0; blk < 2; ++blk) {
    k_copy_cols<<<dim3(gs, R), 256, 0, st>>>(n, R, r + blk * n, ld, tin, (int)n, 1.0);
    KKT_CK(cudaGetLastError());
    rc = mass_inverse(c, tin, (int)n, tout, (int)n, R, deg, scr3, st);
    if (rc) return rc;
    k_copy_cols<<<dim3(gs, R), 256, 0, st>>>(n, R, tout, (int)n, z + blk * n, ld, blk == 0 ? 1.0 : 1.0 / c->beta);
    KKT_CK(cudaGetLastError());
  }
  // S block through the factored Schur solve
  k_copy_cols<<<dim3(gs, R), 256, 0, st>>>(n, R, r + 2 * n, ld, tin, (int)n, 1.0);
  KKT_CK(cudaGetLastError());
  schur_stats sst;
  std::memset(&sst, 0, sizeof(sst));
  for (int r0 = 0; r0 < R; r0 += kMaxR) {
    int RR = std::min(kMaxR, R - r0);
    rc = ctx_schur_inverse(c, tin + (size_t)r0 * n, (int)n, RR, tout + (size_t)r0 * n, (int)n, st, &sst);
    if (rc) return rc;
  }
  k_copy_cols<<<dim3(gs, R), 256, 0, st>>>(n, R, tout, (int)n, z + 2 * n, ld, 1.0);
  KKT_CK(cudaGetLastError());
  return SCHUR_OK;
}

}  // namespace schur

using namespace schur;

extern "C" {

int schur_kkt_apply(schur_ctx* c, const double* v, double* r, int nrhs, int ld, void* stream) {
  if (!c || (nrhs > 0 && (!v || !r)) || nrhs < 0) return set_error(SCHUR_EINVAL, "bad arguments");
  if (nrhs == 0) return SCHUR_OK;
  if ((long long)ld < 3 * c->mp->hm.g.n) return set_error(SCHUR_EINVAL, "ld < 3n");
  return kkt_apply_impl(c, v, r, nrhs, ld, reinterpret_cast<cudaStream_t>(stream));
}

int schur_kkt_precond_apply(schur_ctx* c, const double* r, double* z, int nrhs, int ld, void* stream) {
  if (!c || (nrhs > 0 && (!r || !z)) || nrhs < 0) return set_error(SCHUR_EINVAL, "bad arguments");
  if (nrhs == 0) return SCHUR_OK;
  if ((long long)ld < 3 * c->mp->hm.g.n) return set_error(SCHUR_EINVAL, "ld < 3n");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  for (int r0 = 0; r0 < nrhs; r0 += kMaxR) {
    int R = std::min(kMaxR, nrhs - r0);
    int rc = kkt_precond_impl(c, r + (size_t)r0 * ld, z + (size_t)r0 * ld, R, ld, st);
    if (rc) return rc;
  }
  KKT_CK(cudaStreamSynchronize(st));
  return SCHUR_OK;
}

int schur_apply_S(schur_ctx* c, const double* x, double* y, int nrhs, int ld, void* stream) {
  if (!c || (nrhs > 0 && (!x || !y)) || nrhs < 0) return set_error(SCHUR_EINVAL, "bad arguments");
  if (nrhs == 0) return SCHUR_OK;
  if ((long long)ld < c->mp->hm.g.n) return set_error(SCHUR_EINVAL, "ld < n");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const Geom& g = c->mp->hm.g;
  const long long n = g.n;
  Coef27 sten = make_coef(g, 1.0);
  const int gs = grid_for(n);
  const int deg = cheb_degree(g.dim, 1e-15);
  for (int r0 = 0; r0 < nrhs; r0 += kMaxR) {
    int R = std::min(kMaxR, nrhs - r0);
    int rc = kkt_ws(c, R);
    if (rc) return rc;
    double* t = c->kkt_buf;
    double* w = t + (size_t)n * R;
    double* scr = c->kkt_buf + 3 * (size_t)n * R;
    const double* xr = x + (size_t)r0 * ld;
    double* yr = y + (size_t)r0 * ld;
    k_apply_real<<<dim3(gs, R), 256, 0, st>>>(g, sten, 1, xr, ld, t, (int)n, R, 1.0, 0.0);
    KKT_CK(cudaGetLastError());
    rc = mass_inverse(c, t, (int)n, w, (int)n, R, deg, scr, st);
    if (rc) return rc;
    k_apply_real<<<dim3(gs, R), 256, 0, st>>>(g, sten, 1, w, (int)n, yr, ld, R, 1.0, 0.0);
    k_apply_real<<<dim3(gs, R), 256, 0, st>>>(g, sten, 0, xr, ld, yr, ld, R, 1.0 / c->beta, 1.0);
    KKT_CK(cudaGetLastError());
  }
  KKT_CK(cudaStreamSynchronize(st));
  return SCHUR_OK;
}

// The range-space method of Sec. 3.1 with Dirichlet data (the thermal problem of Sec. 6.1):
// lambda = S^{-1} (K ybar + K_c y_c), y = ybar - M^{-1} K lambda, u = lambda / beta, and the relative
// constraint violation ||K y + K_c y_c - M u|| / ||K y|| of Eq. relativeconstraintviolation.
int schur_control_solve(schur_ctx* c, const double* yfull, int ldf, double* y, double* u, double* lam, int nrhs,
                        int ld, double* viol, void* stream, schur_stats* st) {
  if (!c || nrhs < 0) return set_error(SCHUR_EINVAL, "bad arguments");
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->ms_setup = c->ms_setup;
  }
  if (nrhs == 0) return SCHUR_OK;
  const Geom& g = c->mp->hm.g;
  const long long n = g.n;
  long long nfull = 1;
  for (int a = 0; a < g.dim; ++a) nfull *= (long long)g.nel[a] + 1;
  if (!yfull || !y || !u) return set_error(SCHUR_EINVAL, "NULL vector");
  if ((long long)ldf < nfull) return set_error(SCHUR_EINVAL, "ldf smaller than the number of grid nodes");
  if ((long long)ld < n) return set_error(SCHUR_EINVAL, "ld < n");
  if (c->opts.factor != SCHUR_FACTOR_EXACT)
    return set_error(SCHUR_EINVAL, "the range-space solve needs the exact factor (SCHUR_FACTOR_EXACT)");
  cudaStream_t st_ = reinterpret_cast<cudaStream_t>(stream);
  Coef27 sten = make_coef(g, 1.0);
  const int gs = grid_for(n);
  const int deg = cheb_degree(g.dim, 1e-15);
  int status = SCHUR_OK;
  for (int r0 = 0; r0 < nrhs; r0 += kMaxR) {
    const int R = std::min(kMaxR, nrhs - r0);
    int rc = kkt_ws(c, R);
    if (rc) return rc;
    const size_t nR = (size_t)n * R;
    double* rhs = c->kkt_buf;
    double* lw = rhs + nR;
    double* t = lw + nR;
    double* w = t + nR;
    double* scr = w + nR;  // 3 n R
    double* v = scr + 3 * nR;
    double* ky = v + nR;
    const double* yf = yfull + (size_t)r0 * ldf;
    double* yr = y + (size_t)r0 * ld;
    double* ur = u + (size_t)r0 * ld;
    k_full_stiffness<<<dim3(gs, R), 256, 0, st_>>>(g, sten, yf, ldf, rhs, (int)n, R);
    KKT_CK(cudaGetLastError());
    schur_stats sst;
    std::memset(&sst, 0, sizeof(sst));
    rc = ctx_schur_inverse(c, rhs, (int)n, R, lw, (int)n, st_, &sst);
    if (rc == SCHUR_ENOTCONV) status = rc;
    else if (rc) return rc;
    if (st) {
      st->outer_steps = std::max(st->outer_steps, sst.outer_steps);
      st->iters_total = std::max(st->iters_total, sst.iters_total);
      st->iters_first = std::max(st->iters_first, sst.iters_first);
      st->rel_residual = std::max(st->rel_residual, sst.rel_residual);
    }
    // w = M^{-1} K lambda
    k_apply_real<<<dim3(gs, R), 256, 0, st_>>>(g, sten, 1, lw, (int)n, t, (int)n, R, 1.0, 0.0);
    KKT_CK(cudaGetLastError());
    rc = mass_inverse(c, t, (int)n, w, (int)n, R, deg, scr, st_);
    if (rc) return rc;
    k_control_update<<<dim3(gs, R), 256, 0, st_>>>(g, yf, ldf, w, lw, (int)n, 1.0 / c->beta, yr, ur, ld, R);
    KKT_CK(cudaGetLastError());
    if (lam) {
      k_copy_cols<<<dim3(gs, R), 256, 0, st_>>>(n, R, lw, (int)n, lam + (size_t)r0 * ld, ld, 1.0);
      KKT_CK(cudaGetLastError());
    }
    if (viol) {
      k_constraint<<<dim3(gs, R), 256, 0, st_>>>(g, sten, yr, ur, ld, yf, ldf, v, (int)n, R);
      k_apply_real<<<dim3(gs, R), 256, 0, st_>>>(g, sten, 1, yr, ld, ky, (int)n, R, 1.0, 0.0);
      KKT_CK(cudaGetLastError());
      std::vector<double> vv(R), kk(R);
      rc = dots(c, n, v, (int)n, v, (int)n, R, vv.data(), st_);
      if (rc) return rc;
      rc = dots(c, n, ky, (int)n, ky, (int)n, R, kk.data(), st_);
      if (rc) return rc;
      for (int r = 0; r < R; ++r) viol[r0 + r] = kk[r] > 0 ? std::sqrt(vv[r] / kk[r]) : std::sqrt(vv[r]);
    }
  }
  KKT_CK(cudaStreamSynchronize(st_));
  if (st) st->status = status;
  return status;
}

// Preconditioned MINRES (Lanczos with P_mgw, Givens QR of the tridiagonal), one independent
// recurrence per right-hand side; host scalars, device vectors.
int schur_kkt_minres(schur_ctx* c, const double* rhs, double* sol, int nrhs, int ld, double tol, int max_it,
                     int* iters, void* stream) {
  if (!c || (nrhs > 0 && (!rhs || !sol)) || nrhs < 0 || !(tol > 0) || max_it < 1)
    return set_error(SCHUR_EINVAL, "bad arguments");
  if (iters) *iters = 0;
  if (nrhs == 0) return SCHUR_OK;
  const long long n3 = 3 * c->mp->hm.g.n;
  if ((long long)ld < n3) return set_error(SCHUR_EINVAL, "ld < 3n");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int status = SCHUR_OK, itmax = 0;
  for (int r0 = 0; r0 < nrhs; r0 += kMaxR) {
    const int R = std::min(kMaxR, nrhs - r0);
    int rc = kkt_ws(c, R);
    if (rc) return rc;
    const size_t blk = (size_t)n3 * R;
    double* vprev = c->kkt_buf;
    double* vcur = vprev + blk;
    double* vnext = vcur + blk;
    double* zcur = vnext + blk;
    double* znext = zcur + blk;
    double* q = znext + blk;
    double* wprev = q + blk;
    double* wcur = wprev + blk;
    double* wnext = wcur + blk;
    double* x = wnext + blk;
    const int gs = grid_for(n3);
    const int ldv = (int)n3;
    KKT_CK(cudaMemsetAsync(vprev, 0, blk * sizeof(double), st));
    KKT_CK(cudaMemsetAsync(wprev, 0, blk * sizeof(double), st));
    KKT_CK(cudaMemsetAsync(wcur, 0, blk * sizeof(double), st));
    KKT_CK(cudaMemsetAsync(x, 0, blk * sizeof(double), st));
    k_copy_cols<<<dim3(gs, R), 256, 0, st>>>(n3, R, rhs + (size_t)r0 * ld, ld, vcur, ldv, 1.0);
    KKT_CK(cudaGetLastError());
    rc = kkt_precond_impl(c, vcur, zcur, R, ldv, st);
    if (rc) return rc;
    std::vector<double> gam(R), gam_prev(R, 1.0), eta(R), gam1(R), c0(R, 1.0), c1(R, 1.0), s0(R, 0.0), s1(R, 0.0),
        del(R), tmp(R), coef(3 * R);
    std::vector<int> done(R, 0);
    rc = dots(c, n3, vcur, ldv, zcur, ldv, R, tmp.data(), st);
    if (rc) return rc;
    for (int r = 0; r < R; ++r) {
      if (tmp[r] < 0) return set_error(SCHUR_EBREAKDOWN, "preconditioner not positive definite");
      gam[r] = std::sqrt(tmp[r]);
      eta[r] = gam[r];
      gam1[r] = gam[r];
      if (gam[r] == 0) done[r] = 1;
    }
    int it = 0;
    bool all = std::all_of(done.begin(), done.end(), [](int d) { return d; });
    while (!all && it < max_it) {
      ++it;
      // z_j /= gamma_j
      for (int r = 0; r < R; ++r) {
        coef[3 * r] = gam[r] > 0 ? 1.0 / gam[r] : 0.0;
        coef[3 * r + 1] = coef[3 * r + 2] = 0;
      }
      KKT_CK(cudaMemcpyAsync(c->kkt_coef, coef.data(), 3 * R * sizeof(double), cudaMemcpyHostToDevice, st));
      k_lin3<<<dim3(gs, R), 256, 0, st>>>(n3, R, zcur, ldv, c->kkt_coef, zcur, nullptr, nullptr, ldv);
      KKT_CK(cudaGetLastError());
      rc = kkt_apply_impl(c, zcur, q, R, ldv, st);
      if (rc) return rc;
      rc = dots(c, n3, q, ldv, zcur, ldv, R, del.data(), st);
      if (rc) return rc;
      // v_{j+1} = q - (delta/gamma_j) v_j - (gamma_j/gamma_{j-1}) v_{j-1}
      for (int r = 0; r < R; ++r) {
        coef[3 * r] = 1.0;
        coef[3 * r + 1] = gam[r] > 0 ? -del[r] / gam[r] : 0.0;
        coef[3 * r + 2] = -gam[r] / gam_prev[r];
      }
      KKT_CK(cudaMemcpyAsync(c->kkt_coef, coef.data(), 3 * R * sizeof(double), cudaMemcpyHostToDevice, st));
      k_lin3<<<dim3(gs, R), 256, 0, st>>>(n3, R, vnext, ldv, c->kkt_coef, q, vcur, vprev, ldv);
      KKT_CK(cudaGetLastError());
      rc = kkt_precond_impl(c, vnext, znext, R, ldv, st);
      if (rc) return rc;
      rc = dots(c, n3, vnext, ldv, znext, ldv, R, tmp.data(), st);
      if (rc) return rc;
      std::vector<double> gnext(R), a1v(R), a2v(R), a3v(R), cn(R), sn(R);
      for (int r = 0; r < R; ++r) {
        gnext[r] = std::sqrt(std::max(0.0, tmp[r]));
        double a0 = c1[r] * del[r] - c0[r] * s1[r] * gam[r];
        double a1 = std::sqrt(a0 * a0 + gnext[r] * gnext[r]);
        double a2 = s1[r] * del[r] + c0[r] * c1[r] * gam[r];
        double a3 = s0[r] * gam[r];
        cn[r] = a1 > 0 ? a0 / a1 : 1.0;
        sn[r] = a1 > 0 ? gnext[r] / a1 : 0.0;
        a1v[r] = a1;
        a2v[r] = a2;
        a3v[r] = a3;
      }
      // w_{j+1} = (z_j - a3 w_{j-1} - a2 w_j) / a1
      for (int r = 0; r < R; ++r) {
        double inv = (a1v[r] > 0 && !done[r]) ? 1.0 / a1v[r] : 0.0;
        coef[3 * r] = inv;
        coef[3 * r + 1] = -a3v[r] * inv;
        coef[3 * r + 2] = -a2v[r] * inv;
      }
      KKT_CK(cudaMemcpyAsync(c->kkt_coef, coef.data(), 3 * R * sizeof(double), cudaMemcpyHostToDevice, st));
      k_lin3<<<dim3(gs, R), 256, 0, st>>>(n3, R, wnext, ldv, c->kkt_coef, zcur, wprev, wcur, ldv);
      KKT_CK(cudaGetLastError());
      // x += c_{j+1} eta w_{j+1}
      for (int r = 0; r < R; ++r) {
        coef[3 * r] = 1.0;
        coef[3 * r + 1] = done[r] ? 0.0 : cn[r] * eta[r];
        coef[3 * r + 2] = 0.0;
      }
      KKT_CK(cudaMemcpyAsync(c->kkt_coef, coef.data(), 3 * R * sizeof(double), cudaMemcpyHostToDevice, st));
      k_lin3<<<dim3(gs, R), 256, 0, st>>>(n3, R, x, ldv, c->kkt_coef, x, wnext, nullptr, ldv);
      KKT_CK(cudaGetLastError());
      for (int r = 0; r < R; ++r) {
        if (done[r]) continue;
        eta[r] = -sn[r] * eta[r];
        c0[r] = c1[r];
        c1[r] = cn[r];
        s0[r] = s1[r];
        s1[r] = sn[r];
        gam_prev[r] = gam[r];
        gam[r] = gnext[r];
        if (std::fabs(eta[r]) <= tol * gam1[r] || gnext[r] == 0) done[r] = 1;
      }
      // rotate buffers
      std::swap(vprev, vcur);
      std::swap(vcur, vnext);
      std::swap(zcur, znext);
      std::swap(wprev, wcur);
      std::swap(wcur, wnext);
      all = std::all_of(done.begin(), done.end(), [](int d) { return d; });
    }
    itmax = std::max(itmax, it);
    if (!all) status = set_error(SCHUR_ENOTCONV, "MINRES did not converge within max_it");
    const int gs2 = grid_for(n3);
    k_copy_cols<<<dim3(gs2, R), 256, 0, st>>>(n3, R, x, ldv, sol + (size_t)r0 * ld, ld, 1.0);
    KKT_CK(cudaGetLastError());
  }
  KKT_CK(cudaStreamSynchronize(st));
  if (iters) *iters = itmax;
  return status;
}

}  // extern "C"
