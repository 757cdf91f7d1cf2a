// FP64 scalar side of GMRES on the FETI-DP dual problem (Sec. 5: GMRES for the indefinite
// complex factors): reductions of the Gram-Schmidt coefficients, the Hessenberg column update
// with complex Givens rotations, and the triangular solve for the Krylov coefficients.
// Layouts per right-hand side r:  H[(r*m + k)*(m+1) + j] = H_{j,k};  g[r*(m+1) + j];
// hc[r*kMaxKdev + j];  cs: c real [r*m + k], s complex [r*m + k].
#include "gmres.h"

namespace schur {

__global__ void k_dots_reduce(const cx<double>* __restrict__ part, int nblk, int R, int k, int m,
                              const int* __restrict__ active, cx<double>* H, cx<double>* hc) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int r = wid / (k + 1), j = wid % (k + 1);
  if (r >= R || !active[r]) return;
  double re = 0, im = 0;
  const cx<double>* p = part + ((size_t)r * kMaxKdev + j) * nblk;
  for (int b = lane; b < nblk; b += 32) {
    re += p[b].re;
    im += p[b].im;
  }
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    hc[(size_t)r * kMaxKdev + j] = mkc<double>(re, im);
    cx<double>& h = H[((size_t)r * m + k) * (m + 1) + j];
    h = cadd(h, mkc<double>(re, im));
  }
}

// Sum of the nblk partial sums of right-hand side r, by the whole warp (result in every lane).
__device__ __forceinline__ double warp_sum_parts(const double* __restrict__ part, int nblk) {
  double s = 0;
  for (int b = threadIdx.x; b < nblk; b += 32) s += part[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

// One warp per right-hand side (grid R x 32 threads).
__global__ void k_gmres_init(int R, const double* __restrict__ nrm_part, int nblk, int m, double* beta0,
                             cx<double>* gvec, int* active, int* kk, double* inv_nrm, double* resid) {
  const int r = blockIdx.x;
  if (r >= R) return;
  const double s = warp_sum_parts(nrm_part + (size_t)r * nblk, nblk);
  if (threadIdx.x != 0) return;
  double b0 = sqrt(s);
  beta0[r] = b0;
  for (int j = 0; j <= m; ++j) gvec[(size_t)r * (m + 1) + j] = mkc<double>(0, 0);
  gvec[(size_t)r * (m + 1)] = mkc<double>(b0, 0);
  bool ok = b0 > 0 && isfinite(b0);
  active[r] = ok ? 1 : 0;
  kk[r] = 0;
  inv_nrm[r] = ok ? 1.0 / b0 : 0.0;
  resid[r] = b0;
}

__global__ void k_givens(int R, int k, int m, cx<double>* H, const double* __restrict__ nrm_part, int nblk,
                         double* cs_c, cx<double>* cs_s, cx<double>* gvec, const double* __restrict__ beta0,
                         double tol, int* active, int* kk, double* inv_nrm, double* resid, int* bad) {
  const int r = blockIdx.x;  // one warp per right-hand side
  if (r >= R || !active[r]) return;
  const double s2 = warp_sum_parts(nrm_part + (size_t)r * nblk, nblk);
  if (threadIdx.x != 0) return;
  const double hk1 = sqrt(s2);
  cx<double>* col = H + ((size_t)r * m + k) * (m + 1);
  for (int i = 0; i < k; ++i) {
    double c = cs_c[(size_t)r * m + i];
    cx<double> s = cs_s[(size_t)r * m + i];
    cx<double> a = col[i], b = col[i + 1];
    cx<double> sb = cmul(s, b);
    cx<double> cs = mkc<double>(s.re, -s.im);
    cx<double> t = cmul(cs, a);
    col[i] = mkc<double>(c * a.re + sb.re, c * a.im + sb.im);
    col[i + 1] = mkc<double>(c * b.re - t.re, c * b.im - t.im);
  }
  cx<double> a = col[k];
  double aa = hypot(a.re, a.im);
  double rho = hypot(aa, hk1);
  double c;
  cx<double> s, top;
  if (aa == 0.0) {
    c = 0.0;
    s = mkc<double>(1.0, 0.0);
    top = mkc<double>(rho, 0.0);
  } else {
    cx<double> ph = mkc<double>(a.re / aa, a.im / aa);
    c = aa / rho;
    s = cscale(ph, hk1 / rho);
    top = cscale(ph, rho);
  }
  col[k] = top;
  col[k + 1] = mkc<double>(hk1, 0.0);  // kept for reference; eliminated by the rotation
  cs_c[(size_t)r * m + k] = c;
  cs_s[(size_t)r * m + k] = s;
  cx<double> gk = gvec[(size_t)r * (m + 1) + k];
  cx<double> sc = mkc<double>(s.re, -s.im);
  cx<double> t = cmul(sc, gk);
  gvec[(size_t)r * (m + 1) + k] = cscale(gk, c);
  gvec[(size_t)r * (m + 1) + k + 1] = mkc<double>(-t.re, -t.im);
  double res = hypot(t.re, t.im);
  resid[r] = res;
  kk[r] = k + 1;
  bool finite = isfinite(hk1) && isfinite(res) && isfinite(rho) && rho > 0.0;
  if (!finite) bad[r] = 1;
  if (!finite || res <= tol * beta0[r] || hk1 == 0.0 || k + 1 >= m) active[r] = 0;
  inv_nrm[r] = hk1 > 0.0 ? 1.0 / hk1 : 0.0;
}

__global__ void k_hess_solve(int m, const cx<double>* __restrict__ H, const cx<double>* __restrict__ gvec,
                             const int* __restrict__ kk, cx<double>* y) {
  __shared__ cx<double> rhs[kMaxKdev];
  __shared__ cx<double> yj;
  const int r = blockIdx.x, n = kk[r];
  for (int i = threadIdx.x; i < n; i += blockDim.x) rhs[i] = gvec[(size_t)r * (m + 1) + i];
  __syncthreads();
  for (int j = n - 1; j >= 0; --j) {
    const cx<double>* col = H + ((size_t)r * m + j) * (m + 1);
    if (threadIdx.x == 0) {
      cx<double> d = col[j];
      yj = cmul(rhs[j], cinv(d));
      y[(size_t)r * kMaxKdev + j] = yj;
    }
    __syncthreads();
    cx<double> v = yj;
    for (int i = threadIdx.x; i < j; i += blockDim.x) cfms(rhs[i], col[i], v);
    __syncthreads();
  }
}

}  // namespace schur
