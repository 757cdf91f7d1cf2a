#pragma once
#include "common.cuh"

namespace schur {

// Hessenberg column k of right-hand side r after the Arnoldi step, with h_{k+1,k} = hk1: apply the
// previous complex Givens rotations, form the new one, rotate the residual vector g, and update
// the convergence state (single thread).  Layouts as in gmres.cu.
__device__ __forceinline__ void givens_step(int r, int k, int m, double hk1, cx<double>* H, double* cs_c,
                                            cx<double>* cs_s, cx<double>* gvec, const double* __restrict__ beta0,
                                            double tol, int* active, int* kk, double* inv_nrm, double* resid,
                                            int* bad) {
  cx<double>* col = H + ((size_t)r * m + k) * (m + 1);
  for (int i = 0; i < k; ++i) {
    const double c = cs_c[(size_t)r * m + i];
    const cx<double> s = cs_s[(size_t)r * m + i];
    const cx<double> a = col[i], b = col[i + 1];
    const cx<double> sb = cmul(s, b);
    const cx<double> t = cmul(mkc<double>(s.re, -s.im), a);
    col[i] = mkc<double>(c * a.re + sb.re, c * a.im + sb.im);
    col[i + 1] = mkc<double>(c * b.re - t.re, c * b.im - t.im);
  }
  const cx<double> a = col[k];
  const double aa = hypot(a.re, a.im);
  const double rho = hypot(aa, hk1);
  double c;
  cx<double> s, top;
  if (aa == 0.0) {
    c = 0.0;
    s = mkc<double>(1.0, 0.0);
    top = mkc<double>(rho, 0.0);
  } else {
    const cx<double> ph = mkc<double>(a.re / aa, a.im / aa);
    c = aa / rho;
    s = cscale(ph, hk1 / rho);
    top = cscale(ph, rho);
  }
  col[k] = top;
  col[k + 1] = mkc<double>(hk1, 0.0);  // kept for reference; eliminated by the rotation
  cs_c[(size_t)r * m + k] = c;
  cs_s[(size_t)r * m + k] = s;
  const cx<double> gk = gvec[(size_t)r * (m + 1) + k];
  const cx<double> t = cmul(mkc<double>(s.re, -s.im), gk);
  gvec[(size_t)r * (m + 1) + k] = cscale(gk, c);
  gvec[(size_t)r * (m + 1) + k + 1] = mkc<double>(-t.re, -t.im);
  const double res = hypot(t.re, t.im);
  resid[r] = res;
  kk[r] = k + 1;
  const bool finite = isfinite(hk1) && isfinite(res) && isfinite(rho) && rho > 0.0;
  if (!finite) bad[r] = 1;
  if (!finite || res <= tol * beta0[r] || hk1 == 0.0 || k + 1 >= m) active[r] = 0;
  inv_nrm[r] = hk1 > 0.0 ? 1.0 / hk1 : 0.0;
}

__global__ void k_gmres_init(int R, const double* __restrict__ nrm_part, int nblk, int m, double* beta0,
                             cx<double>* gvec, int* active, int* kk, double* inv_nrm, double* resid);
__global__ void k_hess_solve(int m, const cx<double>* __restrict__ H, const cx<double>* __restrict__ gvec,
                             const int* __restrict__ kk, cx<double>* y);

}  // namespace schur
