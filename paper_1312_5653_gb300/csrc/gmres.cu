// FP64 scalar side of GMRES on the FETI-DP dual problem (Sec. 5: GMRES for the indefinite
// complex factors): the initial residual norm and the triangular solve for the Krylov
// coefficients.  The Givens step on the Hessenberg column (gmres.h) runs inside the fused
// orthogonalisation kernels.
// Layouts per right-hand side r:  H[(r*m + k)*(m+1) + j] = H_{j,k};  g[r*(m+1) + j];
// hc[r*kMaxKdev + j];  cs: c real [r*m + k], s complex [r*m + k].
#include "gmres.h"

namespace schur {

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
