// Dense FP64 inversion of the augmented coarse matrix (Sec. 5: the coarse problem of FETI-DP with
// the face-average augmentation).  Its unknowns (corners and faces) do not form the layered grid
// the corner-only cyclic reduction works on, and the matrix is small (at most 4096 unknowns), so it
// is inverted as a whole by Gauss-Jordan elimination without pivoting in panels of 32 pivots.  For
// the panel K = [k0, k0 + w):
//   P = A[K, K]^{-1}                        (one block)
//   R = P A[K, :]  (R[:, K] = P),  C = A[:, K]
//   A[i, j] <- (j in K ? 0 : A[i, j]) - C[i, :] R[:, j]   for rows i outside K,   A[K, :] <- R
// which is the unblocked elimination applied w pivots at a time.  The real and imaginary parts of
// the corner block are positive definite; the face block enters with the opposite sign (a
// saddle-point system), and its pivots stay nonzero as long as the face constraints are linearly
// independent of the corner ones; a zero or non-finite pivot sets *err.
#include <cuda_runtime.h>

#include <string>

#include "../../include/schur.h"
#include "coarse.h"

namespace schur {
namespace {

constexpr int kPW = 32;  // pivots per panel

__global__ void k_dgj_pivot(const cx<double>* __restrict__ A, int n, int k0, int w, cx<double>* Pb, int* err) {
  __shared__ cx<double> B[kPW][kPW + 1];
  __shared__ cx<double> row[kPW], col[kPW];
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int e = tid; e < w * w; e += nthr) B[e / w][e % w] = A[(size_t)(k0 + e / w) * n + k0 + e % w];
  __syncthreads();
  for (int k = 0; k < w; ++k) {
    const cx<double> p = B[k][k];
    const cx<double> piv = cinv(p);
    if (tid == 0 && !(isfinite(p.re) && isfinite(p.im) && (p.re != 0.0 || p.im != 0.0))) atomicExch(err, 1);
    for (int t = tid; t < w; t += nthr) {
      row[t] = cmul(B[k][t], piv);
      col[t] = B[t][k];
    }
    __syncthreads();
    for (int e = tid; e < w * w; e += nthr) {
      const int i = e / w, j = e % w;
      if (i == k) {
        B[i][j] = j == k ? piv : row[j];
      } else if (j == k) {
        const cx<double> v = cmul(col[i], piv);
        B[i][j] = mkc<double>(-v.re, -v.im);
      } else {
        cfms(B[i][j], col[i], row[j]);
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < w * w; e += nthr) Pb[e] = B[e / w][e % w];
}

// R[k][j] = sum_m P[k][m] A[k0 + m][j] (j outside K), P[k][j - k0] (j inside K)
__global__ void k_dgj_rows(const cx<double>* __restrict__ A, int n, int k0, int w, const cx<double>* __restrict__ Pb,
                           cx<double>* Rb) {
  __shared__ cx<double> Ps[kPW * kPW];
  for (int e = threadIdx.x; e < w * w; e += blockDim.x) Ps[e] = Pb[e];
  __syncthreads();
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  if (j >= k0 && j < k0 + w) {
    for (int k = 0; k < w; ++k) Rb[(size_t)k * n + j] = Ps[k * w + (j - k0)];
    return;
  }
  cx<double> a[kPW];
  for (int m = 0; m < w; ++m) a[m] = A[(size_t)(k0 + m) * n + j];
  for (int k = 0; k < w; ++k) {
    cx<double> s = mkc<double>(0, 0);
    for (int m = 0; m < w; ++m) cfma(s, Ps[k * w + m], a[m]);
    Rb[(size_t)k * n + j] = s;
  }
}

__global__ void k_dgj_cols(const cx<double>* __restrict__ A, int n, int k0, int w, cx<double>* Cb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int m = 0; m < w; ++m) Cb[(size_t)i * kPW + m] = A[(size_t)i * n + k0 + m];
}

// A[i][j] <- (i in K) ? R[i - k0][j] : (j in K ? 0 : A[i][j]) - sum_m C[i][m] R[m][j], 32 x 32 tiles
__global__ void __launch_bounds__(256) k_dgj_update(cx<double>* A, int n, int k0, int w,
                                                    const cx<double>* __restrict__ Cb,
                                                    const cx<double>* __restrict__ Rb) {
  __shared__ cx<double> Cs[32][kPW + 1];
  __shared__ cx<double> Rs[kPW][32 + 1];
  const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32, tid = threadIdx.x;
  for (int e = tid; e < 32 * w; e += 256) {
    const int r = e / w, m = e % w, i = i0 + r;
    Cs[r][m] = i < n ? Cb[(size_t)i * kPW + m] : mkc<double>(0, 0);
  }
  for (int e = tid; e < w * 32; e += 256) {
    const int m = e / 32, c = e % 32, j = j0 + c;
    Rs[m][c] = j < n ? Rb[(size_t)m * n + j] : mkc<double>(0, 0);
  }
  __syncthreads();
  const int c = tid & 31, r0 = tid >> 5;  // column c, rows r0, r0 + 8, r0 + 16, r0 + 24
  const int j = j0 + c;
  if (j >= n) return;
  const bool jin = j >= k0 && j < k0 + w;
  for (int rr = r0; rr < 32; rr += 8) {
    const int i = i0 + rr;
    if (i >= n) break;
    cx<double>* a = A + (size_t)i * n + j;
    if (i >= k0 && i < k0 + w) {
      *a = Rs[i - k0][c];
      continue;
    }
    cx<double> v = jin ? mkc<double>(0, 0) : *a;
    for (int m = 0; m < w; ++m) cfms(v, Cs[rr][m], Rs[m][c]);
    *a = v;
  }
}

}  // namespace

int dense_gj_inverse(cx<double>* A, int n, int* err, cudaStream_t st, std::string* msg, long long* launches) {
  if (n <= 0) return 0;
  cx<double>*Pb = nullptr, *Rb = nullptr, *Cb = nullptr;
  auto fail = [&](cudaError_t e, const char* where) {
    if (msg) *msg = std::string("dense coarse inverse (") + where + "): " + cudaGetErrorString(e);
    if (Pb) cudaFreeAsync(Pb, st);
    if (Rb) cudaFreeAsync(Rb, st);
    if (Cb) cudaFreeAsync(Cb, st);
    return e == cudaErrorMemoryAllocation ? SCHUR_ENOMEM : SCHUR_ECUDA;
  };
  cudaError_t e = cudaMallocAsync((void**)&Pb, sizeof(cx<double>) * kPW * kPW, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&Rb, sizeof(cx<double>) * kPW * (size_t)n, st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&Cb, sizeof(cx<double>) * kPW * (size_t)n, st);
  if (e != cudaSuccess) return fail(e, "alloc");
  const int nb = (n + 255) / 256, nt = (n + 31) / 32;
  for (int k0 = 0; k0 < n; k0 += kPW) {
    const int w = n - k0 < kPW ? n - k0 : kPW;
    k_dgj_pivot<<<1, 256, 0, st>>>(A, n, k0, w, Pb, err);
    k_dgj_rows<<<nb, 256, 0, st>>>(A, n, k0, w, Pb, Rb);
    k_dgj_cols<<<nb, 256, 0, st>>>(A, n, k0, w, Cb);
    k_dgj_update<<<dim3(nt, nt), 256, 0, st>>>(A, n, k0, w, Cb, Rb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(e, "launch");
    if (launches) *launches += 4;
  }
  cudaFreeAsync(Pb, st);
  cudaFreeAsync(Rb, st);
  cudaFreeAsync(Cb, st);
  return 0;
}

}  // namespace schur
