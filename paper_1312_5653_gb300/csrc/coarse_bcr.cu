// Block cyclic reduction (odd-even reduction over layers) of the coarse corner matrix.
//
// The coarse matrix of Sec. 5 is block tridiagonal over the layers of the corner grid.  Instead of
// the sequential layer recursion, every level eliminates every other remaining layer j at once
// (p, q: its remaining neighbours; A_pj = U_p, A_jq = U_j, symmetric blocks):
//   Dinv_j = D_j^{-1},  Lp_j = A_pj Dinv_j,  Lq_j = Dinv_j A_jq,
//   D_p -= Lp_j A_pj^T,  D_q -= A_jq^T Lq_j,  A_pq = -Lp_j A_jq
// so the critical path is log2(L) levels of batched dense work.  The factor is computed in FP64
// (BcrFactor).  The explicit inverse is a cyclic-reduction solve with the identity as right-hand
// side in the working precision (FP32 copies of Dinv, Lp, Lq in the mixed form):
//   forward  X_p -= Lp_j X_j,  X_q -= Lq_j^T X_j
//   backward X_j  = Dinv_j X_j - Lp_j^T X_p - Lq_j X_q
#include <cooperative_groups.h>

#include <algorithm>
#include <vector>

#include "../../include/schur.h"
#include "coarse.h"
#include "prof.h"

namespace cg = cooperative_groups;

namespace schur {

// ------------------------------------------------------------------ batched dense kernels
// Dense layer blocks from the stored sparse coarse blocks: D_K = A_KK, U_K = A_{K,K+1}.
template <class S>
__global__ void k_bcr_densify(StoredProv<double> P, cx<S>* D, cx<S>* U) {
  const int b = P.ly.b, L = P.ly.L, nt = nbr_count(P.ly.dim);
  const size_t bb = (size_t)b * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)L * bb; e += (size_t)gridDim.x * blockDim.x) {
    int K = (int)(e / bb), r = (int)(e % bb), i = r / b, j = r % b;
    int t = nbr_slot(P.ly, i, j);
    D[e] = ccast<S>(t >= 0 ? P.Ad(K, i, t) : mkc<double>(0, 0));
    // A_{K,K+1}[i][j] = A(K, i ; K+1, j) = A(K+1, j ; K, i) = CB[K][j][slot of i from j]
    cx<double> u = mkc<double>(0, 0);
    if (K + 1 < L) {
      int tj = nbr_slot(P.ly, j, i);
      if (tj >= 0) u = P.Al(K, j, tj);
    }
    U[e] = ccast<S>(u);
  }
}

// Gauss-Jordan inversion of a batch of dense b x b blocks, one thread-block cluster per
// block; columns distributed over the cluster, pivot column broadcast through DSMEM.
template <class S>
__global__ void __launch_bounds__(256) k_gj_batch_cluster(const cx<S>* __restrict__ Din, cx<S>* Dout,
                                                          const int* __restrict__ list, int b, int* err) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), me = (int)cluster.block_rank();
  const int which = list[blockIdx.x / CL];
  const int cw = (b + CL - 1) / CL, c0 = me * cw, c1 = min(b, c0 + cw), ncol = max(0, c1 - c0);
  const int tid = threadIdx.x, nthr = blockDim.x;
  extern __shared__ unsigned char smraw[];
  cx<S>* Dl = reinterpret_cast<cx<S>*>(smraw);  // b x cw
  cx<S>* colk = Dl + (size_t)b * cw;                  // b
  cx<S>* bcast = colk + b;                            // 2 x b
  cx<S>* rowk = bcast + 2 * b;                        // cw
  const size_t bb = (size_t)b * b;
  const cx<S>* src = Din + (size_t)which * bb;
  for (int e = tid; e < b * cw; e += nthr) {
    int i = e / cw, jl = e - i * cw;
    Dl[e] = jl < ncol ? src[(size_t)i * b + c0 + jl] : mkc<S>(0, 0);
  }
  __syncthreads();
  for (int k = 0; k < b; ++k) {
    const int owner = k / cw;
    cx<S>* pub = bcast + (k & 1) * b;
    if (me == owner)
      for (int i = tid; i < b; i += nthr) pub[i] = Dl[i * cw + (k - c0)];
    cluster.sync();
    const cx<S>* rs = cluster.map_shared_rank(pub, owner);
    for (int i = tid; i < b; i += nthr) colk[i] = rs[i];
    __syncthreads();
    const cx<S> p = colk[k];
    const cx<S> piv = cinv(p);
    if (tid == 0 && me == 0 && !finite_nonzero(p)) atomicExch(err, 1);
    for (int jl = tid; jl < ncol; jl += nthr) rowk[jl] = cmul(Dl[k * cw + jl], piv);
    __syncthreads();
    for (int e = tid; e < b * ncol; e += nthr) {
      int i = e / ncol, jl = e - i * ncol, j = c0 + jl;
      cx<S>& a = Dl[i * cw + jl];
      if (j == k) {
        if (i == k) {
          a = piv;
        } else {
          cx<S> v = cmul(colk[i], piv);
          a = mkc<S>(-v.re, -v.im);
        }
      } else if (i == k) {
        a = rowk[jl];
      } else {
        cfms(a, colk[i], rowk[jl]);
      }
    }
    __syncthreads();
  }
  cx<S>* dst = Dout + (size_t)which * bb;
  for (int e = tid; e < b * ncol; e += nthr) {
    int i = e / ncol, jl = e - i * ncol;
    dst[(size_t)i * b + c0 + jl] = Dl[i * cw + jl];
  }
  cluster.sync();
}

// Gauss-Jordan inversion by column panels, one thread-block cluster of CL CTAs per matrix (no
// pivoting).  CTA c owns columns [c*cw, c*cw + ncol) in shared memory (row-major, stride cw), and
// panel step k uses the columns of CTA k as the pivot block K.  The owner publishes the panel
// A[:, K] and P = A[K, K]^{-1} in its shared memory; after one cluster barrier every CTA reads them
// through distributed shared memory and updates its own columns:
//   A[K, j] <- P A[K, j],   A[i, j] <- A[i, j] - A[i, K] A[K, j]_new   (i not in K)
// while the owner sets A[i, K] <- -A[i, K] P (i not in K) and A[K, K] <- P.  One cluster barrier
// per panel instead of one per pivot.
template <class S>
__device__ void gj_small_warp(cx<S>* A, int n, int ld, int* err) {
  // in-place inverse of the n x n block A (row stride ld) by one warp, n <= 32
  const int lane = threadIdx.x & 31;
  if (n * n <= 32) {
    // small blocks: lane (i, j) updates entry (i, j) at every pivot, the same arithmetic per entry
    // as the row loop below
    const int i = lane / n, j = lane - i * n;
    for (int k = 0; k < n; ++k) {
      const cx<S> p = A[k * ld + k];
      const cx<S> piv = cinv(p);
      if (lane == 0 && !finite_nonzero(p)) atomicExch(err, 1);
      cx<S> a = mkc<S>(0, 0), ci = a, rk = a;
      if (lane < n * n) {
        a = A[i * ld + j];
        ci = A[i * ld + k];
        rk = cmul(A[k * ld + j], piv);
      }
      __syncwarp();
      if (lane < n * n) {
        if (i == k) {
          a = (j == k) ? piv : rk;
        } else if (j == k) {
          const cx<S> v = cmul(ci, piv);
          a = mkc<S>(-v.re, -v.im);
        } else {
          cfms(a, ci, rk);
        }
        A[i * ld + j] = a;
      }
      __syncwarp();
    }
    return;
  }
  for (int k = 0; k < n; ++k) {
    const cx<S> p = A[k * ld + k];
    const cx<S> piv = cinv(p);
    if (lane == 0 && !finite_nonzero(p)) atomicExch(err, 1);
    cx<S> rk = lane < n ? cmul(A[k * ld + lane], piv) : mkc<S>(0, 0);
    __syncwarp();
    for (int i = 0; i < n; ++i) {
      const cx<S> ci = A[i * ld + k];
      __syncwarp();
      if (lane < n) {
        cx<S>& a = A[i * ld + lane];
        if (i == k) {
          a = (lane == k) ? piv : rk;
        } else if (lane == k) {
          const cx<S> v = cmul(ci, piv);
          a = mkc<S>(-v.re, -v.im);
        } else {
          cfms(a, ci, rk);
        }
      }
      __syncwarp();
    }
  }
}

template <class S>
static size_t gj_blocked_smem(int b, int CL) {
  const size_t cw = (size_t)(b + CL - 1) / CL;
  return (3 * (b * cw + cw * cw) + 2 * cw * cw) * sizeof(cx<S>);
}

template <class S>
__global__ void __launch_bounds__(256) k_gj_blocked(const cx<S>* __restrict__ Din, cx<S>* Dout,
                                                    const int* __restrict__ list, int b, int* err) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), me = (int)cluster.block_rank();
  const int which = list[blockIdx.x / CL];
  const int cw = (b + CL - 1) / CL, c0 = me * cw, ncol = max(0, min(b, c0 + cw) - c0);
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int pnl = b * cw + cw * cw;  // panel (b x cw) followed by P (cw x cw)
  extern __shared__ __align__(16) unsigned char smgjb[];
  cx<S>* Aown = reinterpret_cast<cx<S>*>(smgjb);  // b x cw
  cx<S>* pub = Aown + pnl;                        // published panel + P (owner step only)
  cx<S>* pan = pub + pnl;                         // local copy of the current panel + P
  cx<S>* tmp = pan + pnl;                         // cw x cw: P A[K, own]
  const size_t bb = (size_t)b * b;
  const cx<S>* src = Din + (size_t)which * bb;
  for (int e = tid; e < b * cw; e += nthr) {
    const int i = e / cw, jl = e - i * cw;
    Aown[e] = jl < ncol ? src[(size_t)i * b + c0 + jl] : mkc<S>(0, 0);
  }
  __syncthreads();
  for (int step = 0; step < CL; ++step) {
    const int k0 = step * cw, kp = max(0, min(b, k0 + cw) - k0);
    if (kp == 0) break;  // same for every CTA of the cluster
    if (me == step) {
      // publish the panel and its pivot block (both read from the CTA's own columns), invert the
      // pivot block; the cluster barrier below also orders this CTA's threads
      cx<S>* Pm = pub + b * cw;
      for (int e = tid; e < b * cw; e += nthr) pub[e] = Aown[e];
      for (int e = tid; e < cw * cw; e += nthr) {
        const int r = e / cw, c = e - r * cw;
        Pm[e] = (r < kp && c < kp) ? Aown[(size_t)(k0 + r) * cw + c] : mkc<S>(0, 0);
      }
      __syncthreads();
      if (tid < 32) gj_small_warp(Pm, kp, cw, err);
    }
    cluster.sync();
    const cx<S>* rp = cluster.map_shared_rank(pub, step);
    for (int e = tid; e < pnl; e += nthr) pan[e] = rp[e];
    __syncthreads();
    const cx<S>* Pm = pan + b * cw;
    if (me != step) {
      // tmp = P A[K, own]
      for (int e = tid; e < kp * cw; e += nthr) {
        const int r = e / cw, jl = e - r * cw;
        cx<S> acc = mkc<S>(0, 0);
        for (int m2 = 0; m2 < kp; ++m2) cfma(acc, Pm[r * cw + m2], Aown[(size_t)(k0 + m2) * cw + jl]);
        tmp[e] = acc;
      }
      __syncthreads();
      for (int e = tid; e < b * cw; e += nthr) {
        const int i = e / cw, jl = e - i * cw;
        if (i >= k0 && i < k0 + kp) {
          Aown[e] = tmp[(i - k0) * cw + jl];
        } else {
          cx<S> a = Aown[e];
          for (int m2 = 0; m2 < kp; ++m2) cfms(a, pan[(size_t)i * cw + m2], tmp[m2 * cw + jl]);
          Aown[e] = a;
        }
      }
    } else {
      for (int e = tid; e < b * cw; e += nthr) {
        const int i = e / cw, kl = e - i * cw;
        if (kl >= kp) continue;
        if (i >= k0 && i < k0 + kp) {
          Aown[e] = Pm[(i - k0) * cw + kl];
        } else {
          cx<S> a = mkc<S>(0, 0);
          for (int m2 = 0; m2 < kp; ++m2) cfms(a, pan[(size_t)i * cw + m2], Pm[m2 * cw + kl]);
          Aown[e] = a;
        }
      }
    }
    __syncthreads();
  }
  cx<S>* dst = Dout + (size_t)which * bb;
  for (int e = tid; e < b * ncol; e += nthr) {
    const int i = e / ncol, jl = e - i * ncol;
    dst[(size_t)i * b + c0 + jl] = Aown[(size_t)i * cw + jl];
  }
  cluster.sync();  // keep this CTA's shared memory alive until every remote read is done
}

// One batched complex GEMM task: C (+)= sum_s alpha_s op(A_s) op(B_s) over up to three operand
// pairs (A_s b x b, B_s b x N, N per task), row-major with leading dimensions.  band (level 0 of
// the reduction, where the blocks still have the stencil's band): 1 = op(A_s) banded, 2 = op(B_s)
// banded, half-width w of the launch.
template <class S>
struct GemmPair {
  const cx<S>* A;
  const cx<S>* B;
  int lda, ldb;
  int transA, transB;
  S alpha;  // real scale (+1 / -1)
  int band;
};
template <class S>
struct GemmTask {
  GemmPair<S> p[3];
  int np;
  cx<S>* C;
  int ldc;
  int accumulate;
  int N;
};

// One block copy: dst = src (count entries), src^T for a b x b block when transpose, zero when
// src is null.
template <class S>
struct CopyTask {
  const cx<S>* src;
  cx<S>* dst;
  long long count;
  int transpose;
};

// Dense tasks: TM x TM output tiles per CTA, 16 x 16 threads with (TM/16)^2 outputs each, K in
// steps of 16 staged in shared memory with alpha folded into the A tile.  FP64 uses 16 x 16 tiles:
// its per-SM rate is low (about 2 FMA per clock), so many CTAs per b x b task keep all SMs busy.
template <class S>
struct GemmTile {
  static constexpr int TM = sizeof(S) == 8 ? 16 : 64;
};

template <class S, int TM>
__global__ void __launch_bounds__(256) k_gemm_batch(const GemmTask<S>* __restrict__ tasks, int M, int Kd) {
  constexpr int Q = TM / 16;
  const GemmTask<S>& tk = tasks[blockIdx.z];
  const int N = tk.N;
  const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TM;
  if (col0 >= N) return;  // tasks narrower than the grid
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  __shared__ cx<S> As[16][TM + 1];
  __shared__ cx<S> Bs[16][TM + 1];
  cx<S> acc[Q][Q];
#pragma unroll
  for (int a = 0; a < Q; ++a)
#pragma unroll
    for (int c = 0; c < Q; ++c) acc[a][c] = mkc<S>(0, 0);
  const int np = tk.np;
  for (int s = 0; s < np; ++s) {
    const GemmPair<S> t = tk.p[s];
    for (int k0 = 0; k0 < Kd; k0 += 16) {
      // operands read along their contiguous dimension so consecutive threads touch consecutive
      // addresses
      if (!t.transA) {
        for (int e = threadIdx.x; e < 16 * TM; e += 256) {
          const int r = e >> 4, kk = e & 15, gr = row0 + r, gk = k0 + kk;
          As[kk][r] = (gr < M && gk < Kd) ? cscale(t.A[(size_t)gr * t.lda + gk], t.alpha) : mkc<S>(0, 0);
        }
      } else {
        for (int e = threadIdx.x; e < 16 * TM; e += 256) {
          const int kk = e / TM, r = e % TM, gr = row0 + r, gk = k0 + kk;
          As[kk][r] = (gr < M && gk < Kd) ? cscale(t.A[(size_t)gk * t.lda + gr], t.alpha) : mkc<S>(0, 0);
        }
      }
      if (t.transB) {
        for (int e = threadIdx.x; e < 16 * TM; e += 256) {
          const int c = e >> 4, kk = e & 15, gc = col0 + c, gk = k0 + kk;
          Bs[kk][c] = (gc < N && gk < Kd) ? t.B[(size_t)gc * t.ldb + gk] : mkc<S>(0, 0);
        }
      } else {
        for (int e = threadIdx.x; e < 16 * TM; e += 256) {
          const int kk = e / TM, c = e % TM, gk = k0 + kk, gc = col0 + c;
          Bs[kk][c] = (gc < N && gk < Kd) ? t.B[(size_t)gk * t.ldb + gc] : mkc<S>(0, 0);
        }
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < 16; ++kk) {
        cx<S> a[Q], bq[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) {
          a[q] = As[kk][ty + 16 * q];
          bq[q] = Bs[kk][tx + 16 * q];
        }
#pragma unroll
        for (int q = 0; q < Q; ++q)
#pragma unroll
          for (int c = 0; c < Q; ++c) cfma(acc[q][c], a[q], bq[c]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      int gr = row0 + ty + 16 * q, gc = col0 + tx + 16 * c;
      if (gr < M && gc < N) {
        cx<S>& o = tk.C[(size_t)gr * tk.ldc + gc];
        o = tk.accumulate ? cadd(o, acc[q][c]) : acc[q][c];
      }
    }
}

// Tasks with banded operands: one thread per output entry, the K range of each pair restricted
// to its band; grid (chunks, tasks).
template <class S>
__global__ void k_gemm_band(const GemmTask<S>* __restrict__ tasks, int M, int Kd, int w) {
  const GemmTask<S>& tk = tasks[blockIdx.y];
  const int N = tk.N;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * N; e += gridDim.x * blockDim.x) {
    const int i = e / N, j = e - i * N;
    cx<S> acc = mkc<S>(0, 0);
    for (int s = 0; s < tk.np; ++s) {
      const GemmPair<S> t = tk.p[s];
      int k0 = 0, k1 = Kd - 1;
      if (t.band == 1) {
        k0 = max(0, i - w);
        k1 = min(Kd - 1, i + w);
      } else if (t.band == 2) {
        k0 = max(0, j - w);
        k1 = min(Kd - 1, j + w);
      }
      cx<S> part = mkc<S>(0, 0);
      for (int k = k0; k <= k1; ++k) {
        const cx<S> a = t.transA ? t.A[(size_t)k * t.lda + i] : t.A[(size_t)i * t.lda + k];
        const cx<S> bv = t.transB ? t.B[(size_t)j * t.ldb + k] : t.B[(size_t)k * t.ldb + j];
        cfma(part, a, bv);
      }
      acc = cadd(acc, cscale(part, t.alpha));
    }
    cx<S>& o = tk.C[(size_t)i * tk.ldc + j];
    o = tk.accumulate ? cadd(o, acc) : acc;
  }
}

// Inverses of tridiagonal b x b blocks (listed), one thread per column of the inverse: the Thomas
// recurrence without pivoting, its multipliers shared through shared memory.
template <class S>
__global__ void k_tri_inverse(const cx<S>* __restrict__ Din, cx<S>* Dout, const int* __restrict__ list, int b,
                              int* err) {
  extern __shared__ __align__(16) unsigned char smtri[];
  cx<S>* cp = reinterpret_cast<cx<S>*>(smtri);  // b: modified super-diagonal c'_i
  cx<S>* dp = cp + b;                           // b: 1 / (pivot_i)
  const int which = list[blockIdx.x];
  const cx<S>* D = Din + (size_t)which * b * b;
  if (threadIdx.x == 0) {
    cx<S> cprev = mkc<S>(0, 0);
    for (int i = 0; i < b; ++i) {
      cx<S> piv = D[(size_t)i * b + i];
      if (i > 0) cfms(piv, D[(size_t)i * b + i - 1], cprev);
      if (!finite_nonzero(piv)) atomicExch(err, 1);
      const cx<S> ip = cinv(piv);
      dp[i] = ip;
      cprev = i + 1 < b ? cmul(D[(size_t)i * b + i + 1], ip) : mkc<S>(0, 0);
      cp[i] = cprev;
    }
  }
  __syncthreads();
  cx<S>* X = Dout + (size_t)which * b * b;
  for (int col = threadIdx.x; col < b; col += blockDim.x) {
    // forward: y_i = (e_col,i - l_i y_{i-1}) / pivot_i with l_i = D[i][i-1]
    cx<S> y = mkc<S>(0, 0);
    for (int i = 0; i < b; ++i) {
      cx<S> r = mkc<S>(i == col ? S(1) : S(0), S(0));
      if (i > 0) cfms(r, D[(size_t)i * b + i - 1], y);
      y = cmul(r, dp[i]);
      X[(size_t)i * b + col] = y;
    }
    // backward: x_i = y_i - c'_i x_{i+1}
    cx<S> x = X[(size_t)(b - 1) * b + col];
    for (int i = b - 2; i >= 0; --i) {
      cx<S> v = X[(size_t)i * b + col];
      cfms(v, cp[i], x);
      x = v;
      X[(size_t)i * b + col] = x;
    }
  }
}

// Batched block copies, grid (chunks, tasks).  Transposed copies are b x b blocks (count = b*b).
template <class S>
__global__ void k_copy_blocks(const CopyTask<S>* __restrict__ tasks, int b) {
  const CopyTask<S> t = tasks[blockIdx.y];
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < t.count; e += (long long)gridDim.x * blockDim.x) {
    cx<S> v = mkc<S>(0, 0);
    if (t.src) {
      if (t.transpose) {
        const int i = (int)(e / b), j = (int)(e - (long long)i * b);
        v = t.src[(size_t)j * b + i];
      } else {
        v = t.src[e];
      }
    }
    t.dst[e] = v;
  }
}

// Gauss-Jordan inversion of a batch of dense b x b blocks, one CTA per block with the block in
// shared memory: threads (tx, ty) of a 32 x 8 grid sweep columns j = tx + 32 c and rows
// i = ty + 8 r, so no index division is needed; two barriers per pivot.
template <class S>
__global__ void __launch_bounds__(256) k_gj_block(const cx<S>* __restrict__ Din, cx<S>* Dout,
                                                  const int* __restrict__ list, int b, int* err) {
  extern __shared__ __align__(16) unsigned char smgj[];
  cx<S>* A = reinterpret_cast<cx<S>*>(smgj);  // b x b
  cx<S>* rowk = A + (size_t)b * b;            // b
  cx<S>* colk = rowk + b;                     // b
  const int which = list[blockIdx.x];
  const size_t bb = (size_t)b * b;
  const cx<S>* src = Din + (size_t)which * bb;
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  for (int e = tid; e < (int)bb; e += 256) A[e] = src[e];
  __syncthreads();
  for (int k = 0; k < b; ++k) {
    const cx<S> p = A[k * b + k];
    const cx<S> piv = cinv(p);
    if (tid == 0 && !finite_nonzero(p)) atomicExch(err, 1);
    for (int j = tid; j < b; j += 256) {
      rowk[j] = cmul(A[k * b + j], piv);
      colk[j] = A[j * b + k];
    }
    __syncthreads();
    for (int i = ty; i < b; i += 8) {
      const cx<S> ci = colk[i];
      cx<S>* Ai = A + (size_t)i * b;
      if (i == k) {
        for (int j = tx; j < b; j += 32) Ai[j] = (j == k) ? piv : rowk[j];
      } else {
        for (int j = tx; j < b; j += 32) {
          if (j == k) {
            const cx<S> v = cmul(ci, piv);
            Ai[j] = mkc<S>(-v.re, -v.im);
          } else {
            cfms(Ai[j], ci, rowk[j]);
          }
        }
      }
    }
    __syncthreads();
  }
  cx<S>* dst = Dout + (size_t)which * bb;
  for (int e = tid; e < (int)bb; e += 256) dst[e] = A[e];
}

template <class S>
static size_t gj_block_smem(int b) {
  return ((size_t)b * b + 2 * (size_t)b) * sizeof(cx<S>);
}

template <class S>
static size_t bcr_gj_smem(int b, int CL) {
  int cw = (b + CL - 1) / CL;
  return ((size_t)b * cw + 3 * (size_t)b + cw) * sizeof(cx<S>);
}

// Inversion of the listed blocks: a cluster per block with column panels (k_gj_blocked), else a
// cluster with one barrier per pivot, else one CTA per block with the block in shared memory.
template <class S>
static cudaError_t launch_gj_batch(const cx<S>* Din, cx<S>* Dout, const int* dlist, int nblk, int b, int* err,
                                   cudaStream_t st) {
  cudaError_t last = cudaErrorInvalidConfiguration;
  if (b >= 16) {
    static const int bsizes[] = {16, 8, 4};
    for (int CL : bsizes) {
      if ((b + CL - 1) / CL > 32) continue;  // the pivot block is inverted by one warp
      const size_t smem = gj_blocked_smem<S>(b, CL);
      if (smem > 200 * 1024) continue;
      cudaError_t e = smem_attr((const void*)k_gj_blocked<S>, (int)smem);
      if (e == cudaSuccess && CL > 8)
        e = cudaFuncSetAttribute(k_gj_blocked<S>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) {
        cudaGetLastError();
        last = e;
        continue;
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(nblk * CL, 1, 1);
      cfg.blockDim = dim3(256, 1, 1);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = CL;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      int ncl = 0;
      e = cudaOccupancyMaxActiveClusters(&ncl, k_gj_blocked<S>, &cfg);
      if (e != cudaSuccess || ncl < 1) {
        cudaGetLastError();
        last = e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
        continue;
      }
      e = cudaLaunchKernelEx(&cfg, k_gj_blocked<S>, Din, Dout, dlist, b, err);
      if (e == cudaSuccess) return cudaSuccess;
      cudaGetLastError();
      last = e;
    }
  }
  static const int sizes[] = {16, 8, 4, 2, 1};
  for (int CL : sizes) {
    if (CL > 1 && nblk * CL > 4 * 152 && CL > 4) continue;  // keep many clusters resident at once
    size_t smem = bcr_gj_smem<S>(b, CL);
    if (smem > 200 * 1024) continue;
    cudaError_t e = smem_attr((const void*)k_gj_batch_cluster<S>, (int)smem);
    if (e == cudaSuccess && CL > 8)
      e = cudaFuncSetAttribute(k_gj_batch_cluster<S>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) {
      cudaGetLastError();
      last = e;
      continue;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nblk * CL, 1, 1);
    cfg.blockDim = dim3(256, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int ncl = 0;
    e = cudaOccupancyMaxActiveClusters(&ncl, k_gj_batch_cluster<S>, &cfg);
    if (e != cudaSuccess || ncl < 1) {
      cudaGetLastError();
      last = e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
      continue;
    }
    e = cudaLaunchKernelEx(&cfg, k_gj_batch_cluster<S>, Din, Dout, dlist, b, err);
    if (e == cudaSuccess) return cudaSuccess;
    cudaGetLastError();
    last = e;
  }
  if (gj_block_smem<S>(b) <= 200 * 1024) {
    const size_t smem = gj_block_smem<S>(b);
    cudaError_t e = smem_attr((const void*)k_gj_block<S>, (int)smem);
    if (e != cudaSuccess) return e;
    k_gj_block<S><<<nblk, 256, smem, st>>>(Din, Dout, dlist, b, err);
    return cudaGetLastError();
  }
  return last;
}

template <class S, class I>
__global__ void k_bcr_convert(const cx<I>* __restrict__ in, cx<S>* out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = ccast<S>(in[i]);
}

// X = [I 0]: n rows of ld >= n entries
template <class T>
__global__ void k_bcr_identity(cx<T>* X, int n, int ld) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * ld; e += (size_t)gridDim.x * blockDim.x)
    X[e] = mkc<T>((e / ld) == (e % ld) ? T(1) : T(0), T(0));
}

// dst block k = src block list[k] (count blocks of bb entries)
template <class T>
__global__ void k_bcr_gather_blocks(const cx<T>* __restrict__ src, const int* __restrict__ list, int count, size_t bb,
                                    cx<T>* dst) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)count * bb;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t k = e / bb;
    dst[e] = src[(size_t)list[k] * bb + (e - k * bb)];
  }
}

// ------------------------------------------------------------------ host orchestration
// Levels: lists of (j, p, q) with p, q = remaining neighbours of j (-1 if none).
static void bcr_schedule(int L, std::vector<std::vector<int>>* lev_j, std::vector<std::vector<int>>* lev_p,
                         std::vector<std::vector<int>>* lev_q) {
  std::vector<int> rem(L);
  for (int i = 0; i < L; ++i) rem[i] = i;
  while (!rem.empty()) {
    std::vector<int> J, Pp, Q, next;
    for (size_t t = 0; t < rem.size(); ++t) {
      if (t % 2 == 0) {
        J.push_back(rem[t]);
        Pp.push_back(t > 0 ? rem[t - 1] : -1);
        Q.push_back(t + 1 < rem.size() ? rem[t + 1] : -1);
      } else {
        next.push_back(rem[t]);
      }
    }
    lev_j->push_back(J);
    lev_p->push_back(Pp);
    lev_q->push_back(Q);
    rem.swap(next);
  }
}

void bcr_level0_maps(int L, std::vector<int>* tgt, std::vector<int>* elim, std::vector<int>* rem) {
  std::vector<std::vector<int>> lj, lp, lq;
  bcr_schedule(L, &lj, &lp, &lq);
  tgt->clear();
  elim->clear();
  rem->clear();
  if (lj.empty()) return;
  std::vector<int> cm(L, -1);  // compact index of the layers that survive level 0
  std::vector<char> gone(L, 0);
  for (int j : lj[0]) gone[j] = 1;
  for (int t = 0; t < L; ++t)
    if (!gone[t]) {
      cm[t] = (int)rem->size();
      rem->push_back(t);
    }
  std::vector<int> jr(L, -1), kr(L, -1), jl(L, -1), kl(L, -1);
  for (size_t k = 0; k < lj[0].size(); ++k) {
    const int j = lj[0][k], p = lp[0][k], q = lq[0][k];
    elim->insert(elim->end(), {j, p >= 0 ? cm[p] : -1, q >= 0 ? cm[q] : -1});
    if (p >= 0) {  // j is the right neighbour of p
      jr[p] = j;
      kr[p] = (int)k;
    }
    if (q >= 0) {  // j is the left neighbour of q
      jl[q] = j;
      kl[q] = (int)k;
    }
  }
  for (int t : *rem) tgt->insert(tgt->end(), {t, jr[t], kr[t], jl[t], kl[t]});
}

// The whole reduction as a list of launches over task arrays that are built on the host and
// uploaded once.
enum BcrOpKind { OP_GJ, OP_TRI, OP_GEMM, OP_BAND, OP_COPY };
struct BcrOp {
  BcrOpKind kind;
  size_t off;  // first task (GEMM, BAND, COPY) or list entry (GJ, TRI)
  int count;
  int maxN;  // GEMM/BAND: widest task; COPY: longest copy
};

template <class T>
struct BcrPlan {
  std::vector<GemmTask<T>> gemm;
  std::vector<CopyTask<T>> copy;
  std::vector<int> list;
  std::vector<BcrOp> ops;
  void add_gemm(std::vector<GemmTask<T>>& ts, bool band) {
    if (ts.empty()) return;
    int mx = 0;
    for (auto& t : ts) mx = std::max(mx, t.N);
    ops.push_back({band ? OP_BAND : OP_GEMM, gemm.size(), (int)ts.size(), mx});
    gemm.insert(gemm.end(), ts.begin(), ts.end());
    ts.clear();
  }
  void add_copy(std::vector<CopyTask<T>>& ts) {
    if (ts.empty()) return;
    long long mx = 0;
    for (auto& t : ts) mx = std::max(mx, t.count);
    ops.push_back({OP_COPY, copy.size(), (int)ts.size(), (int)std::min<long long>(mx, 1 << 30)});
    copy.insert(copy.end(), ts.begin(), ts.end());
    ts.clear();
  }
  void add_inv(const std::vector<int>& J, BcrOpKind kind) {
    ops.push_back({kind, list.size(), (int)J.size(), 0});
    list.insert(list.end(), J.begin(), J.end());
  }
};

template <class S>
static GemmPair<S> pair(const cx<S>* A, int lda, int transA, const cx<S>* B, int ldb, int transB, S alpha, int band) {
  GemmPair<S> q;
  q.A = A;
  q.B = B;
  q.lda = lda;
  q.ldb = ldb;
  q.transA = transA;
  q.transB = transB;
  q.alpha = alpha;
  q.band = band;
  return q;
}

template <class S>
static GemmTask<S> task(cx<S>* C, int ldc, int accumulate, int N, std::initializer_list<GemmPair<S>> ps) {
  GemmTask<S> t = {};
  t.np = 0;
  for (const GemmPair<S>& q : ps) t.p[t.np++] = q;
  t.C = C;
  t.ldc = ldc;
  t.accumulate = accumulate;
  t.N = N;
  return t;
}

// Uploads the task arrays of a plan and launches its operations in order (inversions turn blocks
// of Dsrc into Ddst).
template <class S>
static cudaError_t run_plan(const BcrPlan<S>& plan, GemmTask<S>* dG, CopyTask<S>* dC, int* dL, const cx<S>* Dsrc,
                            cx<S>* Ddst, int b, int w, int* err, cudaStream_t st, long long* launches) {
  if (!plan.gemm.empty()) {
    cudaError_t e = cudaMemcpyAsync(dG, plan.gemm.data(), plan.gemm.size() * sizeof(GemmTask<S>), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  if (!plan.copy.empty()) {
    cudaError_t e = cudaMemcpyAsync(dC, plan.copy.data(), plan.copy.size() * sizeof(CopyTask<S>), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  if (!plan.list.empty()) {
    cudaError_t e = cudaMemcpyAsync(dL, plan.list.data(), plan.list.size() * sizeof(int), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
  }
  constexpr int TM = GemmTile<S>::TM;
  for (const BcrOp& op : plan.ops) {
    cudaError_t e;
    if (op.kind == OP_GJ) {
      e = launch_gj_batch<S>(Dsrc, Ddst, dL + op.off, op.count, b, err, st);
    } else if (op.kind == OP_TRI) {
      k_tri_inverse<S><<<op.count, 64, 2 * b * sizeof(cx<S>), st>>>(Dsrc, Ddst, dL + op.off, b, err);
      e = cudaGetLastError();
    } else if (op.kind == OP_BAND) {
      const int chunks = std::max(1, std::min((b * op.maxN + 255) / 256, 64));
      k_gemm_band<S><<<dim3(chunks, op.count), 256, 0, st>>>(dG + op.off, b, b, w);
      e = cudaGetLastError();
    } else if (op.kind == OP_GEMM) {
      dim3 grid((op.maxN + TM - 1) / TM, (b + TM - 1) / TM, (unsigned)op.count);
      k_gemm_batch<S, TM><<<grid, 256, 0, st>>>(dG + op.off, b, b);
      e = cudaGetLastError();
    } else {
      const int chunks = (int)std::min<long long>(((long long)op.maxN + 255) / 256, 256);
      k_copy_blocks<S><<<dim3(chunks, op.count), 256, 0, st>>>(dC + op.off, b);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    ++*launches;
  }
  return cudaSuccess;
}

// Precision of the coarse factorisation (the block cyclic reduction's pivots and Schur updates)
// for a solve in precision T: FP64 in both forms.  (An FP32 factorisation in the mixed form gave
// the same GMRES iterations, refinement steps and errors on the 1024^2 workload; FP64 is kept as
// the precision of the coarse factorisation.)
template <class T>
using BcrFactor = double;

template <class T>
int coarse_bcr(const StoredProv<double>& P, const BcrLevel0<T>* split, cx<T>* Kinv, int ldk, int* err, cudaStream_t st,
               std::string* msg, long long* launches) {
  const int b = P.ly.b, L = P.ly.L;
  const size_t bb = (size_t)b * b;
  std::vector<std::vector<int>> lj, lp, lq;
  bcr_schedule(L, &lj, &lp, &lq);
  // with the level-0 split the explicit inverse covers the layers that survive level 0 (compact
  // numbering cm), and levels 1.. of the reduction
  const size_t lv0 = split ? 1 : 0;
  std::vector<int> cm(L);
  int Lx = L;
  if (split) {
    std::vector<char> gone(L, 0);
    for (int j : lj[0]) gone[j] = 1;
    Lx = 0;
    for (int t = 0; t < L; ++t) cm[t] = gone[t] ? -1 : Lx++;
  } else {
    for (int t = 0; t < L; ++t) cm[t] = t;
  }
  const size_t n = (size_t)b * Lx;
  auto fail = [&](cudaError_t e, const char* where) {
    if (msg) *msg = std::string("coarse reduction (") + where + "): " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SCHUR_ENOMEM : SCHUR_ECUDA;
  };
#define BCR_CK(x, where)                           \
  do {                                             \
    cudaError_t e_ = (x);                          \
    if (e_ != cudaSuccess) return fail(e_, where); \
  } while (0)
  std::vector<void*> mem;
  auto mal = [&](auto** p, size_t bytes) -> cudaError_t {
    cudaError_t e = cudaMallocAsync((void**)p, std::max<size_t>(bytes, 16), st);
    if (e == cudaSuccess) mem.push_back((void*)*p);
    return e;
  };
  struct Guard {
    std::vector<void*>* m;
    cudaStream_t s;
    ~Guard() {
      for (void* p : *m) cudaFreeAsync(p, s);
    }
  } guard{&mem, st};
  using FP = BcrFactor<T>;  // precision of the factorisation
  using D64 = cx<FP>;
  D64 *D = nullptr, *Ucur = nullptr, *Dinv = nullptr, *Lp = nullptr, *Lq = nullptr, *Unew = nullptr;
  BCR_CK(mal(&D, L * bb * sizeof(D64)), "alloc");
  BCR_CK(mal(&Ucur, L * bb * sizeof(D64)), "alloc");
  BCR_CK(mal(&Dinv, L * bb * sizeof(D64)), "alloc");
  BCR_CK(mal(&Lp, L * bb * sizeof(D64)), "alloc");
  BCR_CK(mal(&Lq, L * bb * sizeof(D64)), "alloc");
  BCR_CK(mal(&Unew, L * bb * sizeof(D64)), "alloc");

  // ---- plan: factorisation.  Level 0 still sees the stencil's band (the layer blocks couple
  // in-layer neighbours only): half-width 1 in 2D, a layer row + 1 in 3D, and in 2D the pivot
  // blocks are tridiagonal and are inverted by the Thomas recurrence.
  const int wband = P.ly.dim == 2 ? 1 : P.ly.ext[0] + 1;
  const bool tri0 = P.ly.dim == 2;
  BcrPlan<FP> fp;
  std::vector<GemmTask<FP>> ts;
  std::vector<CopyTask<FP>> cs;
  const long long lbb = (long long)bb;
  auto blk = [&](D64* base, int K) { return base + (size_t)K * bb; };
  for (size_t lv = 0; lv < lj.size(); ++lv) {
    const std::vector<int>& J = lj[lv];
    const bool band = lv == 0;
    const int bA = band ? 1 : 0, bB = band ? 2 : 0;
    fp.add_inv(J, band && tri0 ? OP_TRI : OP_GJ);  // Dinv_j = D_j^{-1}
    // Lp_j = U_p Dinv_j ; Lq_j = Dinv_j U_j
    for (size_t k = 0; k < J.size(); ++k) {
      const int j = J[k], p = lp[lv][k], q = lq[lv][k];
      if (p >= 0) ts.push_back(task<FP>(blk(Lp, j), b, 0, b, {pair<FP>(blk(Ucur, p), b, 0, blk(Dinv, j), b, 0, FP(1), bA)}));
      if (q >= 0) ts.push_back(task<FP>(blk(Lq, j), b, 0, b, {pair<FP>(blk(Dinv, j), b, 0, blk(Ucur, j), b, 0, FP(1), bB)}));
    }
    fp.add_gemm(ts, band);
    // remaining block t: D_t -= Lp_j U_t^T (t = p of j) and U_j'^T Lq_j' (t = q of j'), one task
    // per t; new coupling A_pq = -Lp_j U_j
    std::vector<int> left_of(L, -1), right_of(L, -1);  // eliminated neighbour j of t on each side
    for (size_t k = 0; k < J.size(); ++k) {
      if (lp[lv][k] >= 0) right_of[lp[lv][k]] = J[k];  // t = p: j is its right neighbour
      if (lq[lv][k] >= 0) left_of[lq[lv][k]] = J[k];   // t = q: j is its left neighbour
    }
    for (int t = 0; t < L; ++t) {
      const int jr = right_of[t], jl = left_of[t];
      if (jr < 0 && jl < 0) continue;
      if (jr >= 0 && jl >= 0)
        ts.push_back(task<FP>(blk(D, t), b, 1, b,
                                  {pair<FP>(blk(Lp, jr), b, 0, blk(Ucur, t), b, 1, FP(-1), bB),
                                   pair<FP>(blk(Ucur, jl), b, 1, blk(Lq, jl), b, 0, FP(-1), bA)}));
      else if (jr >= 0)
        ts.push_back(task<FP>(blk(D, t), b, 1, b, {pair<FP>(blk(Lp, jr), b, 0, blk(Ucur, t), b, 1, FP(-1), bB)}));
      else
        ts.push_back(task<FP>(blk(D, t), b, 1, b, {pair<FP>(blk(Ucur, jl), b, 1, blk(Lq, jl), b, 0, FP(-1), bA)}));
    }
    for (size_t k = 0; k < J.size(); ++k) {
      const int j = J[k], p = lp[lv][k], q = lq[lv][k];
      if (p >= 0 && q >= 0)
        ts.push_back(task<FP>(blk(Unew, p), b, 0, b, {pair<FP>(blk(Lp, j), b, 0, blk(Ucur, j), b, 0, FP(-1), bB)}));
    }
    fp.add_gemm(ts, band);
    // the remaining p whose right neighbour j was eliminated now couples to q (or to nothing)
    for (size_t k = 0; k < J.size(); ++k) {
      const int p = lp[lv][k], q = lq[lv][k];
      if (p >= 0) cs.push_back({q >= 0 ? blk(Unew, p) : nullptr, blk(Ucur, p), lbb, 0});
    }
    fp.add_copy(cs);
  }

  // ---- factor operands of the solve in precision T
  cx<T>*DinvT = nullptr, *LpT = nullptr, *LqT = nullptr, *Tmp = nullptr;
  if (sizeof(T) == sizeof(FP)) {
    DinvT = reinterpret_cast<cx<T>*>(Dinv);
    LpT = reinterpret_cast<cx<T>*>(Lp);
    LqT = reinterpret_cast<cx<T>*>(Lq);
  } else {
    BCR_CK(mal(&DinvT, L * bb * sizeof(cx<T>)), "alloc");
    BCR_CK(mal(&LpT, L * bb * sizeof(cx<T>)), "alloc");
    BCR_CK(mal(&LqT, L * bb * sizeof(cx<T>)), "alloc");
  }
  // the backward sweep overwrites X_j in place when one CTA spans the b rows of a tile column;
  // otherwise it writes to Tmp and copies back
  constexpr int TMi = GemmTile<T>::TM;
  const bool inplace = TMi >= b;
  if (!inplace) BCR_CK(mal(&Tmp, n * (size_t)ldk * sizeof(cx<T>)), "alloc");

  // ---- plan: explicit inverse, X = I in place in Kinv.  Forward products only touch the block
  // columns where row block j can be nonzero: [lo_j, hi_j], which starts as {j} and grows by the
  // ranges of the eliminated neighbours.
  BcrPlan<T> ip;
  std::vector<GemmTask<T>> ti;
  std::vector<CopyTask<T>> ci;
  const size_t bN = (size_t)b * ldk;  // one block row of X (row stride ldk)
  const int N = (int)n;
  auto tb = [&](cx<T>* base, int K) { return base + (size_t)K * bb; };
  // row block of layer K (compact numbering), block column c0
  auto xb = [&](cx<T>* base, int K, int c0) { return base + (size_t)cm[K] * bN + (size_t)c0 * b; };
  std::vector<int> lo(L), hi(L);
  for (int i = 0; i < L; ++i) lo[i] = hi[i] = cm[i];
  for (size_t lv = lv0; lv < lj.size(); ++lv) {
    std::vector<int> left_of(L, -1), right_of(L, -1);
    for (size_t k = 0; k < lj[lv].size(); ++k) {
      if (lp[lv][k] >= 0) right_of[lp[lv][k]] = lj[lv][k];
      if (lq[lv][k] >= 0) left_of[lq[lv][k]] = lj[lv][k];
    }
    // X_t -= Lp_jr X_jr (t = p of jr) + Lq_jl^T X_jl (t = q of jl) on the union of their ranges
    for (int t = 0; t < L; ++t) {
      const int jr = right_of[t], jl = left_of[t];
      if (jr < 0 && jl < 0) continue;
      int c0 = 1 << 30, c1 = -1;
      if (jr >= 0) {
        c0 = std::min(c0, lo[jr]);
        c1 = std::max(c1, hi[jr]);
      }
      if (jl >= 0) {
        c0 = std::min(c0, lo[jl]);
        c1 = std::max(c1, hi[jl]);
      }
      const int w = (c1 - c0 + 1) * b;
      if (jr >= 0 && jl >= 0)
        ti.push_back(task<T>(xb(Kinv, t, c0), ldk, 1, w,
                             {pair<T>(tb(LpT, jr), b, 0, xb(Kinv, jr, c0), ldk, 0, T(-1), 0),
                              pair<T>(tb(LqT, jl), b, 1, xb(Kinv, jl, c0), ldk, 0, T(-1), 0)}));
      else if (jr >= 0)
        ti.push_back(task<T>(xb(Kinv, t, c0), ldk, 1, w, {pair<T>(tb(LpT, jr), b, 0, xb(Kinv, jr, c0), ldk, 0, T(-1), 0)}));
      else
        ti.push_back(task<T>(xb(Kinv, t, c0), ldk, 1, w, {pair<T>(tb(LqT, jl), b, 1, xb(Kinv, jl, c0), ldk, 0, T(-1), 0)}));
    }
    ip.add_gemm(ti, false);
    for (int t = 0; t < L; ++t) {
      for (int j : {right_of[t], left_of[t]}) {
        if (j >= 0) {
          lo[t] = std::min(lo[t], lo[j]);
          hi[t] = std::max(hi[t], hi[j]);
        }
      }
    }
  }
  for (int lv = (int)lj.size() - 1; lv >= (int)lv0; --lv) {
    // X_j = Dinv_j X_j - Lp_j^T X_p - Lq_j X_q
    for (size_t k = 0; k < lj[lv].size(); ++k) {
      const int j = lj[lv][k], p = lp[lv][k], q = lq[lv][k];
      cx<T>* out = inplace ? xb(Kinv, j, 0) : xb(Tmp, j, 0);
      GemmTask<T> t = task<T>(out, ldk, 0, N, {pair<T>(tb(DinvT, j), b, 0, xb(Kinv, j, 0), ldk, 0, T(1), 0)});
      if (p >= 0) t.p[t.np++] = pair<T>(tb(LpT, j), b, 1, xb(Kinv, p, 0), ldk, 0, T(-1), 0);
      if (q >= 0) t.p[t.np++] = pair<T>(tb(LqT, j), b, 0, xb(Kinv, q, 0), ldk, 0, T(-1), 0);
      ti.push_back(t);
      if (!inplace) ci.push_back({xb(Tmp, j, 0), xb(Kinv, j, 0), (long long)bN, 0});
    }
    ip.add_gemm(ti, false);
    ip.add_copy(ci);
  }

  // ---- device task arrays
  GemmTask<FP>* dG = nullptr;
  CopyTask<FP>* dC = nullptr;
  int* dL = nullptr;
  GemmTask<T>* dGi = nullptr;
  CopyTask<T>* dCi = nullptr;
  BCR_CK(mal(&dG, fp.gemm.size() * sizeof(GemmTask<FP>)), "alloc");
  BCR_CK(mal(&dC, fp.copy.size() * sizeof(CopyTask<FP>)), "alloc");
  BCR_CK(mal(&dL, fp.list.size() * sizeof(int)), "alloc");
  BCR_CK(mal(&dGi, ip.gemm.size() * sizeof(GemmTask<T>)), "alloc");
  BCR_CK(mal(&dCi, ip.copy.size() * sizeof(CopyTask<T>)), "alloc");

  // ---- run: factorisation
  const int gs = (int)std::min<size_t>((L * bb + 255) / 256, 4096);
  prof_start(KC_COARSE_SETUP, st);
  k_bcr_densify<FP><<<gs, 256, 0, st>>>(P, D, Ucur);
  BCR_CK(cudaGetLastError(), "densify");
  ++*launches;
  BCR_CK(run_plan<FP>(fp, dG, dC, dL, D, Dinv, b, wband, err, st, launches), "factorisation");
  prof_stop(KC_COARSE_SETUP, st);
  // ---- run: explicit inverse
  prof_start(KC_COARSE_INV, st);
  if (sizeof(T) != sizeof(FP)) {
    k_bcr_convert<T><<<gs, 256, 0, st>>>(Dinv, DinvT, L * bb);
    k_bcr_convert<T><<<gs, 256, 0, st>>>(Lp, LpT, L * bb);
    k_bcr_convert<T><<<gs, 256, 0, st>>>(Lq, LqT, L * bb);
    BCR_CK(cudaGetLastError(), "convert");
    *launches += 3;
  }
  if (split) {
    // the level-0 blocks for the per-apply forward and backward steps
    const std::vector<int>& J0 = lj[0];
    int* dJ = nullptr;
    BCR_CK(mal(&dJ, J0.size() * sizeof(int)), "alloc");
    BCR_CK(cudaMemcpyAsync(dJ, J0.data(), J0.size() * sizeof(int), cudaMemcpyHostToDevice, st), "upload");
    const int gg = (int)std::min<size_t>((J0.size() * bb + 255) / 256, 4096);
    k_bcr_gather_blocks<T><<<gg, 256, 0, st>>>(DinvT, dJ, (int)J0.size(), bb, split->D0);
    k_bcr_gather_blocks<T><<<gg, 256, 0, st>>>(LpT, dJ, (int)J0.size(), bb, split->Lp0);
    k_bcr_gather_blocks<T><<<gg, 256, 0, st>>>(LqT, dJ, (int)J0.size(), bb, split->Lq0);
    BCR_CK(cudaGetLastError(), "level-0 blocks");
    *launches += 3;
  }
  k_bcr_identity<T><<<(int)std::min<size_t>((n * ldk + 255) / 256, 8192), 256, 0, st>>>(Kinv, (int)n, ldk);
  BCR_CK(cudaGetLastError(), "identity");
  ++*launches;
  BCR_CK(run_plan<T>(ip, dGi, dCi, nullptr, nullptr, nullptr, b, 0, err, st, launches), "inverse");
  prof_stop(KC_COARSE_INV, st);
  // no synchronisation: the host arrays were pageable (staged when each copy was issued) and the
  // temporaries are released in stream order
  return SCHUR_OK;
#undef BCR_CK
}

template int coarse_bcr<float>(const StoredProv<double>&, const BcrLevel0<float>*, cx<float>*, int, int*, cudaStream_t,
                                std::string*, long long*);
template int coarse_bcr<double>(const StoredProv<double>&, const BcrLevel0<double>*, cx<double>*, int, int*,
                                 cudaStream_t, std::string*, long long*);

}  // namespace schur
