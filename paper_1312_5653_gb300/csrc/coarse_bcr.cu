// Block cyclic reduction (odd-even reduction over layers) of the coarse corner matrix.
//
// The coarse matrix of Sec. 5 is block tridiagonal over the layers of the corner grid.  Instead of
// the sequential layer recursion, every level eliminates every other remaining layer j at once:
//   Dinv_j = D_j^{-1},  Lp = A_pj Dinv_j,  Lq = A_qj Dinv_j,
//   D_p -= Lp A_jp,  D_q -= Lq A_jq,  A_pq = -Lp A_jq          (p, q: remaining neighbours of j)
// so the critical path is log2(L) levels of batched dense work.  The factor and the explicit
// inverse (a cyclic-reduction solve with the identity as right-hand side) are computed in the
// working precision of the solver: FP64, or FP32 for the inner solver of the mixed form, whose
// outer FP64 refinement absorbs the rounding of the coarse problem like that of the local ones.
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

// One batched complex GEMM task: C (+)= alpha * A * op(B), all b x b (or b x N for the solve),
// row-major with leading dimensions; transB: use B^T.
template <class S>
struct GemmTask {
  const cx<S>* A;
  const cx<S>* B;
  cx<S>* C;
  int lda, ldb, ldc;
  int transB;
  S alpha;  // real scale (+1 / -1)
  int accumulate;
};

// C[M x N] (+)= alpha * A[M x Kd] * B[Kd x N]  (B^T when transB), TM x TM output tiles per CTA,
// 16 x 16 threads with (TM/16)^2 outputs each, K in steps of 16 staged in shared memory.  FP64 uses
// 32 x 32 tiles: its per-SM rate is low, so more CTAs per b x b task keep more SMs busy.
template <class S>
struct GemmTile {
  static constexpr int TM = sizeof(S) == 8 ? 32 : 64;
};

template <class S, int TM>
__global__ void __launch_bounds__(256) k_gemm_batch(const GemmTask<S>* __restrict__ tasks, int M, int N, int Kd) {
  constexpr int Q = TM / 16;
  const GemmTask<S> t = tasks[blockIdx.z];
  const int row0 = blockIdx.y * TM, col0 = blockIdx.x * TM;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  __shared__ cx<S> As[16][TM + 1];
  __shared__ cx<S> Bs[16][TM + 1];
  cx<S> acc[Q][Q];
#pragma unroll
  for (int a = 0; a < Q; ++a)
#pragma unroll
    for (int c = 0; c < Q; ++c) acc[a][c] = mkc<S>(0, 0);
  for (int k0 = 0; k0 < Kd; k0 += 16) {
    for (int e = threadIdx.x; e < 16 * TM; e += 256) {
      int kk = e / TM, r = e % TM;
      int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < M && gk < Kd) ? t.A[(size_t)gr * t.lda + gk] : mkc<S>(0, 0);
      int gc = col0 + r;
      cx<S> bv = mkc<S>(0, 0);
      if (gc < N && gk < Kd) bv = t.transB ? t.B[(size_t)gc * t.ldb + gk] : t.B[(size_t)gk * t.ldb + gc];
      Bs[kk][r] = bv;
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
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int c = 0; c < Q; ++c) {
      int gr = row0 + ty + 16 * q, gc = col0 + tx + 16 * c;
      if (gr < M && gc < N) {
        cx<S>& o = t.C[(size_t)gr * t.ldc + gc];
        cx<S> v = cscale(acc[q][c], t.alpha);
        o = t.accumulate ? cadd(o, v) : v;
      }
    }
}

template <class S>
static cudaError_t launch_gemms(const std::vector<GemmTask<S>>& tasks, GemmTask<S>* dtasks, int M, int N, int Kd,
                                cudaStream_t st) {
  if (tasks.empty()) return cudaSuccess;
  cudaError_t e = cudaMemcpyAsync(dtasks, tasks.data(), tasks.size() * sizeof(GemmTask<S>), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  constexpr int TM = GemmTile<S>::TM;
  dim3 grid((N + TM - 1) / TM, (M + TM - 1) / TM, (unsigned)tasks.size());
  k_gemm_batch<S, TM><<<grid, 256, 0, st>>>(dtasks, M, N, Kd);
  return cudaGetLastError();
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

template <class S>
static size_t bcr_gj_smem(int b, int CL) {
  int cw = (b + CL - 1) / CL;
  return ((size_t)b * cw + 3 * (size_t)b + cw) * sizeof(cx<S>);
}

template <class S>
static cudaError_t launch_gj_batch(const cx<S>* Din, cx<S>* Dout, const int* dlist, int nblk, int b, int* err,
                                   cudaStream_t st) {
  static const int sizes[] = {16, 8, 4, 2, 1};
  cudaError_t last = cudaErrorInvalidConfiguration;
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
  return last;
}

template <class T>
__global__ void k_bcr_identity(cx<T>* X, int n) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)n * n; e += (size_t)gridDim.x * blockDim.x)
    X[e] = mkc<T>((e / n) == (e % n) ? T(1) : T(0), T(0));
}

// Solve with the reduction factors for the right-hand side X (n_c x N, row-major, rows grouped by
// layer), in place.  Dinv_j, UP_j = A_pj and UQ_j = A_jq in precision S; UP + L*b*b and
// UQ + L*b*b hold their transposes.  Updates of one block by two neighbours go to separate
// launches, so no launch has two tasks writing the same block.
template <class S>
static cudaError_t bcr_solve(const cx<S>* Dinv, const cx<S>* UP, const cx<S>* UQ, int b, int L,
                             const std::vector<std::vector<int>>& lj, const std::vector<std::vector<int>>& lp,
                             const std::vector<std::vector<int>>& lq, cx<S>* X, cx<S>* Tmp, int N,
                             GemmTask<S>* dt, cudaStream_t st) {
  const size_t bb = (size_t)b * b, bN = (size_t)b * N;
  const cx<S>* UPT = UP + (size_t)L * bb;
  const cx<S>* UQT = UQ + (size_t)L * bb;
  cudaError_t e = cudaSuccess;
  for (size_t lv = 0; lv < lj.size() && e == cudaSuccess; ++lv) {
    std::vector<GemmTask<S>> t1, ta, tb;
    for (size_t k = 0; k < lj[lv].size(); ++k) {
      const int j = lj[lv][k], p = lp[lv][k], q = lq[lv][k];
      t1.push_back({Dinv + j * bb, X + j * bN, Tmp + j * bN, b, N, N, 0, S(1), 0});  // Tmp_j = Dinv_j X_j
      if (p >= 0) ta.push_back({UP + j * bb, Tmp + j * bN, X + p * bN, b, N, N, 0, S(-1), 1});   // X_p -= A_pj Tmp_j
      if (q >= 0) tb.push_back({UQT + j * bb, Tmp + j * bN, X + q * bN, b, N, N, 0, S(-1), 1});  // X_q -= A_qj Tmp_j
    }
    e = launch_gemms(t1, dt, b, N, b, st);
    if (e == cudaSuccess) e = launch_gemms(ta, dt + t1.size(), b, N, b, st);
    if (e == cudaSuccess) e = launch_gemms(tb, dt + t1.size() + ta.size(), b, N, b, st);
  }
  for (int lv = (int)lj.size() - 1; lv >= 0 && e == cudaSuccess; --lv) {
    std::vector<GemmTask<S>> ta, tb, t2;
    for (size_t k = 0; k < lj[lv].size(); ++k) {
      const int j = lj[lv][k], p = lp[lv][k], q = lq[lv][k];
      if (p >= 0) ta.push_back({UPT + j * bb, X + p * bN, X + j * bN, b, N, N, 0, S(-1), 1});  // X_j -= A_jp X_p
      if (q >= 0) tb.push_back({UQ + j * bb, X + q * bN, X + j * bN, b, N, N, 0, S(-1), 1});   // X_j -= A_jq X_q
      t2.push_back({Dinv + j * bb, X + j * bN, Tmp + j * bN, b, N, N, 0, S(1), 0});
    }
    e = launch_gemms(ta, dt, b, N, b, st);
    if (e == cudaSuccess) e = launch_gemms(tb, dt + ta.size(), b, N, b, st);
    if (e == cudaSuccess) e = launch_gemms(t2, dt + ta.size() + tb.size(), b, N, b, st);
    for (size_t k = 0; k < lj[lv].size() && e == cudaSuccess; ++k) {
      const int j = lj[lv][k];
      e = cudaMemcpyAsync(X + j * bN, Tmp + j * bN, bN * sizeof(cx<S>), cudaMemcpyDeviceToDevice, st);
    }
  }
  return e;
}

template <class S>
__global__ void k_bcr_transpose(const cx<S>* __restrict__ in, cx<S>* out, int b, int L) {
  const size_t bb = (size_t)b * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)L * bb; e += (size_t)gridDim.x * blockDim.x) {
    size_t K = e / bb, r = e % bb;
    int i = (int)(r / b), j = (int)(r % b);
    out[K * bb + (size_t)j * b + i] = in[e];
  }
}

template <class T>
int coarse_bcr(const StoredProv<double>& P, cx<T>* Kinv, int* err, cudaStream_t st, std::string* msg,
               long long* launches) {
  const int b = P.ly.b, L = P.ly.L;
  const size_t bb = (size_t)b * b, n = (size_t)b * L;
  std::vector<std::vector<int>> lj, lp, lq;
  bcr_schedule(L, &lj, &lp, &lq);
  cx<T>*D = nullptr, *Ucur = nullptr, *Dinv = nullptr, *UP = nullptr, *UQ = nullptr, *Lp = nullptr, *Lq = nullptr,
        *Unew = nullptr;
  int* dlist = nullptr;
  GemmTask<T>* dtT = nullptr;
  auto fail = [&](cudaError_t e, const char* where) {
    if (msg) *msg = std::string("coarse reduction (") + where + "): " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SCHUR_ENOMEM : SCHUR_ECUDA;
  };
#define BCR_CK(x, where)                    \
  do {                                      \
    cudaError_t e_ = (x);                   \
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
  BCR_CK(mal(&D, L * bb * sizeof(cx<T>)), "alloc");
  BCR_CK(mal(&Ucur, L * bb * sizeof(cx<T>)), "alloc");
  BCR_CK(mal(&Dinv, L * bb * sizeof(cx<T>)), "alloc");
  BCR_CK(mal(&UP, 2 * L * bb * sizeof(cx<T>)), "alloc");  // UP_j, then its transposes
  BCR_CK(mal(&UQ, 2 * L * bb * sizeof(cx<T>)), "alloc");  // UQ_j, then its transposes
  BCR_CK(mal(&Lp, L * bb * sizeof(cx<T>)), "alloc");
  BCR_CK(mal(&Lq, L * bb * sizeof(cx<T>)), "alloc");
  BCR_CK(mal(&Unew, L * bb * sizeof(cx<T>)), "alloc");
  BCR_CK(mal(&dlist, (size_t)L * sizeof(int)), "alloc");
  BCR_CK(mal(&dtT, (size_t)4 * L * sizeof(GemmTask<T>)), "alloc");
  BCR_CK(cudaMemsetAsync(UP, 0, 2 * L * bb * sizeof(cx<T>), st), "memset");
  BCR_CK(cudaMemsetAsync(UQ, 0, 2 * L * bb * sizeof(cx<T>), st), "memset");
  const int gs = (int)std::min<size_t>((L * bb + 255) / 256, 4096);
  k_bcr_densify<T><<<gs, 256, 0, st>>>(P, D, Ucur);
  BCR_CK(cudaGetLastError(), "densify");
  ++*launches;
  // ---- factorisation
  prof_start(KC_COARSE_SETUP, st);
  for (size_t lv = 0; lv < lj.size(); ++lv) {
    const std::vector<int>& J = lj[lv];
    BCR_CK(cudaMemcpyAsync(dlist, J.data(), J.size() * sizeof(int), cudaMemcpyHostToDevice, st), "list");
    BCR_CK(launch_gj_batch<T>(D, Dinv, dlist, (int)J.size(), b, err, st), "inversion");
    ++*launches;
    std::vector<GemmTask<T>> t1;
    for (size_t k = 0; k < J.size(); ++k) {
      int j = J[k], p = lp[lv][k], q = lq[lv][k];
      if (p >= 0) {
        // UP_j = A_pj = Ucur_p ; Lp_j = UP_j Dinv_j
        BCR_CK(cudaMemcpyAsync(UP + j * bb, Ucur + p * bb, bb * sizeof(cx<T>), cudaMemcpyDeviceToDevice, st), "copy");
        t1.push_back({Ucur + p * bb, Dinv + j * bb, Lp + j * bb, b, b, b, 0, T(1), 0});
      }
      if (q >= 0) {
        // UQ_j = A_jq = Ucur_j ; Lq_j = A_qj Dinv_j = UQ_j^T Dinv_j  -> computed as (Dinv_j UQ_j)^T:
        // Dinv_j is symmetric, so Lq_j^T = Dinv_j UQ_j; store W = Dinv_j UQ_j and use its transpose
        BCR_CK(cudaMemcpyAsync(UQ + j * bb, Ucur + j * bb, bb * sizeof(cx<T>), cudaMemcpyDeviceToDevice, st), "copy");
        t1.push_back({Dinv + j * bb, Ucur + j * bb, Lq + j * bb, b, b, b, 0, T(1), 0});  // Lq holds Dinv_j A_jq
      }
    }
    BCR_CK(launch_gemms(t1, dtT, b, b, b, st), "gemm L");
    ++*launches;
    // D_p -= Lp_j A_jp = Lp_j UP_j^T ; D_q -= A_qj Dinv_j A_jq = UQ_j^T (Dinv_j UQ_j) = UQ_j^T Lq_j
    // A_pq (new coupling from p) = -Lp_j A_jq = -Lp_j UQ_j
    // Launch 1: updates from the right neighbour j of p (D_p, Unew_p); launch 2: from the left
    // neighbour j' of q (D_q).  No two tasks of one launch write the same block.
    std::vector<GemmTask<T>> ta, tb;
    for (size_t k = 0; k < J.size(); ++k) {
      int j = J[k], p = lp[lv][k], q = lq[lv][k];
      if (p >= 0) {
        ta.push_back({Lp + j * bb, UP + j * bb, D + p * bb, b, b, b, 1, T(-1), 1});
        if (q >= 0) tb.push_back({Lp + j * bb, UQ + j * bb, Unew + p * bb, b, b, b, 0, T(-1), 0});
      }
    }
    BCR_CK(launch_gemms(ta, dtT, b, b, b, st), "gemm Dp");
    BCR_CK(launch_gemms(tb, dtT + ta.size(), b, b, b, st), "gemm Upq");
    // D_q -= UQ_j^T Lq_j: transpose UQ_j into UQ + L*bb, then a plain GEMM
    k_bcr_transpose<T><<<gs, 256, 0, st>>>(UQ, UQ + (size_t)L * bb, b, L);
    BCR_CK(cudaGetLastError(), "transpose");
    std::vector<GemmTask<T>> tc;
    for (size_t k = 0; k < J.size(); ++k) {
      int j = J[k], q = lq[lv][k];
      if (q >= 0) tc.push_back({UQ + (size_t)L * bb + j * bb, Lq + j * bb, D + q * bb, b, b, b, 0, T(-1), 1});
    }
    BCR_CK(launch_gemms(tc, dtT + ta.size() + tb.size(), b, b, b, st), "gemm Dq");
    *launches += 4;
    // remaining p whose right neighbour j was eliminated now couples to q
    for (size_t k = 0; k < J.size(); ++k) {
      int p = lp[lv][k], q = lq[lv][k];
      if (p >= 0) {
        if (q >= 0)
          BCR_CK(cudaMemcpyAsync(Ucur + p * bb, Unew + p * bb, bb * sizeof(cx<T>), cudaMemcpyDeviceToDevice, st), "copy");
        else
          BCR_CK(cudaMemsetAsync(Ucur + p * bb, 0, bb * sizeof(cx<T>), st), "memset");
      }
    }
  }
  // transposes of UP (for back substitution) and UQ (forward), kept behind the originals
  k_bcr_transpose<T><<<gs, 256, 0, st>>>(UP, UP + (size_t)L * bb, b, L);
  k_bcr_transpose<T><<<gs, 256, 0, st>>>(UQ, UQ + (size_t)L * bb, b, L);
  BCR_CK(cudaGetLastError(), "transpose");
  prof_stop(KC_COARSE_SETUP, st);
  // ---- explicit inverse: solve with the identity
  prof_start(KC_COARSE_INV, st);
  // solved in place in Kinv; the inverse is symmetric, so its rows are the solution columns
  cx<T>* Tmp = nullptr;
  BCR_CK(mal(&Tmp, n * n * sizeof(cx<T>)), "alloc");
  k_bcr_identity<T><<<(int)std::min<size_t>((n * n + 255) / 256, 8192), 256, 0, st>>>(Kinv, (int)n);
  BCR_CK(cudaGetLastError(), "identity");
  BCR_CK(bcr_solve<T>(Dinv, UP, UQ, b, L, lj, lp, lq, Kinv, Tmp, (int)n, dtT, st), "solve");
  prof_stop(KC_COARSE_INV, st);
  BCR_CK(cudaStreamSynchronize(st), "sync");
  *launches += 8;
  return SCHUR_OK;
#undef BCR_CK
}

template int coarse_bcr<float>(const StoredProv<double>&, cx<float>*, int*, cudaStream_t, std::string*, long long*);
template int coarse_bcr<double>(const StoredProv<double>&, cx<double>*, int*, cudaStream_t, std::string*, long long*);

}  // namespace schur
