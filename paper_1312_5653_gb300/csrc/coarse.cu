// FP64 layered block LDL^T of the coarse corner matrix on one thread-block cluster.
//
// The coarse matrix of Sec. 5 (the "extra coarse problem" on the primal corners) is block
// tridiagonal on the corner grid; its layer blocks are dense after a few layers and every layer
// needs one explicit inverse D_K^{-1}.  FP64 throughput per SM is small on this GPU, so each
// Gauss-Jordan pivot step is spread over the CTAs of a cluster: CTA r owns a block of columns
// of D_K in shared memory, the owner of pivot column k publishes it in a double-buffered shared
// buffer, one cluster barrier per pivot orders publication and remote (DSMEM) reads, and every CTA
// updates its own columns.  The Schur update D_{K+1} = A_{K+1,K+1} - A_{K+1,K} D_K^{-1} A_{K,K+1}
// uses the sparse coupling blocks (in-layer 3^(d-1) neighbours) and reads D_K^{-1} columns of other
// CTAs from global memory after a fence and a cluster barrier.
#include <cooperative_groups.h>

#include <algorithm>

#include "coarse.h"

namespace cg = cooperative_groups;

namespace schur {

__global__ void __launch_bounds__(256) k_coarse_factor_cluster(StoredProv<double> P, cx<double>* Dinv, int* err) {
  cg::cluster_group cluster = cg::this_cluster();
  const int CL = (int)cluster.num_blocks(), me = (int)cluster.block_rank();
  const int b = P.ly.b, L = P.ly.L, nt = nbr_count(P.ly.dim);
  const int cw = (b + CL - 1) / CL, c0 = me * cw, c1 = min(b, c0 + cw), ncol = max(0, c1 - c0);
  const int tid = threadIdx.x, nthr = blockDim.x;
  extern __shared__ unsigned char smraw[];
  cx<double>* Dl = reinterpret_cast<cx<double>*>(smraw);  // b x cw, row-major [i*cw + jl]
  cx<double>* Wl = Dl + (size_t)b * cw;                    // b x cw
  cx<double>* colk = Wl + (size_t)b * cw;                  // b
  cx<double>* bcast = colk + b;                            // 2 x b (published pivot column)
  cx<double>* rowk = bcast + 2 * b;                        // cw
  const size_t bb = (size_t)b * b;

  for (int e = tid; e < b * cw; e += nthr) {
    int i = e / cw, jl = e - i * cw, j = c0 + jl;
    cx<double> v = mkc<double>(0, 0);
    if (jl < ncol) {
      int t = nbr_slot(P.ly, i, j);
      if (t >= 0) v = P.Ad(0, i, t);
    }
    Dl[e] = v;
  }
  __syncthreads();
  for (int K = 0; K < L; ++K) {
    // ---- Gauss-Jordan inversion of D_K, columns distributed over the cluster
    for (int k = 0; k < b; ++k) {
      const int owner = k / cw;
      cx<double>* pub = bcast + (k & 1) * b;
      if (me == owner)
        for (int i = tid; i < b; i += nthr) pub[i] = Dl[i * cw + (k - c0)];
      cluster.sync();
      const cx<double>* src = cluster.map_shared_rank(pub, owner);
      for (int i = tid; i < b; i += nthr) colk[i] = src[i];
      __syncthreads();
      const cx<double> p = colk[k];
      const cx<double> piv = cinv(p);
      if (tid == 0 && me == 0 && !finite_nonzero(p)) atomicExch(err, 1);
      for (int jl = tid; jl < ncol; jl += nthr) rowk[jl] = cmul(Dl[k * cw + jl], piv);
      __syncthreads();
      for (int e = tid; e < b * ncol; e += nthr) {
        int i = e / ncol, jl = e - i * ncol, j = c0 + jl;
        cx<double>& a = Dl[i * cw + jl];
        if (j == k) {
          if (i == k) {
            a = piv;
          } else {
            cx<double> v = cmul(colk[i], piv);
            a = mkc<double>(-v.re, -v.im);
          }
        } else if (i == k) {
          a = rowk[jl];
        } else {
          cfms(a, colk[i], rowk[jl]);
        }
      }
      __syncthreads();
    }
    // ---- publish D_K^{-1}
    cx<double>* out = Dinv + (size_t)K * bb;
    for (int e = tid; e < b * ncol; e += nthr) {
      int i = e / ncol, jl = e - i * ncol;
      out[(size_t)i * b + c0 + jl] = Dl[i * cw + jl];
    }
    if (K + 1 == L) break;
    __threadfence();
    cluster.sync();
    // ---- W = D_K^{-1} A_{K,K+1} (own columns), then D_{K+1}
    for (int e = tid; e < b * ncol; e += nthr) {
      int k = e / ncol, jl = e - k * ncol, j = c0 + jl;
      cx<double> acc = mkc<double>(0, 0);
      for (int t = 0; t < nt; ++t) {
        int m = nbr_of(P.ly, j, t);
        if (m >= 0) cfma(acc, out[(size_t)k * b + m], P.Al(K, j, t));
      }
      Wl[k * cw + jl] = acc;
    }
    __syncthreads();
    for (int e = tid; e < b * ncol; e += nthr) {
      int i = e / ncol, jl = e - i * ncol, j = c0 + jl;
      int tj = nbr_slot(P.ly, i, j);
      cx<double> acc = tj >= 0 ? P.Ad(K + 1, i, tj) : mkc<double>(0, 0);
      for (int t = 0; t < nt; ++t) {
        int k = nbr_of(P.ly, i, t);
        if (k >= 0) cfms(acc, P.Al(K, i, t), Wl[k * cw + jl]);
      }
      Dl[i * cw + jl] = acc;
    }
    // the next pivot publication is preceded by this block's barrier and a cluster barrier
    __syncthreads();
  }
  // no CTA may exit while others can still read its shared memory
  cluster.sync();
}

size_t coarse_cluster_smem(int b, int CL) {
  int cw = (b + CL - 1) / CL;
  return ((size_t)2 * b * cw + 3 * (size_t)b + cw) * sizeof(cx<double>);
}

cudaError_t coarse_factor_cluster(const StoredProv<double>& P, cx<double>* Dinv, int* err, cudaStream_t st,
                                  int* cluster_used) {
  static const int sizes[] = {16, 8, 4, 2, 1};
  cudaError_t last = cudaSuccess;
  for (int CL : sizes) {
    size_t smem = coarse_cluster_smem(P.ly.b, CL);
    if (smem > 220 * 1024) continue;
    cudaError_t e = cudaFuncSetAttribute(k_coarse_factor_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) {
      last = e;
      cudaGetLastError();
      continue;
    }
    if (CL > 8) {
      e = cudaFuncSetAttribute(k_coarse_factor_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
      if (e != cudaSuccess) {
        last = e;
        cudaGetLastError();
        continue;
      }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CL, 1, 1);
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
    int nclusters = 0;
    e = cudaOccupancyMaxActiveClusters(&nclusters, k_coarse_factor_cluster, &cfg);
    if (e != cudaSuccess || nclusters < 1) {
      last = e != cudaSuccess ? e : cudaErrorInvalidConfiguration;
      cudaGetLastError();
      continue;
    }
    e = cudaLaunchKernelEx(&cfg, k_coarse_factor_cluster, P, Dinv, err);
    if (e == cudaSuccess) {
      if (cluster_used) *cluster_used = CL;
      return cudaSuccess;
    }
    last = e;
    cudaGetLastError();
  }
  return last;
}

}  // namespace schur
