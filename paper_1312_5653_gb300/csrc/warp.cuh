// Warp-per-subdomain variants of the layered factorisation and solves for layer sizes b <= 32
// (every 2D subdomain with up to 31 elements per side).  Lane i owns row i of the current layer;
// couplings between rows travel by warp shuffles, so a 17 x 17 layer block needs no block-wide
// barrier and one warp processes one subdomain.  Same arithmetic as layered.cuh.
#pragma once
#include "kernels.cuh"

namespace schur {

template <class T>
__device__ __forceinline__ cx<T> shfl_cx(cx<T> v, int src) {
  return mkc<T>(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}

// Asynchronous global -> shared copies (cp.async, L1-allocating), one complex entry per lane.
template <class T>
__device__ __forceinline__ void cp_async_cx(cx<T>* smem, const cx<T>* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  if (sizeof(cx<T>) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Warp-wide asynchronous copy of one b x b layer block into shared memory.
template <class T>
__device__ __forceinline__ void warp_stage_block(cx<T>* dst, const cx<T>* __restrict__ src, int bb) {
  for (int e = threadIdx.x & 31; e < bb; e += 32) cp_async_cx(dst + e, src + e);
}

// Shared memory per warp of warp_layered_solve: two b x b blocks (double buffer).
template <class T>
__host__ __device__ constexpr size_t warp_solve_smem(int b) {
  return 2 * (size_t)b * b * sizeof(cx<T>);
}

// X = A^{-1} B for up to C columns (runtime R <= C used), B given by rhs(K, i, c).
// X (per warp, any address space) holds entry (node K*b + i, column c) at (K*b + i)*rs + c*cs;
// forward results are overwritten by the solution in the backward sweep.  Ds: this warp's
// shared buffer (warp_solve_smem bytes); the D_K^{-1} block of the next layer is copied into it
// asynchronously while the current layer is processed, and the neighbour couplings and right-hand
// side of a layer are loaded before the wait, so one global latency is exposed per layer.
template <class T, int C, class Prov, class RhsF>
__device__ __forceinline__ void warp_layered_solve(const Prov& P, const cx<T>* __restrict__ Dinv, int R, RhsF rhs,
                                                   cx<T>* X, int rs, int cs, cx<T>* Ds) {
  constexpr int kMaxNt = 9;
  const int lane = threadIdx.x & 31, b = P.ly.b, L = P.ly.L, nt = nbr_count(P.ly.dim), bb = b * b;
  const bool act = lane < b;
  cx<T> prev[C];
#pragma unroll
  for (int c = 0; c < C; ++c) prev[c] = czero<T>();
  warp_stage_block(Ds, Dinv, bb);
  cp_async_commit();
  for (int K = 0; K < L; ++K) {
    const cx<T>* Dk = Ds + (size_t)(K & 1) * bb;
    if (K + 1 < L) warp_stage_block(Ds + (size_t)((K + 1) & 1) * bb, Dinv + (size_t)(K + 1) * bb, bb);
    cp_async_commit();
    cx<T> t[C];
#pragma unroll
    for (int c = 0; c < C; ++c) t[c] = (act && c < R) ? rhs(K, lane, c) : czero<T>();
    if (K > 0) {
      cx<T> al[kMaxNt];
      int src[kMaxNt];
#pragma unroll
      for (int tt = 0; tt < kMaxNt; ++tt) {
        int k = (act && tt < nt) ? nbr_of(P.ly, lane, tt) : -1;
        al[tt] = k >= 0 ? P.Al(K - 1, lane, tt) : czero<T>();
        src[tt] = k >= 0 ? k : lane;
      }
#pragma unroll
      for (int tt = 0; tt < kMaxNt; ++tt) {
        if (tt >= nt) break;
#pragma unroll
        for (int c = 0; c < C; ++c) cfms(t[c], al[tt], shfl_cx(prev[c], src[tt]));
      }
    }
    cp_async_wait<1>();
    __syncwarp();
    cx<T> acc[C];
#pragma unroll
    for (int c = 0; c < C; ++c) acc[c] = czero<T>();
    for (int mm = 0; mm < b; ++mm) {
      cx<T> d = act ? Dk[mm * b + lane] : czero<T>();
#pragma unroll
      for (int c = 0; c < C; ++c) cfma(acc[c], d, shfl_cx(t[c], mm));
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      prev[c] = acc[c];
      if (act && c < R) X[(size_t)(K * b + lane) * rs + (size_t)c * cs] = acc[c];
    }
    __syncwarp();
  }
  // backward: prev = E_{L-1} = X_{L-1}
  if (L >= 2) warp_stage_block(Ds, Dinv + (size_t)(L - 2) * bb, bb);
  cp_async_commit();
  for (int K = L - 2, it = 0; K >= 0; --K, ++it) {
    const cx<T>* Dk = Ds + (size_t)(it & 1) * bb;
    if (K >= 1) warp_stage_block(Ds + (size_t)((it + 1) & 1) * bb, Dinv + (size_t)(K - 1) * bb, bb);
    cp_async_commit();
    cx<T> al[kMaxNt];
    int src[kMaxNt];
#pragma unroll
    for (int tt = 0; tt < kMaxNt; ++tt) {
      int k = (act && tt < nt) ? nbr_of(P.ly, lane, tt) : -1;
      al[tt] = k >= 0 ? P.Al(K, k, nt - 1 - tt) : czero<T>();
      src[tt] = k >= 0 ? k : lane;
    }
    cx<T> x[C];
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = (act && c < R) ? X[(size_t)(K * b + lane) * rs + (size_t)c * cs] : czero<T>();
    cx<T> u[C];
#pragma unroll
    for (int c = 0; c < C; ++c) u[c] = czero<T>();
#pragma unroll
    for (int tt = 0; tt < kMaxNt; ++tt) {
      if (tt >= nt) break;
#pragma unroll
      for (int c = 0; c < C; ++c) cfma(u[c], al[tt], shfl_cx(prev[c], src[tt]));
    }
    cp_async_wait<1>();
    __syncwarp();
    for (int mm = 0; mm < b; ++mm) {
      cx<T> d = act ? Dk[mm * b + lane] : czero<T>();
#pragma unroll
      for (int c = 0; c < C; ++c) cfms(x[c], d, shfl_cx(u[c], mm));
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      prev[c] = x[c];
      if (act && c < R) X[(size_t)(K * b + lane) * rs + (size_t)c * cs] = x[c];
    }
    __syncwarp();
  }
  cp_async_wait<0>();
  __syncwarp();
}

// Block LDL^T, one warp per problem (b <= 32): the same steps as k_factor with warp barriers.
template <class T>
__global__ void k_factor_warp(StencilProv<T> P, const int* codes, int nprob, cx<T>* Dinv, int* err) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int q = blockIdx.x * wpb + wib;
  if (q >= nprob) return;
  P.select(q, codes);
  const int b = P.ly.b, L = P.ly.L, bb = b * b, nt = nbr_count(P.ly.dim);
  extern __shared__ unsigned char smraw[];
  cx<T>* Dt = reinterpret_cast<cx<T>*>(smraw) + (size_t)wib * (2 * bb + 2 * b);
  cx<T>* W = Dt + bb;
  cx<T>* rc = W + bb;
  cx<T>* out = Dinv + (size_t)q * L * bb;
  for (int e = lane; e < bb; e += 32) Dt[e] = czero<T>();
  __syncwarp();
  for (int e = lane; e < b * nt; e += 32) {
    int i = e / nt, t = e - i * nt, j = nbr_of(P.ly, i, t);
    if (j >= 0) Dt[i * b + j] = P.Ad(0, i, t);
  }
  __syncwarp();
  for (int K = 0; K < L; ++K) {
    for (int k = 0; k < b; ++k) {
      cx<T> p = Dt[k * b + k];
      cx<T> piv = cinv(p);
      if (lane == 0 && !finite_nonzero(p)) atomicExch(err, 1);
      for (int j = lane; j < b; j += 32) {
        rc[j] = cmul(Dt[k * b + j], piv);
        rc[b + j] = Dt[j * b + k];
      }
      __syncwarp();
      for (int e = lane; e < bb; e += 32) {
        int i = e / b, j = e - i * b;
        if (i == k) {
          Dt[e] = (j == k) ? piv : rc[j];
        } else if (j == k) {
          cx<T> v = cmul(rc[b + i], piv);
          Dt[e] = mkc<T>(-v.re, -v.im);
        } else {
          cfms(Dt[e], rc[b + i], rc[j]);
        }
      }
      __syncwarp();
    }
    for (int e = lane; e < bb; e += 32) {
      int i = e / b, j = e - i * b;
      W[e] = cscale(cadd(Dt[i * b + j], Dt[j * b + i]), T(0.5));
    }
    __syncwarp();
    for (int e = lane; e < bb; e += 32) {
      Dt[e] = W[e];
      out[(size_t)K * bb + e] = W[e];
    }
    __syncwarp();
    if (K + 1 == L) break;
    for (int e = lane; e < bb; e += 32) {
      int k = e / b, j = e - k * b;
      cx<T> acc = czero<T>();
      for (int t = 0; t < nt; ++t) {
        int mm = nbr_of(P.ly, j, t);
        if (mm >= 0) cfma(acc, Dt[k * b + mm], P.Al(K, j, t));
      }
      W[e] = acc;
    }
    __syncwarp();
    for (int e = lane; e < bb; e += 32) {
      int i = e / b, j = e - i * b;
      int tj = nbr_slot(P.ly, i, j);
      cx<T> acc = tj >= 0 ? P.Ad(K + 1, i, tj) : czero<T>();
      for (int t = 0; t < nt; ++t) {
        int k = nbr_of(P.ly, i, t);
        if (k >= 0) cfms(acc, P.Al(K, i, t), W[k * b + j]);
      }
      Dt[e] = acc;
    }
    __syncwarp();
  }
}

// Right-hand side of the remainder problem of subdomain sd at node (K, i), column c:
// f_r (interface entries scaled by 1/multiplicity) - B_r^T lambda - A_rc u_c (lam/uc optional).
template <class T>
__device__ __forceinline__ cx<T> remainder_rhs(const StencilProv<T>& P, const Geom& g, const MapsView& m, int sd,
                                               const int* S, const cx<double>* __restrict__ f, int ldf,
                                               const cx<T>* __restrict__ lam, const cx<T>* __restrict__ uc, int K,
                                               int i, int c) {
  const int dim = g.dim;
  if (P.removed_node(K, i)) return czero<T>();
  int l[3];
  P.crd(K, i, l);
  int G[3] = {S[0] * g.s[0] + l[0], S[1] * g.s[1] + l[1], dim == 3 ? S[2] * g.s[2] + l[2] : 1};
  cx<double> fv = f[(size_t)c * ldf + gidx(g, G)];
  int slot = m.node_slot[K * P.ly.b + i];
  cx<T> v;
  if (slot >= 0) {
    double sc = m.sd_minv[(size_t)sd * g.nD + slot];
    v = mkc<T>((T)(fv.re * sc), (T)(fv.im * sc));
    if (lam) {
      const int* refs = m.sd_lam + ((size_t)sd * g.nD + slot) * g.maxdeg;
      for (int k = 0; k < g.maxdeg; ++k) {
        int ref = refs[k];
        if (ref > 0) v = csub(v, lam[(size_t)c * g.nlam + ref - 1]);
        else if (ref < 0) v = cadd(v, lam[(size_t)c * g.nlam - ref - 1]);
      }
    }
  } else {
    v = mkc<T>((T)fv.re, (T)fv.im);
  }
  if (uc) {
    int ext[3];
    local_ext(g, ext);
    for (int cc = 0; cc < g.nc; ++cc) {
      int ci = m.sd_corner[(size_t)sd * g.nc + cc];
      if (ci < 0) continue;
      int lc[3];
      idx2crd(m.corner_node[cc], ext, dim, lc);
      cfms(v, q1_entry(P.st, g.s, l, lc), uc[(size_t)c * g.ncor + ci]);
    }
  }
  return v;
}

// Per-solve local solves, one warp per subdomain.  VD/Tc extraction when VD != null (right-hand
// side split); otherwise the solution stays in Xs (primal recovery).
template <class T, int C>
__global__ void k_local_solve_warp(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv,
                                   const cx<double>* __restrict__ f, int ldf, const cx<T>* __restrict__ lam,
                                   const cx<T>* __restrict__ uc, int R, cx<T>* Xs, cx<T>* VD, cx<T>* Tc) {
  const int lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
  const int sd = blockIdx.x * wpb + (threadIdx.x >> 5);
  if (sd >= g.nsd) return;
  const int q = m.sd_cls[sd], b = P.ly.b, L = P.ly.L, dim = g.dim, nD = g.nD, nc = g.nc;
  P.select(q, m.cls_code);
  int S[3], ext[3];
  idx2crd(sd, g.nsub, dim, S);
  local_ext(g, ext);
  cx<T>* X = Xs + (size_t)sd * g.nl * R;
  extern __shared__ unsigned char smraw[];
  cx<T>* Ds = reinterpret_cast<cx<T>*>(smraw) + (size_t)(threadIdx.x >> 5) * 2 * b * b;
  auto rhs = [&](int K, int i, int c) -> cx<T> { return remainder_rhs(P, g, m, sd, S, f, ldf, lam, uc, K, i, c); };
  warp_layered_solve<T, C>(P, Dinv + (size_t)q * L * b * b, R, rhs, X, R, 1, Ds);
  if (!VD) return;
  __syncwarp();
  for (int e = lane; e < R * nD; e += 32) {
    int c = e / nD, j = e - c * nD;
    VD[((size_t)sd * R + c) * nD + j] = X[(size_t)m.slot_node[j] * R + c];
  }
  for (int e = lane; e < R * nc; e += 32) {
    int c = e / nc, cc = e - c * nc;
    int lc[3];
    idx2crd(m.corner_node[cc], ext, dim, lc);
    cx<T> v = czero<T>();
    if (!local_dirichlet(P.code, lc, g.s, dim)) {
      const int noff = dim == 2 ? 9 : 27;
      for (int o = 0; o < noff; ++o) {
        int lp[3] = {lc[0] + o % 3 - 1, lc[1] + (o / 3) % 3 - 1, dim == 3 ? lc[2] + o / 9 - 1 : 0};
        bool in = true;
        for (int a = 0; a < dim; ++a) in = in && lp[a] >= 0 && lp[a] <= g.s[a];
        if (!in || P.removed_l(lp)) continue;
        cfma(v, q1_entry(P.st, g.s, lc, lp), X[(size_t)crd2idx(lp, ext, dim) * R + c]);
      }
    }
    Tc[((size_t)sd * R + c) * nc + cc] = v;
  }
}

// F, Frc, Kcc of each class, one warp per (class, chunk of C columns); solution in shared memory.
template <class T, int C>
__global__ void k_form_rr_warp(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv, int ncls,
                               cx<T>* F, cx<T>* Frc, cx<double>* Kcc, cx<T>* Xws) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int nD = g.nD, nc = g.nc, ncol = nD + nc, nchunk = (ncol + C - 1) / C;
  const int b = P.ly.b, L = P.ly.L, dim = g.dim;
  // per-warp solution buffer in global memory (column-major: node fastest), persistent warps;
  // per-warp staging buffer of the layer blocks in shared memory
  cx<T>* X = Xws + (size_t)(blockIdx.x * wpb + wib) * g.nl * C;
  extern __shared__ unsigned char smraw[];
  cx<T>* Ds = reinterpret_cast<cx<T>*>(smraw) + (size_t)wib * 2 * P.ly.b * P.ly.b;
  for (int w = blockIdx.x * wpb + wib; w < ncls * nchunk; w += gridDim.x * wpb) {
  const int q = w / nchunk, col0 = (w % nchunk) * C;
  P.select(q, m.cls_code);
  const int code = P.code;
  int ext[3];
  local_ext(g, ext);
  auto rhs = [&](int K, int i, int c) -> cx<T> {
    int col = col0 + c;
    if (col >= ncol) return czero<T>();
    int l[3];
    P.crd(K, i, l);
    if (P.removed_l(l)) return czero<T>();
    if (col < nD) return mkc<T>(m.slot_node[col] == K * b + i ? T(1) : T(0), T(0));
    int lc[3];
    idx2crd(m.corner_node[col - nD], ext, dim, lc);
    if (local_dirichlet(code, lc, g.s, dim)) return czero<T>();
    return q1_entry(P.st, g.s, l, lc);
  };
  warp_layered_solve<T, C>(P, Dinv + (size_t)q * L * b * b, C, rhs, X, 1, g.nl, Ds);
  __syncwarp();
  for (int e = lane; e < nD * C; e += 32) {
    int j = e / C, c = e - j * C, col = col0 + c;
    if (col >= ncol) continue;
    cx<T> v = X[(size_t)m.slot_node[j] + (size_t)c * g.nl];
    if (col < nD) F[((size_t)q * nD + j) * nD + col] = v;
    else Frc[((size_t)q * nD + j) * nc + (col - nD)] = v;
  }
  for (int e = lane; e < nc * C; e += 32) {
    int c1 = e / C, c = e - c1 * C, col = col0 + c;
    if (col < nD || col >= ncol) continue;
    int c2 = col - nD;
    int l1[3], l2[3];
    idx2crd(m.corner_node[c1], ext, dim, l1);
    idx2crd(m.corner_node[c2], ext, dim, l2);
    cx<T> v = czero<T>();
    if (!local_dirichlet(code, l1, g.s, dim) && !local_dirichlet(code, l2, g.s, dim)) {
      if (c1 == c2) v = q1_entry(P.st, g.s, l1, l1);
      const int noff = dim == 2 ? 9 : 27;
      for (int o = 0; o < noff; ++o) {
        int lp[3] = {l1[0] + o % 3 - 1, l1[1] + (o / 3) % 3 - 1, dim == 3 ? l1[2] + o / 9 - 1 : 0};
        bool in = true;
        for (int a = 0; a < dim; ++a) in = in && lp[a] >= 0 && lp[a] <= g.s[a];
        if (!in || (lp[0] == l1[0] && lp[1] == l1[1] && lp[2] == l1[2])) continue;
        if (P.removed_l(lp)) continue;
        cfms(v, q1_entry(P.st, g.s, l1, lp), X[(size_t)crd2idx(lp, ext, dim) + (size_t)c * g.nl]);
      }
    }
    Kcc[((size_t)q * nc + c1) * nc + c2] = ccast<double>(v);
  }
  __syncwarp();
  }
}

}  // namespace schur
