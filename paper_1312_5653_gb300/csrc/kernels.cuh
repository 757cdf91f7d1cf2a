// FETI-DP kernels for the complex-symmetric factor A = K + i gamma M (Sec. 5 of arXiv 1312.5653),
// templated on the working precision T (double or float).  Notation follows Sec. 5: subdomain
// remainder set r (interior and interface nodes minus corners and Dirichlet nodes), corner set c,
// interface slots Delta, jump operator B, multipliers lambda.
//   local dual operator     F^s   = (A_rr^{-1})_{Delta,Delta}
//   corner coupling         Frc^s = (A_rr^{-1} A_rc)_{Delta,c}
//   corner Schur complement Kcc^s = A_cc - A_cr A_rr^{-1} A_rc
//   Dirichlet operator      S^s   = A_DD - A_Di A_ii^{-1} A_iD          (Eq. WS, b = Delta)
// The dual problem (F_rr + Frc~ Kcc~^{-1} Frc~^T) lambda = d_r - Frc~ Kcc~^{-1} f~_c is solved by
// right-preconditioned GMRES (Sec. 5: GMRES handles the indefinite complex factors) with the
// Dirichlet preconditioner P^{-1} = sum_s B_D^s S^s B_D^s^T, B_D = B / multiplicity (Eq.
// dirichletpreconditioner with W = (sum B B^T)^+).
#pragma once
#include "gmres.h"
#include "layered.cuh"

namespace schur {

struct MapsView {
  const int* slot_node;
  const int* node_slot;
  const int* corner_node;
  const int* sd_cls;
  const int* cls_code;
  const int* sd_lam;
  const int* lam_side;
  const int* sd_corner;
  const double* sd_minv;
  const int* sd_coarse;   // [nsd][nq] coarse unknown of each coupling slot or -1
  const int* face_sd;     // [nface][2] lower and higher subdomain of each face (augmented only)
  const int* lam_face;    // [nlam] face of the multiplier's pair or -1 (augmented only)
  const int* slot_faces;  // [nD] local faces of each slot, bit f = 2a + side (augmented only)
  const int* face_lam_ptr;  // [nface + 1] CSR offsets of the multipliers of each face (augmented only)
  const int* face_lam;      // multipliers of each face (augmented only)
  const int* grp_sd;        // [nsd] subdomains ordered by class
  const int* grp_ptr;       // [ngrp + 1] groups of at most kApplyGroup subdomains of one class
};

__device__ __forceinline__ void local_ext(const Geom& g, int* ext) {
  ext[0] = g.s[0] + 1;
  ext[1] = g.s[1] + 1;
  ext[2] = g.dim == 3 ? g.s[2] + 1 : 1;
}

// global interior index of global node coordinates G (1..nel-1 per axis)
__device__ __forceinline__ long long gidx(const Geom& g, const int* G) {
  long long i = G[0] - 1;
  long long st = g.nel[0] - 1;
  i += st * (G[1] - 1);
  if (g.dim == 3) i += st * (long long)(g.nel[1] - 1) * (G[2] - 1);
  return i;
}

template <class T>
__device__ __forceinline__ cx<T> czero() { return mkc<T>(T(0), T(0)); }

template <class T>
__device__ __forceinline__ cx<T> shfl_cx(cx<T> v, int src) {
  return mkc<T>(__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src));
}
template <class T>
__device__ __forceinline__ cx<T> shfl_xor_cx(cx<T> v, int m) {
  return mkc<T>(__shfl_xor_sync(0xffffffffu, v.re, m), __shfl_xor_sync(0xffffffffu, v.im, m));
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

// 16-byte asynchronous copy (L2 only); both addresses 16-byte aligned.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

// ================================================================================= setup
// F, Frc, Kcc of each class: solve A_rr X = [E_Delta, A_rc] column chunk by chunk.
// Columns [col_begin, nD + nc) only (the leftover columns of the tensor-core formation's tiles).
template <class T>
__global__ void k_form_rr(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv, int ncls, int C,
                          cx<T>* Xws, cx<T>* F, cx<T>* Frc, cx<double>* Kcc, int col_begin) {
  extern __shared__ unsigned char smraw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smraw);
  const int nD = g.nD, nc = g.nc, ncol = nD + nc, nchunk = (ncol - col_begin + C - 1) / C;
  const int b = P.ly.b, L = P.ly.L, dim = g.dim, tid = threadIdx.x, nthr = blockDim.x;
  cx<T>* X = Xws + (size_t)blockIdx.x * g.nl * C;
  int ext[3];
  local_ext(g, ext);
  for (int w = blockIdx.x; w < ncls * nchunk; w += gridDim.x) {
    const int q = w / nchunk, col0 = col_begin + (w % nchunk) * C;
    P.select(q, m.cls_code);
    const int code = P.code;
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
    layered_solve<T>(P, Dinv + (size_t)q * L * b * b, C, rhs, X, C, sm);
    for (int e = tid; e < nD * C; e += nthr) {
      int j = e / C, c = e - j * C, col = col0 + c;
      if (col >= ncol) continue;
      cx<T> v = X[(size_t)m.slot_node[j] * C + c];
      if (col < nD) {
        if (j <= col) F[(size_t)q * sym_ld(nD) + sym_idx(j, col, nD)] = v;
      }
      else Frc[((size_t)q * nD + j) * nc + (col - nD)] = v;
    }
    for (int e = tid; e < nc * C; e += nthr) {
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
          cfms(v, q1_entry(P.st, g.s, l1, lp), X[(size_t)crd2idx(lp, ext, dim) * C + c]);
        }
      }
      Kcc[((size_t)q * nc + c1) * nc + c2] = ccast<double>(v);
    }
    __syncthreads();
  }
}

// S_base = A_DD - A_Di A_ii^{-1} A_iD for all slots (the interior problem is the same for
// every subdomain); classes mask their Dirichlet slots afterwards.
template <class T>
__global__ void k_form_ii(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv, int C, cx<T>* Xws,
                          cx<T>* Sbase) {
  extern __shared__ unsigned char smraw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smraw);
  const int nD = g.nD, nchunk = (nD + C - 1) / C, dim = g.dim, tid = threadIdx.x, nthr = blockDim.x;
  cx<T>* X = Xws + (size_t)blockIdx.x * g.ni * C;
  int ext[3], iext[3];
  local_ext(g, ext);
  for (int a = 0; a < 3; ++a) iext[a] = a < dim ? g.s[a] - 1 : 1;
  for (int w = blockIdx.x; w < nchunk; w += gridDim.x) {
    const int col0 = w * C;
    auto rhs = [&](int K, int i, int c) -> cx<T> {
      int col = col0 + c;
      if (col >= nD) return czero<T>();
      int l[3], ls[3];
      P.crd(K, i, l);
      idx2crd(m.slot_node[col], ext, dim, ls);
      return q1_entry(P.st, g.s, l, ls);
    };
    layered_solve<T>(P, Dinv, C, rhs, X, C, sm);
    for (int e = tid; e < nD * C; e += nthr) {
      int j = e / C, c = e - j * C, col = col0 + c;
      if (col >= nD) continue;
      int lj[3], lc[3];
      idx2crd(m.slot_node[j], ext, dim, lj);
      idx2crd(m.slot_node[col], ext, dim, lc);
      cx<T> v = q1_entry(P.st, g.s, lj, lc);
      const int noff = dim == 2 ? 9 : 27;
      for (int o = 0; o < noff; ++o) {
        int lp[3] = {lj[0] + o % 3 - 1, lj[1] + (o / 3) % 3 - 1, dim == 3 ? lj[2] + o / 9 - 1 : 0};
        bool interior = true;
        for (int a = 0; a < dim; ++a) interior = interior && lp[a] >= 1 && lp[a] <= g.s[a] - 1;
        if (!interior) continue;
        int li[3] = {lp[0] - 1, lp[1] - 1, dim == 3 ? lp[2] - 1 : 0};
        cfms(v, q1_entry(P.st, g.s, lj, lp), X[(size_t)crd2idx(li, iext, dim) * C + c]);
      }
      Sbase[(size_t)j * nD + col] = v;
    }
    __syncthreads();
  }
}

template <class T>
__global__ void k_mask_S(Geom g, MapsView m, int ncls, const cx<T>* __restrict__ Sbase, cx<T>* Sd) {
  const long long tot = (long long)ncls * g.nD * g.nD;
  const long long ld = sym_ld(g.nD);
  int ext[3];
  local_ext(g, ext);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    int q = (int)(e / ((long long)g.nD * g.nD));
    int r = (int)(e % ((long long)g.nD * g.nD));
    int j = r / g.nD, k = r % g.nD;
    if (j > k) continue;  // upper triangle (packed)
    int lj[3], lk[3];
    idx2crd(m.slot_node[j], ext, g.dim, lj);
    idx2crd(m.slot_node[k], ext, g.dim, lk);
    int code = m.cls_code[q];
    bool act = !local_dirichlet(code, lj, g.s, g.dim) && !local_dirichlet(code, lk, g.s, g.dim);
    Sd[(size_t)q * ld + sym_idx(j, k, g.nD)] = act ? Sbase[r] : czero<T>();
  }
}

// Coarse matrix Kcc~ = sum_s B_c^s^T Kcc^s B_c^s in layered storage (CA: in-layer couplings,
// CB: couplings to the previous layer).  One thread per (coarse node, 3^d offset); each entry
// sums the subdomains that hold both corners in a fixed order.
static __global__ void k_coarse_assemble(Geom g, const cx<double>* __restrict__ Kcc, const int* __restrict__ sd_cls,
                                  cx<double>* CA, cx<double>* CB) {
  const int dim = g.dim, noff = dim == 2 ? 9 : 27, nt = nbr_count(dim);
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)g.ncor * noff) return;
  int g1 = (int)(e / noff), o = (int)(e % noff);
  int C1[3], C2[3], d[3] = {o % 3 - 1, (o / 3) % 3 - 1, dim == 3 ? o / 9 - 1 : 0};
  idx2crd(g1, g.ncg, dim, C1);
  for (int a = 0; a < 3; ++a) C2[a] = C1[a] + (a < dim ? d[a] : 0);
  for (int a = 0; a < dim; ++a)
    if (C2[a] < 0 || C2[a] >= g.ncg[a]) return;
  if (d[dim - 1] > 0) return;
  // candidate subdomains per axis: {C1, C1+1} intersect {C2, C2+1}
  int lo[3], hi[3];
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      lo[a] = max(C1[a], C2[a]);
      hi[a] = min(C1[a], C2[a]) + 1;
    } else {
      lo[a] = hi[a] = 0;
    }
  }
  cx<double> sum = mkc<double>(0, 0);
  for (int s2 = lo[2]; s2 <= hi[2]; ++s2)
    for (int s1 = lo[1]; s1 <= hi[1]; ++s1)
      for (int s0 = lo[0]; s0 <= hi[0]; ++s0) {
        int S[3] = {s0, s1, s2};
        int sd = crd2idx(S, g.nsub, dim);
        int c1 = 0, c2 = 0;
        for (int a = 0; a < dim; ++a) {
          c1 |= (C1[a] == S[a]) << a;
          c2 |= (C2[a] == S[a]) << a;
        }
        sum = cadd(sum, Kcc[((size_t)sd_cls[sd] * g.nc + c1) * g.nc + c2]);
      }
  int K1 = C1[dim - 1];
  int i1 = dim == 2 ? C1[0] : C1[0] + g.ncg[0] * C1[1];
  int t = dim == 2 ? d[0] + 1 : (d[0] + 1) + 3 * (d[1] + 1);
  if (d[dim - 1] == 0) CA[((size_t)K1 * g.cb + i1) * nt + t] = sum;
  else CB[((size_t)(K1 - 1) * g.cb + i1) * nt + t] = sum;
}

// Columns of the coarse inverse from the layered factor of the coarse matrix, solved in precision
// S (FP64 for the FP64 path; FP32 copies of the FP64 factor for the mixed path), stored as T.
template <class T, class S>
__global__ void k_coarse_inverse(StoredProv<S> P, const cx<S>* __restrict__ Dinv, int ncor, int C, cx<S>* Xws,
                                 cx<T>* Kinv) {
  extern __shared__ unsigned char smraw[];
  cx<S>* sm = reinterpret_cast<cx<S>*>(smraw);
  const int nchunk = (ncor + C - 1) / C, b = P.ly.b;
  cx<S>* X = Xws + (size_t)blockIdx.x * ncor * C;
  for (int w = blockIdx.x; w < nchunk; w += gridDim.x) {
    const int col0 = w * C;
    auto rhs = [&](int K, int i, int c) -> cx<S> {
      int col = col0 + c;
      return mkc<S>((col < ncor && K * b + i == col) ? S(1) : S(0), S(0));
    };
    layered_solve<S>(P, Dinv, C, rhs, X, C, sm);
    for (int e = threadIdx.x; e < ncor * C; e += blockDim.x) {
      int row = e / C, c = e - row * C, col = col0 + c;
      if (col < ncor) Kinv[(size_t)col * ncor + row] = ccast<T>(X[e]);
    }
    __syncthreads();
  }
}

// The same columns with each layer block D_K^{-1} staged in shared memory (layer size b <= 128):
// a CTA solves 32 columns; thread (row i, group of 8 columns) keeps 8 accumulators, so every
// staged D entry feeds 8 complex multiply-adds.
template <class T, class S>
__global__ void __launch_bounds__(256) k_coarse_inverse_staged(StoredProv<S> P, const cx<S>* __restrict__ Dinv,
                                                               int ncor, cx<S>* Xws, cx<T>* Kinv) {
  constexpr int CS = 32, CG = 8;
  extern __shared__ unsigned char smraw[];
  const int b = P.ly.b, L = P.ly.L, bb = b * b, nt = nbr_count(P.ly.dim), tid = threadIdx.x;
  cx<S>* Dsm = reinterpret_cast<cx<S>*>(smraw);
  cx<S>* Tb = Dsm + bb;
  cx<S>* Ep = Tb + b * CS;
  cx<S>* X = Xws + (size_t)blockIdx.x * ncor * CS;
  const int nchunk = (ncor + CS - 1) / CS;
  const int ri = tid & 63, cg = tid >> 6;  // 4 groups of 8 columns
  for (int w = blockIdx.x; w < nchunk; w += gridDim.x) {
    const int col0 = w * CS;
    for (int K = 0; K < L; ++K) {
      for (int e = tid; e < bb; e += 256) Dsm[e] = Dinv[(size_t)K * bb + e];
      for (int e = tid; e < b * CS; e += 256) {
        int i = e / CS, c = e - i * CS, col = col0 + c;
        cx<S> t = mkc<S>((col < ncor && K * b + i == col) ? S(1) : S(0), S(0));
        if (K > 0)
          for (int tt = 0; tt < nt; ++tt) {
            int k = nbr_of(P.ly, i, tt);
            if (k >= 0) cfms(t, P.Al(K - 1, i, tt), Ep[k * CS + c]);
          }
        Tb[e] = t;
      }
      __syncthreads();
      for (int i0 = 0; i0 < b; i0 += 64) {
        const int i = i0 + ri;
        cx<S> acc[CG];
#pragma unroll
        for (int j = 0; j < CG; ++j) acc[j] = mkc<S>(0, 0);
        if (i < b)
          for (int mm = 0; mm < b; ++mm) {
            const cx<S> d = Dsm[mm * b + i];
#pragma unroll
            for (int j = 0; j < CG; ++j) cfma(acc[j], d, Tb[mm * CS + cg * CG + j]);
          }
        __syncthreads();  // all reads of Ep (coupling) are done before it is overwritten
        if (i < b)
#pragma unroll
          for (int j = 0; j < CG; ++j) {
            Ep[i * CS + cg * CG + j] = acc[j];
            X[(size_t)(K * b + i) * CS + cg * CG + j] = acc[j];
          }
      }
      __syncthreads();
    }
    for (int K = L - 2; K >= 0; --K) {
      for (int e = tid; e < bb; e += 256) Dsm[e] = Dinv[(size_t)K * bb + e];
      for (int e = tid; e < b * CS; e += 256) {
        int i = e / CS, c = e - i * CS;
        cx<S> u = mkc<S>(0, 0);
        for (int tt = 0; tt < nt; ++tt) {
          int k = nbr_of(P.ly, i, tt);
          if (k >= 0) cfma(u, P.Al(K, k, nt - 1 - tt), Ep[k * CS + c]);
        }
        Tb[e] = u;
      }
      __syncthreads();
      for (int i0 = 0; i0 < b; i0 += 64) {
        const int i = i0 + ri;
        cx<S> acc[CG];
#pragma unroll
        for (int j = 0; j < CG; ++j) acc[j] = i < b ? X[(size_t)(K * b + i) * CS + cg * CG + j] : mkc<S>(0, 0);
        if (i < b)
          for (int mm = 0; mm < b; ++mm) {
            const cx<S> d = Dsm[mm * b + i];
#pragma unroll
            for (int j = 0; j < CG; ++j) cfms(acc[j], d, Tb[mm * CS + cg * CG + j]);
          }
        __syncthreads();
        if (i < b)
#pragma unroll
          for (int j = 0; j < CG; ++j) {
            Ep[i * CS + cg * CG + j] = acc[j];
            X[(size_t)(K * b + i) * CS + cg * CG + j] = acc[j];
          }
      }
      __syncthreads();
    }
    for (int e = tid; e < ncor * CS; e += 256) {
      int row = e / CS, c = e - row * CS, col = col0 + c;
      if (col < ncor) Kinv[(size_t)col * ncor + row] = ccast<T>(X[e]);
    }
    __syncthreads();
  }
}

template <class T, class S>
__global__ void k_convert(const cx<S>* __restrict__ in, cx<T>* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = ccast<T>(in[i]);
}

// ================================================================================= solve
// Local right-hand sides f_r^s (interface entries scaled by 1/multiplicity, corners and
// Dirichlet nodes removed), v = A_rr^{-1} f_r, and its restrictions: VD = v on the slots (for
// d_r = sum_s B^s v^s) and Tc = A_cr v (for f~_c = f_c - sum_s B_c^T A_cr A_rr^{-1} f_r).
template <class T>
__global__ void k_local_rhs(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv,
                            const cx<double>* __restrict__ f, int ldf, int R, cx<T>* Xs, cx<T>* VD, cx<T>* Tc) {
  extern __shared__ unsigned char smraw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smraw);
  const int sd = blockIdx.x, dim = g.dim, tid = threadIdx.x, nthr = blockDim.x;
  const int q = m.sd_cls[sd], b = P.ly.b, L = P.ly.L, nD = g.nD, nc = g.nc;
  P.select(q, m.cls_code);
  int S[3], ext[3];
  idx2crd(sd, g.nsub, dim, S);
  local_ext(g, ext);
  cx<T>* X = Xs + (size_t)sd * g.nl * R;
  auto rhs = [&](int K, int i, int c) -> cx<T> {
    int l[3];
    P.crd(K, i, l);
    if (P.removed_l(l)) return czero<T>();
    int G[3] = {S[0] * g.s[0] + l[0], S[1] * g.s[1] + l[1], dim == 3 ? S[2] * g.s[2] + l[2] : 1};
    cx<double> v = f[(size_t)c * ldf + gidx(g, G)];
    int slot = m.node_slot[K * b + i];
    double sc = slot >= 0 ? m.sd_minv[(size_t)sd * nD + slot] : 1.0;
    return mkc<T>((T)(v.re * sc), (T)(v.im * sc));
  };
  layered_solve<T>(P, Dinv + (size_t)q * L * b * b, R, rhs, X, R, sm);
  for (int e = tid; e < R * nD; e += nthr) {
    int c = e / nD, j = e - c * nD;
    VD[((size_t)sd * R + c) * nD + j] = X[(size_t)m.slot_node[j] * R + c];
  }
  for (int e = tid; e < R * nc; e += nthr) {
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
    Tc[((size_t)sd * R + c) * g.nq + cc] = v;
  }
}

// g[r][C] = (add ? add[r][C] : 0) + sign * sum over subdomains holding corner C of Tc; with
// f != null also adds f at the corner node (f~_c = f_c - sum A_cr A_rr^{-1} f_r uses sign -1).
template <class T>
__global__ void k_corner_gather(Geom g, MapsView m, const cx<T>* __restrict__ Tc, int R, const cx<double>* __restrict__ f, int ldf,
                                const cx<T>* __restrict__ add, T sign, cx<T>* out) {
  pdl_wait();
  pdl_trigger();
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= R * g.nco) return;
  int r = e / g.nco, cI = e - r * g.nco, dim = g.dim;
  if (cI >= g.ncor) {
    // face unknown (augmented coarse problem): its two subdomains, at their high and low face slot
    const int f = cI - g.ncor;
    const int lo = m.face_sd[2 * f + 1], hi = m.face_sd[2 * f];
    int A[3], B[3], a = 0;
    idx2crd(lo, g.nsub, dim, A);
    idx2crd(hi, g.nsub, dim, B);
    for (int t = 0; t < dim; ++t)
      if (A[t] != B[t]) a = t;
    cx<T> sum = cadd(Tc[((size_t)lo * R + r) * g.nq + g.nc + 2 * a + 1], Tc[((size_t)hi * R + r) * g.nq + g.nc + 2 * a]);
    cx<T> v = cscale(sum, sign);
    if (add) v = cadd(v, add[(size_t)r * g.nco + cI]);
    out[(size_t)r * g.nco + cI] = v;
    return;
  }
  int C[3];
  idx2crd(cI, g.ncg, dim, C);
  cx<T> sum = czero<T>();
  const int nb = 1 << dim;
  for (int bits = 0; bits < nb; ++bits) {
    // subdomain holding the corner as its vertex `bits` (bit a set: high vertex, S_a = C_a)
    int S[3] = {0, 0, 0};
    for (int a = 0; a < dim; ++a) S[a] = C[a] + 1 - ((bits >> a) & 1);
    int sd = crd2idx(S, g.nsub, dim);
    sum = cadd(sum, Tc[((size_t)sd * R + r) * g.nq + bits]);
  }
  cx<T> v = cscale(sum, sign);
  if (add) v = cadd(v, add[(size_t)r * g.nco + cI]);
  if (f) {
    int G[3] = {(C[0] + 1) * g.s[0], (C[1] + 1) * g.s[1], dim == 3 ? (C[2] + 1) * g.s[2] : 1};
    cx<double> fv = f[(size_t)r * ldf + gidx(g, G)];
    v = cadd(v, mkc<T>((T)fv.re, (T)fv.im));
  }
  out[(size_t)r * g.nco + cI] = v;
}

// ------------------------------------------------------------------ coarse inverse, packed tiles
// The coarse inverse is complex symmetric: only its upper 32 x 32 tiles (I <= J) are kept, tile
// (I, J) at index ctile_idx(I, J) as a row-major 32 x 32 block, zero past n_c.  w = Kinv g is
// formed in two launches: every tile produces its row product T g_J (for w_I) and, off the
// diagonal, its transposed product T^T g_I (for w_J) into a partial buffer; then each row block
// adds its partials in tile order (deterministic).
constexpr int kCT = 32;
__host__ __device__ __forceinline__ long long ctile_idx(int I, int J, int nt) {
  return (long long)I * nt - (long long)I * (I - 1) / 2 + (J - I);
}
__host__ __device__ __forceinline__ long long ctile_count(int nt) { return (long long)nt * (nt + 1) / 2; }

// tiles from the full inverse (n rows of ld entries); one block per tile
template <class T>
__global__ void k_pack_ctiles(const cx<T>* __restrict__ K, int n, int ld, int nt, cx<T>* tiles) {
  for (long long t = blockIdx.x; t < ctile_count(nt); t += gridDim.x) {
    // tile coordinates from the packed index
    int I = 0;
    long long rem = t;
    while (rem >= nt - I) {
      rem -= nt - I;
      ++I;
    }
    const int J = I + (int)rem;
    for (int e = threadIdx.x; e < kCT * kCT; e += blockDim.x) {
      const int r = I * kCT + e / kCT, c = J * kCT + e % kCT;
      tiles[t * kCT * kCT + e] = (r < n && c < n) ? K[(size_t)r * ld + c] : czero<T>();
    }
  }
}

// phase 1: one warp per tile (4 per block).  FP32: the tile stays in registers, lane l holding
// rows 2i + h (h = l / 16, i = 0..15) of columns 2(l % 16) and 2(l % 16) + 1 after sixteen
// coalesced 16-byte loads; the transposed product T^T g_I is accumulated per lane and folded
// across the two row halves, the row product T g_J is reduce-scattered over the 16 lanes of a half.
template <class T>
__global__ void __launch_bounds__(128) k_coarse_tiles(const cx<T>* __restrict__ tiles, int nt, int ncor,
                                                      const cx<T>* __restrict__ gv, int R, const int* __restrict__ active,
                                                      cx<T>* part_u, cx<T>* part_v) {
  pdl_wait();
  pdl_trigger();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long t = (long long)blockIdx.x * 4 + warp;
  const long long ntile = ctile_count(nt);
  if (t >= ntile) return;
  int I = 0;
  long long rem = t;
  while (rem >= nt - I) {
    rem -= nt - I;
    ++I;
  }
  const int J = I + (int)rem;
  const cx<T>* src = tiles + t * kCT * kCT;
  const int h = lane >> 4, c0 = 2 * (lane & 15);
  cx<T> a0[16], a1[16];  // rows 2i + h, columns c0 and c0 + 1
  if constexpr (sizeof(T) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float4 v = s4[i * 32 + lane];
      a0[i] = mkc<T>(v.x, v.y);
      a1[i] = mkc<T>(v.z, v.w);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      a0[i] = src[(2 * i + h) * kCT + c0];
      a1[i] = src[(2 * i + h) * kCT + c0 + 1];
    }
  }
  for (int r = 0; r < R; ++r) {
    if (active && !active[r]) continue;  // active == null: every right-hand side
    const cx<T>* g = gv + (size_t)r * ncor;
    // g_J at columns c0, c0 + 1; g_I at rows 2i + h (from the lane holding index 2i + h)
    const int gj0 = J * kCT + c0;
    const cx<T> gJ0 = gj0 < ncor ? g[gj0] : czero<T>();
    const cx<T> gJ1 = gj0 + 1 < ncor ? g[gj0 + 1] : czero<T>();
    const int gi = I * kCT + lane;
    const cx<T> gIl = gi < ncor ? g[gi] : czero<T>();
    // transposed product: v[c] = sum_rows T[row][c] g_I[row]
    cx<T> v0 = czero<T>(), v1 = czero<T>();
    cx<T> p[16];  // row partials of T g_J for rows 2i + h
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const cx<T> gI = shfl_cx(gIl, 2 * i + h);
      cfma(v0, a0[i], gI);
      cfma(v1, a1[i], gI);
      p[i] = cmul(a0[i], gJ0);
      cfma(p[i], a1[i], gJ1);
    }
    v0 = cadd(v0, shfl_xor_cx(v0, 16));  // add the other row half
    v1 = cadd(v1, shfl_xor_cx(v1, 16));
    // reduce-scatter of p over the 16 lanes of this half (lane bit 3, 2, 1, 0 in turn picks the
    // upper or lower half of the remaining window): lane b = lane & 15 ends with the row-2b+h sum
    const bool u3 = (lane >> 3) & 1, u2 = (lane >> 2) & 1, u1 = (lane >> 1) & 1, u0 = lane & 1;
    cx<T> p8[8], p4[4], p2[2];
#pragma unroll
    for (int i = 0; i < 8; ++i) p8[i] = cadd(u3 ? p[i + 8] : p[i], shfl_xor_cx(u3 ? p[i] : p[i + 8], 8));
#pragma unroll
    for (int i = 0; i < 4; ++i) p4[i] = cadd(u2 ? p8[i + 4] : p8[i], shfl_xor_cx(u2 ? p8[i] : p8[i + 4], 4));
#pragma unroll
    for (int i = 0; i < 2; ++i) p2[i] = cadd(u1 ? p4[i + 2] : p4[i], shfl_xor_cx(u1 ? p4[i] : p4[i + 2], 2));
    const cx<T> p1 = cadd(u0 ? p2[1] : p2[0], shfl_xor_cx(u0 ? p2[0] : p2[1], 1));
    // lane (h, b = lane & 15) now holds row 2 * b + h; rows 0..31 are lanes 2b + h -> reorder
    const cx<T> u = shfl_cx(p1, ((lane & 1) << 4) | (lane >> 1));
    part_u[((size_t)r * ntile + t) * kCT + lane] = u;
    if (I != J) {
      // lane holds v for columns c0, c0 + 1 (duplicated in both halves): lane l writes column l
      const int srcl = (lane >> 1) & 15;
      const cx<T> va = shfl_cx(v0, srcl), vb = shfl_cx(v1, srcl);
      part_v[((size_t)r * ntile + t) * kCT + lane] = (lane & 1) ? vb : va;
    }
  }
}

// phase 2: w_I = sum_{J >= I} part_u(I, J) + sum_{J < I} part_v(J, I); one block of 16 warps per
// (I, rhs), warp q adding a contiguous sixteenth of the J range, the sixteen partials combined in
// order
template <class T>
__global__ void __launch_bounds__(512) k_coarse_reduce(const cx<T>* __restrict__ part_u, const cx<T>* __restrict__ part_v,
                                                       int nt, int ncor, int R, const int* __restrict__ active, cx<T>* w) {
  pdl_wait();
  pdl_trigger();
  __shared__ cx<T> red[16][kCT];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int I = blockIdx.x % nt, r = blockIdx.x / nt;
  if (r >= R || (active && !active[r])) return;
  const long long ntile = ctile_count(nt);
  const cx<T>* pu = part_u + (size_t)r * ntile * kCT;
  const cx<T>* pv = part_v + (size_t)r * ntile * kCT;
  const long long t0 = ctile_idx(I, I, nt);
  const int q0 = (nt * warp) / 16, q1 = (nt * (warp + 1)) / 16;
  cx<T> acc = czero<T>();
  for (int J = q0; J < q1; ++J)
    acc = cadd(acc, J < I ? pv[ctile_idx(J, I, nt) * kCT + lane] : pu[(t0 + (J - I)) * kCT + lane]);
  red[warp][lane] = acc;
  __syncthreads();
  if (warp == 0) {
    cx<T> tot = red[0][lane];
    for (int q = 1; q < 16; ++q) tot = cadd(tot, red[q][lane]);
    const int row = I * kCT + lane;
    if (row < ncor) w[(size_t)r * ncor + row] = tot;
  }
}

// ------------------------------------------------------------------ coarse solve around level 0
// The coarse solve w = K_cc^{-1} g with level 0 of the block cyclic reduction applied explicitly
// around the stored inverse of the reduced matrix on the layers that survive level 0:
//   forward:  f_t = g_t - Lp_jr g_jr - Lq_jl^T g_jl        (every surviving layer t, compact order)
//   reduced:  x_r = K_r^{-1} f_r                            (packed tiles, k_coarse_tiles/reduce)
//   backward: x_j = D_j^{-1} g_j - Lp_j^T x_p - Lq_j x_q    (every layer j eliminated at level 0)
// The blocks used transposed are stored transposed, so every product is M v with M row-major.  CTA
// (layer, 32-row slice, kBcrRC right-hand sides); 256 threads = 32 rows x 8 k-groups, thread
// (il = tid / 8, kg = tid % 8) taking k = kg, kg + 8, ... (a warp reads four 64-byte row segments).
// The operator entries of the first eight k-steps of every term are loaded before the vectors are
// staged, so that their latencies overlap; the k-group partials are added in order.  g is either a
// coarse vector or, with Tc set, assembled on the fly from the subdomains' corner couplings (the
// per-iteration dual operator, without a separate corner gather).
constexpr int kBcrRC = 4;

template <class T>
struct BcrTerm {
  const cx<T>* M;  // b x b row-major block, null: no term
  int src;         // 0: the input g; 1: the reduced solution xr
  int layer;       // layer of g, or compact layer of xr
  bool neg;
};

// coarse right-hand side at corner cI: sum of the corner couplings of the subdomains that hold it
template <class T>
__device__ __forceinline__ cx<T> bcr_corner_sum(const Geom& g, const cx<T>* __restrict__ Tc, int R, int r, int cI) {
  // corner coordinates (axis 0 fastest); the subdomain holding it as vertex `bits` (bit a set:
  // high vertex) has coordinate C_a + 1 - bit_a
  const int c0 = cI % g.ncg[0], c12 = cI / g.ncg[0];
  const int c1 = g.dim == 3 ? c12 % g.ncg[1] : c12, c2 = g.dim == 3 ? c12 / g.ncg[1] : 0;
  cx<T> sum = czero<T>();
  for (int bits = 0; bits < (1 << g.dim); ++bits) {
    const int s0 = c0 + 1 - (bits & 1), s1 = c1 + 1 - ((bits >> 1) & 1), s2 = g.dim == 3 ? c2 + 1 - ((bits >> 2) & 1) : 0;
    const int sd = s0 + g.nsub[0] * (s1 + g.nsub[1] * s2);
    sum = cadd(sum, Tc[((size_t)sd * R + r) * g.nq + bits]);
  }
  return sum;
}

template <class T>
__device__ __forceinline__ cx<T> bcr_g(const Geom& g, const cx<T>* __restrict__ gv, const cx<T>* __restrict__ Tc, int R,
                                       int r, int cI) {
  return Tc ? bcr_corner_sum(g, Tc, R, r, cI) : gv[(size_t)r * g.nco + cI];
}

// sum over the three terms of +-M_s v_s on rows i0 + il < b: threads < 32 kBcrRC return row
// il = tid / kBcrRC, column c = tid % kBcrRC.  vs: 3 x b x kBcrRC staging, red: 8 x 32 x kBcrRC.
template <class T>
__device__ __forceinline__ cx<T> bcr_rows(const Geom& g, int b, int i0, const BcrTerm<T> (&tm)[3],
                                          const cx<T>* __restrict__ gv, const cx<T>* __restrict__ Tc,
                                          const cx<T>* __restrict__ xr, int ldr, int R, int r0, int nc, cx<T>* vs,
                                          cx<T>* red) {
  const int tid = threadIdx.x, il = tid >> 3, kg = tid & 7, i = i0 + il;
  cx<T> mr[3][8];
#pragma unroll
  for (int s = 0; s < 3; ++s)
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int k = kg + 8 * q;
      mr[s][q] = (tm[s].M && i < b && k < b) ? tm[s].M[(size_t)i * b + k] : czero<T>();
    }
#pragma unroll
  for (int s = 0; s < 3; ++s)
    for (int e = tid; tm[s].M && e < b * kBcrRC; e += blockDim.x) {
      const int k = e / kBcrRC, c = e - k * kBcrRC;
      cx<T> v = czero<T>();
      if (c < nc) {
        const int r = r0 + c, cI = tm[s].layer * b + k;
        v = tm[s].src ? xr[(size_t)r * ldr + cI] : bcr_g(g, gv, Tc, R, r, cI);
      }
      vs[((size_t)s * b + k) * kBcrRC + c] = v;
    }
  __syncthreads();
  cx<T> p[kBcrRC];
#pragma unroll
  for (int c = 0; c < kBcrRC; ++c) p[c] = czero<T>();
  for (int q0 = 0; q0 < (b + 7) / 8; q0 += 8) {
    if (q0 > 0) {  // blocks wider than 64: the next eight k-steps
#pragma unroll
      for (int s = 0; s < 3; ++s)
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = kg + 8 * (q0 + q);
          mr[s][q] = (tm[s].M && i < b && k < b) ? tm[s].M[(size_t)i * b + k] : czero<T>();
        }
    }
#pragma unroll
    for (int s = 0; s < 3; ++s)
      if (tm[s].M) {
        const cx<T>* v = vs + (size_t)s * b * kBcrRC;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int k = kg + 8 * (q0 + q);
          if (k < b) {
#pragma unroll
            for (int c = 0; c < kBcrRC; ++c)
              if (c < nc) {
                if (tm[s].neg) cfms(p[c], mr[s][q], v[k * kBcrRC + c]);
                else cfma(p[c], mr[s][q], v[k * kBcrRC + c]);
              }
          }
        }
      }
  }
#pragma unroll
  for (int c = 0; c < kBcrRC; ++c) red[(kg * 32 + il) * kBcrRC + c] = p[c];
  __syncthreads();
  cx<T> out = czero<T>();
  if (tid < 32 * kBcrRC) {
    const int rl = tid / kBcrRC, c = tid - rl * kBcrRC;
#pragma unroll
    for (int q = 0; q < 8; ++q) out = cadd(out, red[(q * 32 + rl) * kBcrRC + c]);
  }
  return out;
}

// forward step of level 0 into the reduced right-hand side fr ([R][ldr], compact layer order);
// tgt[5 c..] = (t, jr, kr, jl, kl) of the c-th surviving layer; Lp0 = A_pj D_j^{-1},
// LqT0 = (D_j^{-1} A_jq)^T
template <class T>
__global__ void __launch_bounds__(256) k_bcr_fwd0(Geom g, const int* __restrict__ tgt, const cx<T>* __restrict__ Lp0,
                                                  const cx<T>* __restrict__ LqT0, const cx<T>* __restrict__ gv,
                                                  const cx<T>* __restrict__ Tc, cx<T>* fr, int ldr, int R,
                                                  const int* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smb[];
  const int b = g.cb;
  cx<T>* vs = reinterpret_cast<cx<T>*>(smb);  // 3 x b x kBcrRC
  cx<T>* red = vs + 3 * (size_t)b * kBcrRC;    // 8 x 32 x kBcrRC
  const int c = blockIdx.x, i0 = blockIdx.y * 32, r0 = blockIdx.z * kBcrRC, nc = min(kBcrRC, R - r0);
  const int t = tgt[5 * c], jr = tgt[5 * c + 1], kr = tgt[5 * c + 2], jl = tgt[5 * c + 3], kl = tgt[5 * c + 4];
  const size_t bb = (size_t)b * b;
  const BcrTerm<T> tm[3] = {{kr >= 0 ? Lp0 + (size_t)kr * bb : nullptr, 0, jr, true},
                            {kl >= 0 ? LqT0 + (size_t)kl * bb : nullptr, 0, jl, true},
                            {nullptr, 0, 0, false}};
  const cx<T> y = bcr_rows(g, b, i0, tm, gv, Tc, (const cx<T>*)nullptr, 0, R, r0, nc, vs, red);
  const int tid = threadIdx.x;
  if (tid < 32 * kBcrRC) {
    const int il = tid / kBcrRC, cc = tid - il * kBcrRC, i = i0 + il, r = r0 + cc;
    if (i < b && cc < nc && (!active || active[r]))
      fr[(size_t)r * ldr + (size_t)c * b + i] = cadd(bcr_g(g, gv, Tc, R, r, t * b + i), y);
  }
}

// backward step of level 0: blocks x < nj solve the eliminated layers (elim[3 x..] = (j, cp, cq)),
// blocks nj + c copy the reduced solution of the c-th surviving layer rem[c] into w ([R][n_c]);
// D0 = D_j^{-1}, LpT0 = (A_pj D_j^{-1})^T, Lq0 = D_j^{-1} A_jq
template <class T>
__global__ void __launch_bounds__(256) k_bcr_bwd0(Geom g, int nj, const int* __restrict__ elim, const int* __restrict__ rem,
                                                  const cx<T>* __restrict__ D0, const cx<T>* __restrict__ LpT0,
                                                  const cx<T>* __restrict__ Lq0, const cx<T>* __restrict__ gv,
                                                  const cx<T>* __restrict__ Tc, const cx<T>* __restrict__ xr, int ldr,
                                                  cx<T>* w, int R, const int* __restrict__ active) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smb[];
  const int b = g.cb;
  cx<T>* vs = reinterpret_cast<cx<T>*>(smb);
  cx<T>* red = vs + 3 * (size_t)b * kBcrRC;
  const int x = blockIdx.x, i0 = blockIdx.y * 32, r0 = blockIdx.z * kBcrRC, nc = min(kBcrRC, R - r0);
  const int tid = threadIdx.x;
  if (x >= nj) {
    const int cidx = x - nj, t = rem[cidx];
    if (tid < 32 * kBcrRC) {
      const int il = tid / kBcrRC, cc = tid - il * kBcrRC, i = i0 + il, r = r0 + cc;
      if (i < b && cc < nc && (!active || active[r]))
        w[(size_t)r * g.nco + (size_t)t * b + i] = xr[(size_t)r * ldr + (size_t)cidx * b + i];
    }
    return;
  }
  const int j = elim[3 * x], cp = elim[3 * x + 1], cq = elim[3 * x + 2];
  const size_t bb = (size_t)b * b;
  const BcrTerm<T> tm[3] = {{D0 + (size_t)x * bb, 0, j, false},
                            {cp >= 0 ? LpT0 + (size_t)x * bb : nullptr, 1, cp, true},
                            {cq >= 0 ? Lq0 + (size_t)x * bb : nullptr, 1, cq, true}};
  const cx<T> y = bcr_rows(g, b, i0, tm, gv, Tc, xr, ldr, R, r0, nc, vs, red);
  if (tid < 32 * kBcrRC) {
    const int il = tid / kBcrRC, cc = tid - il * kBcrRC, i = i0 + il, r = r0 + cc;
    if (i < b && cc < nc && (!active || active[r])) w[(size_t)r * g.nco + (size_t)j * b + i] = y;
  }
}

// dst block k = (src block k)^T for count b x b row-major blocks
template <class T>
__global__ void k_transpose_blocks(const cx<T>* __restrict__ src, int count, int b, cx<T>* dst) {
  const size_t bb = (size_t)b * b;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)count * bb;
       e += (size_t)gridDim.x * blockDim.x) {
    const size_t k = e / bb;
    const int r = (int)(e - k * bb), i = r / b, jx = r - i * b;
    dst[k * bb + (size_t)jx * b + i] = src[e];
  }
}

// Frc^s w_s on slot j of subdomain sd (w: coarse vector of one right-hand side; Frc: the nq
// coupling columns of the class, the corners' and with the augmented coarse problem the faces').
template <class T>
__device__ __forceinline__ cx<T> frc_corr(const Geom& g, const MapsView& m, const cx<T>* __restrict__ Frc,
                                          const cx<T>* __restrict__ w, int sd, int j) {
  cx<T> acc = czero<T>();
  if (!w) return acc;
  const int q = m.sd_cls[sd];
  for (int c = 0; c < g.nq; ++c) {
    int ci = m.sd_coarse[(size_t)sd * g.nq + c];
    if (ci >= 0) cfma(acc, Frc[((size_t)q * g.nD + j) * g.nq + c], w[ci]);
  }
  return acc;
}

// d = d_r - Frc~ Kcc~^{-1} f~_c:  d_lambda = sum over its two sides sigma (VD - Frc w0).
template <class T>
__global__ void k_dual_rhs(Geom g, MapsView m, const cx<T>* __restrict__ VD, const cx<T>* __restrict__ Frc,
                           const cx<T>* __restrict__ w0, int R, cx<T>* d) {
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)R * g.nlam) return;
  int r = (int)(e / g.nlam), lam = (int)(e % g.nlam);
  cx<T> v = czero<T>();
  for (int side = 0; side < 2; ++side) {
    int code = m.lam_side[2 * lam + side];
    int sd = code / g.nD, j = code - sd * g.nD;
    cx<T> t = csub(VD[((size_t)sd * R + r) * g.nD + j], frc_corr(g, m, Frc, w0 ? w0 + (size_t)r * g.nco : nullptr, sd, j));
    v = side == 0 ? cadd(v, t) : csub(v, t);
  }
  d[(size_t)r * g.nlam + lam] = v;
}

// Local dense apply per subdomain with the gather of B^T lambda fused in front:
//   x_j = scale_j * sum_k sign_k lam[idx_k]        (scale = 1/multiplicity for the preconditioner)
//   Y   = Op[cls] x                                 (Op = F or S, nD x nD, symmetric, packed)
//   Tc  = Frc[cls]^T x                              (only when Tc != null)
template <class T, bool SCALE, int MR>
__global__ void k_local_apply(Geom g, MapsView m, const cx<T>* __restrict__ Op, const cx<T>* __restrict__ Frc,
                              const cx<T>* __restrict__ lam, int R, const int* __restrict__ active, cx<T>* Y,
                              cx<T>* Tc, int stage, const double* __restrict__ vscale) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smla[];
  cx<T>* x = reinterpret_cast<cx<T>*>(smla);
  const int sd = blockIdx.x, nD = g.nD, tid = threadIdx.x, nthr = blockDim.x, md = g.maxdeg;
  const int q = m.sd_cls[sd];
  // packed upper triangle of Op[cls]; staged in shared memory by asynchronous 16-byte copies that
  // overlap the gather of x when it fits
  const long long ld = sym_ld(nD);
  const cx<T>* A = Op + (size_t)q * ld;
  if (stage) {
    unsigned char* As = reinterpret_cast<unsigned char*>(x + (((long long)R * nD + 1) & ~1LL));
    const int n16 = (int)(ld * (long long)sizeof(cx<T>) / 16);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(A);
    for (int i = tid; i < n16; i += nthr) cp_async16(As + 16 * (size_t)i, src + 16 * (size_t)i);
    cp_async_commit();
    A = reinterpret_cast<const cx<T>*>(As);
  }
  for (int e = tid; e < R * nD; e += nthr) {
    int r = e / nD, j = e - r * nD;
    cx<T> v = czero<T>();
    if (active[r]) {
      const int* refs = m.sd_lam + ((size_t)sd * nD + j) * md;
      for (int k = 0; k < md; ++k) {
        int ref = refs[k];
        if (ref > 0) v = cadd(v, lam[(size_t)r * g.nlam + ref - 1]);
        else if (ref < 0) v = csub(v, lam[(size_t)r * g.nlam - ref - 1]);
      }
      if (SCALE) v = cscale(v, (T)m.sd_minv[(size_t)sd * nD + j]);
      if (vscale) v = cscale(v, (T)vscale[r]);
    }
    x[e] = v;
  }
  if (stage) cp_async_wait<0>();
  __syncthreads();
  for (int j = tid; j < nD; j += nthr) {
    cx<T> acc[MR];
    for (int r = 0; r < MR; ++r) acc[r] = czero<T>();
    const int offj = sym_off(j, nD);
    int ok = 0;  // sym_off(k, nD)
#pragma unroll 4
    for (int k = 0; k < nD; ++k) {
      const cx<T> a = A[k <= j ? ok + (j - k) : offj + (k - j)];
      ok += nD - k;
#pragma unroll
      for (int r = 0; r < MR; ++r)
        if (r < R) cfma(acc[r], a, x[r * nD + k]);
    }
#pragma unroll
    for (int r = 0; r < MR; ++r)
      if (r < R) Y[((size_t)sd * R + r) * nD + j] = acc[r];
  }
  if (Tc && R * g.nq <= 16) {
    // Tc[r][c] = sum_j Frc[j][c] x[r][j] for all (r, c) at once: per-thread partials over j, warp
    // shuffles, one barrier, the warps' partials added in warp order
    __shared__ cx<T> redf[16][16];
    const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5, nq = g.nq, nrc = R * nq;
    const cx<T>* Fr = Frc + (size_t)q * nD * nq;
    cx<T> p[16];
#pragma unroll
    for (int rc = 0; rc < 16; ++rc) p[rc] = czero<T>();
    for (int j = tid; j < nD; j += nthr) {
#pragma unroll
      for (int rc = 0; rc < 16; ++rc)
        if (rc < nrc) {
          const int r = rc / nq, c = rc - r * nq;
          cfma(p[rc], Fr[(size_t)j * nq + c], x[r * nD + j]);
        }
    }
#pragma unroll
    for (int rc = 0; rc < 16; ++rc)
      if (rc < nrc)
        for (int o = 16; o > 0; o >>= 1) p[rc] = cadd(p[rc], shfl_xor_cx(p[rc], o));
    if (lane == 0)
#pragma unroll
      for (int rc = 0; rc < 16; ++rc)
        if (rc < nrc) redf[warp][rc] = p[rc];
    __syncthreads();
    if (tid < nrc) {
      cx<T> s = czero<T>();
      for (int w = 0; w < nw; ++w) s = cadd(s, redf[w][tid]);
      const int r = tid / nq, c = tid - r * nq;
      Tc[((size_t)sd * R + r) * nq + c] = s;
    }
  } else if (Tc) {
    // Tc[r][c] = sum_j Frc[j][c] x[r][j]: per-thread partials over j, warp shuffles, then warps
    __shared__ cx<T> red[32];
    const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5;
    const cx<T>* Fr = Frc + (size_t)q * nD * g.nq;
    for (int rc = 0; rc < R * g.nq; ++rc) {
      const int r = rc / g.nq, c = rc - r * g.nq;
      cx<T> p = czero<T>();
      for (int j = tid; j < nD; j += nthr) cfma(p, Fr[(size_t)j * g.nq + c], x[r * nD + j]);
      for (int o = 16; o > 0; o >>= 1) {
        p.re += __shfl_xor_sync(0xffffffffu, p.re, o);
        p.im += __shfl_xor_sync(0xffffffffu, p.im, o);
      }
      __syncthreads();
      if (lane == 0) red[warp] = p;
      __syncthreads();
      if (tid == 0) {
        cx<T> s = czero<T>();
        for (int w = 0; w < nw; ++w) s = cadd(s, red[w]);
        Tc[((size_t)sd * R + r) * g.nq + c] = s;
      }
    }
  }
}

// One right-hand side with the packed operator staged in shared memory.  The copies of Op (setup
// data) are issued before waiting on the previous kernel.  Thread j walks two offsets into the
// packed upper triangle: down column j (A[k][j], k < j, step nD - 1 - k) and along row j (A[j][k],
// k >= j, step 1), one select per term, so that
//   y_j = sum_{k<j} A[k][j] x_k + sum_{k>=j} A[j][k] x_k;
// Tc = Frc^T x: each thread's nq products, warp shuffles, one barrier, warps added in order.
template <class T, bool SCALE>
__global__ void __launch_bounds__(128) k_local_apply_1(Geom g, MapsView m, const cx<T>* __restrict__ Op,
                                                       const cx<T>* __restrict__ Frc, const cx<T>* __restrict__ lam,
                                                       const int* __restrict__ active, cx<T>* Y, cx<T>* Tc,
                                                       const double* __restrict__ vscale) {
  extern __shared__ __align__(16) unsigned char smla[];
  const int sd = blockIdx.x, nD = g.nD, tid = threadIdx.x, nthr = blockDim.x, md = g.maxdeg;
  const int q = m.sd_cls[sd];
  const int ld = (int)sym_ld(nD);
  cx<T>* As = reinterpret_cast<cx<T>*>(smla);
  cx<T>* x = As + ld;
  {
    const int n16 = (int)((long long)ld * sizeof(cx<T>) / 16);
    const unsigned char* src = reinterpret_cast<const unsigned char*>(Op + (size_t)q * ld);
    unsigned char* dst = reinterpret_cast<unsigned char*>(As);
    for (int i = tid; i < n16; i += nthr) cp_async16(dst + 16 * (size_t)i, src + 16 * (size_t)i);
    cp_async_commit();
  }
  pdl_wait();
  pdl_trigger();
  const bool on = active[0] != 0;
  for (int j = tid; j < nD; j += nthr) {
    cx<T> v = czero<T>();
    if (on) {
      const int* refs = m.sd_lam + ((size_t)sd * nD + j) * md;
      for (int k = 0; k < md; ++k) {
        const int ref = refs[k];
        if (ref > 0) v = cadd(v, lam[ref - 1]);
        else if (ref < 0) v = csub(v, lam[-ref - 1]);
      }
      if (SCALE) v = cscale(v, (T)m.sd_minv[(size_t)sd * nD + j]);
      if (vscale) v = cscale(v, (T)vscale[0]);
    }
    x[j] = v;
  }
  cp_async_wait<0>();
  __syncthreads();
  const int nq = Tc ? g.nq : 0;
  cx<T> p[16];
#pragma unroll
  for (int c = 0; c < 16; ++c) p[c] = czero<T>();
  for (int j = tid; j < nD; j += nthr) {
    cx<T> acc = czero<T>();
    int oc = j;                        // A[k][j] for k < j
    const int orow = sym_off(j, nD) - j;  // A[j][k] = As[orow + k] for k >= j
#pragma unroll 4
    for (int k = 0; k < nD; ++k) {
      const int o = k < j ? oc : orow + k;
      oc += nD - 1 - k;
      cfma(acc, As[o], x[k]);
    }
    Y[(size_t)sd * nD + j] = acc;
    if (nq) {
      const cx<T>* Fr = Frc + ((size_t)q * nD + j) * nq;
      const cx<T> xj = x[j];
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < nq) cfma(p[c], Fr[c], xj);
    }
  }
  if (nq) {
    __shared__ cx<T> red1[4][16];  // blocks of at most 128 threads
    const int lane = tid & 31, warp = tid >> 5, nw = (nthr + 31) >> 5;
#pragma unroll
    for (int c = 0; c < 16; ++c)
      if (c < nq)
        for (int o = 16; o > 0; o >>= 1) p[c] = cadd(p[c], shfl_xor_cx(p[c], o));
    if (lane == 0)
#pragma unroll
      for (int c = 0; c < 16; ++c)
        if (c < nq) red1[warp][c] = p[c];
    __syncthreads();
    if (tid < nq) {
      cx<T> s = czero<T>();
      for (int w = 0; w < nw; ++w) s = cadd(s, red1[w][tid]);
      Tc[(size_t)sd * nq + tid] = s;
    }
  }
}

// The same apply for a group of subdomains that share their stored operators (one class): the CTA
// unpacks Op[cls] into a full nD x nD array in shared memory and stages Frc[cls] (both written at
// setup, so before waiting on the previous kernel), gathers x for every (member, right-hand side)
// column of the group and forms Y = Op x and Tc = Frc^T x for all of them: each operator entry
// read from L2 serves every column.  Thread (j, cc), j = tid mod TJ (TJ = nD rounded up to a warp),
// takes the CPT consecutive columns cc CPT + s TC CPT; a warp shares cc, so x is read by broadcast
// and Op[k][j] by consecutive j.  Shared memory: (nD^2 + kApplyGroup R nD + nD nq) entries.
template <class T, bool SCALE, int CPT>
__global__ void __launch_bounds__(256) k_local_apply_grp(Geom g, MapsView m, const cx<T>* __restrict__ Op,
                                                         const cx<T>* __restrict__ Frc,
                                                         const cx<T>* __restrict__ lam, int R,
                                                         const int* __restrict__ active, cx<T>* Y, cx<T>* Tc,
                                                         const double* __restrict__ vscale) {
  extern __shared__ __align__(16) unsigned char smla[];
  const int nD = g.nD, nq = g.nq, md = g.maxdeg, tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  const int g0 = m.grp_ptr[blockIdx.x], ncol = (m.grp_ptr[blockIdx.x + 1] - g0) * R;
  const int q = m.sd_cls[m.grp_sd[g0]];
  cx<T>* As = reinterpret_cast<cx<T>*>(smla);   // As[k nD + j] = Op[j][k]
  cx<T>* X = As + (size_t)nD * nD;               // X[c nD + j], column c = member R + r
  cx<T>* Fs = X + (size_t)kApplyGroup * R * nD;  // Fs[j nq + c] = Frc[j][c]
  {
    // packed rows read with consecutive lanes, written to both triangles
    const cx<T>* A = Op + (size_t)q * sym_ld(nD);
    for (int i = warp; i < nD; i += nw) {
      const cx<T>* row = A + sym_off(i, nD) - i;
      for (int k = i + lane; k < nD; k += 32) {
        const cx<T> a = row[k];
        As[(size_t)k * nD + i] = a;
        As[(size_t)i * nD + k] = a;
      }
    }
    if (Tc) {
      const cx<T>* F = Frc + (size_t)q * nD * nq;
      for (int e = tid; e < nD * nq; e += nthr) Fs[e] = F[e];
    }
  }
  pdl_wait();
  pdl_trigger();
  for (int e = tid; e < ncol * nD; e += nthr) {
    const int c = e / nD, j = e - c * nD, mi = c / R, r = c - mi * R;
    const int sd = m.grp_sd[g0 + mi];
    cx<T> v = czero<T>();
    if (active[r]) {
      const int* refs = m.sd_lam + ((size_t)sd * nD + j) * md;
      for (int k = 0; k < md; ++k) {
        const int ref = refs[k];
        if (ref > 0) v = cadd(v, lam[(size_t)r * g.nlam + ref - 1]);
        else if (ref < 0) v = csub(v, lam[(size_t)r * g.nlam - ref - 1]);
      }
      if (SCALE) v = cscale(v, (T)m.sd_minv[(size_t)sd * nD + j]);
      if (vscale) v = cscale(v, (T)vscale[r]);
    }
    X[e] = v;
  }
  __syncthreads();
  const int TJ = (nD + 31) & ~31, TC = nthr / TJ, j = tid % TJ, cc = tid / TJ;
  if (j < nD && cc < TC) {
    for (int c0 = cc * CPT; c0 < ncol; c0 += TC * CPT) {
      cx<T> acc[CPT];
#pragma unroll
      for (int i = 0; i < CPT; ++i) acc[i] = czero<T>();
#pragma unroll 4
      for (int k = 0; k < nD; ++k) {
        const cx<T> a = As[(size_t)k * nD + j];
#pragma unroll
        for (int i = 0; i < CPT; ++i)
          if (c0 + i < ncol) cfma(acc[i], a, X[(size_t)(c0 + i) * nD + k]);
      }
#pragma unroll
      for (int i = 0; i < CPT; ++i)
        if (c0 + i < ncol) {
          const int c = c0 + i, mi = c / R, r = c - mi * R;
          Y[((size_t)m.grp_sd[g0 + mi] * R + r) * nD + j] = acc[i];
        }
    }
  }
  if (Tc) {
    // Tc[sd][r][c] = sum_j Frc[j][c] x[r][j]: L lanes per output, strided over j, xor shuffles
    // within aligned groups of L lanes; every warp runs the same number of passes
    const int nout = ncol * nq;
    int L = 32;
    while (L > 1 && nthr / L < nout) L >>= 1;
    const int per = nthr / L, sub = tid % L, passes = (nout + per - 1) / per;
    for (int p = 0; p < passes; ++p) {
      const int o = p * per + tid / L;
      cx<T> s = czero<T>();
      if (o < nout) {
        const int c = o / nq, cq = o - c * nq;
        for (int jj = sub; jj < nD; jj += L) cfma(s, Fs[jj * nq + cq], X[(size_t)c * nD + jj]);
      }
      for (int off = L >> 1; off > 0; off >>= 1) s = cadd(s, shfl_xor_cx(s, off));
      if (o < nout && sub == 0) {
        const int c = o / nq, cq = o - c * nq, mi = c / R, r = c - mi * R;
        Tc[((size_t)m.grp_sd[g0 + mi] * R + r) * nq + cq] = s;
      }
    }
  }
}

// Single right-hand side, large blocks (3D: nD = 378, 573 KB per packed FP32 operator): the packed
// upper triangle is streamed row by row with coalesced loads.  Warp w takes rows w, w + W, ...; for
// row i its lanes read consecutive entries A[i][k], k >= i, and use each twice: the dot product
// sum_k A[i][k] x_k (-> y_i) and the symmetric update y_k += A[i][k] x_i (k > i) into a per-warp
// partial vector in shared memory.  The partial vectors are summed at the end.
template <class T, bool SCALE>
__global__ void __launch_bounds__(512) k_local_apply_rows(Geom g, MapsView m, const cx<T>* __restrict__ Op,
                                                          const cx<T>* __restrict__ Frc,
                                                          const cx<T>* __restrict__ lam,
                                                          const int* __restrict__ active, cx<T>* Y, cx<T>* Tc,
                                                          const double* __restrict__ vscale) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ __align__(16) unsigned char smla[];
  const int sd = blockIdx.x, nD = g.nD, tid = threadIdx.x, nthr = blockDim.x, md = g.maxdeg;
  const int lane = tid & 31, warp = tid >> 5, nw = nthr >> 5;
  cx<T>* x = reinterpret_cast<cx<T>*>(smla);
  cx<T>* yp = x + ((nD + 1) & ~1);  // [nw][nD] partial results
  const int q = m.sd_cls[sd];
  const cx<T>* A = Op + (size_t)q * sym_ld(nD);
  const bool on = active[0] != 0;
  for (int j = tid; j < nD; j += nthr) {
    cx<T> v = czero<T>();
    if (on) {
      const int* refs = m.sd_lam + ((size_t)sd * nD + j) * md;
      for (int k = 0; k < md; ++k) {
        int ref = refs[k];
        if (ref > 0) v = cadd(v, lam[ref - 1]);
        else if (ref < 0) v = csub(v, lam[-ref - 1]);
      }
      if (SCALE) v = cscale(v, (T)m.sd_minv[(size_t)sd * nD + j]);
      if (vscale) v = cscale(v, (T)vscale[0]);
    }
    x[j] = v;
  }
  for (int e = tid; e < nw * nD; e += nthr) yp[e] = czero<T>();
  __syncthreads();
  cx<T>* y = yp + (size_t)warp * nD;
  for (int i = warp; i < nD; i += nw) {
    const cx<T>* Ai = A + sym_off(i, nD) - i;  // Ai[k] = A[i][k], k >= i
    const cx<T> xi = x[i];
    cx<T> dot = czero<T>();
#pragma unroll 4
    for (int k = i + lane; k < nD; k += 32) {
      const cx<T> a = Ai[k];
      cfma(dot, a, x[k]);
      if (k > i) cfma(y[k], a, xi);
    }
    for (int o = 16; o > 0; o >>= 1) {
      dot.re += __shfl_xor_sync(0xffffffffu, dot.re, o);
      dot.im += __shfl_xor_sync(0xffffffffu, dot.im, o);
    }
    __syncwarp();
    if (lane == 0) y[i] = cadd(y[i], dot);
    __syncwarp();
  }
  __syncthreads();
  for (int j = tid; j < nD; j += nthr) {
    cx<T> s = czero<T>();
    for (int w = 0; w < nw; ++w) s = cadd(s, yp[(size_t)w * nD + j]);
    Y[(size_t)sd * nD + j] = s;
  }
  if (Tc) {
    // Tc[c] = sum_j Frc[j][c] x[j]: one warp per coupling column
    const cx<T>* Fr = Frc + (size_t)q * nD * g.nq;
    for (int c = warp; c < g.nq; c += nw) {
      cx<T> p = czero<T>();
      for (int j = lane; j < nD; j += 32) cfma(p, Fr[(size_t)j * g.nq + c], x[j]);
      for (int o = 16; o > 0; o >>= 1) {
        p.re += __shfl_xor_sync(0xffffffffu, p.re, o);
        p.im += __shfl_xor_sync(0xffffffffu, p.im, o);
      }
      if (lane == 0) Tc[(size_t)sd * g.nq + c] = p;
    }
  }
}

// out_lambda = sum over sides sigma * scale * (Y + Frc wc):  B (Y + Frc wc) for the dual operator,
// B_D Y for the preconditioner (SCALE, wc = null).
template <class T, bool SCALE>
__global__ void k_scatter(Geom g, MapsView m, const cx<T>* __restrict__ Y, const cx<T>* __restrict__ Frc,
                          const cx<T>* __restrict__ wc, int R, const int* __restrict__ active, cx<T>* out) {
  pdl_wait();
  pdl_trigger();
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)R * g.nlam) return;
  int r = (int)(e / g.nlam), lam = (int)(e % g.nlam);
  if (!active[r]) return;
  cx<T> v = czero<T>();
  for (int side = 0; side < 2; ++side) {
    int code = m.lam_side[2 * lam + side];
    int sd = code / g.nD, j = code - sd * g.nD;
    cx<T> t = Y[((size_t)sd * R + r) * g.nD + j];
    if (wc) t = cadd(t, frc_corr(g, m, Frc, wc + (size_t)r * g.nco, sd, j));
    if (SCALE) t = cscale(t, (T)m.sd_minv[(size_t)sd * g.nD + j]);
    v = side == 0 ? cadd(v, t) : csub(v, t);
  }
  out[(size_t)r * g.nlam + lam] = v;
}

// ------------------------------------------------------------------ fused Gram-Schmidt (CGS2)
// Orthogonalisation of w against V_0..V_k for each right-hand side r: grid (nblk, R), block bx
// owns the contiguous slice bx of the vectors.  Each kernel leaves FP64 partial sums per block;
// the last block of r to finish (ticket counter) adds them in block order, so the result does not
// depend on scheduling, and resets the counter for the next launch.
//   k_scatter_orth_dots: w = B (Y + Frc wc); h = V^H w       -> hc, H[:, k] += h
//   k_orth_update_dots: w -= V hc; h = V^H w                -> hc, H[:, k] += h
//   k_orth_update_norm: w -= V hc; h_{k+1,k} = |w|, Givens rotation of column k
struct OrthArgs {
  long long vstride;
  int nlam, k, m, nblk;
  const int* active;
  cx<double>* part;  // [R][kMaxKdev][nblk]
  double* nrm_part;  // [R][nblk]
  int* cnt;          // [R] tickets, zero between launches
  cx<double>* H;
  cx<double>* hc;
  // Givens state
  double* cs_c;
  cx<double>* cs_s;
  cx<double>* gvec;
  const double* beta0;
  double tol;
  int* active_w;
  int* kk;
  double* inv_nrm;
  double* resid;
  int* bad;
  // lazy normalisation: V_k still holds w_k unscaled; the first pass scales its slice by inv_nrm
  int lazy;
};

__device__ __forceinline__ bool orth_last_block(int* cnt, int nblk) {
  __shared__ int is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(cnt, 1) == nblk - 1);
  __syncthreads();
  return is_last != 0;
}

// partial dots of the block slice ws (in shared memory) with V_0..V_k, one warp per j
template <class T>
__device__ __forceinline__ void orth_block_dots(const cx<T>* __restrict__ V, const OrthArgs& a, int r, int lo, int n,
                                                const cx<T>* ws) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j <= a.k; j += nw) {
    const cx<T>* vj = V + j * a.vstride + (size_t)r * a.nlam + lo;
    T pre = 0, pim = 0;  // per-lane partial sums (a few terms) in T, combined in FP64
#pragma unroll 4
    for (int i = lane; i < n; i += 32) {
      const cx<T> x = vj[i], y = ws[i];
      pre += x.re * y.re + x.im * y.im;
      pim += x.re * y.im - x.im * y.re;
    }
    double re = pre, im = pim;
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) a.part[((size_t)r * kMaxKdev + j) * a.nblk + blockIdx.x] = mkc<double>(re, im);
  }
}

// last block: h_j = sum over blocks in order; hc = h, H[:, k] += h
__device__ __forceinline__ void orth_finish_dots(const OrthArgs& a, int r) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = warp; j <= a.k; j += nw) {
    const cx<double>* p = a.part + ((size_t)r * kMaxKdev + j) * a.nblk;
    double re = 0, im = 0;
#pragma unroll 4
    for (int b = lane; b < a.nblk; b += 32) {
      const double2 v = __ldcg(reinterpret_cast<const double2*>(p + b));
      re += v.x;
      im += v.y;
    }
    for (int o = 16; o > 0; o >>= 1) {
      re += __shfl_xor_sync(0xffffffffu, re, o);
      im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0) {
      a.hc[(size_t)r * kMaxKdev + j] = mkc<double>(re, im);
      cx<double>& h = a.H[((size_t)r * a.m + a.k) * (a.m + 1) + j];
      h = cadd(h, mkc<double>(re, im));
    }
  }
  if (threadIdx.x == 0) a.cnt[r] = 0;
}

// slice [lo, lo + n) of block bx
__device__ __forceinline__ void orth_slice(const OrthArgs& a, int* lo, int* n) {
  const int seg = (a.nlam + a.nblk - 1) / a.nblk;
  *lo = blockIdx.x * seg;
  *n = max(0, min(a.nlam, *lo + seg) - *lo);
}

// ws = w - V hc on the slice (written back to w); hc staged in shared memory as T
template <class T>
__device__ __forceinline__ void orth_block_update(const cx<T>* __restrict__ V, const OrthArgs& a, int r, int lo, int n,
                                                  cx<T>* w, cx<T>* ws, cx<T>* h) {
  for (int j = threadIdx.x; j <= a.k; j += blockDim.x) h[j] = ccast<T>(a.hc[(size_t)r * kMaxKdev + j]);
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    cx<T> acc = w[(size_t)r * a.nlam + lo + i];
#pragma unroll 4
    for (int j = 0; j <= a.k; ++j) cfms(acc, h[j], V[j * a.vstride + (size_t)r * a.nlam + lo + i]);
    w[(size_t)r * a.nlam + lo + i] = acc;
    ws[i] = acc;
  }
  __syncthreads();
}

// The dual operator's final scatter fused with the first Gram-Schmidt pass: the block computes
// its slice of w = B (Y + Frc wc) (the new Arnoldi vector, written out) straight into shared memory
// and takes its partial dots with V_0..V_k.
template <class T>
__global__ void __launch_bounds__(256) k_scatter_orth_dots(Geom g, MapsView m, const cx<T>* __restrict__ Y,
                                                           const cx<T>* __restrict__ Frc, const cx<T>* __restrict__ wc,
                                                           cx<T>* V, cx<T>* w, int R, OrthArgs a) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ unsigned char smraw[];
  cx<T>* ws = reinterpret_cast<cx<T>*>(smraw);
  const int r = blockIdx.y;
  if (!a.active[r]) return;
  int lo, n;
  orth_slice(a, &lo, &n);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int lam = lo + i;
    cx<T> v = czero<T>();
    for (int side = 0; side < 2; ++side) {
      const int code = m.lam_side[2 * lam + side];
      const int sd = code / g.nD, j = code - sd * g.nD;
      cx<T> t = Y[((size_t)sd * R + r) * g.nD + j];
      if (wc) t = cadd(t, frc_corr(g, m, Frc, wc + (size_t)r * g.nco, sd, j));
      v = side == 0 ? cadd(v, t) : csub(v, t);
    }
    w[(size_t)r * a.nlam + lam] = v;
    ws[i] = v;
  }
  if (a.lazy) {  // V_k = w_k / ||w_k||: this block's slice, before the dots read it
    cx<T>* vk = V + a.k * a.vstride + (size_t)r * a.nlam + lo;
    const T sc = (T)a.inv_nrm[r];
    for (int i = threadIdx.x; i < n; i += blockDim.x) vk[i] = cscale(vk[i], sc);
  }
  __syncthreads();
  orth_block_dots(V, a, r, lo, n, ws);
  if (orth_last_block(a.cnt + r, a.nblk)) orth_finish_dots(a, r);
}

template <class T>
__global__ void __launch_bounds__(256) k_orth_update_dots(const cx<T>* __restrict__ V, cx<T>* w, OrthArgs a) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ unsigned char smraw[];
  cx<T>* h = reinterpret_cast<cx<T>*>(smraw);  // k + 1
  cx<T>* ws = h + (a.k + 1);                   // slice
  const int r = blockIdx.y;
  if (!a.active[r]) return;
  int lo, n;
  orth_slice(a, &lo, &n);
  orth_block_update(V, a, r, lo, n, w, ws, h);
  orth_block_dots(V, a, r, lo, n, ws);
  if (orth_last_block(a.cnt + r, a.nblk)) orth_finish_dots(a, r);
}

template <class T>
__global__ void __launch_bounds__(256) k_orth_update_norm(const cx<T>* __restrict__ V, cx<T>* w, OrthArgs a) {
  pdl_wait();
  pdl_trigger();
  extern __shared__ unsigned char smraw[];
  cx<T>* h = reinterpret_cast<cx<T>*>(smraw);
  cx<T>* ws = h + (a.k + 1);
  __shared__ double red[32];
  const int r = blockIdx.y;
  if (!a.active[r]) return;
  int lo, n;
  orth_slice(a, &lo, &n);
  orth_block_update(V, a, r, lo, n, w, ws, h);
  T ps = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) ps += ws[i].re * ws[i].re + ws[i].im * ws[i].im;
  double s = ps;
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (int)(blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) a.nrm_part[(size_t)r * a.nblk + blockIdx.x] = s;
  }
  if (orth_last_block(a.cnt + r, a.nblk)) {
    // every thread reads its blocks' partials (one load round), warps and then the block add in order
    __shared__ double fred[32];
    double t = 0;
    for (int b = threadIdx.x; b < a.nblk; b += blockDim.x) t += __ldcg(a.nrm_part + (size_t)r * a.nblk + b);
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) fred[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += fred[w];
      givens_step(r, a.k, a.m, sqrt(s), a.H, a.cs_c, a.cs_s, a.gvec, a.beta0, a.tol, a.active_w, a.kk, a.inv_nrm,
                  a.resid, a.bad);
      a.cnt[r] = 0;
    }
  }
}

// Block partial sums of |w|^2 (FP64 accumulation) per right-hand side.
template <class T>
__global__ void k_norm2(const cx<T>* __restrict__ w, int nlam, int R, const int* __restrict__ active, int nblk,
                        double* part) {
  __shared__ double red[32];
  const int r = blockIdx.y;
  if (active && !active[r]) return;
  double s = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nlam; i += (long long)nblk * blockDim.x) {
    cx<T> a = w[(size_t)r * nlam + i];
    s += (double)a.re * (double)a.re + (double)a.im * (double)a.im;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[(size_t)r * nblk + blockIdx.x] = s;
  }
}

template <class T>
__global__ void k_scale_vec(cx<T>* w, int nlam, int R, const int* __restrict__ active, const double* __restrict__ sc) {
  pdl_wait();
  pdl_trigger();
  const int r = blockIdx.y;
  if (!active[r]) return;
  T s = (T)sc[r];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nlam; i += (long long)gridDim.x * blockDim.x)
    w[(size_t)r * nlam + i] = cscale(w[(size_t)r * nlam + i], s);
}

// u = sum_{j < kk[r]} y_j V_j
template <class T>
__global__ void k_combine(const cx<T>* __restrict__ V, long long vstride, int nlam, int R,
                          const cx<double>* __restrict__ y, const int* __restrict__ kk, cx<T>* u) {
  extern __shared__ unsigned char smraw[];
  cx<T>* ys = reinterpret_cast<cx<T>*>(smraw);
  const int r = blockIdx.y, nk = kk[r];
  for (int j = threadIdx.x; j < nk; j += blockDim.x) ys[j] = ccast<T>(y[(size_t)r * kMaxKdev + j]);
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nlam; i += (long long)gridDim.x * blockDim.x) {
    cx<T> acc = czero<T>();
    for (int j = 0; j < nk; ++j) cfma(acc, ys[j], V[j * vstride + (size_t)r * nlam + i]);
    u[(size_t)r * nlam + i] = acc;
  }
}

// ------------------------------------------------------------------------------- recovery
// u_r^s = A_rr^{-1} (f_r - B_r^T lambda - A_rc u_c)
template <class T>
__global__ void k_recover(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv,
                          const cx<double>* __restrict__ f, int ldf, const cx<T>* __restrict__ lam,
                          const cx<T>* __restrict__ uc, int R, cx<T>* Xs) {
  extern __shared__ unsigned char smraw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smraw);
  const int sd = blockIdx.x, dim = g.dim;
  const int q = m.sd_cls[sd], b = P.ly.b, L = P.ly.L, nD = g.nD, md = g.maxdeg;
  P.select(q, m.cls_code);
  int S[3], ext[3];
  idx2crd(sd, g.nsub, dim, S);
  local_ext(g, ext);
  cx<T>* X = Xs + (size_t)sd * g.nl * R;
  auto rhs = [&](int K, int i, int c) -> cx<T> {
    int l[3];
    P.crd(K, i, l);
    if (P.removed_l(l)) return czero<T>();
    int G[3] = {S[0] * g.s[0] + l[0], S[1] * g.s[1] + l[1], dim == 3 ? S[2] * g.s[2] + l[2] : 1};
    cx<double> fv = f[(size_t)c * ldf + gidx(g, G)];
    int slot = m.node_slot[K * b + i];
    double sc = 1.0;
    cx<T> v;
    if (slot >= 0) {
      sc = m.sd_minv[(size_t)sd * nD + slot];
      v = mkc<T>((T)(fv.re * sc), (T)(fv.im * sc));
      if (lam) {
        const int* refs = m.sd_lam + ((size_t)sd * nD + slot) * md;
        for (int k = 0; k < md; ++k) {
          int ref = refs[k];
          if (ref > 0) v = csub(v, lam[(size_t)c * g.nlam + ref - 1]);
          else if (ref < 0) v = cadd(v, lam[(size_t)c * g.nlam - ref - 1]);
        }
      }
    } else {
      v = mkc<T>((T)fv.re, (T)fv.im);
    }
    if (uc) {
      for (int cc = 0; cc < g.nc; ++cc) {
        int ci = m.sd_corner[(size_t)sd * g.nc + cc];
        if (ci < 0) continue;
        int lc[3];
        idx2crd(m.corner_node[cc], ext, dim, lc);
        cfms(v, q1_entry(P.st, g.s, l, lc), uc[(size_t)c * g.nco + ci]);
      }
    }
    return v;
  };
  layered_solve<T>(P, Dinv + (size_t)q * L * b * b, R, rhs, X, R, sm);
}

// ------------------------------------------------------------------ augmented coarse problem
// Besides the corners, one coarse unknown per pair of face-adjacent subdomains carries the
// constraint that the average jump across that face vanishes, Q^T B u = 0 (Q: one column per face,
// ones on the multipliers between its two subdomains; in the slot space of subdomain s the column
// restricted to its local face f = 2a + side is sigma_f = +1 on the high side, -1 on the low side,
// on the face's non-Dirichlet slots).  With Phi = [F_rc, F_rr Q] the coarse system is
//   [K_cc  -X^T] [u_c]   [f~_c    ]
//   [-X    -Y  ] [mu ] = [-Q^T d_r] + Phi^T lambda,   X = Q^T F_rc,  Y = Q^T F_rr Q,
// the dual operator F_rr + Phi K^{-1} Phi^T keeps the form of the corner-only one, and the
// multipliers of the local problems are lambda + Q mu.

// Per operator class: the coupling columns Phi = [Frc | G], G = F Q_s (G[j][f] = sigma_f * sum of
// F[j][j'] over the active slots j' of face f), and the class's coarse block [[Kcc, -X^T], [-X, -Y]]
// with X = Q_s^T Frc and Y = Q_s^T G, sums accumulated in FP64.  One block per class at a time.
template <class T>
__global__ void k_aug_local(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ F,
                            const cx<T>* __restrict__ Frc0, const cx<double>* __restrict__ Kcc, int ncls, cx<T>* Phi,
                            cx<double>* Kq) {
  extern __shared__ __align__(16) unsigned char smaug[];
  const int nD = g.nD, nc = g.nc, nq = g.nq, ne = nq - nc, b = P.ly.b;
  cx<T>* Gs = reinterpret_cast<cx<T>*>(smaug);         // [nD][ne]
  int* act = reinterpret_cast<int*>(Gs + (size_t)nD * ne);  // [nD] slot active (not Dirichlet)
  const int tid = threadIdx.x, nthr = blockDim.x;
  const long long ld = sym_ld(nD);
  for (int q = blockIdx.x; q < ncls; q += gridDim.x) {
    P.select(q, m.cls_code);
    for (int j = tid; j < nD; j += nthr) {
      const int node = m.slot_node[j];
      act[j] = P.removed_node(node / b, node % b) ? 0 : 1;
    }
    __syncthreads();
    const cx<T>* Fq = F + (size_t)q * ld;
    for (int e = tid; e < nD * ne; e += nthr) {
      const int j = e / ne, f = e - j * ne;
      double re = 0, im = 0;
      if (act[j])
        for (int j2 = 0; j2 < nD; ++j2)
          if (act[j2] && ((m.slot_faces[j2] >> f) & 1)) {
            const cx<T> v = Fq[sym_idx(j, j2, nD)];
            re += (double)v.re;
            im += (double)v.im;
          }
      const double sg = (f & 1) ? 1.0 : -1.0;
      const cx<T> gv = mkc<T>((T)(sg * re), (T)(sg * im));
      Gs[e] = gv;
      Phi[((size_t)q * nD + j) * nq + nc + f] = gv;
    }
    for (int e = tid; e < nD * nc; e += nthr) {
      const int j = e / nc, c = e - j * nc;
      Phi[((size_t)q * nD + j) * nq + c] = Frc0[((size_t)q * nD + j) * nc + c];
    }
    __syncthreads();
    for (int e = tid; e < nq * nq; e += nthr) {
      const int a = e / nq, c = e - a * nq;
      cx<double> v = mkc<double>(0, 0);
      if (a < nc && c < nc) {
        v = Kcc[((size_t)q * nc + a) * nc + c];
      } else {
        // -X[f][corner] = -sigma_f sum_{j in f} Frc[j][corner];  -Y[f][f2] = -sigma_f sum_{j in f} G[j][f2]
        const int f = a >= nc ? a - nc : c - nc, other = a >= nc ? c : a;
        double re = 0, im = 0;
        for (int j = 0; j < nD; ++j)
          if (act[j] && ((m.slot_faces[j] >> f) & 1)) {
            const cx<T> x = other < nc ? Frc0[((size_t)q * nD + j) * nc + other] : Gs[(size_t)j * ne + (other - nc)];
            re += (double)x.re;
            im += (double)x.im;
          }
        const double sg = (f & 1) ? -1.0 : 1.0;  // -sigma_f
        v = mkc<double>(sg * re, sg * im);
      }
      Kq[((size_t)q * nq + a) * nq + c] = v;
    }
    __syncthreads();
  }
}

// Right-hand-side split, face part: Tc[sd][r][nc + f] = sigma_f * sum of VD over the active slots of
// local face f (Q_s^T d_r^s; the coarse gather with sign -1 then gives -Q^T d_r).  One warp per
// (subdomain, right-hand side).
template <class T>
__global__ void k_face_sums(Geom g, MapsView m, const cx<T>* __restrict__ VD, int R, cx<T>* Tc) {
  const int lane = threadIdx.x & 31;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (wid >= (long long)g.nsd * R) return;
  const int sd = (int)(wid / R), r = (int)(wid - (long long)sd * R), ne = g.nq - g.nc;
  cx<T> acc[6];
#pragma unroll
  for (int f = 0; f < 6; ++f) acc[f] = czero<T>();
  const cx<T>* v = VD + ((size_t)sd * R + r) * g.nD;
  for (int j = lane; j < g.nD; j += 32) {
    if (m.sd_minv[(size_t)sd * g.nD + j] == 0.0) continue;  // Dirichlet slot
    const int bits = m.slot_faces[j];
    const cx<T> x = v[j];
#pragma unroll
    for (int f = 0; f < 6; ++f)
      if ((bits >> f) & 1) acc[f] = cadd(acc[f], x);
  }
#pragma unroll
  for (int f = 0; f < 6; ++f)
    for (int o = 16; o > 0; o >>= 1) acc[f] = cadd(acc[f], shfl_xor_cx(acc[f], o));
  if (lane == 0)
    for (int f = 0; f < ne; ++f)
      Tc[((size_t)sd * R + r) * g.nq + g.nc + f] = (f & 1) ? acc[f] : mkc<T>(-acc[f].re, -acc[f].im);
}

// d <- (I - Q (Q^T Q)^{-1} Q^T) d: subtracts from the multipliers of every face their mean.  In exact
// arithmetic the augmented dual right-hand side satisfies Q^T d = 0 (the augmented dual operator
// vanishes on the columns of Q, so the system is consistent only on that complement); in FP32 the
// cancellations in d_r - Phi w leave a component along Q that the Krylov iteration cannot remove
// (its residual would stall near it), so it is projected out.  One warp per (face, column).
template <class T>
__global__ void k_dual_project(Geom g, MapsView m, int R, cx<T>* d) {
  const int lane = threadIdx.x & 31;
  const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  if (wid >= (long long)g.nface * R) return;
  const int f = (int)(wid % g.nface), r = (int)(wid / g.nface);
  const int p0 = m.face_lam_ptr[f], p1 = m.face_lam_ptr[f + 1];
  if (p1 <= p0) return;
  cx<T>* dr = d + (size_t)r * g.nlam;
  double sre = 0, sim = 0;
  for (int k = p0 + lane; k < p1; k += 32) {
    const cx<T> v = dr[m.face_lam[k]];
    sre += (double)v.re;
    sim += (double)v.im;
  }
  for (int o = 16; o > 0; o >>= 1) {
    sre += __shfl_xor_sync(0xffffffffu, sre, o);
    sim += __shfl_xor_sync(0xffffffffu, sim, o);
  }
  const T mre = (T)(sre / (p1 - p0)), mim = (T)(sim / (p1 - p0));
  for (int k = p0 + lane; k < p1; k += 32) {
    cx<T>& v = dr[m.face_lam[k]];
    v = mkc<T>(v.re - mre, v.im - mim);
  }
}

// lambda += Q mu: each multiplier between face neighbours takes its face's coarse unknown
template <class T>
__global__ void k_lam_aug(Geom g, MapsView m, const cx<T>* __restrict__ w, int R, cx<T>* lam) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)R * g.nlam) return;
  const int r = (int)(e / g.nlam), li = (int)(e - (long long)r * g.nlam);
  const int f = m.lam_face[li];
  if (f >= 0) lam[e] = cadd(lam[e], w[(size_t)r * g.nco + g.ncor + f]);
}

// Dense augmented coarse matrix K (nco x nco, FP64, row-major): entry (I, J) is the sum of the class
// blocks Kq of the subdomains holding both unknowns, visited in a fixed order (deterministic).
static __global__ void k_aug_assemble(Geom g, MapsView m, const cx<double>* __restrict__ Kq, cx<double>* K) {
  const long long tot = (long long)g.nco * g.nco;
  const int dim = g.dim, nq = g.nq;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int I = (int)(e / g.nco), J = (int)(e - (long long)I * g.nco);
    int own[8], nown = 0;
    if (I < g.ncor) {
      int C[3];
      idx2crd(I, g.ncg, dim, C);
      for (int bits = 0; bits < (1 << dim); ++bits) {
        int S[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) S[a] = C[a] + 1 - ((bits >> a) & 1);
        own[nown++] = crd2idx(S, g.nsub, dim);
      }
    } else {
      own[nown++] = m.face_sd[2 * (I - g.ncor) + 1];
      own[nown++] = m.face_sd[2 * (I - g.ncor)];
    }
    cx<double> sum = mkc<double>(0, 0);
    for (int k = 0; k < nown; ++k) {
      const int sd = own[k];
      const int* sc = m.sd_coarse + (size_t)sd * nq;
      int a = -1, c = -1;
      for (int t = 0; t < nq; ++t) {
        if (sc[t] == I) a = t;
        if (sc[t] == J) c = t;
      }
      if (a >= 0 && c >= 0) sum = cadd(sum, Kq[((size_t)m.sd_cls[sd] * nq + a) * nq + c]);
    }
    K[e] = sum;
  }
}

// Copy of an FP64 n x n matrix (row stride n) into precision T with row stride ld.
template <class T>
__global__ void k_convert_rows(const cx<double>* __restrict__ A, int n, cx<T>* B, int ld) {
  const long long tot = (long long)n * ld;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / ld), j = (int)(e - (long long)i * ld);
    B[e] = j < n ? ccast<T>(A[(size_t)i * n + j]) : czero<T>();
  }
}

// z[gi][r] += value of node gi: the coarse unknown at corners, else the mean of its subdomain
// copies (equal at convergence).
template <class T>
__global__ void k_assemble_z(Geom g, const cx<T>* __restrict__ Xs, const cx<T>* __restrict__ uc, int R,
                             cx<double>* z, int ldz) {
  long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)R * g.n) return;
  const int dim = g.dim;
  int r = (int)(e / g.n);
  long long gi = e % g.n;
  int G[3] = {0, 0, 0};
  long long t = gi;
  G[0] = (int)(t % (g.nel[0] - 1)) + 1;
  t /= (g.nel[0] - 1);
  if (dim == 2) {
    G[1] = (int)t + 1;
  } else {
    G[1] = (int)(t % (g.nel[1] - 1)) + 1;
    G[2] = (int)(t / (g.nel[1] - 1)) + 1;
  }
  int S0[3], L0[3], twin[3], nshared = 0;
  for (int a = 0; a < 3; ++a) {
    if (a < dim) {
      S0[a] = G[a] / g.s[a];
      L0[a] = G[a] - S0[a] * g.s[a];
      twin[a] = L0[a] == 0;
      nshared += twin[a];
    } else {
      S0[a] = 0;
      L0[a] = 0;
      twin[a] = 0;
    }
  }
  cx<double> val;
  if (nshared == dim) {
    int C[3] = {S0[0] - 1, S0[1] - 1, dim == 3 ? S0[2] - 1 : 0};
    val = uc ? ccast<double>(uc[(size_t)r * g.nco + crd2idx(C, g.ncg, dim)]) : mkc<double>(0, 0);
  } else {
    int ext[3] = {g.s[0] + 1, g.s[1] + 1, dim == 3 ? g.s[2] + 1 : 1};
    cx<double> sum = mkc<double>(0, 0);
    int cnt = 0;
    for (int mask = 0; mask < (1 << dim); ++mask) {
      bool ok = true;
      int S[3], l[3];
      for (int a = 0; a < 3; ++a) {
        int bit = a < dim ? (mask >> a) & 1 : 0;
        if (bit && !twin[a]) ok = false;
        S[a] = S0[a] - bit;
        l[a] = bit ? g.s[a] : L0[a];
      }
      if (!ok) continue;
      int sd = crd2idx(S, g.nsub, dim);
      sum = cadd(sum, ccast<double>(Xs[((size_t)sd * g.nl + crd2idx(l, ext, dim)) * R + r]));
      ++cnt;
    }
    val = cscale(sum, 1.0 / cnt);
  }
  cx<double>& zz = z[(size_t)r * ldz + gi];
  zz = cadd(zz, val);
}

}  // namespace schur
