// Warp-per-subdomain variants of the layered factorisation and solves for layer sizes b <= 32
// (every 2D subdomain with up to 31 elements per side).  Lane i owns row i of the current layer;
// couplings between rows travel by warp shuffles, so a 17 x 17 layer block needs no block-wide
// barrier and one warp processes one subdomain.  Same arithmetic as layered.cuh.
#pragma once
#include "kernels.cuh"

namespace schur {


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

// Local operators F, Frc, Kcc of each class on 2D remainder problems (layer size b <= B), one CTA
// per class and one thread per right-hand-side column c of [E_Delta, A_rc]: the thread keeps its
// column of the current layer in registers (rows unrolled at compile time), the layer block
// D_K^{-1} and the neighbour couplings are staged in shared memory and read as broadcasts, so each
// row update of E_K = D_K^{-1} (b_K - A_{K,K-1} E_{K-1}) is B complex FMAs per loaded entry pair.
// Forward results E_K go to a per-CTA global buffer (layer, row, column; column fastest) and are
// read back by the same thread in the backward sweep X_K = E_K - D_K^{-1} A_{K,K+1} X_{K+1}.
// Outputs: rows of X on the interface slots (F, Frc) and, for the corner columns, the corner
// Schur complement Kcc = A_cc - A_cr X_rc accumulated while the sweep passes the corner layers.
// Only the columns below col1 are formed; with Kcc null the corner Schur complements are not
// written (they come from k_corner_kcc).
template <int B>
struct ColsLayout {
  static constexpr int SB = (B + 1) & ~1;  // row stride of the staged blocks: 16-byte aligned rows
};

template <class T, int B>
__host__ __device__ constexpr size_t form_cols_smem(int b, int L) {
  return (2 * (size_t)B * ColsLayout<B>::SB + 3 * (size_t)B + 12 * (size_t)B) * sizeof(cx<T>) +
         ((size_t)L * b + 12) * sizeof(int);
}

template <class T, int SB>
__device__ __forceinline__ void load_pair(const cx<T>* p, cx<T>& a, cx<T>& b2) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = mkc<T>(v.x, v.y);
    b2 = mkc<T>(v.z, v.w);
  } else {
    a = p[0];
    b2 = p[1];
  }
}

template <class T, int B>
__global__ void __launch_bounds__(128) k_form_rr_cols(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv,
                                                      int ncls, cx<T>* F, cx<T>* Frc, cx<double>* Kcc, cx<T>* Ews,
                                                      int ldE, int col1) {
  constexpr int SB = ColsLayout<B>::SB, NT = 3;
  const int b = P.ly.b, L = P.ly.L, nD = g.nD, nc = g.nc, ncol = nD + nc, bb = b * b;
  const int c = threadIdx.x, nthr = blockDim.x;
  extern __shared__ __align__(16) unsigned char smcols[];
  cx<T>* Db = reinterpret_cast<cx<T>*>(smcols);  // 2 x B x SB
  cx<T>* cf = Db + 2 * B * SB;                  // B x 3 couplings of the current layer
  cx<T>* ct = cf + 3 * B;                       // 4 corners x 3 layers x B: A(node, corner)
  int* slot_s = reinterpret_cast<int*>(ct + 12 * B);  // L x b: interface slot of node or -1
  int* cK = slot_s + L * b;                           // corner layer, row, Dirichlet flag
  int* cI = cK + 4;
  int* cDir = cI + 4;
  for (int e = c; e < 2 * B * SB; e += nthr) Db[e] = czero<T>();
  for (int e = c; e < L * b; e += nthr) slot_s[e] = m.node_slot[e];
  cx<T>* E = Ews + (size_t)blockIdx.x * L * B * ldE;
  const bool is_unit = c < nD && c < col1, is_corner = c >= nD && c < ncol && c < col1;
  const int cc = c - nD;
  for (int q = blockIdx.x; q < ncls; q += gridDim.x) {
    P.select(q, m.cls_code);
    if (c < nc) {
      const int node = m.corner_node[c];
      cK[c] = node / b;
      cI[c] = node % b;
      int lc[3];
      P.crd(node / b, node % b, lc);
      cDir[c] = local_dirichlet(P.code, lc, g.s, 2) ? 1 : 0;
    }
    __syncthreads();
    for (int e = c; e < 12 * B; e += nthr) {
      const int c1 = e / (3 * B), d = (e / B) % 3, i = e % B;
      const int K = cK[c1] - 1 + d;
      cx<T> v = czero<T>();
      if (c1 < nc && !cDir[c1] && i < b && K >= 0 && K < L && abs(i - cI[c1]) <= 1 && !P.removed_node(K, i)) {
        int l[3], lc[3];
        P.crd(K, i, l);
        P.crd(cK[c1], cI[c1], lc);
        v = q1_entry(P.st, g.s, l, lc);
      }
      ct[e] = v;
    }
    int Ku = -1, iu = -1;
    if (is_unit) {
      const int node = m.slot_node[c];
      if (!P.removed_node(node / b, node % b)) {
        Ku = node / b;
        iu = node % b;
      }
    }
    // first layer where this column's right-hand side is nonzero: the forward results E_K of the
    // layers before it are zero, so they are neither stored nor read back (L: the column is zero)
    int K0 = L;
    if (Ku >= 0) K0 = Ku;
    if (is_corner && !cDir[cc]) K0 = max(0, cK[cc] - 1);
    auto stage = [&](int K, int buf) {
      const cx<T>* src = Dinv + ((size_t)q * L + K) * bb;
      cx<T>* dst = Db + buf * B * SB;
      for (int e = c; e < bb; e += nthr) {
        const int mm = e / b, i = e - mm * b;
        cp_async_cx(dst + mm * SB + i, src + e);
      }
    };
    cx<T> prev[B], kacc[4];
#pragma unroll
    for (int i = 0; i < B; ++i) prev[i] = czero<T>();
#pragma unroll
    for (int k = 0; k < 4; ++k) kacc[k] = czero<T>();
    auto emit = [&](int K, const cx<T>(&x)[B]) {
      if (is_unit || is_corner) {
#pragma unroll
        for (int i = 0; i < B; ++i) {
          if (i < b) {
            const int j = slot_s[K * b + i];
            if (j >= 0) {
              if (is_unit) {
                if (j <= c) F[(size_t)q * sym_ld(nD) + sym_idx(j, c, nD)] = x[i];
              }
              else Frc[((size_t)q * nD + j) * nc + cc] = x[i];
            }
          }
        }
      }
      if (is_corner) {
#pragma unroll
        for (int c1 = 0; c1 < 4; ++c1) {
          const int d = K - cK[c1] + 1;
          if (c1 < nc && d >= 0 && d < 3) {
            const cx<T>* a = ct + (c1 * 3 + d) * B;
#pragma unroll
            for (int i = 0; i < B; ++i) cfms(kacc[c1], a[i], x[i]);
          }
        }
      }
    };
    __syncthreads();  // corner tables and cleared blocks visible; previous class fully consumed
    // ---- forward sweep
    stage(0, 0);
    cp_async_commit();
    for (int K = 0; K < L; ++K) {
      if (K + 1 < L) stage(K + 1, (K + 1) & 1);
      cp_async_commit();
      if (K > 0)
        for (int e = c; e < b * NT; e += nthr) cf[e] = P.Al(K - 1, e / NT, e % NT);
      cx<T> t[B];
#pragma unroll
      for (int i = 0; i < B; ++i) t[i] = czero<T>();
      if (K == Ku) {
#pragma unroll
        for (int i = 0; i < B; ++i)
          if (i == iu) t[i] = mkc<T>(T(1), T(0));
      }
      if (is_corner) {
        const int d = K - cK[cc] + 1;
        if (d >= 0 && d < 3) {
#pragma unroll
          for (int i = 0; i < B; ++i) t[i] = ct[(cc * 3 + d) * B + i];
        }
      }
      cp_async_wait<1>();
      __syncthreads();
      if (K > 0) {
#pragma unroll
        for (int i = 0; i < B; ++i) {
          if (i < b) {
            if (i > 0) cfms(t[i], cf[i * NT], prev[i - 1]);
            cfms(t[i], cf[i * NT + 1], prev[i]);
            if (i + 1 < B) cfms(t[i], cf[i * NT + 2], prev[i + 1]);
          }
        }
      }
      const cx<T>* Dk = Db + (K & 1) * B * SB;
#pragma unroll
      for (int i = 0; i < B; ++i) prev[i] = czero<T>();
#pragma unroll
      for (int mm = 0; mm < B; ++mm) {
        const cx<T> tm = t[mm];
#pragma unroll
        for (int i = 0; i + 1 < B; i += 2) {
          cx<T> d0, d1;
          load_pair<T, SB>(Dk + mm * SB + i, d0, d1);
          cfma(prev[i], d0, tm);
          cfma(prev[i + 1], d1, tm);
        }
        if (B & 1) cfma(prev[B - 1], Dk[mm * SB + B - 1], tm);
      }
      if (c < ldE && K >= K0) {
#pragma unroll
        for (int i = 0; i < B; ++i)
          if (i < b) E[((size_t)K * B + i) * ldE + c] = prev[i];
      }
      __syncthreads();
    }
    emit(L - 1, prev);
    // ---- backward sweep: prev = X_{K+1}
    if (L >= 2) stage(L - 2, 0);
    cp_async_commit();
    for (int K = L - 2, it = 0; K >= 0; --K, ++it) {
      if (K >= 1) stage(K - 1, (it + 1) & 1);
      cp_async_commit();
      for (int e = c; e < b * NT; e += nthr) {
        const int i = e / NT, tt = e - i * NT, k = i + tt - 1;
        cf[e] = (k >= 0 && k < b) ? P.Al(K, k, NT - 1 - tt) : czero<T>();
      }
      cx<T> x[B];
#pragma unroll
      for (int i = 0; i < B; ++i) x[i] = (c < ldE && i < b && K >= K0) ? E[((size_t)K * B + i) * ldE + c] : czero<T>();
      cp_async_wait<1>();
      __syncthreads();
      cx<T> u[B];
#pragma unroll
      for (int i = 0; i < B; ++i) {
        u[i] = czero<T>();
        if (i < b) {
          if (i > 0) cfma(u[i], cf[i * NT], prev[i - 1]);
          cfma(u[i], cf[i * NT + 1], prev[i]);
          if (i + 1 < B) cfma(u[i], cf[i * NT + 2], prev[i + 1]);
        }
      }
      const cx<T>* Dk = Db + (it & 1) * B * SB;
#pragma unroll
      for (int mm = 0; mm < B; ++mm) {
        const cx<T> um = u[mm];
#pragma unroll
        for (int i = 0; i + 1 < B; i += 2) {
          cx<T> d0, d1;
          load_pair<T, SB>(Dk + mm * SB + i, d0, d1);
          cfms(x[i], d0, um);
          cfms(x[i + 1], d1, um);
        }
        if (B & 1) cfms(x[B - 1], Dk[mm * SB + B - 1], um);
      }
      emit(K, x);
#pragma unroll
      for (int i = 0; i < B; ++i) prev[i] = x[i];
      __syncthreads();
    }
    cp_async_wait<0>();
    if (is_corner) {
      int lc2[3];
      P.crd(cK[cc], cI[cc], lc2);
#pragma unroll
      for (int c1 = 0; c1 < 4; ++c1) {
        if (c1 < nc) {
          cx<T> v = kacc[c1];
          if (c1 == cc) v = cadd(v, q1_entry(P.st, g.s, lc2, lc2));
          if (cDir[c1] || cDir[cc]) v = czero<T>();
          if (Kcc) Kcc[((size_t)q * nc + c1) * nc + cc] = ccast<double>(v);
        }
      }
    }
    __syncthreads();
  }
}

// Corner Schur complements K_cc = A_cc - A_cr A_rr^{-1} A_rc of every class (2D, layer size b <= B)
// from the forward layer sweep alone: with the block LDL^T factor A_rr = L D L^T by layers (pivot
// blocks D_K, L_{K,K-1} = A_{K,K-1} D_{K-1}^{-1}) and W = L^{-1} A_rc,
//   A_cr A_rr^{-1} A_rc = W^T D^{-1} W = sum_K W_K^T E_K,  E_K = D_K^{-1} W_K,
//   W_K = (A_rc)_K - A_{K,K-1} E_{K-1}
// (plain transposes: the matrices are complex symmetric).  One warp per class, lane i = row i of
// the layer, the four corner columns in registers; D_K^{-1} read by rows (coalesced), the layer
// couplings through shuffles.  It lets the coarse factorisation start before the local operators
// are formed.
template <class T, int B>
__global__ void __launch_bounds__(128) k_corner_kcc(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv,
                                                    int ncls, cx<double>* Kcc) {
  constexpr int NC = 4;  // corners of a 2D subdomain
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int b = P.ly.b, L = P.ly.L, bb = b * b;
  const bool act = lane < b;
  for (int q = blockIdx.x * wpb + wib; q < ncls; q += gridDim.x * wpb) {
    P.select(q, m.cls_code);
    int cK[NC], cI[NC], lc[NC][3];
    bool cDir[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int node = m.corner_node[c];
      cK[c] = node / b;
      cI[c] = node % b;
      P.crd(cK[c], cI[c], lc[c]);
      cDir[c] = local_dirichlet(P.code, lc[c], g.s, 2);
    }
    cx<T> ep[NC], kacc[NC][NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      ep[c] = czero<T>();
#pragma unroll
      for (int c2 = 0; c2 < NC; ++c2) kacc[c][c2] = czero<T>();
    }
    for (int K = 0; K < L; ++K) {
      const cx<T>* Dk = Dinv + ((size_t)q * L + K) * bb;
      cx<T> d[B];
#pragma unroll
      for (int mm = 0; mm < B; ++mm) d[mm] = (act && mm < b) ? Dk[mm * b + lane] : czero<T>();
      cx<T> w[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        w[c] = czero<T>();
        if (act && !cDir[c] && abs(K - cK[c]) <= 1 && abs(lane - cI[c]) <= 1 && !P.removed_node(K, lane)) {
          int l[3];
          P.crd(K, lane, l);
          w[c] = q1_entry(P.st, g.s, l, lc[c]);
        }
      }
      if (K > 0) {
        const cx<T> a0 = act ? P.Al(K - 1, lane, 0) : czero<T>();
        const cx<T> a1 = act ? P.Al(K - 1, lane, 1) : czero<T>();
        const cx<T> a2 = act ? P.Al(K - 1, lane, 2) : czero<T>();
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          const cx<T> em = shfl_cx(ep[c], lane > 0 ? lane - 1 : 0);
          const cx<T> en = shfl_cx(ep[c], lane < 31 ? lane + 1 : 31);
          cfms(w[c], a0, em);
          cfms(w[c], a1, ep[c]);
          cfms(w[c], a2, en);
        }
      }
      cx<T> e[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) e[c] = czero<T>();
#pragma unroll
      for (int mm = 0; mm < B; ++mm)
        if (mm < b) {
#pragma unroll
          for (int c = 0; c < NC; ++c) cfma(e[c], d[mm], shfl_cx(w[c], mm));
        }
#pragma unroll
      for (int c1 = 0; c1 < NC; ++c1)
#pragma unroll
        for (int c2 = 0; c2 < NC; ++c2) cfma(kacc[c1][c2], w[c1], e[c2]);
#pragma unroll
      for (int c = 0; c < NC; ++c) ep[c] = e[c];
    }
#pragma unroll
    for (int c1 = 0; c1 < NC; ++c1)
#pragma unroll
      for (int c2 = 0; c2 < NC; ++c2) {
        cx<T> v = kacc[c1][c2];
        for (int o = 16; o > 0; o >>= 1) v = cadd(v, shfl_xor_cx(v, o));
        if (lane == 0) {
          cx<T> r = mkc<T>(-v.re, -v.im);
          if (c1 == c2) r = cadd(r, q1_entry(P.st, g.s, lc[c1], lc[c1]));
          if (cDir[c1] || cDir[c2]) r = czero<T>();
          Kcc[((size_t)q * NC + c1) * NC + c2] = ccast<double>(r);
        }
      }
  }
}

// Block LDL^T of 2D remainder problems (layer size b <= B), one warp per problem: lane j holds
// column j of the current pivot block in registers (rows unrolled at compile time).  Gauss-Jordan
// pivots broadcast the pivot column by shuffles; the product with the tridiagonal layer coupling
// takes the neighbouring columns by uniform shuffles up / down; the transpose for the symmetric
// average goes through a padded per-warp shared tile.  Same steps as k_factor_warp.
template <int B>
struct FacLayout {
  static constexpr int TS = B | 1;  // odd row stride: conflict-free column reads of 8-byte entries
};

template <class T, int B>
__host__ __device__ constexpr size_t factor_cols_smem_per_warp() {
  return ((size_t)B * FacLayout<B>::TS + 3 * (size_t)B) * sizeof(cx<T>);
}

template <class T>
__device__ __forceinline__ cx<T> shfl_up_cx(cx<T> v, int d) {
  return mkc<T>(__shfl_up_sync(0xffffffffu, v.re, d), __shfl_up_sync(0xffffffffu, v.im, d));
}
template <class T>
__device__ __forceinline__ cx<T> shfl_down_cx(cx<T> v, int d) {
  return mkc<T>(__shfl_down_sync(0xffffffffu, v.re, d), __shfl_down_sync(0xffffffffu, v.im, d));
}

template <class T, int B>
__global__ void __launch_bounds__(128) k_factor_cols(StencilProv<T> P, const int* codes, int nprob, cx<T>* Dinv,
                                                     int* err) {
  constexpr int TS = FacLayout<B>::TS, NT = 3;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int q = blockIdx.x * wpb + wib;
  if (q >= nprob) return;
  P.select(q, codes);
  const int b = P.ly.b, L = P.ly.L, bb = b * b;
  extern __shared__ __align__(16) unsigned char smfac[];
  cx<T>* Tr = reinterpret_cast<cx<T>*>(smfac) + (size_t)wib * (B * TS + 3 * B);  // B x TS tile
  cx<T>* cf = Tr + B * TS;                                                        // B x 3 couplings
  const bool act = lane < b;
  cx<T>* out = Dinv + (size_t)q * L * bb;
  cx<T> d[B];
  // pivot block of layer K from the stencil: column j has rows j-1, j, j+1
  auto diag_block = [&](int K) {
#pragma unroll
    for (int i = 0; i < B; ++i) {
      const int dl = i - lane;
      d[i] = (act && i < b && dl >= -1 && dl <= 1) ? P.Ad(K, i, 1 - dl) : czero<T>();
    }
  };
  diag_block(0);
  for (int K = 0; K < L; ++K) {
    // ---- explicit inverse of the pivot block (Gauss-Jordan, no pivoting).  After each pivot the
    // rows rotate by one register, so the pivot row is always d[0] and the pivot loop stays rolled
    // (small code); B rotations in total restore the row order.
    for (int k = 0; k < b; ++k) {
      const cx<T> p = shfl_cx(d[0], k);
      const cx<T> piv = cinv(p);
      if (lane == 0 && !finite_nonzero(p)) atomicExch(err, 1);
      const cx<T> rk = cmul(d[0], piv);
      d[0] = (lane == k) ? piv : rk;
#pragma unroll
      for (int i = 1; i < B; ++i) {
        const cx<T> ci = shfl_cx(d[i], k);
        if (lane == k) {
          const cx<T> v = cmul(ci, piv);
          d[i] = mkc<T>(-v.re, -v.im);
        } else {
          cfms(d[i], ci, rk);
        }
      }
      const cx<T> t0 = d[0];
#pragma unroll
      for (int i = 0; i + 1 < B; ++i) d[i] = d[i + 1];
      d[B - 1] = t0;
    }
    for (int k = b; k < B; ++k) {
      const cx<T> t0 = d[0];
#pragma unroll
      for (int i = 0; i + 1 < B; ++i) d[i] = d[i + 1];
      d[B - 1] = t0;
    }
    // ---- symmetric average (D + D^T) / 2 through the shared tile; store D_K^{-1}
    if (lane < B) {
#pragma unroll
      for (int i = 0; i < B; ++i) Tr[i * TS + lane] = d[i];
    }
    __syncwarp();
    if (act) {
#pragma unroll
      for (int i = 0; i < B; ++i) {
        const cx<T> t = Tr[lane * TS + i];
        d[i] = cscale(cadd(d[i], t), T(0.5));
      }
    }
    if (act) {
#pragma unroll
      for (int i = 0; i < B; ++i)
        if (i < b) out[(size_t)K * bb + (size_t)i * b + lane] = d[i];
    }
    __syncwarp();
    if (K + 1 == L) break;
    // ---- W = D_K^{-1} A_{K,K+1}: column j = sum_t Al(K, j, t) * (column j + t - 1 of D_K^{-1})
    const cx<T> a0 = act ? P.Al(K, lane, 0) : czero<T>();
    const cx<T> a1 = act ? P.Al(K, lane, 1) : czero<T>();
    const cx<T> a2 = act ? P.Al(K, lane, 2) : czero<T>();
    for (int e = lane; e < b * NT; e += 32) cf[e] = P.Al(K, e / NT, e % NT);
    cx<T> w[B];
#pragma unroll
    for (int m = 0; m < B; ++m) {
      const cx<T> left = shfl_up_cx(d[m], 1), right = shfl_down_cx(d[m], 1);
      cx<T> v = cmul(a1, d[m]);
      if (lane > 0) cfma(v, a0, left);
      if (lane + 1 < 32) cfma(v, a2, right);
      w[m] = v;
    }
    __syncwarp();
    // ---- D_{K+1} = A_{K+1,K+1} - A_{K+1,K} W: row i couples to rows i-1, i, i+1 of W
    diag_block(K + 1);
#pragma unroll
    for (int i = 0; i < B; ++i) {
      if (i < b) {
        if (i > 0) cfms(d[i], cf[i * NT], w[i - 1]);
        cfms(d[i], cf[i * NT + 1], w[i]);
        if (i + 1 < B) cfms(d[i], cf[i * NT + 2], w[i + 1]);
      }
    }
    __syncwarp();
  }
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
      cfms(v, q1_entry(P.st, g.s, l, lc), uc[(size_t)c * g.nco + ci]);
    }
  }
  return v;
}

// Remainder right-hand sides of every subdomain node and column, one thread each, into the
// per-subdomain solution buffers (layout [sd][node][R]) ahead of the layered solves.
template <class T>
__global__ void k_remainder_rhs(StencilProv<T> P, Geom g, MapsView m, const cx<double>* __restrict__ f, int ldf,
                                const cx<T>* __restrict__ lam, const cx<T>* __restrict__ uc, int R, cx<T>* Xs) {
  const int nl = P.ly.L * P.ly.b;
  const long long tot = (long long)g.nsd * nl * R;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
    const int sd = (int)(e / ((long long)nl * R));
    const int rem = (int)(e - (long long)sd * nl * R);
    const int node = rem / R, c = rem - node * R, K = node / P.ly.b, i = node - K * P.ly.b;
    StencilProv<T> Pq = P;
    Pq.select(m.sd_cls[sd], m.cls_code);
    int S[3];
    idx2crd(sd, g.nsub, g.dim, S);
    Xs[(size_t)sd * g.nl * R + rem] = remainder_rhs(Pq, g, m, sd, S, f, ldf, lam, uc, K, i, c);
  }
}

// Per-solve local solves, one warp per subdomain.  VD/Tc extraction when VD != null (right-hand
// side split); otherwise the solution stays in Xs (primal recovery).
template <class T, int C>
__global__ void k_local_solve_warp(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv,
                                   const cx<double>* __restrict__ f, int ldf, const cx<T>* __restrict__ lam,
                                   const cx<T>* __restrict__ uc, int R, cx<T>* Xs, cx<T>* VD, cx<T>* Tc, int rhs_pre) {
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
  if (rhs_pre) {  // right-hand sides already in X (k_remainder_rhs); read back layer by layer
    auto rhs = [&](int K, int i, int c) -> cx<T> { return X[(size_t)(K * b + i) * R + c]; };
    warp_layered_solve<T, C>(P, Dinv + (size_t)q * L * b * b, R, rhs, X, R, 1, Ds);
  } else {
    auto rhs = [&](int K, int i, int c) -> cx<T> { return remainder_rhs(P, g, m, sd, S, f, ldf, lam, uc, K, i, c); };
    warp_layered_solve<T, C>(P, Dinv + (size_t)q * L * b * b, R, rhs, X, R, 1, Ds);
  }
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
    Tc[((size_t)sd * R + c) * g.nq + cc] = v;
  }
}

// F, Frc, Kcc of each class, one warp per (class, chunk of C columns); solution in shared memory.
template <class T, int C>
__global__ void k_form_rr_warp(StencilProv<T> P, Geom g, MapsView m, const cx<T>* __restrict__ Dinv, int ncls,
                               cx<T>* F, cx<T>* Frc, cx<double>* Kcc, cx<T>* Xws, int chunk0, int nrun) {
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int nD = g.nD, nc = g.nc, ncol = nD + nc, nchunk = (ncol + C - 1) / C;
  const int b = P.ly.b, L = P.ly.L, dim = g.dim;
  // per-warp solution buffer in global memory (column-major: node fastest), persistent warps;
  // per-warp staging buffer of the layer blocks in shared memory
  cx<T>* X = Xws + (size_t)(blockIdx.x * wpb + wib) * g.nl * C;
  extern __shared__ unsigned char smraw[];
  cx<T>* Ds = reinterpret_cast<cx<T>*>(smraw) + (size_t)wib * 2 * P.ly.b * P.ly.b;
  // chunks [chunk0, chunk0 + nrun) of C columns of every class (all: 0, nchunk)
  (void)nchunk;
  for (int w = blockIdx.x * wpb + wib; w < ncls * nrun; w += gridDim.x * wpb) {
  const int q = w / nrun, col0 = (chunk0 + w % nrun) * C;
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
    if (col < nD) {
      if (j <= col) F[(size_t)q * sym_ld(nD) + sym_idx(j, col, nD)] = v;
    }
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
