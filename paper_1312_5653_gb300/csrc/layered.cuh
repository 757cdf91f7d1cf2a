// Block LDL^T of complex-symmetric matrices on box grids, layered along the last axis.
//
// A box problem with ext[a] nodes per axis, numbered lexicographically (axis 0 fastest), has a
// block-tridiagonal matrix when grouped by layers of the last axis: b = prod_{a<dim-1} ext[a]
// nodes per layer, L = ext[dim-1] layers, and every node couples only to in-layer offsets in
// {-1,0,1}^(dim-1) of its own and the two adjacent layers (Q1 stencil).  The block LDL^T
//   D_0 = A_00,  D_{K+1} = A_{K+1,K+1} - A_{K+1,K} D_K^{-1} A_{K,K+1}
// is computed with explicit, symmetrised D_K^{-1} (Gauss-Jordan without pivoting).  For the
// subdomain matrices A_rr = K_rr + i gamma M_rr the real and imaginary parts are positive
// definite, a class closed under Schur complements, so every D_K has positive definite real and
// imaginary parts and no pivot vanishes.  The solve needs only D_K^{-1} and the sparse A blocks:
//   forward   E_K = D_K^{-1} (b_K - A_{K,K-1} E_{K-1})
//   backward  X_K = E_K - D_K^{-1} A_{K,K+1} X_{K+1}
// (the unit lower factor is A_{K+1,K} D_K^{-1}; its products are re-associated above).
#pragma once
#include "common.cuh"

namespace schur {

struct Layer {
  int dim;
  int ext[3];
  int b, L;
};

__host__ __device__ __forceinline__ int nbr_count(int dim) { return dim == 2 ? 3 : 9; }

// In-layer neighbour t of in-layer node i (offset digit a = (t / 3^a) % 3 - 1), or -1.
__device__ __forceinline__ int nbr_of(const Layer& ly, int i, int t) {
  int c0 = i % ly.ext[0];
  int n0 = c0 + (t % 3) - 1;
  if (n0 < 0 || n0 >= ly.ext[0]) return -1;
  if (ly.dim == 2) return n0;
  int c1 = i / ly.ext[0];
  int n1 = c1 + (t / 3) - 1;
  if (n1 < 0 || n1 >= ly.ext[1]) return -1;
  return n0 + ly.ext[0] * n1;
}
// Slot t with nbr_of(i, t) == j, or -1 if j is not an in-layer neighbour of i.
__device__ __forceinline__ int nbr_slot(const Layer& ly, int i, int j) {
  int d0 = j % ly.ext[0] - i % ly.ext[0];
  if (d0 < -1 || d0 > 1) return -1;
  if (ly.dim == 2) return d0 + 1;
  int d1 = j / ly.ext[0] - i / ly.ext[0];
  if (d1 < -1 || d1 > 1) return -1;
  return (d0 + 1) + 3 * (d1 + 1);
}

// Entries of a subdomain problem.  Node (K, i) has subdomain-local coordinates off + (in-layer
// coords, K).  The unmasked Neumann entries are read from tables built once per problem from the
// closed-form Q1 stencil (tad: in-layer couplings, tal: couplings to the previous layer, both
// [(K*b + i)*nt + t]); flags[K*b + i] marks subdomain vertices (bit 7) and the faces a node lies on
// (bit 2a: low face of axis a, bit 2a+1: high face).  masked: remainder problem, whose vertices
// and Dirichlet nodes (face bit set in the subdomain's boundary code) become identity rows.
template <class T>
struct StencilProv {
  Layer ly;
  Stencil<T> st;
  int s[3];
  int off;
  int masked;
  int code;
  const cx<T>* tad;
  const cx<T>* tal;
  const unsigned char* flags;
  __device__ __forceinline__ void select(int q, const int* codes) { code = masked ? codes[q] : 0; }
  __device__ __forceinline__ void crd(int K, int i, int* l) const {
    l[0] = i % ly.ext[0] + off;
    if (ly.dim == 3) {
      l[1] = i / ly.ext[0] + off;
      l[2] = K + off;
    } else {
      l[1] = K + off;
      l[2] = 0;
    }
  }
  __device__ __forceinline__ bool removed_node(int K, int i) const {
    if (!masked) return false;
    unsigned f = flags[K * ly.b + i];
    return (f & 0x80u) || (f & (unsigned)code);
  }
  __device__ __forceinline__ bool removed_l(const int* l) const {
    return masked && (local_vertex(l, s, ly.dim) || local_dirichlet(code, l, s, ly.dim));
  }
  __device__ __forceinline__ cx<T> Ad(int K, int i, int t) const {
    int j = nbr_of(ly, i, t);
    if (j < 0) return mkc<T>(0, 0);
    if (removed_node(K, i) || removed_node(K, j)) return mkc<T>(i == j ? T(1) : T(0), T(0));
    return tad[((size_t)K * ly.b + i) * nbr_count(ly.dim) + t];
  }
  // A(K+1, i ; K, nbr(i, t))
  __device__ __forceinline__ cx<T> Al(int K, int i, int t) const {
    int j = nbr_of(ly, i, t);
    if (j < 0 || removed_node(K + 1, i) || removed_node(K, j)) return mkc<T>(0, 0);
    return tal[((size_t)K * ly.b + i) * nbr_count(ly.dim) + t];
  }
};

// Builds tad, tal and flags of a box problem from the closed-form Q1 stencil (no masking).
template <class T>
__global__ void k_stencil_tables(StencilProv<T> P, cx<T>* tad, cx<T>* tal, unsigned char* flags) {
  const int b = P.ly.b, L = P.ly.L, nt = nbr_count(P.ly.dim), dim = P.ly.dim;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < L * b * nt; e += gridDim.x * blockDim.x) {
    int t = e % nt, i = (e / nt) % b, K = e / (nt * b);
    int j = nbr_of(P.ly, i, t);
    int p[3], q[3];
    P.crd(K, i, p);
    cx<T> ad = mkc<T>(0, 0), al = mkc<T>(0, 0);
    if (j >= 0) {
      P.crd(K, j, q);
      ad = q1_entry(P.st, P.s, p, q);
      if (K + 1 < L) {
        int p1[3];
        P.crd(K + 1, i, p1);
        al = q1_entry(P.st, P.s, p1, q);
      }
    }
    tad[e] = ad;
    tal[e] = al;
    if (t == 0) {
      unsigned f = local_vertex(p, P.s, dim) ? 0x80u : 0u;
      for (int a = 0; a < dim; ++a) {
        if (p[a] == 0) f |= 1u << (2 * a);
        if (p[a] == P.s[a]) f |= 1u << (2 * a + 1);
      }
      flags[K * b + i] = (unsigned char)f;
    }
  }
}

// Entries stored per (layer, node, neighbour slot): CA = diagonal blocks, CB = A_{K+1,K}.
template <class T>
struct StoredProv {
  Layer ly;
  const cx<T>* CA;
  const cx<T>* CB;
  __device__ __forceinline__ void select(int, const int*) {}
  __device__ __forceinline__ cx<T> Ad(int K, int i, int t) const {
    return CA[((size_t)K * ly.b + i) * nbr_count(ly.dim) + t];
  }
  __device__ __forceinline__ cx<T> Al(int K, int i, int t) const {
    return CB[((size_t)K * ly.b + i) * nbr_count(ly.dim) + t];
  }
};

template <class T>
__device__ __forceinline__ bool finite_nonzero(cx<T> p) {
  return isfinite(p.re) && isfinite(p.im) && (p.re != T(0) || p.im != T(0));
}

// In-place Gauss-Jordan inversion without pivoting of the b x b matrix A (whole block).
// rc: 2b scratch entries.  Sets *err on a zero or non-finite pivot.  With at least b threads,
// thread (j, g) = (tid mod b, tid div b) updates column j of the rows g, g + Gn, ... (Gn =
// floor(threads / b)), so no index is divided inside the pivot loop.
template <class T>
__device__ void gj_invert(cx<T>* A, int b, cx<T>* rc, int* err) {
  const int nthr = blockDim.x, tid = threadIdx.x, bb = b * b;
  const int Gn = nthr / b, j = tid % b, g = tid / b;
  for (int k = 0; k < b; ++k) {
    cx<T> p = A[k * b + k];
    cx<T> piv = cinv(p);
    if (tid == 0 && !finite_nonzero(p)) atomicExch(err, 1);
    for (int jj = tid; jj < b; jj += nthr) {
      rc[jj] = cmul(A[k * b + jj], piv);
      rc[b + jj] = A[jj * b + k];
    }
    __syncthreads();
    if (Gn >= 1) {
      if (g < Gn) {
        const cx<T> rj = rc[j];
        for (int i = g; i < b; i += Gn) {
          cx<T>& a = A[i * b + j];
          if (i == k) {
            a = (j == k) ? piv : rj;
          } else if (j == k) {
            cx<T> v = cmul(rc[b + i], piv);
            a = mkc<T>(-v.re, -v.im);
          } else {
            cfms(a, rc[b + i], rj);
          }
        }
      }
    } else {
      for (int e = tid; e < bb; e += nthr) {
        int i = e / b, jj = e - i * b;
        if (i == k) {
          A[e] = (jj == k) ? piv : rc[jj];
        } else if (jj == k) {
          cx<T> v = cmul(rc[b + i], piv);
          A[e] = mkc<T>(-v.re, -v.im);
        } else {
          cfms(A[e], rc[b + i], rc[jj]);
        }
      }
    }
    __syncthreads();
  }
}

// Block LDL^T of one layered problem per block (blockIdx.x = problem).  Writes the L explicit
// inverses D_K^{-1} (b x b, symmetric) to Dinv + q*L*b*b.  Workspace: 2 b^2 + 2 b entries in
// shared memory when use_smem (+ b * nbr_count entries for the couplings of the current layer
// when use_tab), else the (2 b^2 per block) global buffer gws (+2b in shared).
// Optionally (non-null G, H, same layout as Dinv) also the dense layer couplings of the solve,
//   G_K = D_K^{-1} A_{K,K+1}  (K < L-1),   H_K = D_K^{-1} A_{K,K-1}  (K > 0),
// with which forward and backward sweeps become one dense product per layer:
//   V_K = D_K^{-1} b_K - H_K V_{K-1},   X_K = V_K - G_K X_{K+1}.
// Matrix loops use the thread -> (column, row group) map of gj_invert when there are at least b
// threads.
template <class T, class Prov>
__global__ void k_factor(Prov P, const int* codes, cx<T>* Dinv, cx<T>* gws, int use_smem, int* err,
                         cx<T>* G = nullptr, cx<T>* H = nullptr, int use_tab = 0) {
  const int q = blockIdx.x;
  P.select(q, codes);
  const int b = P.ly.b, L = P.ly.L, bb = b * b, nt = nbr_count(P.ly.dim);
  const int tid = threadIdx.x, nthr = blockDim.x;
  extern __shared__ unsigned char smraw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smraw);
  cx<T>*Dt, *W, *rc;
  if (use_smem) {
    Dt = sm;
    W = sm + bb;
    rc = sm + 2 * bb;
  } else {
    Dt = gws + (size_t)q * 2 * bb;
    W = Dt + bb;
    rc = sm;
  }
  // couplings A(K+1, i ; K, nbr(i, t)) of the current layer K: a shared table or the provider
  cx<T>* tab = use_tab ? rc + 2 * b : nullptr;
  auto al = [&](int K, int i, int t) -> cx<T> { return tab ? tab[i * nt + t] : P.Al(K, i, t); };
  const int Gn = nthr / b, jc = tid % b, gc = tid / b;
  const bool map2d = Gn >= 1;
  // visits the entries (i, j) of a b x b matrix owned by this thread
  auto for_entries = [&](auto f) {
    if (map2d) {
      if (gc < Gn)
        for (int i = gc; i < b; i += Gn) f(i, jc);
    } else {
      for (int e = tid; e < bb; e += nthr) f(e / b, e % b);
    }
  };
  cx<T>* out = Dinv + (size_t)q * L * bb;
  for (int e = tid; e < bb; e += nthr) Dt[e] = mkc<T>(0, 0);
  __syncthreads();
  for (int e = tid; e < b * nt; e += nthr) {
    int i = e / nt, t = e - i * nt;
    int j = nbr_of(P.ly, i, t);
    if (j >= 0) Dt[i * b + j] = P.Ad(0, i, t);
  }
  __syncthreads();
  for (int K = 0; K < L; ++K) {
    gj_invert(Dt, b, rc, err);
    for_entries([&](int i, int j) { W[i * b + j] = cscale(cadd(Dt[i * b + j], Dt[j * b + i]), T(0.5)); });
    __syncthreads();
    for_entries([&](int i, int j) {
      const cx<T> v = W[i * b + j];
      Dt[i * b + j] = v;
      out[(size_t)K * bb + i * b + j] = v;
    });
    __syncthreads();
    if (H && K > 0) {
      // H_K[k][j] = sum_t Dt[k][m] A(K, m ; K-1, j), m = nbr(j, t) (the reverse slot of m reaches j);
      // the table still holds layer K-1
      cx<T>* Hk = H + ((size_t)q * L + K) * bb;
      for_entries([&](int k, int j) {
        cx<T> acc = mkc<T>(0, 0);
        for (int t = 0; t < nt; ++t) {
          int m = nbr_of(P.ly, j, t);
          if (m >= 0) cfma(acc, Dt[k * b + m], al(K - 1, m, nt - 1 - t));
        }
        Hk[(size_t)k * b + j] = acc;
      });
    }
    if (K + 1 == L) break;
    if (tab) {
      __syncthreads();  // H has read the previous layer's table
      for (int e = tid; e < b * nt; e += nthr) tab[e] = P.Al(K, e / nt, e % nt);
      __syncthreads();
    }
    // W = D_K^{-1} A_{K,K+1}:  W[k][j] = sum_t Dt[k][nbr(j,t)] A(K+1, j ; K, nbr(j,t))
    cx<T>* Gk = G ? G + ((size_t)q * L + K) * bb : nullptr;
    for_entries([&](int k, int j) {
      cx<T> acc = mkc<T>(0, 0);
      for (int t = 0; t < nt; ++t) {
        int m = nbr_of(P.ly, j, t);
        if (m >= 0) cfma(acc, Dt[k * b + m], al(K, j, t));
      }
      W[k * b + j] = acc;
      if (Gk) Gk[(size_t)k * b + j] = acc;
    });
    __syncthreads();
    // D_{K+1} = A_{K+1,K+1} - A_{K+1,K} W
    for_entries([&](int i, int j) {
      int tj = nbr_slot(P.ly, i, j);
      cx<T> acc = tj >= 0 ? P.Ad(K + 1, i, tj) : mkc<T>(0, 0);
      for (int t = 0; t < nt; ++t) {
        int k = nbr_of(P.ly, i, t);
        if (k >= 0) cfms(acc, al(K, i, t), W[k * b + j]);
      }
      Dt[i * b + j] = acc;
    });
    __syncthreads();
  }
}

// Multi-column solve with a layered factor, executed by one whole block.
//   rhs(K, i, c)   right-hand side entry of node (K, i), column c (must be 0 on removed nodes)
//   X              solution, X[(K*b + i) * ldx + c] (global memory, written here)
//   sm             2 * b * C shared entries
template <class T, class Prov, class RhsF>
__device__ void layered_solve(const Prov& P, const cx<T>* __restrict__ Dinv, int C, RhsF rhs, cx<T>* X,
                              int ldx, cx<T>* sm) {
  const int b = P.ly.b, L = P.ly.L, bb = b * b, nt = nbr_count(P.ly.dim);
  const int tid = threadIdx.x, nthr = blockDim.x, bc = b * C;
  cx<T>* Tb = sm;
  cx<T>* Ep = sm + bc;
  for (int K = 0; K < L; ++K) {
    for (int e = tid; e < bc; e += nthr) {
      int i = e / C, c = e - i * C;
      cx<T> t = rhs(K, i, c);
      if (K > 0)
        for (int tt = 0; tt < nt; ++tt) {
          int k = nbr_of(P.ly, i, tt);
          if (k >= 0) cfms(t, P.Al(K - 1, i, tt), Ep[k * C + c]);
        }
      Tb[e] = t;
    }
    __syncthreads();
    const cx<T>* D = Dinv + (size_t)K * bb;
    for (int e = tid; e < bc; e += nthr) {
      int i = e / C, c = e - i * C;
      cx<T> acc = mkc<T>(0, 0);
      for (int m = 0; m < b; ++m) cfma(acc, D[m * b + i], Tb[m * C + c]);
      Ep[e] = acc;
      X[(size_t)(K * b + i) * ldx + c] = acc;
    }
    __syncthreads();
  }
  for (int K = L - 1; K >= 0; --K) {
    for (int e = tid; e < bc; e += nthr) {
      int i = e / C, c = e - i * C;
      cx<T> u = mkc<T>(0, 0);
      if (K < L - 1)
        for (int tt = 0; tt < nt; ++tt) {
          int k = nbr_of(P.ly, i, tt);
          // A(K, i ; K+1, k) = A(K+1, k ; K, i) = Al(K, k, reverse slot)
          if (k >= 0) cfma(u, P.Al(K, k, nt - 1 - tt), Ep[k * C + c]);
        }
      Tb[e] = u;
    }
    __syncthreads();
    const cx<T>* D = Dinv + (size_t)K * bb;
    for (int e = tid; e < bc; e += nthr) {
      int i = e / C, c = e - i * C;
      cx<T> x = X[(size_t)(K * b + i) * ldx + c];
      for (int m = 0; m < b; ++m) cfms(x, D[m * b + i], Tb[m * C + c]);
      X[(size_t)(K * b + i) * ldx + c] = x;
      Ep[e] = x;
    }
    __syncthreads();
  }
}

}  // namespace schur
