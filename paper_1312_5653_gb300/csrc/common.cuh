// Shared device/host definitions of libschur: complex arithmetic, the subdomain geometry, and the
// closed-form Q1 entries of the shifted operator A = K + i gamma M on a subdomain.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>

namespace schur {

// Raises the dynamic shared-memory limit of kernel `func` to at least `bytes`.  The limit is a
// per-process attribute shared by every thread, so it only ever grows (under a lock): a thread
// configuring a smaller launch never undercuts a concurrent larger one.
cudaError_t smem_attr(const void* func, int bytes);

constexpr int kMaxRdev = 16;   // right-hand sides per FETI-DP solve
constexpr int kMaxKdev = 512;  // Krylov basis size bound (max_iter < kMaxKdev)
constexpr int kApplyGroup = 8;  // subdomains of one class that share a staged local operator

// Programmatic dependent launch: a kernel launched by launch_pdl may start while its predecessor
// in the stream is still running; it calls pdl_wait() before anything else (which returns once the
// predecessor has completed and its memory is visible; a no-op for an ordinary launch) and
// pdl_trigger() to let its own successor start launching.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <class R>
struct alignas(2 * sizeof(R)) cx {
  R re, im;
};

template <class R>
__host__ __device__ __forceinline__ cx<R> mkc(R a, R b) {
  cx<R> c;
  c.re = a;
  c.im = b;
  return c;
}
template <class R>
__host__ __device__ __forceinline__ cx<R> cadd(cx<R> a, cx<R> b) { return mkc<R>(a.re + b.re, a.im + b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> csub(cx<R> a, cx<R> b) { return mkc<R>(a.re - b.re, a.im - b.im); }
template <class R>
__host__ __device__ __forceinline__ cx<R> cmul(cx<R> a, cx<R> b) {
  return mkc<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
// acc += a * b
template <class R>
__host__ __device__ __forceinline__ void cfma(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// acc -= a * b
template <class R>
__host__ __device__ __forceinline__ void cfms(cx<R>& acc, cx<R> a, cx<R> b) {
  acc.re = fma(-a.re, b.re, acc.re);
  acc.re = fma(a.im, b.im, acc.re);
  acc.im = fma(-a.re, b.im, acc.im);
  acc.im = fma(-a.im, b.re, acc.im);
}
template <class R>
__host__ __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return mkc<R>(a.re * s, a.im * s); }
template <class R>
__host__ __device__ __forceinline__ cx<R> cinv(cx<R> a) {
  const R s = R(1) / (a.re * a.re + a.im * a.im);  // one division
  return mkc<R>(a.re * s, -a.im * s);
}
template <class R, class S>
__host__ __device__ __forceinline__ cx<R> ccast(cx<S> a) { return mkc<R>((R)a.re, (R)a.im); }

// ------------------------------------------------------------------ symmetric packed storage
// Complex symmetric n x n matrices (the local F and S) keep their upper triangle row by row:
// entry (i, j), i <= j, at sym_off(i, n) + j - i.  Each matrix takes sym_ld(n) entries, an even
// count, so consecutive FP32 matrices start on 16-byte boundaries.
__host__ __device__ __forceinline__ int sym_off(int i, int n) { return i * n - (i * (i - 1)) / 2; }
__host__ __device__ __forceinline__ int sym_idx(int i, int j, int n) {
  return i <= j ? sym_off(i, n) + (j - i) : sym_off(j, n) + (i - j);
}
__host__ __device__ __forceinline__ long long sym_ld(int n) { return (((long long)n * (n + 1) / 2) + 1) & ~1LL; }

// --------------------------------------------------------------------------------- geometry
// One uniform Q1 mesh on [0,1]^dim split into nsub[a] boxes of s[a] elements per axis.
// Node numbering everywhere: lexicographic with axis 0 fastest.
//   local grid of a subdomain: (s+1)^dim nodes, coordinates l in [0, s]
//   global interior nodes: coordinates g in [1, nel-1]
//   interface slots: local boundary nodes that are not subdomain vertices (same list for every
//     subdomain); corners: the 2^dim subdomain vertices (bit a set <=> l_a = s_a)
//   coarse grid: interior subdomain vertices, (nsub[a]-1) per axis
struct Geom {
  int dim;
  int nel[3], nsub[3], s[3];
  double h[3];
  int nsd;        // subdomains
  int nl;         // local nodes
  int lb, lL;     // remainder problem: nodes per layer, layers (layer = last axis)
  int ib, iL, ni; // interior problem: nodes per layer, layers, nodes
  int nD;         // interface slots per subdomain
  int nc;         // local corners (2^dim)
  long long n;    // global interior nodes
  int nlam;       // dual unknowns
  int ncg[3];     // coarse grid per axis
  int ncor;       // primal corners (coarse unknowns of the unaugmented coarse problem)
  int cb, cL;     // coarse layered structure of the corners
  int maxdeg;     // multipliers per interface slot at most (1 in 2D, 3 in 3D)
  // coarse couplings per subdomain (nq) and coarse unknowns (nco): the corners, plus with the
  // augmented coarse problem one average constraint per pair of face-adjacent subdomains, faces
  // numbered after the corners (nface of them); a subdomain's face slot f = 2a + side (side 1 =
  // the face at l_a = s_a) follows its corner slots
  int nq, nco, nface;
};

// Per-axis assembled 1D factors of the Q1 stiffness (k) and mass (m), in the working precision.
// For nodes p, q on a segment of `s` elements: same node -> (count of elements containing it) *
// (1/h, h/3); neighbours -> (-1/h, h/6).  A d-dimensional entry is
//   K_pq = sum_t k_t(p_t,q_t) prod_{u != t} m_u(p_u,q_u),   M_pq = prod_u m_u(p_u,q_u).
template <class R>
struct Stencil {
  R k_one[3], k_two[3], k_off[3];  // diagonal with 1 or 2 elements, off-diagonal
  R m_one[3], m_two[3], m_off[3];
  R gamma;  // imaginary mass shift: entries of K + i gamma M
  R sre;    // real mass shift (0 for K + i gamma M; gamma for the real factor K + gamma M)
  int dim;
};

template <class R>
inline Stencil<R> make_stencil(const Geom& g, double gamma, double sre = 0.0) {
  Stencil<R> st;
  st.dim = g.dim;
  st.gamma = (R)gamma;
  st.sre = (R)sre;
  for (int a = 0; a < 3; ++a) {
    double h = a < g.dim ? g.h[a] : 1.0;
    st.k_one[a] = (R)(1.0 / h);
    st.k_two[a] = (R)(2.0 / h);
    st.k_off[a] = (R)(-1.0 / h);
    st.m_one[a] = (R)(h / 3.0);
    st.m_two[a] = (R)(2.0 * h / 3.0);
    st.m_off[a] = (R)(h / 6.0);
  }
  return st;
}

// Entry (p, q) of the subdomain Neumann matrix K + (sre + i gamma) M for local node coordinates p, q
// (|p_a - q_a| <= 1 assumed by callers that pass neighbours; others give 0).  s = elements per
// axis of the segment the counts refer to; pass a huge s for interior (two-element) counts.
template <class R>
__host__ __device__ __forceinline__ cx<R> q1_entry(const Stencil<R>& st, const int* s, const int* p,
                                                   const int* q) {
  R k1[3], m1[3];
  for (int a = 0; a < st.dim; ++a) {
    int d = p[a] - q[a];
    if (d > 1 || d < -1) return mkc<R>(0, 0);
    if (d == 0) {
      bool two = p[a] > 0 && p[a] < s[a];
      k1[a] = two ? st.k_two[a] : st.k_one[a];
      m1[a] = two ? st.m_two[a] : st.m_one[a];
    } else {
      k1[a] = st.k_off[a];
      m1[a] = st.m_off[a];
    }
  }
  R kk, mm;
  if (st.dim == 2) {
    kk = k1[0] * m1[1] + m1[0] * k1[1];
    mm = m1[0] * m1[1];
  } else {
    kk = k1[0] * m1[1] * m1[2] + m1[0] * k1[1] * m1[2] + m1[0] * m1[1] * k1[2];
    mm = m1[0] * m1[1] * m1[2];
  }
  return mkc<R>(kk + st.sre * mm, st.gamma * mm);
}

// Local node <-> coordinates on a box with `ext` nodes per axis.
__host__ __device__ __forceinline__ void idx2crd(int idx, const int* ext, int dim, int* c) {
  c[0] = idx % ext[0];
  idx /= ext[0];
  c[1] = idx % ext[1];
  if (dim == 3) c[2] = idx / ext[1];
  else c[2] = 0;
}
__host__ __device__ __forceinline__ int crd2idx(const int* c, const int* ext, int dim) {
  return dim == 2 ? c[0] + ext[0] * c[1] : c[0] + ext[0] * (c[1] + ext[1] * c[2]);
}

// Boundary-type code of a subdomain: bit 2a = its low face on axis a is Dirichlet, bit 2a+1 =
// its high face is.  A local node is removed from the remainder set if it is a subdomain vertex
// (primal corner or Dirichlet) or lies on a Dirichlet face.
__host__ __device__ __forceinline__ bool local_dirichlet(int code, const int* l, const int* s, int dim) {
  for (int a = 0; a < dim; ++a) {
    if (l[a] == 0 && (code >> (2 * a) & 1)) return true;
    if (l[a] == s[a] && (code >> (2 * a + 1) & 1)) return true;
  }
  return false;
}
__host__ __device__ __forceinline__ bool local_vertex(const int* l, const int* s, int dim) {
  for (int a = 0; a < dim; ++a)
    if (l[a] != 0 && l[a] != s[a]) return false;
  return true;
}
__host__ __device__ __forceinline__ bool local_on_boundary(const int* l, const int* s, int dim) {
  for (int a = 0; a < dim; ++a)
    if (l[a] == 0 || l[a] == s[a]) return true;
  return false;
}

}  // namespace schur
