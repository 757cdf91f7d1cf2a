// FP64 whole-mesh kernels: matrix-free Q1 stencils for K, M and A = K + i gamma M on the interior
// nodes, the refinement residual b - A z, the real-input shortcut x = -Im(z)/gamma, and small
// vector reductions.  (Sec. 2 operators; Sec. 3.1 iterative refinement in higher precision;
// shortcut from the factorisation of Sec. 4.)
#include "outer.h"

namespace schur {

__device__ __forceinline__ void node_crd(const Geom& g, long long gi, int* G) {
  G[0] = (int)(gi % (g.nel[0] - 1)) + 1;
  long long t = gi / (g.nel[0] - 1);
  if (g.dim == 2) {
    G[1] = (int)t + 1;
    G[2] = 0;
  } else {
    G[1] = (int)(t % (g.nel[1] - 1)) + 1;
    G[2] = (int)(t / (g.nel[1] - 1)) + 1;
  }
}

Coef27 make_coef(const Geom& g, double gamma, double sre) {
  // every interior node has two elements per axis, so the assembled coefficient of a neighbour
  // depends only on the offset
  Stencil<double> st = make_stencil<double>(g, gamma, sre);
  Coef27 cf;
  int G[3] = {1, 1, 1};
  for (int o = 0; o < 27; ++o) {
    int Q[3] = {1 + o % 3 - 1, 1 + (o / 3) % 3 - 1, 1 + o / 9 - 1};
    cf.c[o] = q1_entry(st, g.nel, G, Q);
  }
  return cf;
}

// calls fn(offset index o, neighbour index) for the interior neighbours of interior node G
template <class F>
__device__ __forceinline__ void for_neighbours(const Geom& g, const int* G, F fn) {
  const int noff = g.dim == 2 ? 9 : 27;
  long long s1 = g.nel[0] - 1, s2 = s1 * (g.nel[1] - 1);
  for (int o = 0; o < noff; ++o) {
    int Q[3] = {G[0] + o % 3 - 1, G[1] + (o / 3) % 3 - 1, g.dim == 3 ? G[2] + o / 9 - 1 : 0};
    bool in = true;
    for (int a = 0; a < g.dim; ++a) in = in && Q[a] >= 1 && Q[a] <= g.nel[a] - 1;
    if (!in) continue;
    long long qi = (Q[0] - 1) + s1 * (Q[1] - 1) + (g.dim == 3 ? s2 * (Q[2] - 1) : 0);
    fn(o, qi);
  }
}

// (A z) at interior node G.  On the uniform mesh mirrored neighbours share their coefficient, so
// the neighbours are first summed per offset class (which axes the offset moves along) and each
// class sum then takes one complex product: 2^dim products instead of 3^dim.  Neighbours on the
// Dirichlet boundary (outside the interior nodes) contribute nothing.
template <int DIM>
__device__ __forceinline__ cx<double> apply_A_node(const Geom& g, const Coef27& cf, const cx<double>* __restrict__ zr,
                                                   const int* G) {
  constexpr int NC = 1 << DIM;
  cx<double> s[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) s[c] = mkc<double>(0, 0);
  const long long s1 = g.nel[0] - 1, s2 = s1 * (g.nel[1] - 1);
#pragma unroll
  for (int o = 0; o < (DIM == 2 ? 9 : 27); ++o) {
    const int d0 = o % 3 - 1, d1 = (o / 3) % 3 - 1, d2 = DIM == 3 ? o / 9 - 1 : 0;
    const int Q0 = G[0] + d0, Q1 = G[1] + d1, Q2 = G[2] + d2;
    bool in = Q0 >= 1 && Q0 <= g.nel[0] - 1 && Q1 >= 1 && Q1 <= g.nel[1] - 1;
    if (DIM == 3) in = in && Q2 >= 1 && Q2 <= g.nel[2] - 1;
    if (!in) continue;
    const long long qi = (Q0 - 1) + s1 * (Q1 - 1) + (DIM == 3 ? s2 * (Q2 - 1) : 0);
    const int c = (d0 != 0 ? 1 : 0) | (d1 != 0 ? 2 : 0) | (d2 != 0 ? 4 : 0);
    s[c] = cadd(s[c], zr[qi]);
  }
  cx<double> acc = mkc<double>(0, 0);
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    // the coefficient of the class's neighbour at +1 along each of its axes
    const int o = (1 + (c & 1)) + 3 * (1 + ((c >> 1) & 1)) + (DIM == 3 ? 9 * (1 + ((c >> 2) & 1)) : 0);
    cfma(acc, cf.c[o], s[c]);
  }
  return acc;
}

// res = b - A z and the block partial sums of |res|^2 and |b|^2; zero != 0 takes z = 0 (the first
// refinement step) and reads no z.
__global__ void k_residual(Geom g, Coef27 cf, const double* __restrict__ bre, const double* __restrict__ bim,
                           int ldb, const cx<double>* __restrict__ z, int ldz, int R, cx<double>* res,
                           double* part, int nblk, int zero) {
  __shared__ double red[2][32];
  const int r = blockIdx.y;
  double s_r = 0, s_b = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.n; i += (long long)nblk * blockDim.x) {
    cx<double> acc = mkc<double>(0, 0);
    if (!zero) {
      int G[3];
      node_crd(g, i, G);
      const cx<double>* zr = z + (size_t)r * ldz;
      acc = g.dim == 2 ? apply_A_node<2>(g, cf, zr, G) : apply_A_node<3>(g, cf, zr, G);
    }
    double br = bre[(size_t)r * ldb + i], bi = bim ? bim[(size_t)r * ldb + i] : 0.0;
    cx<double> rr = mkc<double>(br - acc.re, bi - acc.im);
    res[(size_t)r * g.n + i] = rr;
    s_r += rr.re * rr.re + rr.im * rr.im;
    s_b += br * br + bi * bi;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s_r += __shfl_xor_sync(0xffffffffu, s_r, o);
    s_b += __shfl_xor_sync(0xffffffffu, s_b, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s_r;
    red[1][threadIdx.x >> 5] = s_b;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    int nw = blockDim.x >> 5;
    s_r = threadIdx.x < nw ? red[0][threadIdx.x] : 0.0;
    s_b = threadIdx.x < nw ? red[1][threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      s_r += __shfl_xor_sync(0xffffffffu, s_r, o);
      s_b += __shfl_xor_sync(0xffffffffu, s_b, o);
    }
    if (threadIdx.x == 0) {
      part[((size_t)r * nblk + blockIdx.x) * 2] = s_r;
      part[((size_t)r * nblk + blockIdx.x) * 2 + 1] = s_b;
    }
  }
}

__global__ void k_shortcut(long long n, const cx<double>* __restrict__ z, int ldz, int R, double inv_gamma, double* x,
                           int ldx) {
  const int r = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[(size_t)r * ldx + i] = -z[(size_t)r * ldz + i].im * inv_gamma;
}

__global__ void k_real_part(long long n, const cx<double>* __restrict__ z, int ldz, int R, double scale, double* x,
                            int ldx) {
  const int r = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    x[(size_t)r * ldx + i] = z[(size_t)r * ldz + i].re * scale;
}

__global__ void k_split_complex(long long n, const cx<double>* __restrict__ z, int ldz, int R, double* out, int ldo) {
  const int r = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    cx<double> v = z[(size_t)r * ldz + i];
    out[((size_t)r * ldo + i) * 2] = v.re;
    out[((size_t)r * ldo + i) * 2 + 1] = v.im;
  }
}

// y = alpha * Op x + beta * y, Op = M (mode 0), K (mode 1), real FP64
__global__ void k_apply_real(Geom g, Coef27 cf, int mode, const double* __restrict__ x, int ldx, double* y,
                             int ldy, int R, double alpha, double beta) {
  const int r = blockIdx.y;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < g.n; i += (long long)gridDim.x * blockDim.x) {
    int G[3];
    node_crd(g, i, G);
    double acc = 0;
    const double* xr = x + (size_t)r * ldx;
    for_neighbours(g, G, [&](int o, long long qi) { acc += (mode == 0 ? cf.c[o].im : cf.c[o].re) * xr[qi]; });
    double* yy = y + (size_t)r * ldy + i;
    *yy = alpha * acc + (beta == 0.0 ? 0.0 : beta * *yy);
  }
}

// diagonal of M (mode 0) or K (mode 1) at an interior node (the same for every node)
double stencil_diag(const Geom& g, int mode) {
  Stencil<double> st = make_stencil<double>(g, 1.0);
  int G[3] = {1, 1, 1};
  cx<double> c = q1_entry(st, g.nel, G, G);
  return mode == 0 ? c.im : c.re;
}

__global__ void k_dot_real(long long n, const double* __restrict__ x, int ldx, const double* __restrict__ y, int ldy,
                           int R, double* part, int nblk) {
  __shared__ double red[32];
  const int r = blockIdx.y;
  double s = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)nblk * blockDim.x)
    s += x[(size_t)r * ldx + i] * y[(size_t)r * ldy + i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) part[(size_t)r * nblk + blockIdx.x] = s;
  }
}

// y = a[r] * x + b[r] * y  (coefficient arrays on the device, per right-hand side)
__global__ void k_axpby(long long n, const double* __restrict__ a, const double* __restrict__ x, int ldx,
                        const double* __restrict__ b, double* y, int ldy, int R) {
  const int r = blockIdx.y;
  const double ar = a[r], br = b[r];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double* yy = y + (size_t)r * ldy + i;
    *yy = ar * x[(size_t)r * ldx + i] + (br == 0.0 ? 0.0 : br * *yy);
  }
}

}  // namespace schur
