/*
 * Reference oracle (TEST INFRASTRUCTURE ONLY; see oracle.h for scope and conventions).
 *
 * Paper passages followed, by function:
 *   or_element / or_assemble  Sec. 2 (K, V=M from a Q1 finite element discretisation of the
 *                             Poisson-constrained control problem, homogeneous Dirichlet data).
 *   or_kkt_solve              Sec. 2, the 3x3 KKT optimality system.  The control is eliminated
 *                             exactly from its own block row (beta*M*u - M*l = ru), which leaves
 *                             the symmetric quasi-definite system [M K; K -M/beta] (y, l) =
 *                             (ry, rl + ru/beta); u = (l + M^{-1} ru)/beta.
 *   or_schur_solve_kkt        Sec. 3.1, Eq. "schurcomplementsystem": the multiplier block of the
 *                             KKT solution with right-hand side (0, 0, -b) solves S l = b.
 *   or_schur_apply            Sec. 3.1: S = K M^{-1} K + M/beta, product form.
 *   or_fd_*                   the same operators in the sine eigenbasis of Q1 K and M.
 */
#include "oracle.h"
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

static int check_mesh(int dim, const int* nel) {
  if (dim != 2 && dim != 3) return -1;
  for (int a = 0; a < dim; ++a)
    if (nel[a] < 2) return -1;
  return 0;
}

long or_ndof(int dim, const int* nel) {
  if (check_mesh(dim, nel)) return -1;
  long n = 1;
  for (int a = 0; a < dim; ++a) n *= (nel[a] - 1);
  return n;
}

int or_bandwidth(int dim, const int* nel) {
  if (check_mesh(dim, nel)) return -1;
  int nx = nel[0] - 1, ny = nel[1] - 1;
  return dim == 2 ? nx + 1 : nx * ny + nx + 1;
}

/* ---------------------------------------------------------------- element matrices ---- */
/* Reference element [0,1]^d, node alpha in {0,1}^d (bit a of the node number = alpha_a),
 * phi_alpha(xi) = prod_a (alpha_a ? xi_a : 1 - xi_a).  Two Gauss points per axis on [0,1]:
 * xi = 1/2 -+ 1/(2 sqrt 3), weight 1/2 each; exact for the Q1 stiffness and mass integrands. */
int or_element(int dim, const double* h, double* Ke, double* Me) {
  if (dim != 2 && dim != 3) return -1;
  int nn = 1 << dim;
  double gp[2] = {0.5 - 0.5 / sqrt(3.0), 0.5 + 0.5 / sqrt(3.0)};
  double jac = 1.0;
  for (int a = 0; a < dim; ++a) jac *= h[a];
  memset(Ke, 0, sizeof(double) * nn * nn);
  memset(Me, 0, sizeof(double) * nn * nn);
  int ngp = 1 << dim;
  for (int g = 0; g < ngp; ++g) {
    double xi[3], w = 1.0;
    for (int a = 0; a < dim; ++a) { xi[a] = gp[(g >> a) & 1]; w *= 0.5; }
    double phi[8], grad[8][3];
    for (int p = 0; p < nn; ++p) {
      double v = 1.0;
      for (int a = 0; a < dim; ++a) v *= ((p >> a) & 1) ? xi[a] : 1.0 - xi[a];
      phi[p] = v;
      for (int t = 0; t < dim; ++t) {
        double d = ((p >> t) & 1) ? 1.0 : -1.0; /* d/dxi_t of the factor for axis t */
        for (int a = 0; a < dim; ++a)
          if (a != t) d *= ((p >> a) & 1) ? xi[a] : 1.0 - xi[a];
        grad[p][t] = d / h[t];
      }
    }
    for (int p = 0; p < nn; ++p)
      for (int q = 0; q < nn; ++q) {
        double kk = 0.0;
        for (int t = 0; t < dim; ++t) kk += grad[p][t] * grad[q][t];
        Ke[p * nn + q] += w * jac * kk;
        Me[p * nn + q] += w * jac * phi[p] * phi[q];
      }
  }
  return 0;
}

/* ---------------------------------------------------------------- assembly ------------- */
static long node_index(int dim, const int* nel, const int* g) {
  /* interior node with global grid coordinates g (1..nel-1), or -1 if on the boundary */
  long idx = 0, stride = 1;
  for (int a = 0; a < dim; ++a) {
    if (g[a] <= 0 || g[a] >= nel[a]) return -1;
    idx += (long)(g[a] - 1) * stride;
    stride *= (nel[a] - 1);
  }
  return idx;
}

int or_assemble(int dim, const int* nel, double* Kband, double* Mband) {
  if (check_mesh(dim, nel)) return -1;
  long n = or_ndof(dim, nel);
  int w = or_bandwidth(dim, nel);
  double h[3] = {1.0, 1.0, 1.0};
  for (int a = 0; a < dim; ++a) h[a] = 1.0 / nel[a];
  double Ke[64], Me[64];
  or_element(dim, h, Ke, Me);
  if (Kband) memset(Kband, 0, sizeof(double) * n * (w + 1));
  if (Mband) memset(Mband, 0, sizeof(double) * n * (w + 1));
  int nn = 1 << dim;
  int e[3] = {0, 0, 0};
  int ez = dim == 3 ? nel[2] : 1;
  for (e[2] = 0; e[2] < ez; ++e[2])
    for (e[1] = 0; e[1] < nel[1]; ++e[1])
      for (e[0] = 0; e[0] < nel[0]; ++e[0])
        for (int p = 0; p < nn; ++p) {
          int gp[3];
          for (int a = 0; a < dim; ++a) gp[a] = e[a] + ((p >> a) & 1);
          long ip = node_index(dim, nel, gp);
          if (ip < 0) continue;
          for (int q = 0; q < nn; ++q) {
            int gq[3];
            for (int a = 0; a < dim; ++a) gq[a] = e[a] + ((q >> a) & 1);
            long iq = node_index(dim, nel, gq);
            if (iq < 0 || iq > ip) continue; /* lower triangle only */
            long k = ip - iq;
            if (Kband) Kband[ip * (w + 1) + k] += Ke[p * nn + q];
            if (Mband) Mband[ip * (w + 1) + k] += Me[p * nn + q];
          }
        }
  return 0;
}

static void band_matvec(long n, int w, const double* band, const double* x, double* y) {
  for (long i = 0; i < n; ++i) y[i] = 0.0;
  for (long i = 0; i < n; ++i) {
    y[i] += band[i * (w + 1)] * x[i];
    for (int k = 1; k <= w && k <= i; ++k) {
      double a = band[i * (w + 1) + k];
      y[i] += a * x[i - k];
      y[i - k] += a * x[i];
    }
  }
}

/* Matrix-free products by the element loop: y = sum_e P_e^T A_e P_e x (memory O(n), any mesh). */
int or_apply_KM(int dim, const int* nel, int nrhs, const double* x, double* Kx, double* Mx) {
  if (check_mesh(dim, nel) || nrhs < 0) return -1;
  long n = or_ndof(dim, nel);
  double h[3] = {1.0, 1.0, 1.0};
  for (int a = 0; a < dim; ++a) h[a] = 1.0 / nel[a];
  double Ke[64], Me[64];
  or_element(dim, h, Ke, Me);
  int nn = 1 << dim;
  for (int r = 0; r < nrhs; ++r) {
    const double* xr = x + (long)r * n;
    double* kr = Kx ? Kx + (long)r * n : NULL;
    double* mr = Mx ? Mx + (long)r * n : NULL;
    if (kr) memset(kr, 0, sizeof(double) * n);
    if (mr) memset(mr, 0, sizeof(double) * n);
    int e[3] = {0, 0, 0};
    int ez = dim == 3 ? nel[2] : 1;
    for (e[2] = 0; e[2] < ez; ++e[2])
      for (e[1] = 0; e[1] < nel[1]; ++e[1])
        for (e[0] = 0; e[0] < nel[0]; ++e[0]) {
          long idx[8];
          double xe[8];
          for (int p = 0; p < nn; ++p) {
            int gp[3];
            for (int a = 0; a < dim; ++a) gp[a] = e[a] + ((p >> a) & 1);
            idx[p] = node_index(dim, nel, gp);
            xe[p] = idx[p] >= 0 ? xr[idx[p]] : 0.0;
          }
          for (int p = 0; p < nn; ++p) {
            if (idx[p] < 0) continue;
            double sk = 0.0, sm = 0.0;
            for (int q = 0; q < nn; ++q) {
              sk += Ke[p * nn + q] * xe[q];
              sm += Me[p * nn + q] * xe[q];
            }
            if (kr) kr[idx[p]] += sk;
            if (mr) mr[idx[p]] += sm;
          }
        }
  }
  return 0;
}

/* Sec. 2 with Dirichlet data: the stiffness rows of the interior nodes applied to a vector over all
 * prod(nel[a]+1) grid nodes (lexicographic, axis 0 fastest; boundary values = the data y_c), i.e.
 * out = K y + K_c y_c on the interior nodes, by the element loop over the whole grid. */
int or_full_stiffness(int dim, const int* nel, int nrhs, const double* yfull, double* out) {
  if (check_mesh(dim, nel) || nrhs < 0) return -1;
  long n = or_ndof(dim, nel), nf = 1;
  for (int a = 0; a < dim; ++a) nf *= nel[a] + 1;
  double h[3] = {1.0, 1.0, 1.0};
  for (int a = 0; a < dim; ++a) h[a] = 1.0 / nel[a];
  double Ke[64], Me[64];
  or_element(dim, h, Ke, Me);
  int nn = 1 << dim;
  for (int r = 0; r < nrhs; ++r) {
    const double* yr = yfull + (long)r * nf;
    double* o = out + (long)r * n;
    memset(o, 0, sizeof(double) * n);
    int e[3] = {0, 0, 0};
    int ez = dim == 3 ? nel[2] : 1;
    for (e[2] = 0; e[2] < ez; ++e[2])
      for (e[1] = 0; e[1] < nel[1]; ++e[1])
        for (e[0] = 0; e[0] < nel[0]; ++e[0]) {
          long ip[8];
          double ye[8];
          for (int p = 0; p < nn; ++p) {
            int gp[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) gp[a] = e[a] + ((p >> a) & 1);
            ip[p] = node_index(dim, nel, gp);
            long f = gp[0] + (long)(nel[0] + 1) * (gp[1] + (long)(nel[1] + 1) * gp[2]);
            ye[p] = yr[f];
          }
          for (int p = 0; p < nn; ++p) {
            if (ip[p] < 0) continue;
            double s = 0.0;
            for (int q = 0; q < nn; ++q) s += Ke[p * nn + q] * ye[q];
            o[ip[p]] += s;
          }
        }
  }
  return 0;
}

/* ---------------------------------------------------------------- banded LDL^T --------- */
/* In-place LDL^T without pivoting of a symmetric band matrix (lower-band storage, half
 * bandwidth w).  On exit band[i*(w+1)] = D_i and band[i*(w+1)+k] = L[i][i-k]. */
static int band_ldlt(long n, int w, double* band) {
  for (long j = 0; j < n; ++j) {
    double d = band[j * (w + 1)];
    if (d == 0.0 || !isfinite(d)) return -3;
    long iend = j + w < n - 1 ? j + w : n - 1;
    /* trailing update with the unscaled column, then scale it */
    for (long i = j + 1; i <= iend; ++i) {
      double aij = band[i * (w + 1) + (i - j)];
      if (aij == 0.0) continue;
      double f = aij / d;
      for (long k = j + 1; k <= i; ++k) {
        double akj = band[k * (w + 1) + (k - j)];
        band[i * (w + 1) + (i - k)] -= f * akj;
      }
    }
    for (long i = j + 1; i <= iend; ++i) band[i * (w + 1) + (i - j)] /= d;
  }
  return 0;
}

static void band_ldlt_solve(long n, int w, const double* band, double* x) {
  for (long i = 0; i < n; ++i) { /* L y = x */
    double s = x[i];
    for (int k = 1; k <= w && k <= i; ++k) s -= band[i * (w + 1) + k] * x[i - k];
    x[i] = s;
  }
  for (long i = 0; i < n; ++i) x[i] /= band[i * (w + 1)];
  for (long i = n - 1; i >= 0; --i) { /* L^T x = y */
    double s = x[i];
    for (int k = 1; k <= w && i + k < n; ++k) s -= band[(i + k) * (w + 1) + k] * x[i + k];
    x[i] = s;
  }
}

/* ---------------------------------------------------------------- O1: KKT ------------- */
int or_kkt_solve(int dim, const int* nel, double beta, int nrhs, const double* ry, const double* ru,
                 const double* rl, double* y, double* u, double* l) {
  if (check_mesh(dim, nel) || !(beta > 0.0) || nrhs < 0) return -1;
  long n = or_ndof(dim, nel);
  int w = or_bandwidth(dim, nel);
  double* Kb = (double*)malloc(sizeof(double) * n * (w + 1));
  double* Mb = (double*)malloc(sizeof(double) * n * (w + 1));
  /* interleaved unknowns (y_0, l_0, y_1, l_1, ...): half bandwidth 2w+1 */
  long N2 = 2 * n;
  int W2 = 2 * w + 1;
  double* Q = (double*)calloc((size_t)N2 * (W2 + 1), sizeof(double));
  double* Mf = (double*)malloc(sizeof(double) * n * (w + 1));
  double* rhs = (double*)malloc(sizeof(double) * N2);
  double* tmp = (double*)malloc(sizeof(double) * n);
  if (!Kb || !Mb || !Q || !Mf || !rhs || !tmp) {
    free(Kb); free(Mb); free(Q); free(Mf); free(rhs); free(tmp);
    return -2;
  }
  or_assemble(dim, nel, Kb, Mb);
  /* Q = [M K; K -M/beta] in interleaved order, lower band: Q[I][I-k] */
  for (long i = 0; i < n; ++i)
    for (int k = 0; k <= w && k <= i; ++k) {
      long j = i - k;
      double m = Mb[i * (w + 1) + k], kk = Kb[i * (w + 1) + k];
      /* (y_i, y_j): M ; (l_i, l_j): -M/beta ; (l_i, y_j): K ; (y_i, l_j): K (only if lower) */
      long Iy = 2 * i, Il = 2 * i + 1, Jy = 2 * j, Jl = 2 * j + 1;
      Q[Iy * (W2 + 1) + (Iy - Jy)] = m;
      Q[Il * (W2 + 1) + (Il - Jl)] = -m / beta;
      Q[Il * (W2 + 1) + (Il - Jy)] = kk;
      if (Iy > Jl) Q[Iy * (W2 + 1) + (Iy - Jl)] = kk;
    }
  int rc = band_ldlt(N2, W2, Q);
  if (rc == 0 && ru) {
    memcpy(Mf, Mb, sizeof(double) * n * (w + 1));
    rc = band_ldlt(n, w, Mf);
  }
  for (int r = 0; rc == 0 && r < nrhs; ++r) {
    long off = (long)r * n;
    for (long i = 0; i < n; ++i) {
      rhs[2 * i] = ry ? ry[off + i] : 0.0;
      rhs[2 * i + 1] = (rl ? rl[off + i] : 0.0) + (ru ? ru[off + i] / beta : 0.0);
    }
    band_ldlt_solve(N2, W2, Q, rhs);
    for (long i = 0; i < n; ++i) {
      if (y) y[off + i] = rhs[2 * i];
      if (l) l[off + i] = rhs[2 * i + 1];
    }
    if (u) {
      if (ru) {
        memcpy(tmp, ru + off, sizeof(double) * n);
        band_ldlt_solve(n, w, Mf, tmp);
      } else {
        memset(tmp, 0, sizeof(double) * n);
      }
      for (long i = 0; i < n; ++i) u[off + i] = (rhs[2 * i + 1] + tmp[i]) / beta;
    }
  }
  free(Kb); free(Mb); free(Q); free(Mf); free(rhs); free(tmp);
  return rc;
}

int or_schur_solve_kkt(int dim, const int* nel, double beta, int nrhs, const double* b, double* x) {
  if (check_mesh(dim, nel) || nrhs < 0) return -1;
  long n = or_ndof(dim, nel);
  double* rl = (double*)malloc(sizeof(double) * n * (nrhs > 0 ? nrhs : 1));
  if (!rl) return -2;
  for (long i = 0; i < n * nrhs; ++i) rl[i] = -b[i];
  int rc = or_kkt_solve(dim, nel, beta, nrhs, NULL, NULL, rl, NULL, NULL, x);
  free(rl);
  return rc;
}

int or_schur_apply(int dim, const int* nel, double beta, int nrhs, const double* x, double* y) {
  if (check_mesh(dim, nel) || !(beta > 0.0) || nrhs < 0) return -1;
  long n = or_ndof(dim, nel);
  int w = or_bandwidth(dim, nel);
  double* Kb = (double*)malloc(sizeof(double) * n * (w + 1));
  double* Mb = (double*)malloc(sizeof(double) * n * (w + 1));
  double* Mf = (double*)malloc(sizeof(double) * n * (w + 1));
  double* t = (double*)malloc(sizeof(double) * n);
  double* t2 = (double*)malloc(sizeof(double) * n);
  if (!Kb || !Mb || !Mf || !t || !t2) {
    free(Kb); free(Mb); free(Mf); free(t); free(t2);
    return -2;
  }
  or_assemble(dim, nel, Kb, Mb);
  memcpy(Mf, Mb, sizeof(double) * n * (w + 1));
  int rc = band_ldlt(n, w, Mf);
  for (int r = 0; rc == 0 && r < nrhs; ++r) {
    const double* xr = x + (long)r * n;
    double* yr = y + (long)r * n;
    band_matvec(n, w, Kb, xr, t);   /* t = K x        */
    band_ldlt_solve(n, w, Mf, t);   /* t = M^{-1} K x */
    band_matvec(n, w, Kb, t, yr);   /* y = K M^-1 K x */
    band_matvec(n, w, Mb, xr, t2);  /* t2 = M x       */
    for (long i = 0; i < n; ++i) yr[i] += t2[i] / beta;
  }
  free(Kb); free(Mb); free(Mf); free(t); free(t2);
  return rc;
}

/* ---------------------------------------------------------------- O2: sine basis ------- */
/* Orthonormal DST-I matrix for m = N-1 interior nodes: V[a][j] = sqrt(2/N) sin(pi a j / N),
 * a, j = 1..m.  It is symmetric and orthogonal, so it is its own inverse. */
static double* sine_matrix(int N) {
  int m = N - 1;
  double* V = (double*)malloc(sizeof(double) * m * m);
  if (!V) return NULL;
  double s = sqrt(2.0 / N);
  for (int a = 1; a <= m; ++a)
    for (int j = 1; j <= m; ++j) V[(a - 1) * m + (j - 1)] = s * sin(M_PI * (double)a * (double)j / N);
  return V;
}

/* Apply V along axis `ax` of an array with dims m[0..dim-1] (axis 0 fastest), in place.  The
 * lines along the axis are independent; with OpenMP they are shared out among the threads, each
 * line's arithmetic unchanged (the same products summed in the same order), so the result does
 * not depend on the thread count. */
static int transform_axis(int dim, const int* m, int ax, const double* V, double* x) {
  long stride = 1;
  for (int a = 0; a < ax; ++a) stride *= m[a];
  long len = m[ax];
  long outer = 1;
  for (int a = ax + 1; a < dim; ++a) outer *= m[a];
  long nlines = outer * stride;
  int fail = 0;
#pragma omp parallel
  {
    double* line = (double*)malloc(sizeof(double) * len);
    double* out = (double*)malloc(sizeof(double) * len);
    if (!line || !out) {
#pragma omp atomic write
      fail = 1;
    } else {
#pragma omp for schedule(static)
      for (long q = 0; q < nlines; ++q) {
        long o = q / stride, in = q % stride;
        long base = o * stride * len + in;
        for (long a = 0; a < len; ++a) line[a] = x[base + a * stride];
        for (long j = 0; j < len; ++j) {
          double s = 0.0;
          const double* row = V + j * len;
          for (long a = 0; a < len; ++a) s += row[a] * line[a];
          out[j] = s;
        }
        for (long a = 0; a < len; ++a) x[base + a * stride] = out[a];
      }
    }
    free(line);
    free(out);
  }
  return fail ? -2 : 0;
}

/* Threads of the sine transforms (OpenMP); 1 = single-threaded.  Returns the count in effect. */
int or_set_threads(int nthreads) {
#ifdef _OPENMP
  if (nthreads >= 1) omp_set_num_threads(nthreads);
  return omp_get_max_threads();
#else
  (void)nthreads;
  return 1;
#endif
}

static int sine_transform(int dim, const int* nel, double* const* Vs, double* x) {
  int m[3];
  for (int a = 0; a < dim; ++a) m[a] = nel[a] - 1;
  for (int a = 0; a < dim; ++a) {
    int rc = transform_axis(dim, m, a, Vs[a], x);
    if (rc) return rc;
  }
  return 0;
}

/* 1D Q1 eigenvalues on a uniform Dirichlet grid, mode j: stiffness (2/h)(1 - cos(j pi h)),
 * mass (h/3)(2 + cos(j pi h)).  In d dimensions K = sum_t (K_t (x) prod_{u != t} M_u) and
 * M = prod_u M_u as Kronecker products, so kappa and mu follow per mode. */
int or_fd_eigs(int dim, const int* nel, double* kappa, double* mu) {
  if (check_mesh(dim, nel)) return -1;
  int m[3] = {1, 1, 1};
  for (int a = 0; a < dim; ++a) m[a] = nel[a] - 1;
  long n = or_ndof(dim, nel);
  for (long idx = 0; idx < n; ++idx) {
    long r = idx;
    double k1[3], m1[3];
    for (int a = 0; a < dim; ++a) {
      int j = (int)(r % m[a]) + 1;
      r /= m[a];
      double h = 1.0 / nel[a], c = cos(M_PI * j * h);
      k1[a] = 2.0 / h * (1.0 - c);
      m1[a] = h / 3.0 * (2.0 + c);
    }
    double kk = 0.0, mm = 1.0;
    for (int t = 0; t < dim; ++t) {
      double p = k1[t];
      for (int u = 0; u < dim; ++u)
        if (u != t) p *= m1[u];
      kk += p;
      mm *= m1[t];
    }
    kappa[idx] = kk;
    mu[idx] = mm;
  }
  return 0;
}

typedef struct {
  int dim;
  int nel[3];
  long n;
  double* V[3];
  double* kappa;
  double* mu;
} fd_ctx;

static void fd_free(fd_ctx* c) {
  for (int a = 0; a < 3; ++a) {
    int dup = 0;
    for (int b = 0; b < a; ++b)
      if (c->V[b] == c->V[a]) dup = 1;
    if (!dup) free(c->V[a]);
  }
  free(c->kappa);
  free(c->mu);
}

static int fd_init(fd_ctx* c, int dim, const int* nel) {
  memset(c, 0, sizeof(*c));
  if (check_mesh(dim, nel)) return -1;
  c->dim = dim;
  for (int a = 0; a < dim; ++a) c->nel[a] = nel[a];
  c->n = or_ndof(dim, nel);
  for (int a = 0; a < dim; ++a) {
    for (int b = 0; b < a; ++b)
      if (nel[b] == nel[a]) c->V[a] = c->V[b];
    if (!c->V[a]) c->V[a] = sine_matrix(nel[a]);
    if (!c->V[a]) { fd_free(c); return -2; }
  }
  c->kappa = (double*)malloc(sizeof(double) * c->n);
  c->mu = (double*)malloc(sizeof(double) * c->n);
  if (!c->kappa || !c->mu) { fd_free(c); return -2; }
  or_fd_eigs(dim, nel, c->kappa, c->mu);
  return 0;
}

/* y = f(mode) * x in the sine basis, f(kappa, mu) = scale for each mode */
typedef double (*mode_fn)(double kappa, double mu, double beta);

static double f_schur_inv(double k, double m, double beta) { return 1.0 / (k * k / m + m / beta); }
static double f_schur(double k, double m, double beta) { return k * k / m + m / beta; }
/* Sec. 3.2, Eq. pearsonapproximation: S_p = (K + M/sqrt(beta)) M^{-1} (K + M/sqrt(beta)), per mode
 * (kappa + mu/sqrt(beta))^2 / mu */
static double f_pw_inv(double k, double m, double beta) {
  double s = k + m / sqrt(beta);
  return m / (s * s);
}

static int fd_diag_op(int dim, const int* nel, double beta, int nrhs, const double* x, double* y, mode_fn f) {
  fd_ctx c;
  int rc = fd_init(&c, dim, nel);
  if (rc) return rc;
  for (int r = 0; r < nrhs && rc == 0; ++r) {
    double* yr = y + (long)r * c.n;
    memcpy(yr, x + (long)r * c.n, sizeof(double) * c.n);
    rc = sine_transform(dim, nel, c.V, yr);
    for (long i = 0; rc == 0 && i < c.n; ++i) yr[i] *= f(c.kappa[i], c.mu[i], beta);
    if (rc == 0) rc = sine_transform(dim, nel, c.V, yr);
  }
  fd_free(&c);
  return rc;
}

int or_fd_schur_solve(int dim, const int* nel, double beta, int nrhs, const double* b, double* x) {
  if (!(beta > 0.0) || nrhs < 0) return -1;
  return fd_diag_op(dim, nel, beta, nrhs, b, x, f_schur_inv);
}

int or_fd_pw_solve(int dim, const int* nel, double beta, int nrhs, const double* b, double* x) {
  if (!(beta > 0.0) || nrhs < 0) return -1;
  return fd_diag_op(dim, nel, beta, nrhs, b, x, f_pw_inv);
}

int or_fd_schur_apply(int dim, const int* nel, double beta, int nrhs, const double* x, double* y) {
  if (!(beta > 0.0) || nrhs < 0) return -1;
  return fd_diag_op(dim, nel, beta, nrhs, x, y, f_schur);
}

int or_fd_complex_solve(int dim, const int* nel, double gamma, int sgn, int nrhs, const double* bre,
                        const double* bim, double* zre, double* zim) {
  if (nrhs < 0 || (sgn != 1 && sgn != -1)) return -1;
  fd_ctx c;
  int rc = fd_init(&c, dim, nel);
  if (rc) return rc;
  for (int r = 0; r < nrhs && rc == 0; ++r) {
    long off = (long)r * c.n;
    memcpy(zre + off, bre + off, sizeof(double) * c.n);
    if (bim) memcpy(zim + off, bim + off, sizeof(double) * c.n);
    else memset(zim + off, 0, sizeof(double) * c.n);
    rc = sine_transform(dim, nel, c.V, zre + off);
    if (rc == 0) rc = sine_transform(dim, nel, c.V, zim + off);
    for (long i = 0; rc == 0 && i < c.n; ++i) {
      /* (br + i bi) / (kappa + i sgn gamma mu) */
      double a = c.kappa[i], bb = sgn * gamma * c.mu[i];
      double den = a * a + bb * bb;
      double br = zre[off + i], bi = zim[off + i];
      zre[off + i] = (br * a + bi * bb) / den;
      zim[off + i] = (bi * a - br * bb) / den;
    }
    if (rc == 0) rc = sine_transform(dim, nel, c.V, zre + off);
    if (rc == 0) rc = sine_transform(dim, nel, c.V, zim + off);
  }
  fd_free(&c);
  return rc;
}

int or_fd_kkt_solve(int dim, const int* nel, double beta, int nrhs, const double* ry, const double* ru,
                    const double* rl, double* y, double* u, double* l) {
  if (!(beta > 0.0) || nrhs < 0) return -1;
  fd_ctx c;
  int rc = fd_init(&c, dim, nel);
  if (rc) return rc;
  long n = c.n;
  double* t = (double*)malloc(sizeof(double) * 3 * n);
  if (!t) { fd_free(&c); return -2; }
  double *ty = t, *tu = t + n, *tl = t + 2 * n;
  for (int r = 0; r < nrhs && rc == 0; ++r) {
    long off = (long)r * n;
    if (ry) memcpy(ty, ry + off, sizeof(double) * n); else memset(ty, 0, sizeof(double) * n);
    if (ru) memcpy(tu, ru + off, sizeof(double) * n); else memset(tu, 0, sizeof(double) * n);
    if (rl) memcpy(tl, rl + off, sizeof(double) * n); else memset(tl, 0, sizeof(double) * n);
    rc = sine_transform(dim, nel, c.V, ty);
    if (!rc) rc = sine_transform(dim, nel, c.V, tu);
    if (!rc) rc = sine_transform(dim, nel, c.V, tl);
    for (long i = 0; rc == 0 && i < n; ++i) {
      /* per mode: [mu 0 k; 0 beta mu -mu; k -mu 0] (y, u, l) = (a, b, c).  Eliminate u from the
       * second row: u = (l + b/mu)/beta; then [mu k; k -mu/beta] (y, l) = (a, c + b/beta). */
      double k = c.kappa[i], m = c.mu[i];
      double a = ty[i], b = tu[i], cc = tl[i] + tu[i] / beta;
      double det = -m * m / beta - k * k;
      double yy = (-(m / beta) * a - k * cc) / det;
      double ll = (m * cc - k * a) / det;
      ty[i] = yy;
      tl[i] = ll;
      tu[i] = (ll + b / m) / beta;
    }
    if (!rc) rc = sine_transform(dim, nel, c.V, ty);
    if (!rc) rc = sine_transform(dim, nel, c.V, tu);
    if (!rc) rc = sine_transform(dim, nel, c.V, tl);
    if (y) memcpy(y + off, ty, sizeof(double) * n);
    if (u) memcpy(u + off, tu, sizeof(double) * n);
    if (l) memcpy(l + off, tl, sizeof(double) * n);
  }
  free(t);
  fd_free(&c);
  return rc;
}
