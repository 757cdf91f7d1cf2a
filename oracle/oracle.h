/*
 * Reference oracle for the factored Schur complement solve of distributed optimal control
 * (Choi, Farhat, Murray, Saunders, arXiv 1312.5653).  TEST INFRASTRUCTURE ONLY: plain, slow
 * FP64 C (single-threaded, except that the independent lines of the O2 sine transforms may be
 * shared out over OpenMP threads with unchanged arithmetic; see or_set_threads).  Only the test suite, the smoke check and the CPU-baseline leg of the
 * benchmark may call it; the product library never links or loads it, and this code shares
 * nothing (no header, helper, table or constant) with the CUDA path.
 *
 * Problem (Sec. 2, Eq. "discretizedoptimalheatcontrol" and the KKT system after it): on the
 * unit box [0,1]^d (d = 2, 3) with a uniform grid of nel[a] Q1 elements per axis and homogeneous
 * Dirichlet conditions on the whole boundary, K (stiffness) and M (consistent mass, the paper's
 * volume matrix V) act on the n = prod(nel[a]-1) interior nodes, numbered lexicographically with
 * axis 0 fastest.  beta is the paper's regularisation phi; gamma = 1/sqrt(beta).
 *   KKT (Sec. 2):  [M 0 K; 0 beta*M -M; K -M 0] (y,u,l) = (ry, ru, rl)
 *   S = K M^{-1} K + M / beta              (Sec. 3.1, negative Schur complement)
 *
 * Two independent solvers:
 *   O1 (or_kkt_solve)   element-loop assembly by 2-point Gauss quadrature, exact elimination
 *                       of u, banded LDL^T (no pivoting) of the quasi-definite 2n system.
 *   O2 (or_fd_*)        fast diagonalisation: the discrete sine vectors are exact eigenvectors
 *                       of Q1 K and M on uniform grids, so every operator above is diagonal in
 *                       the sine basis.  Transforms are dense products (no FFT library).
 * All arrays are column-major with leading dimension n when nrhs > 1.
 * Return value: 0 on success, -1 on bad arguments, -2 on allocation failure, -3 on a zero pivot.
 */
#ifndef SCHUR_ORACLE_H
#define SCHUR_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

long or_ndof(int dim, const int* nel);
int or_bandwidth(int dim, const int* nel);
/* Q1 element matrices (2^d x 2^d, row-major, element nodes lexicographic) by 2-pt Gauss. */
int or_element(int dim, const double* h, double* Ke, double* Me);
/* Assembled K and M in lower-band storage: band[i*(w+1)+k] = A[i][i-k], k = 0..w. */
int or_assemble(int dim, const int* nel, double* Kband, double* Mband);
/* Kx = K x and Mx = M x (either output may be NULL). */
int or_apply_KM(int dim, const int* nel, int nrhs, const double* x, double* Kx, double* Mx);
/* O1: KKT solve for general right-hand sides (any of ry, ru, rl may be NULL = zero). */
int or_kkt_solve(int dim, const int* nel, double beta, int nrhs, const double* ry, const double* ru,
                 const double* rl, double* y, double* u, double* l);
/* O1: x = S^{-1} b through the KKT system with right-hand side (0, 0, -b), x = lambda. */
int or_schur_solve_kkt(int dim, const int* nel, double beta, int nrhs, const double* b, double* x);
/* y = S x with M^{-1} applied by banded Cholesky (LDL^T) of M. */
int or_schur_apply(int dim, const int* nel, double beta, int nrhs, const double* x, double* y);

/* O2: x = S^{-1} b. */
int or_fd_schur_solve(int dim, const int* nel, double beta, int nrhs, const double* b, double* x);
/* O2: x = S_p^{-1} b, S_p = (K + M/sqrt(beta)) M^{-1} (K + M/sqrt(beta)) (Sec. 3.2). */
int or_fd_pw_solve(int dim, const int* nel, double beta, int nrhs, const double* b, double* x);
/* O2: y = S x. */
int or_fd_schur_apply(int dim, const int* nel, double beta, int nrhs, const double* x, double* y);
/* O2: z = (K + i*sgn*gamma*M)^{-1} (bre + i*bim); bim may be NULL. */
int or_fd_complex_solve(int dim, const int* nel, double gamma, int sgn, int nrhs, const double* bre,
                        const double* bim, double* zre, double* zim);
/* O2: KKT solve (any right-hand side pointer may be NULL = zero). */
int or_fd_kkt_solve(int dim, const int* nel, double beta, int nrhs, const double* ry, const double* ru,
                    const double* rl, double* y, double* u, double* l);
/* O2: eigenvalues of K and M for each sine vector (arrays of length n). */
int or_fd_eigs(int dim, const int* nel, double* kappa, double* mu);
/* Threads used by the O2 sine transforms (OpenMP over independent transform lines; the result
 * does not depend on the count).  nthreads < 1 leaves it unchanged.  Returns the count in effect. */
int or_set_threads(int nthreads);
/* Sec. 2 with Dirichlet data: out = K y + K_c y_c on the interior nodes, from a vector over all
 * prod(nel[a]+1) grid nodes whose boundary values are y_c (element loop over the whole grid). */
int or_full_stiffness(int dim, const int* nel, int nrhs, const double* yfull, double* out);

#ifdef __cplusplus
}
#endif
#endif
