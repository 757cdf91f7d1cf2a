#pragma once
#include "common.cuh"

namespace schur {

// assembled Q1 coefficients (K + (sre + i gamma) M) of an interior node towards its 3^dim offsets
struct Coef27 {
  cx<double> c[27];
};
Coef27 make_coef(const Geom& g, double gamma, double sre = 0.0);

__global__ void k_residual(Geom g, Coef27 cf, const double* __restrict__ bre, const double* __restrict__ bim,
                           int ldb, const cx<double>* __restrict__ z, int ldz, int R, cx<double>* res,
                           double* part, int nblk, int zero);
__global__ void k_shortcut(long long n, const cx<double>* __restrict__ z, int ldz, int R, double inv_gamma, double* x,
                           int ldx);
// x = scale * Re(z) (the solution of a real factor K + gamma M; its imaginary part is zero)
__global__ void k_real_part(long long n, const cx<double>* __restrict__ z, int ldz, int R, double scale, double* x,
                            int ldx);
__global__ void k_split_complex(long long n, const cx<double>* __restrict__ z, int ldz, int R, double* out, int ldo);
__global__ void k_apply_real(Geom g, Coef27 cf, int mode, const double* __restrict__ x, int ldx, double* y,
                             int ldy, int R, double alpha, double beta);
__global__ void k_dot_real(long long n, const double* __restrict__ x, int ldx, const double* __restrict__ y, int ldy,
                           int R, double* part, int nblk);
__global__ void k_axpby(long long n, const double* __restrict__ a, const double* __restrict__ x, int ldx,
                        const double* __restrict__ b, double* y, int ldy, int R);
double stencil_diag(const Geom& g, int mode);

}  // namespace schur
