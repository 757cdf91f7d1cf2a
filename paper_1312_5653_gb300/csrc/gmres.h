#pragma once
#include "common.cuh"

namespace schur {

__global__ void k_dots_reduce(const cx<double>* __restrict__ part, int nblk, int R, int k, int m,
                              const int* __restrict__ active, cx<double>* H, cx<double>* hc);
__global__ void k_gmres_init(int R, const double* __restrict__ nrm_part, int nblk, int m, double* beta0,
                             cx<double>* gvec, int* active, int* kk, double* inv_nrm, double* resid);
__global__ void k_givens(int R, int k, int m, cx<double>* H, const double* __restrict__ nrm_part, int nblk,
                         double* cs_c, cx<double>* cs_s, cx<double>* gvec, const double* __restrict__ beta0,
                         double tol, int* active, int* kk, double* inv_nrm, double* resid, int* bad);
__global__ void k_hess_solve(int m, const cx<double>* __restrict__ H, const cx<double>* __restrict__ gvec,
                             const int* __restrict__ kk, cx<double>* y);

}  // namespace schur
