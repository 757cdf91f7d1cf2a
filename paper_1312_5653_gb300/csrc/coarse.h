// Coarse problems: block cyclic reduction of the corner problem and its explicit inverse
// (coarse_bcr.cu); dense inversion of the augmented coarse matrix (coarse_dense.cu).
#pragma once
#include <string>

#include "layered.cuh"

namespace schur {
// Block cyclic reduction of the coarse matrix (assembled in FP64) and its explicit inverse, both in
// precision T; the inverse is written to Kinv (n_c rows of ldk >= n_c entries; entries past n_c in
// a row are not defined).  Returns SCHUR_* code; *launches counts kernel launches.
template <class T>
int coarse_bcr(const StoredProv<double>& P, cx<T>* Kinv, int ldk, int* err, cudaStream_t st, std::string* msg,
               long long* launches);
// In-place inverse of the dense complex n x n matrix A (row-major, FP64) by Gauss-Jordan elimination
// without pivoting in panels of 32 pivots; *err is set on a zero or non-finite pivot.  Returns 0,
// SCHUR_ENOMEM or SCHUR_ECUDA.
int dense_gj_inverse(cx<double>* A, int n, int* err, cudaStream_t st, std::string* msg, long long* launches);
}  // namespace schur
