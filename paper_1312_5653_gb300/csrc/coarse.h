// Coarse problems: block cyclic reduction of the corner problem and its explicit inverse
// (coarse_bcr.cu); dense inversion of the augmented coarse matrix (coarse_dense.cu).
#pragma once
#include <string>
#include <vector>

#include "layered.cuh"

namespace schur {
// Level 0 of the reduction kept as blocks for the solve (precision T, b x b row-major blocks, one
// per layer eliminated at level 0, in elimination order): D0 = D_j^{-1}, Lp0 = A_pj D_j^{-1},
// Lq0 = D_j^{-1} A_jq (undefined where j has no such neighbour).
template <class T>
struct BcrLevel0 {
  cx<T>* D0;
  cx<T>* Lp0;
  cx<T>* Lq0;
};
// Block cyclic reduction of the coarse matrix (assembled and factorised in FP64) and the explicit
// inverse in precision T.  Without split the inverse of the whole coarse matrix is written to Kinv
// (n_c rows of ldk >= n_c entries); with split the level-0 blocks go to *split and Kinv receives the
// inverse of the reduced matrix on the layers that survive level 0 (b * Lr rows, compact layer
// order).  Entries past the row length are not defined.  Returns SCHUR_* code; *launches counts
// kernel launches.
template <class T>
int coarse_bcr(const StoredProv<double>& P, const BcrLevel0<T>* split, cx<T>* Kinv, int ldk, int* err, cudaStream_t st,
               std::string* msg, long long* launches);
// Level 0 of the reduction over L layers: tgt[5 c..] = (t, jr, kr, jl, kl) for the c-th surviving
// layer t with its eliminated right neighbour jr (k-th entry kr of the elimination order, t = p of
// jr) and left neighbour jl (kl, t = q of jl), -1 if none; elim[3 k..] = (j, cp, cq) for the k-th
// eliminated layer with the compact indices of its neighbours p, q (-1 if none); rem = surviving
// layers in order.
void bcr_level0_maps(int L, std::vector<int>* tgt, std::vector<int>* elim, std::vector<int>* rem);
// In-place inverse of the dense complex n x n matrix A (row-major, FP64) by Gauss-Jordan elimination
// without pivoting in panels of 32 pivots; *err is set on a zero or non-finite pivot.  Returns 0,
// SCHUR_ENOMEM or SCHUR_ECUDA.
int dense_gj_inverse(cx<double>* A, int n, int* err, cudaStream_t st, std::string* msg, long long* launches);
}  // namespace schur
