// Coarse corner problem: block cyclic reduction and its explicit inverse (coarse_bcr.cu).
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
}  // namespace schur
