// Cluster-parallel FP64 layered factorisation of the coarse corner matrix (see coarse.cu).
#pragma once
#include <string>

#include "layered.cuh"

namespace schur {

size_t coarse_cluster_smem(int b, int cluster);
// Launches the factorisation on the largest cluster size (16, 8, ...) the device accepts.
cudaError_t coarse_factor_cluster(const StoredProv<double>& P, cx<double>* Dinv, int* err, cudaStream_t st,
                                  int* cluster_used);

}  // namespace schur

namespace schur {
// Block cyclic reduction of the coarse matrix (FP64 factor) and its explicit inverse in precision
// T written to Kinv (n_c x n_c).  Returns SCHUR_* code; *launches counts kernel launches.
template <class T>
int coarse_bcr(const StoredProv<double>& P, cx<T>* Kinv, int* err, cudaStream_t st, std::string* msg,
               long long* launches);
}  // namespace schur
