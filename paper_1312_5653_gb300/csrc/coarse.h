// Cluster-parallel FP64 layered factorisation of the coarse corner matrix (see coarse.cu).
#pragma once
#include "layered.cuh"

namespace schur {

size_t coarse_cluster_smem(int b, int cluster);
// Launches the factorisation on the largest cluster size (16, 8, ...) the device accepts.
cudaError_t coarse_factor_cluster(const StoredProv<double>& P, cx<double>* Dinv, int* err, cudaStream_t st,
                                  int* cluster_used);

}  // namespace schur
