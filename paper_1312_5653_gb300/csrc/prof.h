// Optional per-category kernel timing with CUDA events recorded on the launching stream.
#pragma once
#include <cuda_runtime.h>

namespace schur {

enum KCat {
  KC_FACTOR = 0,      // batched block LDL^T of subdomain matrices
  KC_FORM = 1,        // local operator formation (multi-RHS layered solves)
  KC_COARSE_SETUP = 2,// coarse assembly and block cyclic reduction
  KC_LOCAL_RHS = 3,   // local right-hand-side solves
  KC_APPLY_F = 4,     // local dual operator apply (gather fused)
  KC_APPLY_S = 5,     // local Dirichlet operator apply (gather fused)
  KC_SCATTER = 6,     // jump-operator scatter (and dual right-hand side)
  KC_COARSE_APPLY = 7,// coarse inverse apply
  KC_CORNER = 8,      // corner gathers
  KC_GMRES_DOTS = 9,  // Gram-Schmidt dot products
  KC_GMRES_UPDATE = 10,
  KC_GMRES_OTHER = 11,// norms, Givens, scaling, combination
  KC_RECOVER = 12,    // primal recovery solves
  KC_ASSEMBLE = 13,   // z assembly
  KC_RESIDUAL = 14,   // FP64 refinement residual and shortcut
  KC_COARSE_INV = 15, // coarse inverse columns (and precision conversion)
  KC_INTERIOR = 16,   // interior factor and Dirichlet S (second setup stream)
  KC_FORM_CORNER = 17,// corner columns of the local operators formed ahead of F (2D, corner coarse)
  KC_N = 18
};

// start/stop brackets around one launch; no-ops unless the category is enabled
void prof_start(int cat, cudaStream_t st);
void prof_stop(int cat, cudaStream_t st);

}  // namespace schur
