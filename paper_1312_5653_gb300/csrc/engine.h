// Host interface of the FETI-DP engine (one per context and working precision).
#pragma once
#include <cuda_runtime.h>

#include <string>

#include "maps.h"

namespace schur {

// Device copies of the index maps (uploaded once per context).
struct DevMaps {
  int* slot_node = nullptr;
  int* node_slot = nullptr;
  int* corner_node = nullptr;
  int* sd_code = nullptr;
  int* sd_cls = nullptr;
  int* cls_code = nullptr;
  int* sd_lam = nullptr;
  int* lam_side = nullptr;
  int* sd_corner = nullptr;
  double* sd_minv = nullptr;
  int* sd_coarse = nullptr;
  int* face_sd = nullptr;
  int* lam_face = nullptr;
  int* slot_faces = nullptr;
  int* face_lam_ptr = nullptr;
  int* face_lam = nullptr;
  int* grp_sd = nullptr;
  int* grp_ptr = nullptr;
};

int upload_maps(const HostMaps& hm, DevMaps* dm, std::string* msg);
void free_maps(DevMaps* dm);

struct InnerResult {
  int iters = 0;        // GMRES iterations (max over right-hand sides)
  int converged = 1;    // all right-hand sides met the inner tolerance
};

class EngineBase {
 public:
  virtual ~EngineBase() {}
  // Builds factors and operators (synchronises `st`).  Returns SCHUR_* code.
  virtual int setup(cudaStream_t st, std::string* msg) = 0;
  // One FETI-DP solve of A dz = f for R <= kMaxR columns; f, z interleaved complex FP64 with
  // leading dimensions ldf, ldz (complex entries); z += dz.  Synchronises `st`.
  virtual int inner_solve(const double* f, int ldf, double* z, int ldz, int R, double tol, int max_iter,
                          cudaStream_t st, InnerResult* res, std::string* msg) = 0;
  virtual long long op_bytes() const = 0;
  virtual int debug_operator(int which, int cls, double* out, long long cap, cudaStream_t st,
                             std::string* msg) = 0;
  // Kernel launches issued by the most recent inner_solve.
  long long launches = 0;
  // Tensor-core products per layer chunk of the 3D FP32 formation: 3 (TF32 split, FP32 accuracy) or 1.
  int tc_terms = 3;
};

constexpr int kMaxR = 16;
// Largest augmented coarse problem (corners + faces): inverted densely in FP64.
constexpr int kMaxAugCoarse = 4096;

// Keeps freed blocks of the current device's default memory pool cached in the process
// (release threshold = unlimited), once per device.
void configure_pool();

// The engine solves with A = K + (sre + i gamma) M: sre = 0 for the complex factor of Sec. 4,
// sre = gamma, gamma = 0 for the real factor K + gamma M of the Pearson-Wathen S_p (Sec. 3.2).
EngineBase* make_engine_f64(const HostMaps* hm, const DevMaps* dm, double gamma, double sre);
EngineBase* make_engine_f32(const HostMaps* hm, const DevMaps* dm, double gamma, double sre);

}  // namespace schur
