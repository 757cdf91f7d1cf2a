// Internal layout of the opaque schur_ctx and helpers shared by the C-ABI translation units.
#pragma once
#include <memory>
#include <string>

#include "../../include/schur.h"
#include "engine.h"
#include "maps.h"


namespace schur {
// Partition of one (mesh, nsub, local_mode): host maps and their device copies, shared by every
// context on the same device that uses that partition (it does not depend on beta).
struct MapEntry {
  HostMaps hm;
  DevMaps dm;
  int device = 0;
  ~MapEntry();
};
}  // namespace schur

struct schur_ctx {
  std::shared_ptr<schur::MapEntry> mp;
  schur::EngineBase* eng = nullptr;
  schur_mesh mesh;
  schur_opts opts;
  double beta = 0, gamma = 0, ms_setup = 0;
  // the factor the engine solves with: A = K + (sre + i sim) M (sim = gamma, sre = 0 for the complex
  // factor of Sec. 4; sre = gamma, sim = 0 for the real factor of the Pearson-Wathen S_p)
  double sre = 0, sim = 0;
  // S_p solves: the first factor solve's result and its mass product (n x kMaxR each)
  double* pw_buf = nullptr;
  long long launches = 0;        // kernels launched by the most recent solve call
  long long total_launches = 0;  // kernels launched through this context since setup
  // FP64 outer refinement workspace
  int wsR = 0, nblk = 1;
  double* z = nullptr;      // complex, n x wsR
  double* res = nullptr;    // complex, n x wsR
  double* part = nullptr;   // norm partials
  double* h_part = nullptr; // pinned host copy
  // host-buffer entry points
  double* hb = nullptr;
  double* hx = nullptr;
  size_t host_cap = 0;
  // full-space (KKT) workspace
  int kkt_R = 0;
  double* kkt_buf = nullptr;
  double* kkt_part = nullptr;
  double* kkt_hpart = nullptr;
  double* kkt_coef = nullptr;
};

namespace schur {
int set_error(int code, const std::string& msg);
int ctx_ensure_outer(schur_ctx* c, int R);
int ctx_outer(schur_ctx* c, const double* bre, const double* bim, int ldb, int R, double* x, int ldx, double* zout,
              int ldz, cudaStream_t st, schur_stats* stats);
// x = S^{-1} b (exact factor) or x = S_p^{-1} b (Pearson-Wathen factor) for R <= kMaxR columns
int ctx_schur_inverse(schur_ctx* c, const double* b, int ldb, int R, double* x, int ldx, cudaStream_t st,
                      schur_stats* stats);
void kkt_free(schur_ctx* c);
int get_partition(const schur_mesh* mesh, const schur_opts* opts, std::shared_ptr<MapEntry>* out, std::string* msg);
}  // namespace schur
