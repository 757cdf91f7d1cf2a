// Per-category kernel timing: an event pair recorded on the launching stream around each launch of
// an enabled category; totals are read after a device synchronisation.
#include <mutex>
#include <vector>

#include "../../include/schur.h"
#include "prof.h"

namespace schur {
namespace {
std::mutex g_mu;
unsigned g_mask = 0;
struct Pair {
  int cat;
  cudaEvent_t a, b;
};
std::vector<Pair> g_open[KC_N];  // started, not stopped (stack per category)
std::vector<Pair> g_done;
std::vector<cudaEvent_t> g_pool;
const char* kNames[KC_N] = {"factor",         "form",        "coarse_setup", "local_rhs",   "apply_F",
                            "apply_S",        "scatter",     "coarse_apply", "corner",      "gmres_dots",
                            "gmres_update",   "gmres_other", "recover",      "assemble_z",  "residual",
                            "coarse_inverse", "interior",    "form_corner"};

cudaEvent_t take() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void prof_start(int cat, cudaStream_t st) {
  if (!(g_mask >> cat & 1u)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  Pair p{cat, take(), nullptr};
  cudaEventRecord(p.a, st);
  g_open[cat].push_back(p);
}

void prof_stop(int cat, cudaStream_t st) {
  if (!(g_mask >> cat & 1u)) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_open[cat].empty()) return;
  Pair p = g_open[cat].back();
  g_open[cat].pop_back();
  p.b = take();
  cudaEventRecord(p.b, st);
  g_done.push_back(p);
}

}  // namespace schur

using namespace schur;

extern "C" {

int schur_profile_begin(unsigned mask) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_mask = mask;
  return SCHUR_OK;
}

int schur_profile_end(schur_kernel_time* out, int cap, int* count) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_mask = 0;
  cudaError_t e = cudaDeviceSynchronize();
  double tot[KC_N] = {0};
  long long cnt[KC_N] = {0};
  for (auto& p : g_done) {
    float ms = 0;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) {
      tot[p.cat] += ms;
      cnt[p.cat] += 1;
    }
    g_pool.push_back(p.a);
    g_pool.push_back(p.b);
  }
  g_done.clear();
  for (int c = 0; c < KC_N; ++c) {
    for (auto& p : g_open[c]) g_pool.push_back(p.a);
    g_open[c].clear();
  }
  int n = 0;
  for (int c = 0; c < KC_N; ++c) {
    if (!cnt[c]) continue;
    if (out && n < cap) {
      out[n].category = c;
      out[n].launches = cnt[c];
      out[n].total_ms = tot[c];
    }
    ++n;
  }
  if (count) *count = n;
  return e == cudaSuccess ? SCHUR_OK : SCHUR_ECUDA;
}

const char* schur_kernel_category_name(int category) {
  return (category >= 0 && category < KC_N) ? kNames[category] : "unknown";
}

}  // extern "C"
