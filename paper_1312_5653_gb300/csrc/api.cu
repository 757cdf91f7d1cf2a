// C-ABI of libschur (declared in include/schur.h): context management, the FP64 outer
// refinement around the FETI-DP engine, the real-input shortcut, and host-buffer entry points.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/schur.h"
#include "engine.h"
#include "outer.h"
#include "api_internal.h"
#include "prof.h"

namespace {
thread_local std::string g_last_error;
}

namespace schur {

int set_error(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define API_CK(call)                                                                 \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      return set_error(e_ == cudaErrorMemoryAllocation ? SCHUR_ENOMEM : SCHUR_ECUDA, \
                       std::string(#call) + ": " + cudaGetErrorString(e_));          \
  } while (0)

template <class V>
static cudaError_t upload(V** dst, const std::vector<V>& src) {
  size_t bytes = std::max<size_t>(src.size() * sizeof(V), 16);
  cudaError_t e = cudaMalloc(dst, bytes);
  if (e != cudaSuccess) return e;
  if (!src.empty()) e = cudaMemcpy(*dst, src.data(), src.size() * sizeof(V), cudaMemcpyHostToDevice);
  return e;
}

int upload_maps(const HostMaps& hm, DevMaps* dm, std::string* msg) {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = upload(&dm->slot_node, hm.slot_node);
  if (e == cudaSuccess) e = upload(&dm->node_slot, hm.node_slot);
  if (e == cudaSuccess) e = upload(&dm->corner_node, hm.corner_node);
  if (e == cudaSuccess) e = upload(&dm->sd_code, hm.sd_code);
  if (e == cudaSuccess) e = upload(&dm->sd_cls, hm.sd_cls);
  if (e == cudaSuccess) e = upload(&dm->cls_code, hm.cls_code);
  if (e == cudaSuccess) e = upload(&dm->sd_lam, hm.sd_lam);
  if (e == cudaSuccess) e = upload(&dm->lam_side, hm.lam_side);
  if (e == cudaSuccess) e = upload(&dm->sd_corner, hm.sd_corner);
  if (e == cudaSuccess) e = upload(&dm->sd_minv, hm.sd_minv);
  if (e == cudaSuccess) e = upload(&dm->sd_coarse, hm.sd_coarse);
  if (e == cudaSuccess) e = upload(&dm->face_sd, hm.face_sd);
  if (e == cudaSuccess) e = upload(&dm->lam_face, hm.lam_face);
  if (e == cudaSuccess) e = upload(&dm->slot_faces, hm.slot_faces);
  if (e == cudaSuccess) e = upload(&dm->face_lam_ptr, hm.face_lam_ptr);
  if (e == cudaSuccess) e = upload(&dm->face_lam, hm.face_lam);
  if (e == cudaSuccess) e = upload(&dm->grp_sd, hm.grp_sd);
  if (e == cudaSuccess) e = upload(&dm->grp_ptr, hm.grp_ptr);
  if (e != cudaSuccess) {
    if (msg) *msg = std::string("uploading index maps: ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? SCHUR_ENOMEM : SCHUR_ECUDA;
  }
  return SCHUR_OK;
}

void free_maps(DevMaps* dm) {
  void* ps[] = {dm->slot_node, dm->node_slot, dm->corner_node, dm->sd_code, dm->sd_cls,
                dm->cls_code,  dm->sd_lam,    dm->lam_side,    dm->sd_corner, dm->sd_minv,
                dm->sd_coarse, dm->face_sd,   dm->lam_face,    dm->slot_faces, dm->face_lam_ptr, dm->face_lam,
                dm->grp_sd,    dm->grp_ptr};
  for (void* p : ps)
    if (p) cudaFree(p);
  *dm = DevMaps();
}

cudaError_t smem_attr(const void* func, int bytes) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, int>> set;  // (kernel, limit set so far)
  std::lock_guard<std::mutex> lk(mu);
  for (auto& kv : set)
    if (kv.first == func) {
      if (kv.second >= bytes) return cudaSuccess;
      cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      if (e == cudaSuccess) kv.second = bytes;
      return e;
    }
  cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) set.push_back({func, bytes});
  return e;
}

void configure_pool() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  cudaGetLastError();
  done[dev] = true;
}

MapEntry::~MapEntry() {
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != device) cudaSetDevice(device);
  free_maps(&dm);
  if (cur != device) cudaSetDevice(cur);
}

// Process-wide cache of partitions (host maps + device copies), keyed by device, mesh, nsub and
// local_mode; the most recently used kPartitionCache entries stay alive after their contexts.
namespace {
constexpr size_t kPartitionCache = 8;
std::mutex g_part_mu;
std::vector<std::pair<std::string, std::shared_ptr<MapEntry>>> g_parts;  // most recent last
}  // namespace

int get_partition(const schur_mesh* mesh, const schur_opts* opts, std::shared_ptr<MapEntry>* out, std::string* msg) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = -1;
  char key[160];
  const int d = mesh->dim;
  snprintf(key, sizeof(key), "%d|%d|%d,%d,%d|%d,%d,%d|%d|%d", dev, d, mesh->nel[0], mesh->nel[1],
           d == 3 ? mesh->nel[2] : 1, opts->nsub[0], opts->nsub[1], d == 3 ? opts->nsub[2] : 1, opts->local_mode,
           opts->augment);
  std::lock_guard<std::mutex> lk(g_part_mu);
  for (size_t i = 0; i < g_parts.size(); ++i)
    if (g_parts[i].first == key) {
      auto e = g_parts[i];
      g_parts.erase(g_parts.begin() + i);
      g_parts.push_back(e);
      *out = e.second;
      return SCHUR_OK;
    }
  auto e = std::make_shared<MapEntry>();
  e->device = dev;
  std::string m = build_maps(mesh->dim, mesh->nel, opts->nsub, opts->local_mode, &e->hm, opts->augment);
  if (!m.empty()) {
    if (msg) *msg = m;
    return SCHUR_EINVAL;
  }
  int rc = upload_maps(e->hm, &e->dm, msg);
  if (rc) return rc;
  g_parts.push_back({key, e});
  if (g_parts.size() > kPartitionCache) g_parts.erase(g_parts.begin());
  *out = e;
  return SCHUR_OK;
}

static double now_ms() {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int ctx_ensure_outer(schur_ctx* c, int R) {
  if (R <= c->wsR) return SCHUR_OK;
  if (c->z) cudaFree(c->z);
  if (c->res) cudaFree(c->res);
  if (c->part) cudaFree(c->part);
  if (c->h_part) cudaFreeHost(c->h_part);
  c->z = c->res = c->part = c->h_part = nullptr;
  const size_t n = (size_t)c->mp->hm.g.n;
  API_CK(cudaMalloc(&c->z, n * R * 2 * sizeof(double)));
  API_CK(cudaMalloc(&c->res, n * R * 2 * sizeof(double)));
  c->nblk = (int)std::min<long long>(4LL * 152, (c->mp->hm.g.n + 255) / 256);
  if (c->nblk < 1) c->nblk = 1;
  API_CK(cudaMalloc(&c->part, (size_t)R * c->nblk * 2 * sizeof(double)));
  API_CK(cudaMallocHost(&c->h_part, (size_t)R * c->nblk * 2 * sizeof(double)));
  c->wsR = R;
  return SCHUR_OK;
}

// Relative residuals ||f - A z|| / ||f|| for R columns (synchronises).  Leaves res = f - A z.
// z_zero: z is known to be zero (the first refinement step), so res = f without the stencil.
int ctx_residual(schur_ctx* c, const double* bre, const double* bim, int ldb, int R, cudaStream_t st, double* rel,
                 bool z_zero) {
  const Geom& g = c->mp->hm.g;
  Coef27 sten = make_coef(g, c->sim, c->sre);
  prof_start(KC_RESIDUAL, st);
  k_residual<<<dim3(c->nblk, R), 256, 0, st>>>(g, sten, bre, bim, ldb, reinterpret_cast<const cx<double>*>(c->z),
                                               (int)g.n, R, reinterpret_cast<cx<double>*>(c->res), c->part, c->nblk,
                                               z_zero ? 1 : 0);
  prof_stop(KC_RESIDUAL, st);
  API_CK(cudaGetLastError());
  ++c->launches;
  ++c->total_launches;
  API_CK(cudaMemcpyAsync(c->h_part, c->part, (size_t)R * c->nblk * 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  API_CK(cudaStreamSynchronize(st));
  for (int r = 0; r < R; ++r) {
    double sr = 0, sb = 0;
    for (int b = 0; b < c->nblk; ++b) {
      sr += c->h_part[((size_t)r * c->nblk + b) * 2];
      sb += c->h_part[((size_t)r * c->nblk + b) * 2 + 1];
    }
    rel[r] = sb > 0 ? std::sqrt(sr / sb) : (sr > 0 ? INFINITY : 0.0);
    if (!std::isfinite(sr)) rel[r] = NAN;
  }
  return SCHUR_OK;
}

// Outer refinement for R <= kMaxR columns: z accumulates in FP64 with z += FETI(b - A z) until
// ||b - A z|| / ||b|| <= tol.  Output: x (x != null) = -Im(z)/gamma for the complex factor (the
// real-input shortcut), Re(z) for the real factor K + gamma M; and/or z itself (zout != null).
int ctx_outer(schur_ctx* c, const double* bre, const double* bim, int ldb, int R, double* x, int ldx, double* zout,
              int ldz, cudaStream_t st, schur_stats* stats) {
  const Geom& g = c->mp->hm.g;
  int rc = ctx_ensure_outer(c, R);
  if (rc) return rc;
  API_CK(cudaMemsetAsync(c->z, 0, (size_t)g.n * R * 2 * sizeof(double), st));
  double rel[kMaxR];
  int steps = 0, iters_total = 0, iters_first = -1;
  int status = SCHUR_OK;
  const double inner_tol = c->opts.inner_tol > 0 ? c->opts.inner_tol : (c->opts.precision == SCHUR_MIXED ? 3e-5 : 1e-12);
  while (true) {
    rc = ctx_residual(c, bre, bim, ldb, R, st, rel, steps == 0);
    if (rc) return rc;
    double worst = 0;
    bool nan = false;
    for (int r = 0; r < R; ++r) {
      if (std::isnan(rel[r])) nan = true;
      worst = std::max(worst, rel[r]);
    }
    if (nan) {
      status = set_error(SCHUR_EBREAKDOWN, "non-finite residual");
      break;
    }
    if (stats) stats->rel_residual = worst;
    if (worst <= c->opts.tol) break;
    if (steps >= c->opts.max_refine) {
      status = set_error(SCHUR_ENOTCONV, "refinement did not reach the tolerance within max_refine steps");
      break;
    }
    InnerResult ir;
    std::string msg;
    rc = c->eng->inner_solve(c->res, (int)g.n, c->z, (int)g.n, R, inner_tol, c->opts.max_iter, st, &ir, &msg);
    c->launches += c->eng->launches;
    c->total_launches += c->eng->launches;
    if (rc) return set_error(rc, msg);
    ++steps;
    iters_total += ir.iters;
    if (iters_first < 0) iters_first = ir.iters;
  }
  if (x) {
    const dim3 grid(std::max(1, (int)std::min<long long>((g.n + 255) / 256, 4 * 152)), R);
    prof_start(KC_RESIDUAL, st);
    if (c->opts.factor == SCHUR_FACTOR_PW)
      k_real_part<<<grid, 256, 0, st>>>(g.n, reinterpret_cast<const cx<double>*>(c->z), (int)g.n, R, 1.0, x, ldx);
    else
      k_shortcut<<<grid, 256, 0, st>>>(g.n, reinterpret_cast<const cx<double>*>(c->z), (int)g.n, R, 1.0 / c->gamma,
                                       x, ldx);
    prof_stop(KC_RESIDUAL, st);
    API_CK(cudaGetLastError());
    ++c->launches;
    ++c->total_launches;
  }
  if (zout) {
    k_split_complex<<<dim3(std::max(1, (int)std::min<long long>((g.n + 255) / 256, 4 * 152)), R), 256, 0, st>>>(
        g.n, reinterpret_cast<const cx<double>*>(c->z), (int)g.n, R, zout, ldz);
    API_CK(cudaGetLastError());
    ++c->launches;
  }
  if (stats) {
    stats->outer_steps = std::max(stats->outer_steps, steps);
    stats->iters_total = std::max(stats->iters_total, iters_total);
    stats->iters_first = std::max(stats->iters_first, iters_first < 0 ? 0 : iters_first);
  }
  return status;
}

// S^{-1} b by the complex factor: one outer-refined complex solve and the shortcut.  S_p^{-1} b by
// the real factor A = K + gamma M (Sec. 3.2): w = A^{-1} b, t = M w, x = A^{-1} t, each solve
// refined in FP64 to the context's tolerance.
int ctx_schur_inverse(schur_ctx* c, const double* b, int ldb, int R, double* x, int ldx, cudaStream_t st,
                      schur_stats* stats) {
  if (c->opts.factor != SCHUR_FACTOR_PW) return ctx_outer(c, b, nullptr, ldb, R, x, ldx, nullptr, 0, st, stats);
  const Geom& g = c->mp->hm.g;
  const size_t n = (size_t)g.n;
  if (!c->pw_buf) API_CK(cudaMalloc(&c->pw_buf, 2 * n * kMaxR * sizeof(double)));
  double* w = c->pw_buf;
  double* t = c->pw_buf + n * kMaxR;
  schur_stats s1, s2;
  std::memset(&s1, 0, sizeof(s1));
  std::memset(&s2, 0, sizeof(s2));
  int rc1 = ctx_outer(c, b, nullptr, ldb, R, w, (int)n, nullptr, 0, st, &s1);
  if (rc1 && rc1 != SCHUR_ENOTCONV) return rc1;
  Coef27 sten = make_coef(g, 1.0);
  const int grid = std::max(1, (int)std::min<long long>((g.n + 255) / 256, 8 * 152));
  k_apply_real<<<dim3(grid, R), 256, 0, st>>>(g, sten, 0, w, (int)n, t, (int)n, R, 1.0, 0.0);
  API_CK(cudaGetLastError());
  ++c->launches;
  ++c->total_launches;
  int rc2 = ctx_outer(c, t, nullptr, (int)n, R, x, ldx, nullptr, 0, st, &s2);
  if (rc2 && rc2 != SCHUR_ENOTCONV) return rc2;
  if (stats) {
    stats->outer_steps = std::max(stats->outer_steps, s1.outer_steps + s2.outer_steps);
    stats->iters_total = std::max(stats->iters_total, s1.iters_total + s2.iters_total);
    stats->iters_first = std::max(stats->iters_first, s1.iters_first);
    stats->rel_residual = std::max(s1.rel_residual, s2.rel_residual);
  }
  return rc1 ? rc1 : rc2;
}

}  // namespace schur

using namespace schur;

extern "C" {

void schur_default_opts(schur_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->nsub[0] = o->nsub[1] = o->nsub[2] = 4;
  o->precision = SCHUR_FP64;
  o->tol = 1e-12;
  o->inner_tol = 0;
  o->max_iter = 300;
  o->max_refine = 8;
  o->local_mode = SCHUR_LOCAL_PER_SUBDOMAIN;
}

const char* schur_strerror(int code) {
  switch (code) {
    case SCHUR_OK: return "ok";
    case SCHUR_EINVAL: return "invalid argument";
    case SCHUR_ENOMEM: return "out of memory";
    case SCHUR_ENOTCONV: return "tolerance not reached";
    case SCHUR_EBREAKDOWN: return "numerical breakdown";
    case SCHUR_ETIMEOUT: return "timeout";
    case SCHUR_ECUDA: return "CUDA error";
    case SCHUR_EBUSY: return "busy";
    default: return "unknown error";
  }
}

const char* schur_last_error(void) { return g_last_error.c_str(); }

long long schur_ndof(const schur_mesh* mesh) {
  if (!mesh || (mesh->dim != 2 && mesh->dim != 3)) return -1;
  long long n = 1;
  for (int a = 0; a < mesh->dim; ++a) {
    if (mesh->nel[a] < 2) return -1;
    n *= mesh->nel[a] - 1;
  }
  return n;
}

int schur_setup(const schur_mesh* mesh, double beta, const schur_opts* opts, void* stream, schur_ctx** out) {
  if (!out) return set_error(SCHUR_EINVAL, "out is NULL");
  *out = nullptr;
  if (!mesh || !opts) return set_error(SCHUR_EINVAL, "mesh or opts is NULL");
  if (!(beta > 0) || !std::isfinite(beta)) return set_error(SCHUR_EINVAL, "beta must be positive and finite");
  if (opts->precision != SCHUR_FP64 && opts->precision != SCHUR_MIXED)
    return set_error(SCHUR_EINVAL, "unknown precision");
  if (opts->local_mode != SCHUR_LOCAL_PER_SUBDOMAIN && opts->local_mode != SCHUR_LOCAL_SHARED)
    return set_error(SCHUR_EINVAL, "unknown local_mode");
  if (!(opts->tol > 0) || opts->max_iter < 1 || opts->max_iter >= kMaxKdev || opts->max_refine < 0)
    return set_error(SCHUR_EINVAL, "tol must be > 0, 1 <= max_iter < 512, max_refine >= 0");
  if (opts->tc_split != 0 && opts->tc_split != 1 && opts->tc_split != 3)
    return set_error(SCHUR_EINVAL, "tc_split must be 0, 1 or 3");
  if (opts->factor != SCHUR_FACTOR_EXACT && opts->factor != SCHUR_FACTOR_PW)
    return set_error(SCHUR_EINVAL, "factor must be SCHUR_FACTOR_EXACT or SCHUR_FACTOR_PW");
  if (opts->augment != 0 && opts->augment != 1) return set_error(SCHUR_EINVAL, "augment must be 0 or 1");
  for (int i = 0; i < 2; ++i)
    if (opts->reserved[i]) return set_error(SCHUR_EINVAL, "reserved option fields must be zero");
  double t0 = now_ms();
  schur_ctx* c = new (std::nothrow) schur_ctx();
  if (!c) return set_error(SCHUR_ENOMEM, "host allocation failed");
  c->mesh = *mesh;
  c->opts = *opts;
  c->beta = beta;
  c->gamma = 1.0 / std::sqrt(beta);
  c->sre = opts->factor == SCHUR_FACTOR_PW ? c->gamma : 0.0;
  c->sim = opts->factor == SCHUR_FACTOR_PW ? 0.0 : c->gamma;
  std::string msg;
  int rc = get_partition(mesh, opts, &c->mp, &msg);
  if (rc) {
    delete c;
    return set_error(rc, msg);
  }
  c->eng = opts->precision == SCHUR_MIXED ? make_engine_f32(&c->mp->hm, &c->mp->dm, c->sim, c->sre)
                                          : make_engine_f64(&c->mp->hm, &c->mp->dm, c->sim, c->sre);
  if (!c->eng) {
    schur_destroy(c);
    return set_error(SCHUR_ENOMEM, "engine allocation failed");
  }
  c->eng->tc_terms = opts->tc_split == 1 ? 1 : 3;
  rc = c->eng->setup(reinterpret_cast<cudaStream_t>(stream), &msg);
  if (rc) {
    schur_destroy(c);
    return set_error(rc, msg);
  }
  c->ms_setup = now_ms() - t0;
  c->total_launches = c->eng->launches;
  *out = c;
  return SCHUR_OK;
}

static int check_vec_args(schur_ctx* c, const void* a, const void* b, int nrhs, int ld, long long mult) {
  if (!c) return set_error(SCHUR_EINVAL, "ctx is NULL");
  if (nrhs < 0) return set_error(SCHUR_EINVAL, "nrhs < 0");
  if (nrhs == 0) return SCHUR_OK;
  if (!a || !b) return set_error(SCHUR_EINVAL, "NULL vector");
  if ((long long)ld < mult * c->mp->hm.g.n) return set_error(SCHUR_EINVAL, "ld smaller than the vector length");
  return SCHUR_OK;
}

int schur_solve(schur_ctx* c, const double* b, double* x, int nrhs, int ld, void* stream, schur_stats* st) {
  int rc = check_vec_args(c, b, x, nrhs, ld, 1);
  if (rc) return rc;
  double t0 = now_ms();
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->ms_setup = c->ms_setup;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  c->launches = 0;
  int status = SCHUR_OK;
  for (int r0 = 0; r0 < nrhs; r0 += kMaxR) {
    int R = std::min(kMaxR, nrhs - r0);
    rc = ctx_schur_inverse(c, b + (size_t)r0 * ld, ld, R, x + (size_t)r0 * ld, ld, s, st);
    if (rc == SCHUR_ENOTCONV) status = rc;
    else if (rc) {
      if (st) st->status = rc;
      return rc;
    }
  }
  if (st) {
    st->status = status;
    st->ms_solve = now_ms() - t0;
  }
  return status;
}

int schur_complex_solve(schur_ctx* c, const double* bre, const double* bim, double* z, int nrhs, int ld, void* stream,
                        schur_stats* st) {
  int rc = check_vec_args(c, bre, z, nrhs, ld, 1);
  if (rc) return rc;
  double t0 = now_ms();
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->ms_setup = c->ms_setup;
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  c->launches = 0;
  int status = SCHUR_OK;
  for (int r0 = 0; r0 < nrhs; r0 += kMaxR) {
    int R = std::min(kMaxR, nrhs - r0);
    rc = ctx_outer(c, bre + (size_t)r0 * ld, bim ? bim + (size_t)r0 * ld : nullptr, ld, R, nullptr, 0,
                   z + (size_t)r0 * ld * 2, ld, s, st);
    if (rc == SCHUR_ENOTCONV) status = rc;
    else if (rc) return rc;
  }
  API_CK(cudaStreamSynchronize(s));
  if (st) {
    st->status = status;
    st->ms_solve = now_ms() - t0;
  }
  return status;
}

int schur_solve_host(schur_ctx* c, const double* bh, double* xh, int nrhs, int ld, void* stream, schur_stats* st) {
  int rc = check_vec_args(c, bh, xh, nrhs, ld, 1);
  if (rc || nrhs == 0) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  size_t bytes = (size_t)ld * nrhs * sizeof(double);
  if (bytes > c->host_cap) {
    if (c->hb) cudaFree(c->hb);
    if (c->hx) cudaFree(c->hx);
    c->hb = c->hx = nullptr;
    c->host_cap = 0;
    API_CK(cudaMalloc(&c->hb, bytes));
    API_CK(cudaMalloc(&c->hx, bytes));
    c->host_cap = bytes;
  }
  double t0 = now_ms();
  API_CK(cudaMemcpyAsync(c->hb, bh, bytes, cudaMemcpyHostToDevice, s));
  rc = schur_solve(c, c->hb, c->hx, nrhs, ld, stream, st);
  if (rc && rc != SCHUR_ENOTCONV) return rc;
  API_CK(cudaMemcpyAsync(xh, c->hx, bytes, cudaMemcpyDeviceToHost, s));
  API_CK(cudaStreamSynchronize(s));
  if (st) st->ms_solve = now_ms() - t0;
  return rc;
}

static int apply_real(schur_ctx* c, int mode, const double* x, double* y, int nrhs, int ld, void* stream) {
  int rc = check_vec_args(c, x, y, nrhs, ld, 1);
  if (rc || nrhs == 0) return rc;
  const Geom& g = c->mp->hm.g;
  Coef27 sten = make_coef(g, 1.0);
  int grid = std::max(1, (int)std::min<long long>((g.n + 255) / 256, 8 * 152));
  k_apply_real<<<dim3(grid, nrhs), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(g, sten, mode, x, ld, y, ld, nrhs,
                                                                                       1.0, 0.0);
  API_CK(cudaGetLastError());
  return SCHUR_OK;
}

int schur_apply_mass(schur_ctx* c, const double* x, double* y, int nrhs, int ld, void* stream) {
  return apply_real(c, 0, x, y, nrhs, ld, stream);
}
int schur_apply_stiffness(schur_ctx* c, const double* x, double* y, int nrhs, int ld, void* stream) {
  return apply_real(c, 1, x, y, nrhs, ld, stream);
}

long long schur_launch_count(const schur_ctx* c) { return c ? c->total_launches : -1; }

int schur_get_info(const schur_ctx* c, schur_info_t* info) {
  if (!c || !info) return set_error(SCHUR_EINVAL, "NULL argument");
  const Geom& g = c->mp->hm.g;
  info->n = g.n;
  info->n_sub = g.nsd;
  info->n_classes = c->mp->hm.ncls;
  info->n_lambda = g.nlam;
  info->n_coarse = g.nco;
  info->n_delta = g.nD;
  info->n_local = g.nl;
  info->bytes_operators = c->eng ? c->eng->op_bytes() : 0;
  return SCHUR_OK;
}

int schur_debug_operator(schur_ctx* c, int which, int cls, double* out, long long cap) {
  if (!c || !out) return set_error(SCHUR_EINVAL, "NULL argument");
  std::string msg;
  int rc = c->eng->debug_operator(which, cls, out, cap, nullptr, &msg);
  if (rc) return set_error(rc, msg.empty() ? "bad operator request" : msg);
  return SCHUR_OK;
}

void schur_destroy(schur_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  delete c->eng;
  c->mp.reset();
  if (c->z) cudaFree(c->z);
  if (c->res) cudaFree(c->res);
  if (c->part) cudaFree(c->part);
  if (c->h_part) cudaFreeHost(c->h_part);
  if (c->hb) cudaFree(c->hb);
  if (c->hx) cudaFree(c->hx);
  if (c->pw_buf) cudaFree(c->pw_buf);
  kkt_free(c);
  delete c;
}

}  // extern "C"
