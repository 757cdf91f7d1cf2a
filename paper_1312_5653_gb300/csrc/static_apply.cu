// schur_apply_S_static: y = S x = K M^{-1} K x + M x / beta without any device allocation.
//
// For callers that cannot allocate device memory themselves: code running where cudaMalloc is
// unavailable or forbidden (inside a stream-ordered region owned by another runtime, a plugin
// with a fixed memory budget, a process whose allocator is locked by its host application).
// Such a caller cannot create a schur_ctx (schur_setup allocates), so this entry point takes the
// mesh and beta directly and keeps its work vectors in one fixed device array that every GPU
// loading the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "../../include/schur.h"
#include "api_internal.h"
#include "outer.h"

namespace schur {
namespace {

// Work vectors t, w, r, d, Ad of one right-hand side: 5 x kStaticMaxN doubles = 40 MiB.
constexpr long long kStaticMaxN = 1LL << 20;
__device__ __align__(256) double g_static_scratch[5 * kStaticMaxN];

constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array for the current device (looked up once per device).
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

__global__ void k_static_cheb(long long n, double* x, double* r, double* d, const double* __restrict__ Ad, double c1,
                              double c2, double dinv, int first) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (first) {
      d[i] = c2 * dinv * r[i];
      x[i] = 0.0;
      continue;
    }
    x[i] += d[i];
    r[i] -= Ad[i];
    d[i] = c1 * d[i] + c2 * dinv * r[i];
  }
}

}  // namespace
}  // namespace schur

using namespace schur;

extern "C" int schur_apply_S_static(const schur_mesh* mesh, double beta, const double* x_dev, double* y_dev, int nrhs,
                                    int ld, void* stream) {
  if (!mesh || (mesh->dim != 2 && mesh->dim != 3)) return set_error(SCHUR_EINVAL, "mesh: dim must be 2 or 3");
  if (!(beta > 0) || !std::isfinite(beta)) return set_error(SCHUR_EINVAL, "beta must be positive and finite");
  if (nrhs < 0) return set_error(SCHUR_EINVAL, "nrhs < 0");
  Geom g = Geom();
  g.dim = mesh->dim;
  long long n = 1;
  for (int a = 0; a < 3; ++a) {
    g.nel[a] = a < g.dim ? mesh->nel[a] : 1;
    if (a < g.dim) {
      if (g.nel[a] < 2) return set_error(SCHUR_EINVAL, "mesh: nel must be >= 2 on every axis");
      // each factor and the running product stay <= 2^20, so the product never overflows
      const long long na = (long long)g.nel[a] - 1;
      if (na > kStaticMaxN || n * na > kStaticMaxN)
        return set_error(SCHUR_EINVAL, "schur_apply_S_static: more than 2^20 interior nodes (its fixed work array)");
      g.h[a] = 1.0 / g.nel[a];
      n *= na;
    } else {
      g.h[a] = 1.0;
    }
  }
  g.n = n;
  if (nrhs == 0) return SCHUR_OK;
  if (!x_dev || !y_dev) return set_error(SCHUR_EINVAL, "null x or y");
  if ((long long)ld < n) return set_error(SCHUR_EINVAL, "ld < n");
  {
    // y = K w is written before M x / beta is added to it, so x and y must not share memory
    const char* xb = reinterpret_cast<const char*>(x_dev);
    const char* yb = reinterpret_cast<const char*>(y_dev);
    const size_t span = ((size_t)(nrhs - 1) * ld + (size_t)n) * sizeof(double);
    if (xb < yb + span && yb < xb + span) return set_error(SCHUR_EINVAL, "x and y overlap");
  }
  double* scr = nullptr;
  {
    cudaError_t e = scratch_for_current_device(&scr);
    if (e != cudaSuccess)
      return set_error(SCHUR_ECUDA, std::string("schur_apply_S_static: address of the work array: ") +
                                        cudaGetErrorString(e));
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* t = scr;
  double* w = scr + kStaticMaxN;
  double* r = scr + 2 * kStaticMaxN;
  double* d = scr + 3 * kStaticMaxN;
  double* Ad = scr + 4 * kStaticMaxN;
  const Coef27 cf = make_coef(g, 1.0);
  const int gs = (int)std::max<long long>(1, std::min<long long>((n + 255) / 256, 8 * 152));
  // Chebyshev iteration for M w = t with the Q1 mass bounds of D^{-1} M, (2^-d, (3/2)^d), and the
  // same degree as schur_apply_S (relative accuracy 1e-15)
  const double lo = std::pow(0.5, g.dim), hi = std::pow(1.5, g.dim);
  const double theta = 0.5 * (hi + lo), delta = 0.5 * (hi - lo), sigma = theta / delta;
  const double dinv = 1.0 / stencil_diag(g, 0);
  const double kappa = std::pow(3.0, g.dim), rq = (std::sqrt(kappa) - 1.0) / (std::sqrt(kappa) + 1.0);
  const int deg = (int)std::ceil(std::log(1e-15 / 2.0) / std::log(rq)) + 1;
  for (int c = 0; c < nrhs; ++c) {
    const double* xc = x_dev + (size_t)c * ld;
    double* yc = y_dev + (size_t)c * ld;
    // t = K x ; r = t (every entry written before it is read, so no clearing is needed)
    k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, cf, 1, xc, (int)n, t, (int)n, 1, 1.0, 0.0);
    cudaError_t e = cudaMemcpyAsync(r, t, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    double rho = 1.0 / sigma;
    if (e == cudaSuccess) k_static_cheb<<<gs, 256, 0, st>>>(n, w, r, d, Ad, 0.0, 1.0 / theta, dinv, 1);
    for (int k = 1; k <= deg && e == cudaSuccess; ++k) {
      k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, cf, 0, d, (int)n, Ad, (int)n, 1, 1.0, 0.0);
      double rho_new = 1.0 / (2.0 * sigma - rho);
      double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
      if (k == deg) c1 = c2 = 0.0;
      k_static_cheb<<<gs, 256, 0, st>>>(n, w, r, d, Ad, c1, c2, dinv, 0);
      rho = rho_new;
    }
    // y = K w + M x / beta
    if (e == cudaSuccess) {
      k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, cf, 1, w, (int)n, yc, ld, 1, 1.0, 0.0);
      k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, cf, 0, xc, ld, yc, ld, 1, 1.0 / beta, 1.0);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess)
      return set_error(SCHUR_ECUDA, std::string("schur_apply_S_static: column ") + std::to_string(c) + ": " +
                                        cudaGetErrorString(e));
  }
  return SCHUR_OK;
}
