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

#include "../../include/schur.h"
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
  if (!mesh || (mesh->dim != 2 && mesh->dim != 3) || !(beta > 0) || !std::isfinite(beta) || nrhs < 0)
    return SCHUR_EINVAL;
  Geom g = Geom();
  g.dim = mesh->dim;
  long long n = 1;
  for (int a = 0; a < 3; ++a) {
    g.nel[a] = a < g.dim ? mesh->nel[a] : 1;
    if (a < g.dim) {
      if (g.nel[a] < 2) return SCHUR_EINVAL;
      g.h[a] = 1.0 / g.nel[a];
      n *= g.nel[a] - 1;
    } else {
      g.h[a] = 1.0;
    }
  }
  g.n = n;
  if (n > kStaticMaxN) return SCHUR_EINVAL;  // the fixed scratch holds one vector set of 2^20 nodes
  if (nrhs == 0) return SCHUR_OK;
  if (!x_dev || !y_dev || (long long)ld < n) return SCHUR_EINVAL;
  double* scr = nullptr;
  if (scratch_for_current_device(&scr) != cudaSuccess) return SCHUR_ECUDA;
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
    if (cudaMemcpyAsync(r, t, (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
      return SCHUR_ECUDA;
    double rho = 1.0 / sigma;
    k_static_cheb<<<gs, 256, 0, st>>>(n, w, r, d, Ad, 0.0, 1.0 / theta, dinv, 1);
    for (int k = 1; k <= deg; ++k) {
      k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, cf, 0, d, (int)n, Ad, (int)n, 1, 1.0, 0.0);
      double rho_new = 1.0 / (2.0 * sigma - rho);
      double c1 = rho_new * rho, c2 = 2.0 * rho_new / delta;
      if (k == deg) c1 = c2 = 0.0;
      k_static_cheb<<<gs, 256, 0, st>>>(n, w, r, d, Ad, c1, c2, dinv, 0);
      rho = rho_new;
    }
    // y = K w + M x / beta
    k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, cf, 1, w, (int)n, yc, ld, 1, 1.0, 0.0);
    k_apply_real<<<dim3(gs, 1), 256, 0, st>>>(g, cf, 0, xc, ld, yc, ld, 1, 1.0 / beta, 1.0);
    if (cudaGetLastError() != cudaSuccess) return SCHUR_ECUDA;
  }
  return SCHUR_OK;
}
