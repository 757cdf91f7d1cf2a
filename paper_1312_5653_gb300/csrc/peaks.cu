// Arithmetic peak probes: the denominators of the ALU and tensor rooflines of this library's
// kernels, measured on the GPU that runs them instead of taken from a datasheet.
//
//   kind 0  FP64 FMA on the CUDA cores (DFMA)           independent FMA chains per thread
//   kind 1  FP32 FMA on the CUDA cores (FFMA)           independent FMA chains per thread
//   kind 2  FP64 tensor MMA (DMMA, mma.sync m8n8k4)      independent accumulators per warp
//   kind 3  TF32 tensor MMA (tcgen05.mma kind::tf32)     M = 128, N = 256, K = 8 from shared
//                                                        memory into tensor memory, one CTA per SM
//
// Every probe keeps its operands in registers or shared memory (no global traffic in the loop)
// and stores one value per thread or CTA so the work cannot be dropped.  The tensor-core probe
// waits for its MMAs with a bounded mbarrier poll and reports a timeout instead of hanging.
#include <cuda_runtime.h>

#include <string>

#include "../../include/schur.h"
#include "api_internal.h"
#include "tc.cuh"

namespace schur {
namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) k_peak_ffma(float* out, int iters, float seed) {
  float a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3f * (threadIdx.x + c);
  const float b = 0.999999f, d = 1e-7f;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fmaf(a[c], b, d);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dfma(double* out, int iters, double seed) {
  double a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double b = 0.9999999999, d = 1e-12;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], b, d);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// D (8x8) += A (8x4) B (4x8) in FP64 on the tensor cores; each lane holds one A and one B value and
// two accumulator values.  Four independent accumulators per warp.
__global__ void __launch_bounds__(256) k_peak_dmma(double* out, int iters, double seed) {
  const double a = seed + 1e-3 * (threadIdx.x & 31), b = 0.5 - 1e-4 * (threadIdx.x & 31);
  double acc[4][2];
#pragma unroll
  for (int q = 0; q < 4; ++q) acc[q][0] = acc[q][1] = 0.0;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                     : "+d"(acc[q][0]), "+d"(acc[q][1])
                     : "d"(a), "d"(b));
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) s += acc[q][0] + acc[q][1];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

constexpr int kPkM = 128, kPkN = 256;
constexpr long long kPkWait = 1LL << 28;

// One CTA per SM: A (128 x 16 FP32) and B (256 x 16 FP32) in 64-byte-swizzled K-major tiles, `iters`
// MMAs of 128 x 256 x 8 issued back to back by one thread (alternating the two K halves of the
// tiles) into one tensor-memory accumulator, then one commit and a bounded wait.
__global__ void __launch_bounds__(128, 1) k_peak_tf32_tc(float* out, int iters, int* err) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  unsigned char* As = sm;                  // 128 rows x 64 B
  unsigned char* Bs = sm + kPkM * 64;      // 256 rows x 64 B
  __shared__ uint64_t done;
  __shared__ uint32_t tbase;
  __shared__ int timed_out;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tc::tmem_alloc(&tbase, kPkN);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&done, 1);
    tc::mbar_fence_init();
    timed_out = 0;
  }
  for (int e = tid; e < kPkM * 16; e += blockDim.x)
    *reinterpret_cast<float*>(As + tc::sw64_off(e / 16, e % 16)) = 1.0f / (1 + (e % 13));
  for (int e = tid; e < kPkN * 16; e += blockDim.x)
    *reinterpret_cast<float*>(Bs + tc::sw64_off(e / 16, e % 16)) = 1.0f / (2 + (e % 7));
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  if (tid == 0) {
    const uint32_t idesc = tc::idesc_tf32(kPkM, kPkN);
    const uint64_t da = tc::desc_sw64(tc::smem_u32(As)), db = tc::desc_sw64(tc::smem_u32(Bs));
    const uint64_t k_off = 32 >> 4;
    for (int it = 0; it < iters; ++it) {
      const uint64_t o = (uint64_t)(it & 1) * k_off;
      tc::mma_tf32(tmem, da + o, db + o, idesc, it > 0 ? 1 : 0);
    }
    tc::commit(&done);
    if (!tc::mbar_wait(&done, 0, kPkWait)) {
      timed_out = 1;
      atomicExch(err, 1);
      // the MMAs may still be running: give them a second bounded wait before the memory is freed
      tc::mbar_wait(&done, 0, kPkWait);
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (!timed_out) {
    float v[16];
    tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16), v);
    if (tid == 0) out[blockIdx.x] = v[0];
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kPkN);
}

}  // namespace
}  // namespace schur

using namespace schur;

#define PK_CK(call)                                                                                   \
  do {                                                                                                \
    cudaError_t e_ = (call);                                                                          \
    if (e_ != cudaSuccess) {                                                                          \
      rc = set_error(e_ == cudaErrorMemoryAllocation ? SCHUR_ENOMEM : SCHUR_ECUDA,                    \
                     std::string("schur_peak_probe: ") + #call + ": " + cudaGetErrorString(e_));     \
      goto done;                                                                                      \
    }                                                                                                 \
  } while (0)

extern "C" int schur_peak_probe(int kind, int iters, double* tflops, void* stream) {
  if (!tflops || kind < 0 || kind > 3 || iters < 1) return set_error(SCHUR_EINVAL, "schur_peak_probe: bad arguments");
  *tflops = 0.0;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0, nsm = 0, rc = SCHUR_OK;
  void* out = nullptr;
  int* err = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double flops = 0.0;
  float ms = 0.f;
  int herr = 0;
  PK_CK(cudaGetDevice(&dev));
  PK_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  PK_CK(cudaMalloc(&out, (size_t)nsm * 8 * 256 * sizeof(double)));
  PK_CK(cudaMalloc(&err, sizeof(int)));
  PK_CK(cudaMemsetAsync(err, 0, sizeof(int), st));
  PK_CK(cudaEventCreate(&e0));
  PK_CK(cudaEventCreate(&e1));
  for (int pass = 0; pass < 2; ++pass) {  // pass 0 warms up (clocks, module load); pass 1 is timed
    PK_CK(cudaEventRecord(e0, st));
    const int grid = nsm * 8, thr = 256;
    if (kind == 0) {
      k_peak_dfma<<<grid, thr, 0, st>>>(static_cast<double*>(out), iters, 1.0);
      flops = 2.0 * kChains * 16 * (double)iters * grid * thr;
    } else if (kind == 1) {
      k_peak_ffma<<<grid, thr, 0, st>>>(static_cast<float*>(out), iters, 1.0f);
      flops = 2.0 * kChains * 16 * (double)iters * grid * thr;
    } else if (kind == 2) {
      k_peak_dmma<<<grid, thr, 0, st>>>(static_cast<double*>(out), iters, 1.0);
      flops = 2.0 * 8 * 8 * 4 * 4 * 4 * (double)iters * (grid * thr / 32);
    } else {
      const size_t smem = 1024 + (size_t)(kPkM + kPkN) * 64;
      PK_CK(cudaFuncSetAttribute(k_peak_tf32_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_peak_tf32_tc<<<nsm, 128, smem, st>>>(static_cast<float*>(out), iters, err);
      flops = 2.0 * kPkM * kPkN * 8 * (double)iters * nsm;
    }
    PK_CK(cudaGetLastError());
    PK_CK(cudaEventRecord(e1, st));
    PK_CK(cudaEventSynchronize(e1));
  }
  PK_CK(cudaEventElapsedTime(&ms, e0, e1));
  PK_CK(cudaMemcpy(&herr, err, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr) {
    rc = set_error(SCHUR_ETIMEOUT, "schur_peak_probe: tensor-core completion wait timed out");
    goto done;
  }
  *tflops = flops / (ms * 1e-3) / 1e12;
done:
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (err) cudaFree(err);
  return rc;
}
