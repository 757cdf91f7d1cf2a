// Local dual operators F^s, F_rc^s and K~_cc^s (Sec. 5) by multi-column layered solves with the
// remainder factor, the dense layer products on the tensor cores (tcgen05, 3xTF32).
//
// One CTA of 128 threads owns a tile of 128 right-hand-side columns of one class (thread t =
// column t = accumulator lane t).  The forward and backward sweeps of the block LDL^T solve
//   forward   V_K = D_K^{-1} (R_K - A_{K,K-1} V_{K-1})
//   backward  X_K = V_K - D_K^{-1} (A_{K,K+1} X_{K+1})
// alternate a sparse coupling step, done per column on the CUDA cores from the column's own
// previous layer, with the dense product by D_K^{-1}, done as one real GEMM per layer:
//   out[t][2i+c'] = sum_j  W[t][2j+c] * B[2i+c'][2j+c],  B = [[Re D, -Im D], [Im D, Re D]] interleaved,
// M = 128 columns, N = 2b rounded up to 16, K = 2b in chunks of 8 nodes (16 values, one 64-byte
// swizzled row).  Each operand is split x = hi + lo into TF32 parts and the product is accumulated
// in FP32 as hi*hi + hi*lo + lo*hi, which keeps FP32 accuracy.  Chunks are double-buffered in
// shared memory: the threads build chunk c+1 while the tensor core multiplies chunk c.
// The column solutions live in a per-CTA global scratch X[node][128] (coalesced per node).
#pragma once
#include "kernels.cuh"
#include "tc.cuh"

namespace schur {

constexpr int kTcCols = 128;         // columns per tile (MMA M)
constexpr int kTcTmemCols = 256;     // tensor-memory columns per CTA (accumulator N <= 256)
constexpr long long kTcWaitLimit = 1LL << 26;

__host__ __device__ inline int tc_nb(int b) { return ((2 * b + 15) / 16) * 16; }
__host__ __device__ inline int tc_stage_bytes(int b) { return ((2 * 8192 + 2 * 64 * tc_nb(b)) + 1023) & ~1023; }
// Dynamic shared memory of k_form_rr_tc: 2 operand stages, the layer coupling table, alignment slack.
__host__ inline size_t form_tc_smem(int b, int nt) {
  return 1024 + 2 * (size_t)tc_stage_bytes(b) + (size_t)b * nt * (sizeof(cx<float>) + sizeof(int));
}

// Writes the 16 values v (8 complex entries) of one operand row, split into TF32 hi/lo parts.
__device__ __forceinline__ void tc_put_row(unsigned char* hi, unsigned char* lo, int r, const float* v) {
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) tc::tf32_split(v[4 * p + e], h[e], l[e]);
    const uint32_t o = tc::sw64_off(r, 4 * p);
    *reinterpret_cast<float4*>(hi + o) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4*>(lo + o) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

template <class T>
__global__ void __launch_bounds__(kTcCols) k_form_rr_tc(StencilProv<T> P, Geom g, MapsView m,
                                                        const cx<T>* __restrict__ Dinv, int ncls, cx<T>* Xws,
                                                        cx<T>* F, cx<T>* Frc, cx<double>* Kcc, int* err) {
  static_assert(sizeof(T) == 4, "TF32 tensor-core path: FP32 working precision only");
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int b = P.ly.b, L = P.ly.L, nt = nbr_count(P.ly.dim), dim = g.dim;
  const int NB = tc_nb(b), SB = tc_stage_bytes(b), nch = (b + 7) / 8;
  const int nD = g.nD, nc = g.nc, ncol = nD + nc, ntile = (ncol + kTcCols - 1) / kTcCols;
  const int tid = threadIdx.x, warp = tid >> 5;
  cx<float>* cf = reinterpret_cast<cx<float>*>(sm + 2 * SB);
  int* nb = reinterpret_cast<int*>(cf + b * nt);
  __shared__ uint64_t bar[2];
  __shared__ uint32_t tbase;

  if (warp == 0) {
    tc::tmem_alloc(&tbase, kTcTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_fence_init();
  }
  // operand rows past 2b are never written again: zero them once in both stages
  for (int s = 0; s < 2; ++s)
    for (int e = tid; e < (NB - 2 * b) * 16; e += kTcCols) {
      const int r = 2 * b + e / 16, f = e % 16;
      *reinterpret_cast<float*>(sm + s * SB + 16384 + tc::sw64_off(r, f)) = 0.f;
      *reinterpret_cast<float*>(sm + s * SB + 16384 + 64 * NB + tc::sw64_off(r, f)) = 0.f;
    }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
  const uint32_t idesc = tc::idesc_tf32(kTcCols, NB);
  cx<float>* X = Xws + (size_t)blockIdx.x * g.nl * kTcCols;
  int ext[3];
  local_ext(g, ext);
  unsigned gc = 0;  // chunks issued so far (stage = gc & 1, per-stage phase = gc >> 1)
  bool ok = true;

  // One layer product: out = D_K^{-1} * (column values produced by `val(i)` for node i).
  auto layer_gemm = [&](const cx<float>* D, auto val) -> bool {
    for (int c = 0; c < nch; ++c) {
      const int s = gc & 1;
      const bool timed_out = gc >= 2 && !tc::mbar_wait(&bar[s], ((gc - 2) >> 1) & 1, kTcWaitLimit);
      unsigned char* Ah = sm + s * SB;
      unsigned char* Al = Ah + 8192;
      unsigned char* Bh = Ah + 16384;
      unsigned char* Bl = Bh + 64 * NB;
      float v[16];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = 8 * c + k;
        cx<float> w = i < b ? val(i) : czero<float>();
        v[2 * k] = w.re;
        v[2 * k + 1] = w.im;
      }
      tc_put_row(Ah, Al, tid, v);
      for (int e = tid; e < 4 * b; e += kTcCols) {
        const int i = e >> 2, p = e & 3, j0 = 8 * c + 2 * p;
        const cx<float> d0 = j0 < b ? D[i * b + j0] : czero<float>();
        const cx<float> d1 = j0 + 1 < b ? D[i * b + j0 + 1] : czero<float>();
        float r0[4] = {d0.re, -d0.im, d1.re, -d1.im}, r1[4] = {d0.im, d0.re, d1.im, d1.re};
        float h[4], l[4];
        uint32_t o = tc::sw64_off(2 * i, 4 * p);
#pragma unroll
        for (int q = 0; q < 4; ++q) tc::tf32_split(r0[q], h[q], l[q]);
        *reinterpret_cast<float4*>(Bh + o) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(Bl + o) = make_float4(l[0], l[1], l[2], l[3]);
        o = tc::sw64_off(2 * i + 1, 4 * p);
#pragma unroll
        for (int q = 0; q < 4; ++q) tc::tf32_split(r1[q], h[q], l[q]);
        *reinterpret_cast<float4*>(Bh + o) = make_float4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<float4*>(Bl + o) = make_float4(l[0], l[1], l[2], l[3]);
      }
      tc::fence_proxy_async();
      if (__syncthreads_or(timed_out)) return false;
      if (tid == 0) {
        tc::fence_after();
        const int ksteps = (2 * (b - 8 * c) + 7) / 8 < 2 ? (2 * (b - 8 * c) + 7) / 8 : 2;
        for (int st = 0; st < ksteps; ++st) {
          const uint64_t ah = tc::desc_sw64(tc::smem_u32(Ah) + 32 * st);
          const uint64_t al = tc::desc_sw64(tc::smem_u32(Al) + 32 * st);
          const uint64_t bh = tc::desc_sw64(tc::smem_u32(Bh) + 32 * st);
          const uint64_t bl = tc::desc_sw64(tc::smem_u32(Bl) + 32 * st);
          tc::mma_tf32(tmem, ah, bh, idesc, (c > 0 || st > 0) ? 1 : 0);
          tc::mma_tf32(tmem, ah, bl, idesc, 1);
          tc::mma_tf32(tmem, al, bh, idesc, 1);
        }
        tc::commit(&bar[s]);
      }
      ++gc;
    }
    const bool timed_out = !tc::mbar_wait(&bar[(gc - 1) & 1], ((gc - 1) >> 1) & 1, kTcWaitLimit);
    if (__syncthreads_or(timed_out)) return false;
    tc::fence_after();
    return true;
  };
  // Reads the accumulator row of this column: node values out(i), i < b, passed to `use(i, v)`.
  auto drain = [&](auto use) {
    for (int n0 = 0; n0 < 2 * b; n0 += 16) {
      float v[16];
      tc::tmem_ld16(tlane + n0, v);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int i = n0 / 2 + k;
        if (i < b) use(i, mkc<float>(v[2 * k], v[2 * k + 1]));
      }
    }
    tc::fence_before();
    __syncthreads();
  };

  for (int w = blockIdx.x; w < ncls * ntile && ok; w += gridDim.x) {
    const int q = w / ntile, col = (w % ntile) * kTcCols + tid;
    P.select(q, m.cls_code);
    const int code = P.code;
    // this column's right-hand side: a unit vector at an interface node, or a column of A_rc
    int my_node = -1, corner = -1;
    int lc[3] = {0, 0, 0};
    if (col < nD) {
      int l[3];
      my_node = m.slot_node[col];
      idx2crd(my_node, ext, dim, l);
      if (P.removed_l(l)) my_node = -1;
    } else if (col < ncol) {
      idx2crd(m.corner_node[col - nD], ext, dim, lc);
      if (!local_dirichlet(code, lc, g.s, dim)) corner = col - nD;
    }
    const cx<float>* Dq = Dinv + (size_t)q * L * b * b;
    // ---- forward sweep
    for (int K = 0; K < L && ok; ++K) {
      if (K > 0) {
        for (int e = tid; e < b * nt; e += kTcCols) {
          const int i = e / nt, t = e - i * nt, j = nbr_of(P.ly, i, t);
          cf[e] = P.Al(K - 1, i, t);
          nb[e] = j < 0 ? 0 : j;
        }
        __syncthreads();
      }
      const cx<float>* Xp = X + (size_t)(K > 0 ? K - 1 : 0) * b * kTcCols + tid;
      auto val = [&](int i) -> cx<float> {
        cx<float> r = czero<float>();
        const int node = K * b + i;
        if (node == my_node) r.re = 1.f;
        if (corner >= 0) {
          int l[3];
          P.crd(K, i, l);
          if (!P.removed_l(l)) r = q1_entry(P.st, g.s, l, lc);
        }
        if (K > 0)
          for (int t = 0; t < nt; ++t) cfms(r, cf[i * nt + t], Xp[(size_t)nb[i * nt + t] * kTcCols]);
        return r;
      };
      if (!layer_gemm(Dq + (size_t)K * b * b, val)) {
        ok = false;
        break;
      }
      cx<float>* Xk = X + (size_t)K * b * kTcCols + tid;
      drain([&](int i, cx<float> v) { Xk[(size_t)i * kTcCols] = v; });
    }
    // ---- backward sweep
    for (int K = L - 2; K >= 0 && ok; --K) {
      for (int e = tid; e < b * nt; e += kTcCols) {
        const int i = e / nt, t = e - i * nt, k = nbr_of(P.ly, i, t);
        cf[e] = k < 0 ? czero<float>() : P.Al(K, k, nt - 1 - t);
        nb[e] = k < 0 ? 0 : k;
      }
      __syncthreads();
      const cx<float>* Xn = X + (size_t)(K + 1) * b * kTcCols + tid;
      auto val = [&](int i) -> cx<float> {
        cx<float> r = czero<float>();
        for (int t = 0; t < nt; ++t) cfma(r, cf[i * nt + t], Xn[(size_t)nb[i * nt + t] * kTcCols]);
        return r;
      };
      if (!layer_gemm(Dq + (size_t)K * b * b, val)) {
        ok = false;
        break;
      }
      cx<float>* Xk = X + (size_t)K * b * kTcCols + tid;
      drain([&](int i, cx<float> v) { Xk[(size_t)i * kTcCols] = csub(Xk[(size_t)i * kTcCols], v); });
    }
    if (!ok) break;
    // ---- F (packed upper triangle), F_rc and K~_cc of this column
    const cx<float>* Xc = X + tid;
    if (col < nD) {
      cx<float>* Fq = F + (size_t)q * sym_ld(nD);
      for (int j = 0; j <= col; ++j) Fq[sym_idx(j, col, nD)] = Xc[(size_t)m.slot_node[j] * kTcCols];
    } else if (col < ncol) {
      const int c2 = col - nD;
      for (int j = 0; j < nD; ++j) Frc[((size_t)q * nD + j) * nc + c2] = Xc[(size_t)m.slot_node[j] * kTcCols];
      for (int c1 = 0; c1 < nc; ++c1) {
        int l1[3], l2[3];
        idx2crd(m.corner_node[c1], ext, dim, l1);
        idx2crd(m.corner_node[c2], ext, dim, l2);
        cx<float> v = czero<float>();
        if (!local_dirichlet(code, l1, g.s, dim) && !local_dirichlet(code, l2, g.s, dim)) {
          if (c1 == c2) v = q1_entry(P.st, g.s, l1, l1);
          const int noff = dim == 2 ? 9 : 27;
          for (int o = 0; o < noff; ++o) {
            int lp[3] = {l1[0] + o % 3 - 1, l1[1] + (o / 3) % 3 - 1, dim == 3 ? l1[2] + o / 9 - 1 : 0};
            bool in = true;
            for (int a = 0; a < dim; ++a) in = in && lp[a] >= 0 && lp[a] <= g.s[a];
            if (!in || (lp[0] == l1[0] && lp[1] == l1[1] && lp[2] == l1[2])) continue;
            if (P.removed_l(lp)) continue;
            cfms(v, q1_entry(P.st, g.s, l1, lp), Xc[(size_t)crd2idx(lp, ext, dim) * kTcCols]);
          }
        }
        Kcc[((size_t)q * nc + c1) * nc + c2] = ccast<double>(v);
      }
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  // every MMA this CTA issued has completed once the last commit has arrived
  if (tid == 0 && gc > 0) tc::mbar_wait(&bar[(gc - 1) & 1], ((gc - 1) >> 1) & 1, kTcWaitLimit);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTcTmemCols);
}

}  // namespace schur
