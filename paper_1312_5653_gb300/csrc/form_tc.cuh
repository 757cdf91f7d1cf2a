// Local dual operators F^s, F_rc^s and K~_cc^s (Sec. 5) by multi-column layered solves with the
// remainder factor, the dense layer products on the tensor cores (tcgen05, 3xTF32).
//
// With the layer couplings of the factorisation, G_K = D_K^{-1} A_{K,K+1} and
// H_K = D_K^{-1} A_{K,K-1}, the block LDL^T solve of A_rr X = R is one dense product per layer:
//   forward   V_0 = D_0^{-1} R_0,   V_K = D_K^{-1} R_K - H_K V_{K-1}
//   backward  X_{L-1} = V_{L-1},    X_K = V_K - G_K X_{K+1}.
// One CTA owns a tile of 128 right-hand-side columns of one class: 512 producer threads (column t =
// accumulator lane t; the four threads t + 128 u share its work) and one issuer warp that only
// launches the MMAs, so that issuing (which waits for the tensor pipe) never holds up the operand
// builds.  Per layer the tensor core forms
//   out[t][2i+c'] = sum_j  Y[t][2j+c] * B[2i+c'][2j+c],  B = -[[Re M, -Im M], [Im M, Re M]] interleaved,
// M = H_K or G_K, Y = the previous layer of the column (V_{K-1} or X_{K+1}): M = 128 columns,
// N = 2b rounded up to 16, K = 2b.  Every operand value is split x = hi + lo into TF32 parts and
// the product accumulates hi*hi + hi*lo + lo*hi in FP32, which keeps FP32 accuracy.  Y stays in
// shared memory for the whole layer (the operand of the next layer is written by the drain of the
// accumulator); B is built chunk by chunk (8 nodes = one 64-byte swizzled row per chunk) into two
// stages, so the threads build chunk c+1 while the tensor core multiplies chunk c: a stage is
// marked written through an mbarrier (one arrival per producer warp) and free again through the
// tcgen05.commit of its MMAs.  The layers V_K go to a per-CTA global scratch X[node][128] for the
// backward sweep and the corner rows; F and F_rc are stored from the drains of the final layers.
#pragma once
#include "kernels.cuh"
#include "tc.cuh"

namespace schur {

constexpr int kTcCols = 128;                // columns per tile (MMA M)
constexpr int kTcProducers = 512;           // four producer threads per column
constexpr int kTcThreads = kTcProducers + 32;  // + the MMA issuer warp
constexpr int kTcTmemCols = 256;            // tensor-memory columns per CTA (accumulator N <= 256)
constexpr int kTcRhs = 8;                   // nonzeros of one right-hand-side column at most
constexpr long long kTcWaitLimit = 1LL << 26;

__host__ __device__ inline int tc_nb(int b) { return ((2 * b + 15) / 16) * 16; }
__host__ __device__ inline int tc_bstage_bytes(int b) { return (2 * 64 * tc_nb(b) + 1023) & ~1023; }
// Dynamic shared memory of k_form_rr_tc: the layer operand (hi/lo, 16 KB per chunk of 8 nodes),
// two B stages, the slot numbers of one layer, alignment slack.
__host__ inline size_t form_tc_smem(int b) {
  return 1024 + (size_t)((b + 7) / 8) * 16384 + 2 * (size_t)tc_bstage_bytes(b) + (size_t)b * sizeof(int);
}

// Named barrier 1: the producers only (the issuer warp never waits on it).
__device__ __forceinline__ void tc_producers_sync() {
  asm volatile("bar.sync 1, %0;\n" ::"n"(kTcProducers) : "memory");
}

// Writes 4 values (2 complex entries) as one 16-byte chunk of an operand row, split into TF32 hi/lo.
__device__ __forceinline__ void tc_put4(unsigned char* hi, unsigned char* lo, uint32_t o, const float* v) {
  float a[4], c[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) tc::tf32_split(v[e], a[e], c[e]);
  *reinterpret_cast<float4*>(hi + o) = make_float4(a[0], a[1], a[2], a[3]);
  *reinterpret_cast<float4*>(lo + o) = make_float4(c[0], c[1], c[2], c[3]);
}

// Nonzeros of one right-hand-side column (kept in registers: indexed with constants only).
struct TcRhs {
  int n[kTcRhs];
  cx<float> v[kTcRhs];
  unsigned layers;  // bit K: a nonzero lies in layer K
};

// Entries j0, j0 + 1 (j0 = 8c + 2p) of row i of a b x b layer matrix M, zero past b.
__device__ __forceinline__ void tc_load_m(const cx<float>* __restrict__ M, int b, int c, int i, int p, bool has,
                                          cx<float>* d) {
  const int j0 = 8 * c + 2 * p;
  d[0] = has && j0 < b ? M[i * b + j0] : czero<float>();
  d[1] = has && j0 + 1 < b ? M[i * b + j0 + 1] : czero<float>();
}

__device__ __forceinline__ void tc_prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p));
}

// Producer side of one chunk: waits until the stage of chunk gc is free (its MMAs of two chunks
// ago completed), builds the B chunk (16-byte chunk bp of rows 2 bi, 2 bi + 1 of
// B = -[[Re M, -Im M], [Im M, Re M]]) from `use`, loads the entries of the next chunk into `nxt`
// (from Mn, chunk cn) and signals the issuer: one arrival per warp on bfull[stage] (16 per chunk)
// once the warp's writes are visible to the tensor core.  A timed-out wait sets *bad (later waits
// are skipped).
__device__ __forceinline__ void tc_produce(int b, int NB, int BS, unsigned char* Bst, uint64_t* bar, uint64_t* bfull,
                                           unsigned& gc, int bi, int bp, bool has_b, const cx<float>* use,
                                           cx<float>* nxt, const cx<float>* __restrict__ Mn, int cn,
                                           volatile int* bad) {
  const int s = gc & 1;
  unsigned char* Bh = Bst + s * BS;
  unsigned char* Bl = Bh + 64 * NB;
  nxt[0] = czero<float>();
  nxt[1] = czero<float>();
  if (Mn) tc_load_m(Mn, b, cn, bi, bp, has_b, nxt);
  if (gc >= 2 && !*bad && !tc::mbar_wait(&bar[s], ((gc - 2) >> 1) & 1, kTcWaitLimit)) *bad = 1;
  if (has_b) {
    const float r0[4] = {-use[0].re, use[0].im, -use[1].re, use[1].im};
    const float r1[4] = {-use[0].im, -use[0].re, -use[1].im, -use[1].re};
    tc_put4(Bh, Bl, tc::sw64_off(2 * bi, 4 * bp), r0);
    tc_put4(Bh, Bl, tc::sw64_off(2 * bi + 1, 4 * bp), r1);
  }
  tc::fence_proxy_async();
  __syncwarp();
  if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&bfull[s]);
  ++gc;
}

template <class T>
__global__ void __launch_bounds__(kTcThreads, 1) k_form_rr_tc(StencilProv<T> P, Geom g, MapsView m,
                                                              const cx<T>* __restrict__ Dinv,
                                                              const cx<T>* __restrict__ Gc,
                                                              const cx<T>* __restrict__ Hc, int ncls, cx<T>* Xws,
                                                              cx<T>* F, cx<T>* Frc, cx<double>* Kcc, int* err,
                                                              int nterms, int ncol_tc) {
  static_assert(sizeof(T) == 4, "TF32 tensor-core path: FP32 working precision only");
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const int b = P.ly.b, L = P.ly.L, dim = g.dim;
  const int NB = tc_nb(b), nch = (b + 7) / 8;
  // the first ncol_tc of the nD + nc right-hand-side columns (the rest go to the CUDA-core kernel)
  const int nD = g.nD, nc = g.nc, ncol = nD + nc, ntile = (ncol_tc + kTcCols - 1) / kTcCols;
  const int tid = threadIdx.x, warp = tid >> 5, ct = tid & (kTcCols - 1), qq = tid >> 7;
  const size_t bb = (size_t)b * b;
  unsigned char* Ybuf = sm;                       // chunk c: hi at c*16K, lo at c*16K + 8K
  unsigned char* Bst = sm + (size_t)nch * 16384;  // two B stages (hi, lo)
  const int BS = tc_bstage_bytes(b);
  int* ns = reinterpret_cast<int*>(Bst + 2 * BS);  // slot numbers of the drained layer
  __shared__ uint64_t bar[2];    // stage s: the MMAs of its last chunk completed (tcgen05.commit)
  __shared__ uint64_t bfull[2];  // stage s: its B chunk written (one arrival per producer warp)
  __shared__ uint32_t tbase;
  __shared__ volatile int bad;

  if (warp == 0) {
    tc::tmem_alloc(&tbase, kTcTmemCols);
    tc::tmem_relinquish();
  }
  if (tid == 0) {
    tc::mbar_init(&bar[0], 1);
    tc::mbar_init(&bar[1], 1);
    tc::mbar_init(&bfull[0], kTcProducers / 32);
    tc::mbar_init(&bfull[1], kTcProducers / 32);
    tc::mbar_fence_init();
    bad = 0;
  }
  // B rows past 2b are never written again: zero them once in both stages
  for (int st = 0; st < 2; ++st)
    for (int e = tid; e < (NB - 2 * b) * 16; e += kTcThreads) {
      const int r = 2 * b + e / 16, f = e % 16;
      *reinterpret_cast<float*>(Bst + st * BS + tc::sw64_off(r, f)) = 0.f;
      *reinterpret_cast<float*>(Bst + st * BS + 64 * NB + tc::sw64_off(r, f)) = 0.f;
    }
  tc::fence_proxy_async();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  const int nwork = ncls * ntile, nphase = 2 * L - 2;
  const int nmine = (nwork - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // items of this CTA

  if (warp == kTcProducers / 32) {
    // ---------------- issuer warp: every chunk of every GEMM phase, in the producers' order
    const uint32_t idesc = tc::idesc_tf32(kTcCols, NB);
    const int lane = tid & 31;
    // descriptors of operand chunk 0 and of the two B stages (start-address field in 16-byte
    // units: chunk c of Y starts 1024 units further, the lo parts 512 and 4 NB units, the
    // second K step 2 units)
    const uint64_t ya0 = tc::desc_sw64(tc::smem_u32(Ybuf));
    const uint64_t bst[2] = {tc::desc_sw64(tc::smem_u32(Bst)), tc::desc_sw64(tc::smem_u32(Bst + BS))};
    const uint64_t lo_off = 8192 >> 4, bl_off = (uint64_t)(64 * NB) >> 4, k_off = 32 >> 4;
    unsigned gi = 0;
    for (int it = 0; it < nmine; ++it)
      for (int ph = 0; ph < nphase; ++ph)
        for (int c = 0; c < nch; ++c, ++gi) {
          const int s = gi & 1;
          if (lane == 0 && !bad && !tc::mbar_wait(&bfull[s], (gi >> 1) & 1, kTcWaitLimit)) bad = 1;
          __syncwarp();
          if (lane == 0 && !bad) {
            // the first chunk of a layer overwrites the accumulator the drain has just read
            if (c == 0) tc::fence_after();
            const int left = 2 * (b - 8 * c), ksteps = left >= 16 ? 2 : (left + 7) / 8;
            const uint64_t ah = ya0 + (uint64_t)c * (16384 >> 4), bh = bst[s];
            for (int st = 0; st < ksteps; ++st) {
              const uint64_t o = (uint64_t)st * k_off;
              tc::mma_tf32(tmem, ah + o, bh + o, idesc, (c > 0 || st > 0) ? 1 : 0);
              if (nterms == 3) {
                tc::mma_tf32(tmem, ah + o, bh + bl_off + o, idesc, 1);
                tc::mma_tf32(tmem, ah + lo_off + o, bh + o, idesc, 1);
              }
            }
            tc::commit(&bar[s]);
          }
          __syncwarp();
        }
  } else {
    // ---------------- producers
    const uint32_t tlane = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    cx<float>* X = Xws + (size_t)blockIdx.x * g.nl * kTcCols + ct;  // this column's scratch, stride 128
    int ext[3];
    local_ext(g, ext);
    unsigned gc = 0;  // chunks produced so far (stage = gc & 1, per-stage phase = gc >> 1)
    // B operand item of this thread: rows 2 bi, 2 bi + 1, 16-byte chunk bp (entries j0, j0 + 1 of row bi)
    const int bi = tid >> 2, bp = tid & 3;
    const bool has_b = tid < 4 * b;
    cx<float> mcur[2] = {czero<float>(), czero<float>()}, maux[2] = {czero<float>(), czero<float>()};
    // layer matrix of GEMM phase ph (forward K = ph + 1 uses H_K, backward K = 2L - 3 - ph uses G_K)
    auto phase_m = [&](const cx<float>* Gq, const cx<float>* Hq, int ph) -> const cx<float>* {
      return ph < L - 1 ? Hq + (size_t)(ph + 1) * bb : Gq + (size_t)(2 * L - 3 - ph) * bb;
    };

    // Drain of layer K: x = base(i) + accumulator (none for the first forward layer), written to
    // the operand buffer (TF32 hi/lo) and to the scratch.  base = D_K^{-1} R_K (forward) or V_K
    // (backward, read back from the scratch).  Thread u of a column handles chunks u, u + 4, ...
    // Final layers (every backward layer and the last forward one) also store this column's
    // entries of F (packed upper triangle; interface columns) or F_rc (corner columns).
    auto drain = [&](int K, bool fwd, bool acc, const cx<float>* __restrict__ Dk, const TcRhs& R, int col,
                     cx<float>* Fq, cx<float>* Frcq) {
      cx<float>* Xk = X + (size_t)K * b * kTcCols;
      const bool fin = !fwd || K == L - 1;
      if (fin) {
        for (int i = tid; i < b; i += kTcProducers) ns[i] = m.node_slot[K * b + i];
      }
      tc_producers_sync();
      for (int gq = qq; gq < nch; gq += 4) {
        cx<float> x[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] = czero<float>();
        if (!fwd) {
#pragma unroll
          for (int k = 0; k < 8; ++k)
            if (8 * gq + k < b) x[k] = Xk[(size_t)(8 * gq + k) * kTcCols];
        } else if (R.layers >> K & 1) {
          // D_K^{-1} R_K: sum over this column's nonzeros in layer K of value * row n of D_K^{-1}
#pragma unroll
          for (int e = 0; e < kTcRhs; ++e) {
            const int n = R.n[e] - K * b;
            if (n >= 0 && n < b) {
              const cx<float>* Dr = Dk + (size_t)n * b;
#pragma unroll
              for (int k = 0; k < 8; ++k)
                if (8 * gq + k < b) cfma(x[k], R.v[e], Dr[8 * gq + k]);
            }
          }
        }
        if (acc) {
          float v[16];
          tc::tmem_ld16(tlane + 16 * gq, v);
#pragma unroll
          for (int k = 0; k < 8; ++k) x[k] = mkc<float>(x[k].re + v[2 * k], x[k].im + v[2 * k + 1]);
        }
        unsigned char* hi = Ybuf + (size_t)gq * 16384;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
          const float va[4] = {x[2 * p].re, x[2 * p].im, x[2 * p + 1].re, x[2 * p + 1].im};
          tc_put4(hi, hi + 8192, tc::sw64_off(ct, 4 * p), va);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int i = 8 * gq + k;
          if (i < b) {
            Xk[(size_t)i * kTcCols] = x[k];
            if (fin) {
              const int j = ns[i];
              if (j >= 0) {
                if (col < nD) {
                  if (j <= col) Fq[sym_idx(j, col, nD)] = x[k];
                } else if (col < ncol) {
                  Frcq[(size_t)j * nc + (col - nD)] = x[k];
                }
              }
            }
          }
        }
      }
      tc::fence_before();
      tc_producers_sync();  // the slot table is reused by the next drain
    };

    for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
      const int q = w / ntile, col = (w % ntile) * kTcCols + ct;
      P.select(q, m.cls_code);
      const int code = P.code;
      // nonzeros of this column's right-hand side: a unit vector at an interface node, or the
      // column of A_rc of a corner (its neighbours in the remainder set)
      TcRhs R;
      R.layers = 0;
#pragma unroll
      for (int e = 0; e < kTcRhs; ++e) {
        R.n[e] = -1000000;
        R.v[e] = czero<float>();
      }
      if (col < nD) {
        int l[3];
        idx2crd(m.slot_node[col], ext, dim, l);
        if (!P.removed_l(l)) {
          R.n[0] = m.slot_node[col];
          R.v[0] = mkc<float>(1.f, 0.f);
          R.layers = 1u << (R.n[0] / b);
        }
      } else if (col < ncol) {
        int lc[3];
        idx2crd(m.corner_node[col - nD], ext, dim, lc);
        if (!local_dirichlet(code, lc, g.s, dim)) {
          int k = 0;
          for (int o = 0; o < (dim == 2 ? 9 : 27); ++o) {
            int lp[3] = {lc[0] + o % 3 - 1, lc[1] + (o / 3) % 3 - 1, dim == 3 ? lc[2] + o / 9 - 1 : 0};
            bool in = true;
            for (int a = 0; a < dim; ++a) in = in && lp[a] >= 0 && lp[a] <= g.s[a];
            if (!in || P.removed_l(lp)) continue;
            const int node = crd2idx(lp, ext, dim);
            const cx<float> a = q1_entry(P.st, g.s, lp, lc);
#pragma unroll
            for (int e = 0; e < kTcRhs; ++e)
              if (e == k) {
                R.n[e] = node;
                R.v[e] = a;
              }
            R.layers |= 1u << (node / b);
            ++k;
          }
        }
      }
      const size_t qoff = (size_t)q * L * bb;
      const cx<float>* Dq = Dinv + qoff;
      const cx<float>* Gq = Gc + qoff;
      const cx<float>* Hq = Hc + qoff;
      if (w == (int)blockIdx.x && nphase > 0) tc_load_m(phase_m(Gq, Hq, 0), b, 0, bi, bp, has_b, mcur);
      const int wn = w + (int)gridDim.x;
      const cx<float>* Mnext =
          wn < nwork && nphase > 0
              ? phase_m(Gc + (size_t)(wn / ntile) * L * bb, Hc + (size_t)(wn / ntile) * L * bb, 0)
              : nullptr;
      cx<float>* Fq = F + (size_t)q * sym_ld(nD);
      cx<float>* Frcq = Frc + (size_t)q * nD * nc;
      // first forward layer: V_0 = D_0^{-1} R_0
      drain(0, true, false, Dq, R, col, Fq, Frcq);
      // GEMM phases: forward K = 1..L-1, then backward K = L-2..0
      for (int ph = 0; ph < nphase; ++ph) {
        const bool fwd = ph < L - 1;
        const int K = fwd ? ph + 1 : 2 * L - 3 - ph;
        const cx<float>* M = phase_m(Gq, Hq, ph);
        const cx<float>* Mn = ph + 1 < nphase ? phase_m(Gq, Hq, ph + 1) : Mnext;
        // the next layer matrix (52 KB at b = 81) and, backward, the V_K this drain reads back are
        // pulled into L2 while the layer is multiplied
        if (Mn && tid * 16 < (int)bb) tc_prefetch_l2(Mn + (size_t)tid * 16);
        if (!fwd) {
          const char* xb = reinterpret_cast<const char*>(X - ct + (size_t)K * b * kTcCols);
          for (int ln = tid; ln < b * kTcCols * 8 / 128; ln += kTcProducers) tc_prefetch_l2(xb + (size_t)ln * 128);
        }
        // chunks in pairs: the entries of chunk c + 1 are loaded into the other register set while
        // chunk c is built, so no load result is waited for in the chunk that issues it
        for (int c = 0; c < nch; c += 2) {
          tc_produce(b, NB, BS, Bst, bar, bfull, gc, bi, bp, has_b, mcur, maux, c + 1 < nch ? M : Mn,
                     c + 1 < nch ? c + 1 : 0, &bad);
          if (c + 1 >= nch) break;
          tc_produce(b, NB, BS, Bst, bar, bfull, gc, bi, bp, has_b, maux, mcur, c + 2 < nch ? M : Mn,
                     c + 2 < nch ? c + 2 : 0, &bad);
        }
        if (nch & 1) {  // odd chunk count: the next chunk's entries are in maux
          mcur[0] = maux[0];
          mcur[1] = maux[1];
        }
        // every MMA of this layer has completed once its last chunk's commit has arrived
        if (!bad && !tc::mbar_wait(&bar[(gc - 1) & 1], ((gc - 1) >> 1) & 1, kTcWaitLimit)) bad = 1;
        tc::fence_after();
        drain(K, fwd, true, Dq + (size_t)K * bb, R, col, Fq, Frcq);
      }
      // ---- K~_cc of corner columns (F and F_rc were stored by the drains); the four threads of a
      // column split the rows.  Every value read was written by this column's threads before the
      // last barrier.
      if (col >= nD && col < ncol) {
        const int c2 = col - nD;
        for (int c1 = qq; c1 < nc; c1 += 4) {
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
              cfms(v, q1_entry(P.st, g.s, l1, lp), X[(size_t)crd2idx(lp, ext, dim) * kTcCols]);
            }
          }
          Kcc[((size_t)q * nc + c1) * nc + c2] = ccast<double>(v);
        }
      }
      tc_producers_sync();  // the next item rewrites the operand buffer
    }
    if (bad && tid == 0) atomicExch(err, 1);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, kTcTmemCols);
}

}  // namespace schur
