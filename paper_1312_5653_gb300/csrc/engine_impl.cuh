// Engine<T>: device storage and host orchestration of one FETI-DP solver for A = K + i gamma M in
// working precision T.  Included by engine_f64.cu and engine_f32.cu (one instantiation each).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/schur.h"
#include "engine.h"
#include "gmres.h"
#include "kernels.cuh"
#include "warp.cuh"
#include "form_tc.cuh"
#include "prof.h"
#include "coarse.h"

namespace schur {

#define ENG_CK(call)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      if (msg) *msg = std::string(#call) + ": " + cudaGetErrorString(e_);              \
      return e_ == cudaErrorMemoryAllocation ? SCHUR_ENOMEM : SCHUR_ECUDA;             \
    }                                                                                  \
  } while (0)

#define ENG_LAUNCH()                                                                   \
  do {                                                                                 \
    ++launches;                                                                        \
    cudaError_t e_ = cudaGetLastError();                                               \
    if (e_ != cudaSuccess) {                                                           \
      if (msg) *msg = std::string("kernel launch at line ") + std::to_string(__LINE__) + \
                      ": " + cudaGetErrorString(e_);                                   \
      return SCHUR_ECUDA;                                                              \
    }                                                                                  \
  } while (0)

// Launch of the column-per-thread local operator formation (2D, layer size b <= B).
template <class T, int B>
static cudaError_t launch_form_cols(const StencilProv<T>& P, const Geom& g, const MapsView& mv, const cx<T>* Dinv,
                                    int ncls, cx<T>* F, cx<T>* Frc, cx<double>* Kcc, cx<T>* Ews, int grid, int ldE,
                                    int col1, cudaStream_t st) {
  const size_t smem = form_cols_smem<T, B>(g.lb, g.lL);
  cudaError_t e = smem_attr((const void*)k_form_rr_cols<T, B>, (int)smem);
  if (e != cudaSuccess) return e;
  k_form_rr_cols<T, B><<<grid, ldE, smem, st>>>(P, g, mv, Dinv, ncls, F, Frc, Kcc, Ews, ldE, col1);
  return cudaGetLastError();
}

// Launch of the column-per-lane layered factorisation (2D, layer size b <= B), 4 warps per block.
template <class T, int B>
static cudaError_t launch_factor_cols(const StencilProv<T>& P, const int* codes, int nprob, cx<T>* Dinv, int* err,
                                      cudaStream_t st) {
  const int wpb = 4;
  const size_t smem = wpb * factor_cols_smem_per_warp<T, B>();
  cudaError_t e = smem_attr((const void*)k_factor_cols<T, B>, (int)smem);
  if (e != cudaSuccess) return e;
  k_factor_cols<T, B><<<(nprob + wpb - 1) / wpb, 32 * wpb, smem, st>>>(P, codes, nprob, Dinv, err);
  return cudaGetLastError();
}

template <class T>
class Engine : public EngineBase {
 public:
  Engine(const HostMaps* hm, const DevMaps* dm, double gamma, double sre)
      : hm_(hm), dm_(dm), g_(hm->g), gamma_(gamma) {
    mv_.slot_node = dm->slot_node;
    mv_.node_slot = dm->node_slot;
    mv_.corner_node = dm->corner_node;
    mv_.sd_cls = dm->sd_cls;
    mv_.cls_code = dm->cls_code;
    mv_.sd_lam = dm->sd_lam;
    mv_.lam_side = dm->lam_side;
    mv_.sd_corner = dm->sd_corner;
    mv_.sd_minv = dm->sd_minv;
    mv_.sd_coarse = dm->sd_coarse;
    mv_.face_sd = dm->face_sd;
    mv_.lam_face = dm->lam_face;
    mv_.slot_faces = dm->slot_faces;
    mv_.face_lam_ptr = dm->face_lam_ptr;
    mv_.face_lam = dm->face_lam;
    mv_.grp_sd = dm->grp_sd;
    mv_.grp_ptr = dm->grp_ptr;
    ngrp_ = (int)hm->grp_ptr.size() - 1;
    st_ = make_stencil<T>(g_, gamma, sre);
    ncls_ = hm->ncls;
    // remainder problem: full local grid, vertices and Dirichlet nodes removed
    prr_.ly.dim = g_.dim;
    pii_.ly.dim = g_.dim;
    for (int a = 0; a < 3; ++a) {
      prr_.ly.ext[a] = a < g_.dim ? g_.s[a] + 1 : 1;
      pii_.ly.ext[a] = a < g_.dim ? g_.s[a] - 1 : 1;
      prr_.s[a] = g_.s[a];
      pii_.s[a] = g_.s[a];
    }
    prr_.ly.b = g_.lb;
    prr_.ly.L = g_.lL;
    prr_.st = st_;
    prr_.off = 0;
    prr_.masked = 1;
    prr_.code = 0;
    pii_.ly.b = g_.ib;
    pii_.ly.L = g_.iL;
    pii_.st = st_;
    pii_.off = 1;
    pii_.masked = 0;
    pii_.code = 0;
    cudaDeviceGetAttribute(&nsm_, cudaDevAttrMultiProcessorCount, 0);
    if (nsm_ <= 0) nsm_ = 152;
  }

  // The stream of the last call may no longer exist (a server worker that created the context can
  // have exited); schur_destroy synchronises the device first, so free on the default stream.
  ~Engine() override {
    for (void* p : allocs_) cudaFreeAsync(p, nullptr);
    cudaStreamSynchronize(nullptr);
    if (h_active_) cudaFreeHost(h_active_);
    if (side_) cudaStreamDestroy(side_);
    if (fork_) cudaEventDestroy(fork_);
    if (join_) cudaEventDestroy(join_);
    if (corner_ev_) cudaEventDestroy(corner_ev_);
  }

  long long op_bytes() const override { return op_bytes_; }

  int setup(cudaStream_t st, std::string* msg) override {
    const Geom& g = g_;
    ast_ = st;
    configure_pool();
    const size_t cxT = sizeof(cx<T>);
    const int bb = g.lb * g.lb;
    ENG_CK(alloc(&err_, 4 * sizeof(int)));
    ENG_CK(cudaMemsetAsync(err_, 0, 4 * sizeof(int), st));
    ENG_CK(alloc(&ones_, kMaxRdev * sizeof(int)));
    {
      int h1[kMaxRdev];
      for (int i = 0; i < kMaxRdev; ++i) h1[i] = 1;
      ENG_CK(cudaMemcpyAsync(ones_, h1, sizeof(h1), cudaMemcpyHostToDevice, st));
    }
    // ---- stencil tables of the remainder and interior problems
    {
      const int nt = nbr_count(g.dim);
      StencilProv<T>* probs[2] = {&prr_, &pii_};
      for (StencilProv<T>* P : probs) {
        const size_t ne = (size_t)P->ly.L * P->ly.b * nt;
        cx<T>*tad = nullptr, *tal = nullptr;
        unsigned char* fl = nullptr;
        ENG_CK(alloc(&tad, ne * cxT));
        ENG_CK(alloc(&tal, ne * cxT));
        ENG_CK(alloc(&fl, (size_t)P->ly.L * P->ly.b));
        P->tad = tad;
        P->tal = tal;
        P->flags = fl;
        prof_start(KC_FACTOR, st);
        k_stencil_tables<T><<<(int)std::min<size_t>((ne + 255) / 256, 1024), 256, 0, st>>>(*P, tad, tal, fl);
        prof_stop(KC_FACTOR, st);
        ENG_LAUNCH();
      }
    }
    // ---- local operator storage
    ENG_CK(alloc(&F_, (size_t)ncls_ * sym_ld(g.nD) * cxT));  // packed symmetric
    // coupling columns: the corners' from the formation; with the augmented coarse problem the
    // formation writes them to a temporary and Frc_ receives [Frc | F Q] (k_aug_local)
    const bool aug = g.nq > g.nc;
    if (aug && g.nco > kMaxAugCoarse) {
      if (msg) *msg = "augmented coarse problem larger than " + std::to_string(kMaxAugCoarse) + " unknowns";
      return SCHUR_EINVAL;
    }
    cx<T>* Frc0 = nullptr;
    ENG_CK(alloc(&Frc_, (size_t)ncls_ * g.nD * g.nq * cxT));
    if (aug) ENG_CK(alloc(&Frc0, (size_t)ncls_ * g.nD * g.nc * cxT));
    cx<T>* FrcF = aug ? Frc0 : Frc_;
    ENG_CK(alloc(&Sd_, (size_t)ncls_ * sym_ld(g.nD) * cxT));  // packed symmetric
    ENG_CK(alloc(&Kcc_, (size_t)ncls_ * g.nc * g.nc * sizeof(cx<double>)));
    op_bytes_ += (long long)ncls_ * (2 * sym_ld(g.nD) + (long long)g.nD * g.nq) * cxT;
    // ---- interior branch on a second stream: the interior problem is independent of the
    // remainder problems, so its factor and the Dirichlet S run beside the remainder factors and F
    const int C = 32;
    const int nchunk2 = (g.nD + C - 1) / C;
    cx<T>* Xi = nullptr;
    cx<T>* Sbase = nullptr;
    ENG_CK(alloc(&Xi, (size_t)nchunk2 * g.ni * C * cxT));
    ENG_CK(alloc(&Sbase, (size_t)g.nD * g.nD * cxT));
    // interior factor (identical for all subdomains)
    const int ibb = g.ib * g.ib;
    cx<T>* Dii = nullptr;
    ENG_CK(alloc(&Dii, (size_t)g.iL * ibb * cxT));
    if (!side_) {
      // the second stream carries latency-bound branches (the interior factor and S, the coarse
      // problem): its blocks are scheduled before those of the main stream
      int lo_pri = 0, hi_pri = 0;
      ENG_CK(cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri));
      ENG_CK(cudaStreamCreateWithPriority(&side_, cudaStreamNonBlocking, hi_pri));
      ENG_CK(cudaEventCreateWithFlags(&fork_, cudaEventDisableTiming));
      ENG_CK(cudaEventCreateWithFlags(&join_, cudaEventDisableTiming));
    }
    // every buffer the side stream touches is allocated (stream-ordered on st) before the fork
    const bool cols_if = sizeof(T) == 4 && g.dim == 2 && g.ib <= 32;
    const size_t need_if = (2 * (size_t)ibb + 2 * g.ib) * cxT;
    const int use_smem_if = need_if <= 200 * 1024;
    cx<T>* gws_if = nullptr;
    if (!cols_if && !use_smem_if) ENG_CK(alloc(&gws_if, 2 * (size_t)ibb * cxT));
    ENG_CK(cudaEventRecord(fork_, st));
    ENG_CK(cudaStreamWaitEvent(side_, fork_, 0));
    bool ifactored = false;
    if constexpr (sizeof(T) == 4) {
      if (cols_if) {
        const int Bp = g.ib == 9 ? 9 : g.ib == 17 ? 17 : ((g.ib + 7) / 8) * 8;
        prof_start(KC_INTERIOR, side_);
        cudaError_t fe = cudaErrorInvalidValue;
#define FK_CASE(BV) \
  case BV: fe = launch_factor_cols<T, BV>(pii_, dm_->cls_code, 1, Dii, err_ + 1, side_); break
        switch (Bp) {
          FK_CASE(8);
          FK_CASE(9);
          FK_CASE(16);
          FK_CASE(17);
          FK_CASE(24);
          FK_CASE(32);
          default: break;
        }
#undef FK_CASE
        ENG_CK(fe);
        prof_stop(KC_INTERIOR, side_);
        ENG_LAUNCH();
        ifactored = true;
      }
    }
    if (!ifactored) {
      size_t smem = use_smem_if ? need_if : 2 * g.ib * cxT;
      ENG_CK(smem_attr((const void*)k_factor<T, StencilProv<T>>, (int)smem));
      prof_start(KC_INTERIOR, side_);
      k_factor<T, StencilProv<T>><<<1, ibb >= 1024 ? 512 : 256, smem, side_>>>(pii_, dm_->cls_code, Dii, gws_if, use_smem_if,
                                                                               err_ + 1);
      prof_stop(KC_INTERIOR, side_);
      ENG_LAUNCH();
    }
    {
      size_t smem2 = 2 * (size_t)g.ib * C * cxT;
      ENG_CK(smem_attr((const void*)k_form_ii<T>, (int)smem2));
      prof_start(KC_INTERIOR, side_);
      k_form_ii<T><<<nchunk2, 256, smem2, side_>>>(pii_, g, mv_, Dii, C, Xi, Sbase);
      prof_stop(KC_INTERIOR, side_);
      ENG_LAUNCH();
      long long tot = (long long)ncls_ * g.nD * g.nD;
      int gs = (int)std::min<long long>((tot + 255) / 256, 16LL * nsm_);
      prof_start(KC_INTERIOR, side_);
      k_mask_S<T><<<gs, 256, 0, side_>>>(g, mv_, ncls_, Sbase, Sd_);
      prof_stop(KC_INTERIOR, side_);
      ENG_LAUNCH();
    }
    // ---- remainder factors, one per class
    ENG_CK(alloc(&Dinv_, (size_t)ncls_ * g.lL * bb * cxT));
    op_bytes_ += (long long)ncls_ * g.lL * bb * cxT;
    // 3D FP32: the local operators are formed on the tensor cores from the layer couplings G, H
    // of the factorisation (temporaries, released after the formation)
    const bool tc_form = sizeof(T) == 4 && g.dim == 3 && g.lL <= 32 && tc_nb(g.lb) <= kTcTmemCols &&
                         form_tc_smem(g.lb) <= (size_t)227 * 1024;
    cx<T>*Gc = nullptr, *Hc = nullptr;
    if (tc_form) {
      ENG_CK(alloc(&Gc, (size_t)ncls_ * g.lL * bb * cxT));
      ENG_CK(alloc(&Hc, (size_t)ncls_ * g.lL * bb * cxT));
    }
    bool factored = false;
    if constexpr (sizeof(T) == 4) {
      if (g.dim == 2 && g.lb <= 32) {
        const int Bp = g.lb == 9 ? 9 : g.lb == 17 ? 17 : ((g.lb + 7) / 8) * 8;
        prof_start(KC_FACTOR, st);
        cudaError_t fe = cudaErrorInvalidValue;
#define FK_CASE(BV) \
  case BV: fe = launch_factor_cols<T, BV>(prr_, dm_->cls_code, ncls_, Dinv_, err_, st); break
        switch (Bp) {
          FK_CASE(8);
          FK_CASE(9);
          FK_CASE(16);
          FK_CASE(17);
          FK_CASE(24);
          FK_CASE(32);
          default: break;
        }
#undef FK_CASE
        ENG_CK(fe);
        prof_stop(KC_FACTOR, st);
        ENG_LAUNCH();
        factored = true;
      }
    }
    if (factored) {
    } else if (g.lb <= 32 && !tc_form) {
      const size_t per_warp = (2 * (size_t)bb + 2 * g.lb) * cxT;
      const int wpb = (int)std::max<size_t>(1, std::min<size_t>(8, ((size_t)160 << 10) / per_warp));
      size_t smem = (size_t)wpb * per_warp;
      ENG_CK(smem_attr((const void*)k_factor_warp<T>, (int)smem));
      prof_start(KC_FACTOR, st);
      k_factor_warp<T><<<(ncls_ + wpb - 1) / wpb, 32 * wpb, smem, st>>>(prr_, dm_->cls_code, ncls_, Dinv_, err_);
      prof_stop(KC_FACTOR, st);
      ENG_LAUNCH();
    } else {
      size_t need = (2 * (size_t)bb + 2 * g.lb) * cxT;
      int use_smem = need <= 200 * 1024;
      // the coupling table of the current layer fits beside the two blocks: FP32 up to two blocks
      // per SM (113 KB each), FP64 one (up to 227 KB)
      const size_t tabb = (size_t)g.lb * nbr_count(g.dim) * cxT;
      const int use_tab = use_smem && need + tabb <= (sizeof(T) == 4 ? (size_t)113 << 10 : (size_t)227 << 10);
      size_t smem = use_smem ? need + (use_tab ? tabb : 0) : 2 * g.lb * cxT;
      cx<T>* gws = nullptr;
      if (!use_smem) ENG_CK(alloc(&gws, (size_t)ncls_ * 2 * bb * cxT));
      ENG_CK(smem_attr((const void*)k_factor<T, StencilProv<T>>, (int)smem));
      int thr = bb >= 1024 ? 512 : 256;
      prof_start(KC_FACTOR, st);
      k_factor<T, StencilProv<T>><<<ncls_, thr, smem, st>>>(prr_, dm_->cls_code, Dinv_, gws, use_smem, err_, Gc, Hc,
                                                            use_tab);
      prof_stop(KC_FACTOR, st);
      ENG_LAUNCH();
    }
    // ---- local operators
    bool early_coarse = false;
    {
      cx<T>* Xws = nullptr;
      bool formed = false;
      if constexpr (sizeof(T) == 4) {
        const int ncol = g.nD + g.nc, ldE = ((ncol + 31) / 32) * 32;
        if (tc_form) {
          // layer products on the tensor cores, 128 columns per CTA, one CTA per SM; a last tile of at
          // most 16 columns (3D 8^3 subdomains: 386 = 3 x 128 + 2) goes to the CUDA-core kernel, so the
          // tensor pipe does not spend a whole tile on it
          const int rem = ncol % kTcCols;
          const int ncol_tc = (rem > 0 && rem <= 16 && ncol > kTcCols) ? ncol - rem : ncol;
          const int ntile = (ncol_tc + kTcCols - 1) / kTcCols;
          const size_t smem = form_tc_smem(g.lb);
          const int grid = std::max(1, std::min(ncls_ * ntile, nsm_));
          ENG_CK(alloc(&Xws, (size_t)grid * g.nl * kTcCols * cxT));
          ENG_CK(smem_attr((const void*)k_form_rr_tc<T>, (int)smem));
          prof_start(KC_FORM, st);
          k_form_rr_tc<T><<<grid, kTcThreads, smem, st>>>(prr_, g, mv_, Dinv_, Gc, Hc, ncls_, Xws, F_, FrcF, Kcc_,
                                                          err_ + 3, tc_terms, ncol_tc);
          prof_stop(KC_FORM, st);
          ENG_LAUNCH();
          if (ncol_tc < ncol) {
            const int Cr = ncol - ncol_tc;
            const int grid2 = std::min(ncls_, 8 * nsm_);
            cx<T>* Xr = nullptr;
            ENG_CK(alloc(&Xr, (size_t)grid2 * g.nl * Cr * cxT));
            const size_t smem2 = 2 * (size_t)g.lb * Cr * cxT;
            ENG_CK(smem_attr((const void*)k_form_rr<T>, (int)smem2));
            prof_start(KC_FORM, st);
            k_form_rr<T><<<grid2, 256, smem2, st>>>(prr_, g, mv_, Dinv_, ncls_, Cr, Xr, F_, FrcF, Kcc_, ncol_tc);
            prof_stop(KC_FORM, st);
            ENG_LAUNCH();
            free_one(Xr);
          }
          formed = true;
        } else if (g.dim == 2 && g.lb <= 32 && ldE <= 128) {
          const int Bp = g.lb == 9 ? 9 : g.lb == 17 ? 17 : ((g.lb + 7) / 8) * 8;
          // With the corner coarse problem (not augmented) K_cc is formed first, so that the FP64
          // coarse factorisation and inverse run on the second (higher-priority) stream while one
          // CTA per class forms F and F_rc
          early_coarse = !aug && g.ncor > 0 && g.nc == 4 && g.nD > 0;
          const int col1 = g.nD + g.nc;
          if (early_coarse) {
            // K_cc of every class from the forward sweep of its four corner columns (k_corner_kcc);
            // F and F_rc then come from the formation below, which leaves K_cc alone
            const int wpb = 4, gridk = std::max(1, (ncls_ + wpb - 1) / wpb);
            prof_start(KC_FORM_CORNER, st);
            cudaError_t ke = cudaErrorInvalidValue;
#define KC_CASE(BV) \
  case BV: k_corner_kcc<T, BV><<<gridk, 32 * wpb, 0, st>>>(prr_, g, mv_, Dinv_, ncls_, Kcc_); ke = cudaGetLastError(); break
            switch (Bp) {
              KC_CASE(8);
              KC_CASE(9);
              KC_CASE(16);
              KC_CASE(17);
              KC_CASE(24);
              KC_CASE(32);
              default: break;
            }
#undef KC_CASE
            ENG_CK(ke);
            prof_stop(KC_FORM_CORNER, st);
            ENG_LAUNCH();
            if (!corner_ev_) ENG_CK(cudaEventCreateWithFlags(&corner_ev_, cudaEventDisableTiming));
            ENG_CK(cudaEventRecord(corner_ev_, st));
          }
          // one CTA per class when the coarse setup runs beside it, so that its blocks retire often
          // and the second stream's blocks are scheduled in between; else persistent CTAs
          const size_t per_cta = (size_t)g.lL * Bp * ldE * cxT;
          int grid = early_coarse ? ncls_ : std::min(ncls_, 8 * nsm_);
          const size_t cap = early_coarse ? ((size_t)1 << 30) : ((size_t)256 << 20);
          grid = std::max(1, (int)std::min<size_t>((size_t)grid, cap / per_cta));
          ENG_CK(alloc(&Xws, (size_t)grid * per_cta));
          prof_start(KC_FORM, st);
          cudaError_t fe = cudaErrorInvalidValue;
#define FC_CASE(BV) \
  case BV: fe = launch_form_cols<T, BV>(prr_, g, mv_, Dinv_, ncls_, F_, FrcF, early_coarse ? nullptr : Kcc_, Xws, grid, ldE, col1, st); break
          switch (Bp) {
            FC_CASE(8);
            FC_CASE(9);
            FC_CASE(16);
            FC_CASE(17);
            FC_CASE(24);
            FC_CASE(32);
            default: break;
          }
#undef FC_CASE
          ENG_CK(fe);
          prof_stop(KC_FORM, st);
          ENG_LAUNCH();
          formed = true;
        }
      }
      if (formed) {
      } else if (g.lb <= 32) {
        constexpr int CW = 4;
        const int ncol = g.nD + g.nc, nchunk = (ncol + CW - 1) / CW, nwork = ncls_ * nchunk;
        const int wpb = 4;
        const int grid = std::max(1, std::min((nwork + wpb - 1) / wpb, 4 * nsm_));
        const size_t smem = wpb * warp_solve_smem<T>(g.lb);
        ENG_CK(alloc(&Xws, (size_t)grid * wpb * g.nl * CW * cxT));
        ENG_CK(smem_attr((const void*)k_form_rr_warp<T, CW>, (int)smem));
        prof_start(KC_FORM, st);
        k_form_rr_warp<T, CW><<<grid, 32 * wpb, smem, st>>>(prr_, g, mv_, Dinv_, ncls_, F_, FrcF, Kcc_, Xws, 0, nchunk);
        prof_stop(KC_FORM, st);
        ENG_LAUNCH();
      } else {
        const int ncol = g.nD + g.nc, nchunk = (ncol + C - 1) / C;
        int grid = std::min(ncls_ * nchunk, 8 * nsm_);
        ENG_CK(alloc(&Xws, (size_t)grid * g.nl * C * cxT));
        size_t smem = 2 * (size_t)g.lb * C * cxT;
        ENG_CK(smem_attr((const void*)k_form_rr<T>, (int)smem));
        prof_start(KC_FORM, st);
        k_form_rr<T><<<grid, 256, smem, st>>>(prr_, g, mv_, Dinv_, ncls_, C, Xws, F_, FrcF, Kcc_, 0);
        prof_stop(KC_FORM, st);
        ENG_LAUNCH();
      }
      if (early_coarse) {
        // coarse factorisation and inverse on the second stream once the corner columns are formed
        // (its allocations are ordered on that stream; joined below)
        ENG_CK(cudaStreamWaitEvent(side_, corner_ev_, 0));
        ast_ = side_;
        const int crc = coarse_setup_bcr(side_, msg);
        ast_ = st;
        if (crc) return crc;
      }
      // join the interior branch (S) and the coarse setup before the buffers are released
      ENG_CK(cudaEventRecord(join_, side_));
      ENG_CK(cudaStreamWaitEvent(st, join_, 0));
      ENG_CK(cudaStreamSynchronize(st));
      if (Xws) free_one(Xws);
      if (Gc) free_one(Gc);
      if (Hc) free_one(Hc);
      free_one(Xi);
      free_one(Sbase);
      free_one(Dii);
    }
    if (aug) {
      // ---- augmented coarse problem: class couplings [Frc | F Q] and coarse blocks, the dense
      // coarse matrix (FP64), its inverse (FP64 Gauss-Jordan), kept as packed tiles in precision T
      const int nq = g.nq;
      cx<double>* Kq = nullptr;
      cx<double>* Kd = nullptr;
      ENG_CK(alloc(&Kq, (size_t)ncls_ * nq * nq * sizeof(cx<double>)));
      const size_t smem = (size_t)g.nD * (nq - g.nc) * cxT + (size_t)g.nD * sizeof(int);
      ENG_CK(smem_attr((const void*)k_aug_local<T>, (int)smem));
      prof_start(KC_COARSE_SETUP, st);
      k_aug_local<T><<<std::max(1, std::min(ncls_, 8 * nsm_)), 256, smem, st>>>(prr_, g, mv_, F_, Frc0, Kcc_, ncls_,
                                                                                 Frc_, Kq);
      ENG_LAUNCH();
      const size_t nn = (size_t)g.nco * g.nco;
      ENG_CK(alloc(&Kd, nn * sizeof(cx<double>)));
      k_aug_assemble<<<(int)std::min<size_t>((nn + 255) / 256, 64 * nsm_), 256, 0, st>>>(g, mv_, Kq, Kd);
      ENG_LAUNCH();
      int crc = dense_gj_inverse(Kd, g.nco, err_ + 2, st, msg, &launches);
      prof_stop(KC_COARSE_SETUP, st);
      if (crc) return crc;
      ncr_ = g.nco;
      ldk_ = (g.nco + 1) & ~1;
      nct_ = (g.nco + kCT - 1) / kCT;
      ENG_CK(alloc(&Kinv_, (size_t)g.nco * ldk_ * cxT));
      ENG_CK(alloc(&Kt_, (size_t)ctile_count(nct_) * kCT * kCT * cxT));
      op_bytes_ += (long long)ctile_count(nct_) * kCT * kCT * cxT;
      prof_start(KC_COARSE_INV, st);
      k_convert_rows<T><<<(int)std::min<size_t>(((size_t)g.nco * ldk_ + 255) / 256, 64 * nsm_), 256, 0, st>>>(
          Kd, g.nco, Kinv_, ldk_);
      ENG_LAUNCH();
      k_pack_ctiles<T><<<(int)std::min<long long>(ctile_count(nct_), 8 * nsm_), 256, 0, st>>>(Kinv_, g.nco, ldk_,
                                                                                            nct_, Kt_);
      prof_stop(KC_COARSE_INV, st);
      ENG_LAUNCH();
      free_one(Kinv_);
      Kinv_ = nullptr;
      free_one(Kd);
      free_one(Kq);
      free_one(Frc0);
    } else if (g.ncor > 0 && !early_coarse) {
      const int crc = coarse_setup_bcr(st, msg);
      if (crc) return crc;
    }
    ENG_CK(cudaStreamSynchronize(st));
    int herr[4];
    ENG_CK(cudaMemcpy(herr, err_, sizeof(herr), cudaMemcpyDeviceToHost));
    if (herr[0] || herr[1] || herr[2]) {
      if (msg) *msg = "zero or non-finite pivot in a subdomain or coarse factorisation";
      return SCHUR_EBREAKDOWN;
    }
    if (herr[3]) {
      if (msg) *msg = "tensor-core local operator formation: completion wait timed out";
      return SCHUR_ETIMEOUT;
    }
    return SCHUR_OK;
  }

  // Corner coarse problem: FP64 block cyclic reduction and the stored inverse in precision T, all
  // work on stream cs (allocations follow ast_); the host does not wait for it.
  int coarse_setup_bcr(cudaStream_t cs, std::string* msg) {
    const Geom& g = g_;
    const size_t cxT = sizeof(cx<T>);
    // ---- coarse problem (FP64 factorisation, inverse stored in T)
    const int nt = nbr_count(g.dim), cbb = g.cb * g.cb;
    ENG_CK(alloc(&CA_, (size_t)g.cL * g.cb * nt * sizeof(cx<double>)));
    ENG_CK(alloc(&CB_, (size_t)std::max(1, g.cL) * g.cb * nt * sizeof(cx<double>)));
    ENG_CK(cudaMemsetAsync(CA_, 0, (size_t)g.cL * g.cb * nt * sizeof(cx<double>), cs));
    ENG_CK(cudaMemsetAsync(CB_, 0, (size_t)std::max(1, g.cL) * g.cb * nt * sizeof(cx<double>), cs));
    const int noff = g.dim == 2 ? 9 : 27;
    long long tot = (long long)g.ncor * noff;
    prof_start(KC_COARSE_SETUP, cs);
    k_coarse_assemble<<<(int)((tot + 255) / 256), 256, 0, cs>>>(g, Kcc_, dm_->sd_cls, CA_, CB_);
    prof_stop(KC_COARSE_SETUP, cs);
    ENG_LAUNCH();
    cprov_.ly.dim = g.dim;
    for (int a = 0; a < 3; ++a) cprov_.ly.ext[a] = a < g.dim ? g.ncg[a] : 1;
    cprov_.ly.b = g.cb;
    cprov_.ly.L = g.cL;
    cprov_.CA = CA_;
    cprov_.CB = CB_;
    // FP64 block cyclic reduction over the coarse layers.  With at least two layers, level 0 is
    // kept as blocks (applied by k_bcr_fwd0 / k_bcr_bwd0 around each coarse solve) and the
    // explicit inverse in precision T covers only the reduced matrix on the surviving layers
    split_ = g.cL >= 2;
    BcrLevel0<T> l0{nullptr, nullptr, nullptr};
    ncr_ = g.ncor;
    if (split_) {
      std::vector<int> tgt, elim, rem;
      bcr_level0_maps(g.cL, &tgt, &elim, &rem);
      nj0_ = (int)elim.size() / 3;
      nr0_ = (int)rem.size();
      ncr_ = g.cb * nr0_;
      auto up = [&](int** d, const std::vector<int>& h) -> cudaError_t {
        cudaError_t e = alloc(d, std::max<size_t>(h.size(), 1) * sizeof(int));
        if (e == cudaSuccess && !h.empty())
          e = cudaMemcpyAsync(*d, h.data(), h.size() * sizeof(int), cudaMemcpyHostToDevice, cs);
        return e;
      };
      ENG_CK(up(&bcr_tgt_, tgt));
      ENG_CK(up(&bcr_elim_, elim));
      ENG_CK(up(&bcr_rem_, rem));  // pageable host tables: staged when the copy is issued
      const size_t nb0 = (size_t)nj0_ * cbb;
      ENG_CK(alloc(&D0_, nb0 * cxT));
      ENG_CK(alloc(&Lp0_, nb0 * cxT));
      ENG_CK(alloc(&Lq0_, nb0 * cxT));
      ENG_CK(alloc(&LpT0_, nb0 * cxT));
      ENG_CK(alloc(&LqT0_, nb0 * cxT));
      op_bytes_ += 5 * (long long)nb0 * cxT;
      l0 = BcrLevel0<T>{D0_, Lp0_, Lq0_};
    }
    ldk_ = (ncr_ + 1) & ~1;  // even row stride of the explicit inverse (temporary)
    nct_ = (ncr_ + kCT - 1) / kCT;
    ENG_CK(alloc(&Kinv_, (size_t)ncr_ * ldk_ * cxT));
    ENG_CK(alloc(&Kt_, (size_t)ctile_count(nct_) * kCT * kCT * cxT));
    op_bytes_ += (long long)ctile_count(nct_) * kCT * kCT * cxT;
    int crc = coarse_bcr<T>(cprov_, split_ ? &l0 : nullptr, Kinv_, ldk_, err_ + 2, cs, msg, &launches);
    if (crc) return crc;
    if (split_) {  // the blocks used transposed by the solve, stored transposed
      const size_t nb0 = (size_t)nj0_ * cbb;
      const int gt = (int)std::min<size_t>((nb0 + 255) / 256, 4096);
      k_transpose_blocks<T><<<gt, 256, 0, cs>>>(Lp0_, nj0_, g.cb, LpT0_);
      ENG_LAUNCH();
      k_transpose_blocks<T><<<gt, 256, 0, cs>>>(Lq0_, nj0_, g.cb, LqT0_);
      ENG_LAUNCH();
    }
    // keep the upper 32 x 32 tiles of the symmetric inverse; the full matrix is released
    prof_start(KC_COARSE_INV, cs);
    k_pack_ctiles<T><<<(int)std::min<long long>(ctile_count(nct_), 8 * nsm_), 256, 0, cs>>>(Kinv_, ncr_, ldk_,
                                                                                          nct_, Kt_);
    prof_stop(KC_COARSE_INV, cs);
    ENG_LAUNCH();
    free_one(Kinv_);
    Kinv_ = nullptr;
    return SCHUR_OK;
  }

  int inner_solve(const double* f, int ldf, double* z, int ldz, int R, double tol, int max_iter, cudaStream_t st,
                  InnerResult* res, std::string* msg) override {
    const Geom& g = g_;
    if (R < 1 || R > kMaxRdev) {
      if (msg) *msg = "inner_solve: R out of range";
      return SCHUR_EINVAL;
    }
    const int m = std::max(1, std::min(max_iter, kMaxKdev - 1));
    ast_ = st;
    int rc = ensure_ws(R, m, msg);
    if (rc) return rc;
    launches = 0;
    const cx<double>* fc = reinterpret_cast<const cx<double>*>(f);
    cx<double>* zc = reinterpret_cast<cx<double>*>(z);
    const size_t cxT = sizeof(cx<T>);
    const bool coarse = g.nco > 0, aug = g.nq > g.nc;
    // ---- local right-hand sides
    rc = local_solves(fc, ldf, nullptr, nullptr, R, true, st, msg);
    if (rc) return rc;
    if (aug) {  // face part of the coarse right-hand side: Q_s^T d_r^s
      const long long nw = (long long)g.nsd * R;
      prof_start(KC_CORNER, st);
      k_face_sums<T><<<(int)((nw * 32 + 255) / 256), 256, 0, st>>>(g, mv_, VD_, R, Tc_);
      prof_stop(KC_CORNER, st);
      ENG_LAUNCH();
    }
    if (coarse) {
      int tot = R * g.nco;
      prof_start(KC_CORNER, st);
      k_corner_gather<T><<<(tot + 255) / 256, 256, 0, st>>>(g, mv_, Tc_, R, fc, ldf, nullptr, T(-1), ftc_);
      prof_stop(KC_CORNER, st);
      ENG_LAUNCH();
      rc = coarse_apply(ftc_, R, nullptr, wc_, st, msg);
      if (rc) return rc;
    }
    int iters = 0, conv = 1;
    // breakdown flags: cleared here too, since a problem without multipliers runs no Krylov loop
    ENG_CK(cudaMemsetAsync(bad_, 0, kMaxRdev * sizeof(int), st));
    if (g.nlam > 0) {
      long long tot = (long long)R * g.nlam;
      prof_start(KC_SCATTER, st);
      k_dual_rhs<T><<<(int)((tot + 255) / 256), 256, 0, st>>>(g, mv_, VD_, Frc_, coarse ? wc_ : nullptr, R, d_);
      prof_stop(KC_SCATTER, st);
      ENG_LAUNCH();
      if (aug && g.nface > 0) {
        const long long nw = (long long)g.nface * R;
        prof_start(KC_SCATTER, st);
        k_dual_project<T><<<(int)((nw * 32 + 255) / 256), 256, 0, st>>>(g, mv_, R, d_);
        prof_stop(KC_SCATTER, st);
        ENG_LAUNCH();
      }
      rc = gmres(R, m, tol, st, &iters, &conv, msg);
      if (rc) return rc;
    }
    // ---- primal recovery
    if (g.nlam > 0) {
      rc = local_apply(false, F_, lam_, R, ones_, coarse, st, msg);  // Tc = Frc^T B^T lambda
      if (rc) return rc;
    }
    if (coarse) {
      int tot = R * g.nco;
      if (g.nlam > 0) {
        prof_start(KC_CORNER, st);
        k_corner_gather<T><<<(tot + 255) / 256, 256, 0, st>>>(g, mv_, Tc_, R, nullptr, 0, ftc_, T(1), gc_);
        prof_stop(KC_CORNER, st);
        ENG_LAUNCH();
        rc = coarse_apply(gc_, R, nullptr, uc_, st, msg);
      } else {
        rc = coarse_apply(ftc_, R, nullptr, uc_, st, msg);
      }
      if (rc) return rc;
      if (aug && g.nlam > 0) {  // multipliers of the local problems: lambda + Q mu
        long long tl = (long long)R * g.nlam;
        prof_start(KC_CORNER, st);
        k_lam_aug<T><<<(int)((tl + 255) / 256), 256, 0, st>>>(g, mv_, uc_, R, lam_);
        prof_stop(KC_CORNER, st);
        ENG_LAUNCH();
      }
    }
    {
      rc = local_solves(fc, ldf, g.nlam > 0 ? lam_ : nullptr, coarse ? uc_ : nullptr, R, false, st, msg);
      if (rc) return rc;
      long long tot = (long long)R * g.n;
      prof_start(KC_ASSEMBLE, st);
      k_assemble_z<T><<<(int)((tot + 255) / 256), 256, 0, st>>>(g, Xs_, coarse ? uc_ : nullptr, R, zc, ldz);
      prof_stop(KC_ASSEMBLE, st);
      ENG_LAUNCH();
    }
    ENG_CK(cudaStreamSynchronize(st));
    int hb[kMaxRdev];
    ENG_CK(cudaMemcpy(hb, bad_, sizeof(int) * R, cudaMemcpyDeviceToHost));
    for (int r = 0; r < R; ++r)
      if (hb[r]) {
        if (msg) *msg = "non-finite value in the Krylov iteration";
        return SCHUR_EBREAKDOWN;
      }
    if (res) {
      res->iters = iters;
      res->converged = conv;
    }
    return SCHUR_OK;
  }

  int debug_operator(int which, int cls, double* out, long long cap, cudaStream_t st, std::string* msg) override {
    const Geom& g = g_;
    ENG_CK(cudaStreamSynchronize(st));
    std::vector<cx<double>> host;
    auto fetch = [&](const cx<T>* src, size_t cnt) -> int {
      std::vector<cx<T>> tmp(cnt);
      cudaError_t e = cudaMemcpy(tmp.data(), src, cnt * sizeof(cx<T>), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return SCHUR_ECUDA;
      host.resize(cnt);
      for (size_t i = 0; i < cnt; ++i) host[i] = ccast<double>(tmp[i]);
      return 0;
    };
    int rc = 0;
    if ((which <= 2 || which == 5 || which == 6) && (cls < 0 || cls >= ncls_)) return SCHUR_EINVAL;
    auto unpack = [&]() {  // packed upper triangle -> full symmetric matrix
      std::vector<cx<double>> full((size_t)g.nD * g.nD);
      for (int i = 0; i < g.nD; ++i)
        for (int j = 0; j < g.nD; ++j) full[(size_t)i * g.nD + j] = host[sym_idx(i, j, g.nD)];
      host.swap(full);
    };
    if (which == 0) {
      rc = fetch(F_ + (size_t)cls * sym_ld(g.nD), (size_t)sym_ld(g.nD));
      if (!rc) unpack();
    } else if (which == 1 || which == 5) {
      // coupling columns of the class (nD x nq); which = 1 keeps the corner columns
      rc = fetch(Frc_ + (size_t)cls * g.nD * g.nq, (size_t)g.nD * g.nq);
      if (!rc && which == 1 && g.nq != g.nc) {
        std::vector<cx<double>> fr((size_t)g.nD * g.nc);
        for (int j = 0; j < g.nD; ++j)
          for (int c = 0; c < g.nc; ++c) fr[(size_t)j * g.nc + c] = host[(size_t)j * g.nq + c];
        host.swap(fr);
      }
    } else if (which == 2) {
      rc = fetch(Sd_ + (size_t)cls * sym_ld(g.nD), (size_t)sym_ld(g.nD));
      if (!rc) unpack();
    }
    else if (which == 3 || which == 4) {
      if (g.nco == 0 || (which == 3 && g.nq != g.nc)) return SCHUR_EINVAL;
      if (which == 4 && split_) {
        // the coarse solve applied to the identity, kMaxRdev columns at a time
        int erc = ensure_ws(kMaxRdev, std::max(1, wsM_), msg);
        if (erc) return erc;
        const int n = g.nco;
        host.assign((size_t)n * n, mkc<double>(0, 0));
        std::vector<cx<T>> e((size_t)kMaxRdev * n), wv((size_t)kMaxRdev * n);
        for (int c0 = 0; c0 < n; c0 += kMaxRdev) {
          const int R = std::min(kMaxRdev, n - c0);
          std::fill(e.begin(), e.end(), mkc<T>(T(0), T(0)));
          for (int r = 0; r < R; ++r) e[(size_t)r * n + c0 + r] = mkc<T>(T(1), T(0));
          ENG_CK(cudaMemcpy(gc_, e.data(), (size_t)R * n * sizeof(cx<T>), cudaMemcpyHostToDevice));
          erc = coarse_apply(gc_, R, nullptr, wc_, st, msg);
          if (erc) return erc;
          ENG_CK(cudaStreamSynchronize(st));
          ENG_CK(cudaMemcpy(wv.data(), wc_, (size_t)R * n * sizeof(cx<T>), cudaMemcpyDeviceToHost));
          for (int r = 0; r < R; ++r)
            for (int i = 0; i < n; ++i) host[(size_t)i * n + c0 + r] = ccast<double>(wv[(size_t)r * n + i]);
        }
      } else if (which == 4) {
        rc = fetch(Kt_, (size_t)ctile_count(nct_) * kCT * kCT);
        if (!rc) {  // upper tiles -> full symmetric matrix (lower tiles are the transposes)
          std::vector<cx<double>> full((size_t)g.nco * g.nco);
          for (int i = 0; i < g.nco; ++i)
            for (int j = 0; j < g.nco; ++j) {
              const int I = i / kCT, J = j / kCT;
              const size_t e = I <= J ? (size_t)ctile_idx(I, J, nct_) * kCT * kCT + (i % kCT) * kCT + j % kCT
                                      : (size_t)ctile_idx(J, I, nct_) * kCT * kCT + (j % kCT) * kCT + i % kCT;
              full[(size_t)i * g.nco + j] = host[e];
            }
          host.swap(full);
        }
      } else {
        const int nt = nbr_count(g.dim);
        std::vector<cx<double>> ca((size_t)g.cL * g.cb * nt), cb((size_t)g.cL * g.cb * nt);
        if (cudaMemcpy(ca.data(), CA_, ca.size() * sizeof(cx<double>), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(cb.data(), CB_, cb.size() * sizeof(cx<double>), cudaMemcpyDeviceToHost) != cudaSuccess)
          return SCHUR_ECUDA;
        host.assign((size_t)g.ncor * g.ncor, mkc<double>(0, 0));
        int ext0 = g.ncg[0], ext1 = g.dim == 3 ? g.ncg[1] : 1;
        for (int K = 0; K < g.cL; ++K)
          for (int i = 0; i < g.cb; ++i)
            for (int t = 0; t < nt; ++t) {
              int d0 = t % 3 - 1, d1 = g.dim == 3 ? t / 3 - 1 : 0;
              int c0 = i % ext0 + d0, c1 = (g.dim == 3 ? i / ext0 : 0) + d1;
              if (c0 < 0 || c0 >= ext0 || c1 < 0 || c1 >= ext1) continue;
              int j = c0 + ext0 * c1;
              size_t row = (size_t)K * g.cb + i;
              host[row * g.ncor + (size_t)K * g.cb + j] = ca[((size_t)K * g.cb + i) * nt + t];
              if (K > 0) {
                cx<double> v = cb[((size_t)(K - 1) * g.cb + i) * nt + t];
                size_t col = (size_t)(K - 1) * g.cb + j;
                host[row * g.ncor + col] = v;
                host[col * g.ncor + row] = v;
              }
            }
      }
    } else if (which == 6) {
      // layer pivot inverses D_K^{-1} of the remainder factorisation (L blocks of b x b)
      const size_t blk = (size_t)g.lL * g.lb * g.lb;
      rc = fetch(Dinv_ + (size_t)cls * blk, blk);
    } else {
      return SCHUR_EINVAL;
    }
    if (rc) return rc;
    if ((long long)host.size() > cap) return SCHUR_EINVAL;
    std::memcpy(out, host.data(), host.size() * sizeof(cx<double>));
    return SCHUR_OK;
  }

 private:
  template <class P>
  // Stream-ordered allocations from the device's default memory pool (kept by the pool after a
  // context is destroyed, so the next setup on the same device does not map memory again).
  cudaError_t alloc(P** p, size_t bytes) {
    void* v = nullptr;
    cudaError_t e = cudaMallocAsync(&v, std::max<size_t>(bytes, 16), ast_);
    if (e == cudaSuccess) {
      allocs_.push_back(v);
      *p = reinterpret_cast<P*>(v);
    }
    return e;
  }
  void free_one(void* p) {
    auto it = std::find(allocs_.begin(), allocs_.end(), p);
    if (it != allocs_.end()) {
      cudaFreeAsync(p, ast_);
      allocs_.erase(it);
    }
  }

  int ensure_ws(int R, int m, std::string* msg) {
    if (R <= wsR_ && m <= wsM_) return SCHUR_OK;
    for (void* p : ws_) free_one(p);
    ws_.clear();
    const Geom& g = g_;
    R = std::max(R, wsR_);
    m = std::max(m, wsM_);
    const size_t cxT = sizeof(cx<T>);
    auto wa = [&](auto** p, size_t bytes) -> cudaError_t {
      cudaError_t e = alloc(p, bytes);
      if (e == cudaSuccess) ws_.push_back((void*)*p);
      return e;
    };
    const size_t nl = std::max(1, g.nlam), nco = std::max(1, g.nco);
    ENG_CK(wa(&Xs_, (size_t)g.nsd * g.nl * R * cxT));
    ENG_CK(wa(&VD_, (size_t)g.nsd * R * g.nD * cxT));
    ENG_CK(wa(&Y_, (size_t)g.nsd * R * g.nD * cxT));
    ENG_CK(wa(&Tc_, (size_t)g.nsd * R * g.nq * cxT));
    ENG_CK(wa(&d_, nl * R * cxT));
    ENG_CK(wa(&zv_, nl * R * cxT));
    ENG_CK(wa(&lam_, nl * R * cxT));
    ENG_CK(wa(&V_, nl * R * (m + 1) * cxT));
    ENG_CK(wa(&ftc_, nco * R * cxT));
    ENG_CK(wa(&gc_, nco * R * cxT));
    ENG_CK(wa(&wc_, nco * R * cxT));
    ENG_CK(wa(&uc_, nco * R * cxT));
    if (g.nco > 0) {
      const size_t np = (size_t)ctile_count(nct_) * kCT * R;
      ENG_CK(wa(&cpu_, np * cxT));
      ENG_CK(wa(&cpv_, np * cxT));
    }
    if (split_) {
      ENG_CK(wa(&cfr_, (size_t)ncr_ * R * cxT));
      ENG_CK(wa(&cxr_, (size_t)ncr_ * R * cxT));
    }
    nblk_ = std::max(1, std::min((int)((nl + 255) / 256), 2 * nsm_));
    nblk_ = std::max(nblk_, (int)((nl + 2047) / 2048));
    ENG_CK(wa(&part_, (size_t)kMaxRdev * kMaxKdev * nblk_ * sizeof(cx<double>)));
    ENG_CK(wa(&H_, (size_t)R * m * (m + 1) * sizeof(cx<double>)));
    ENG_CK(wa(&hc_, (size_t)kMaxRdev * kMaxKdev * sizeof(cx<double>)));
    ENG_CK(wa(&gvec_, (size_t)R * (m + 1) * sizeof(cx<double>)));
    ENG_CK(wa(&cs_s_, (size_t)R * m * sizeof(cx<double>)));
    ENG_CK(wa(&cs_c_, (size_t)R * m * sizeof(double)));
    ENG_CK(wa(&y_, (size_t)kMaxRdev * kMaxKdev * sizeof(cx<double>)));
    ENG_CK(wa(&nrm_part_, (size_t)kMaxRdev * nblk_ * sizeof(double)));
    ENG_CK(wa(&beta0_, kMaxRdev * sizeof(double)));
    ENG_CK(wa(&inv_nrm_, kMaxRdev * sizeof(double)));
    ENG_CK(wa(&resid_, kMaxRdev * sizeof(double)));
    ENG_CK(wa(&active_, kMaxRdev * sizeof(int)));
    ENG_CK(wa(&kk_, kMaxRdev * sizeof(int)));
    ENG_CK(wa(&bad_, kMaxRdev * sizeof(int)));
    ENG_CK(wa(&cnt_, kMaxRdev * sizeof(int)));
    ENG_CK(cudaMemsetAsync(cnt_, 0, kMaxRdev * sizeof(int), ast_));  // tickets of the fused reductions
    if (!h_active_) ENG_CK(cudaMallocHost(&h_active_, 2 * kMaxRdev * sizeof(int)));
    wsR_ = R;
    wsM_ = m;
    return SCHUR_OK;
  }

  // Local remainder solves of every subdomain: the right-hand-side split (rhs_split: VD, Tc) or the
  // primal recovery (lam, uc given; solution left in Xs).
  int local_solves(const cx<double>* fc, int ldf, const cx<T>* lam, const cx<T>* uc, int R, bool rhs_split,
                   cudaStream_t st, std::string* msg) {
    const Geom& g = g_;
    const int cat = rhs_split ? KC_LOCAL_RHS : KC_RECOVER;
    if (g.lb <= 32) {
      const int wpb = 4, grid = (g.nsd + wpb - 1) / wpb;
      const size_t smem = wpb * warp_solve_smem<T>(g.lb);
      cx<T>* vd = rhs_split ? VD_ : nullptr;
      cx<T>* tc = rhs_split ? Tc_ : nullptr;
#define LS_ATTR(C) ENG_CK(smem_attr((const void*)k_local_solve_warp<T, C>, (int)smem))
      if (R == 1) LS_ATTR(1);
      else if (R == 2) LS_ATTR(2);
      else if (R <= 4) LS_ATTR(4);
      else if (R <= 8) LS_ATTR(8);
      else LS_ATTR(16);
#undef LS_ATTR
      prof_start(cat, st);
      {  // all remainder right-hand sides first, one thread per (subdomain, node, column)
        const long long tot = (long long)g.nsd * g.nl * R;
        k_remainder_rhs<T><<<(int)std::min<long long>((tot + 255) / 256, 16LL * nsm_), 256, 0, st>>>(prr_, g, mv_, fc, ldf,
                                                                                                   lam, uc, R, Xs_);
        ENG_LAUNCH();
      }
      if (R == 1) k_local_solve_warp<T, 1><<<grid, 32 * wpb, smem, st>>>(prr_, g, mv_, Dinv_, fc, ldf, lam, uc, R, Xs_, vd, tc, 1);
      else if (R == 2) k_local_solve_warp<T, 2><<<grid, 32 * wpb, smem, st>>>(prr_, g, mv_, Dinv_, fc, ldf, lam, uc, R, Xs_, vd, tc, 1);
      else if (R <= 4) k_local_solve_warp<T, 4><<<grid, 32 * wpb, smem, st>>>(prr_, g, mv_, Dinv_, fc, ldf, lam, uc, R, Xs_, vd, tc, 1);
      else if (R <= 8) k_local_solve_warp<T, 8><<<grid, 32 * wpb, smem, st>>>(prr_, g, mv_, Dinv_, fc, ldf, lam, uc, R, Xs_, vd, tc, 1);
      else k_local_solve_warp<T, 16><<<grid, 32 * wpb, smem, st>>>(prr_, g, mv_, Dinv_, fc, ldf, lam, uc, R, Xs_, vd, tc, 1);
      prof_stop(cat, st);
      ENG_LAUNCH();
      return SCHUR_OK;
    }
    int thr = std::min(256, ((g.lb * R + 31) / 32) * 32);
    size_t smem = 2 * (size_t)g.lb * R * sizeof(cx<T>);
    if (rhs_split) {
      ENG_CK(smem_attr((const void*)k_local_rhs<T>, (int)smem));
      prof_start(cat, st);
      k_local_rhs<T><<<g.nsd, thr, smem, st>>>(prr_, g, mv_, Dinv_, fc, ldf, R, Xs_, VD_, Tc_);
      prof_stop(cat, st);
    } else {
      ENG_CK(smem_attr((const void*)k_recover<T>, (int)smem));
      prof_start(cat, st);
      k_recover<T><<<g.nsd, thr, smem, st>>>(prr_, g, mv_, Dinv_, fc, ldf, lam, uc, R, Xs_);
      prof_stop(cat, st);
    }
    ENG_LAUNCH();
    return SCHUR_OK;
  }

  // w = K_cc^{-1} g with g = gv, or (split form only, gv null) assembled from the corner couplings Tcs
  int coarse_apply(const cx<T>* gv, int R, const int* active, cx<T>* w, cudaStream_t st, std::string* msg,
                   const cx<T>* Tcs = nullptr) {
    const long long ntile = ctile_count(nct_);
    prof_start(KC_COARSE_APPLY, st);
    if (split_) {
      // level-0 forward step, reduced inverse, level-0 backward step
      const int b = g_.cb, ns = (b + 31) / 32, nz = (R + kBcrRC - 1) / kBcrRC;
      const size_t sm = (size_t)kBcrRC * (3 * (size_t)b + 256) * sizeof(cx<T>);
      ENG_CK(smem_attr((const void*)k_bcr_fwd0<T>, (int)sm));
      ENG_CK(smem_attr((const void*)k_bcr_bwd0<T>, (int)sm));
      ENG_CK(launch_pdl(k_bcr_fwd0<T>, dim3(nr0_, ns, nz), dim3(256), sm, st, g_, (const int*)bcr_tgt_,
                        (const cx<T>*)Lp0_, (const cx<T>*)LqT0_, gv, Tcs, cfr_, ncr_, R, active));
      ENG_CK(launch_pdl(k_coarse_tiles<T>, dim3((unsigned)((ntile + 3) / 4)), dim3(128), 0, st, Kt_, nct_, ncr_,
                        (const cx<T>*)cfr_, R, active, cpu_, cpv_));
      ENG_CK(launch_pdl(k_coarse_reduce<T>, dim3(nct_ * R), dim3(512), 0, st, cpu_, cpv_, nct_, ncr_, R, active, cxr_));
      ENG_CK(launch_pdl(k_bcr_bwd0<T>, dim3(nj0_ + nr0_, ns, nz), dim3(256), sm, st, g_, nj0_, (const int*)bcr_elim_,
                        (const int*)bcr_rem_, (const cx<T>*)D0_, (const cx<T>*)LpT0_, (const cx<T>*)Lq0_, gv, Tcs,
                        (const cx<T>*)cxr_, ncr_, w, R, active));
      prof_stop(KC_COARSE_APPLY, st);
      ENG_LAUNCH();
      ENG_LAUNCH();
      ENG_LAUNCH();
      ENG_LAUNCH();
      return SCHUR_OK;
    }
    ENG_CK(launch_pdl(k_coarse_tiles<T>, dim3((unsigned)((ntile + 3) / 4)), dim3(128), 0, st, Kt_, nct_, g_.nco, gv, R,
                      active, cpu_, cpv_));
    ENG_CK(launch_pdl(k_coarse_reduce<T>, dim3(nct_ * R), dim3(512), 0, st, cpu_, cpv_, nct_, g_.nco, R, active, w));
    prof_stop(KC_COARSE_APPLY, st);
    ENG_LAUNCH();
    ENG_LAUNCH();
    return SCHUR_OK;
  }

  // Y = Op x with x = (scaled) B^T v gathered per subdomain; Tc = Frc^T x when want_tc.
  // vscale (optional, per right-hand side) multiplies the gathered vector.
  int local_apply(bool precond, const cx<T>* Op, const cx<T>* v, int R, const int* active, bool want_tc,
                  cudaStream_t st, std::string* msg, const double* vscale = nullptr) {
    const Geom& g = g_;
    if (R == 1 && g.nD > 128) {
      // one right-hand side, large blocks: rows streamed with coalesced loads
      const int thr = 512;
      const size_t smem = (((size_t)g.nD + 1) & ~(size_t)1) * sizeof(cx<T>) + (size_t)(thr / 32) * g.nD * sizeof(cx<T>);
      cx<T>* tc = want_tc ? Tc_ : nullptr;
      if (precond) {
        ENG_CK(smem_attr((const void*)k_local_apply_rows<T, true>, (int)smem));
        prof_start(KC_APPLY_S, st);
        ENG_CK(launch_pdl(k_local_apply_rows<T, true>, dim3(g.nsd), dim3(thr), smem, st, g, mv_, Op, Frc_, v, active, Y_,
                          tc, vscale));
        prof_stop(KC_APPLY_S, st);
      } else {
        ENG_CK(smem_attr((const void*)k_local_apply_rows<T, false>, (int)smem));
        prof_start(KC_APPLY_F, st);
        ENG_CK(launch_pdl(k_local_apply_rows<T, false>, dim3(g.nsd), dim3(thr), smem, st, g, mv_, Op, Frc_, v, active,
                          Y_, tc, vscale));
        prof_stop(KC_APPLY_F, st);
      }
      ENG_LAUNCH();
      return SCHUR_OK;
    }
    if (R <= 2 && ngrp_ > 0 && 2 * (long long)ngrp_ <= g.nsd && g.nD <= 256) {
      // subdomains of one class in groups: each staged operator serves the whole group
      const size_t smem = ((size_t)g.nD * g.nD + (size_t)kApplyGroup * R * g.nD +
                           (want_tc ? (size_t)g.nD * g.nq : 0)) * sizeof(cx<T>);
      if (smem <= ((size_t)100 << 10)) {
        cx<T>* tc = want_tc ? Tc_ : nullptr;
#define LG_CASE(SC)                                                                                           \
  do {                                                                                                        \
    ENG_CK(smem_attr((const void*)k_local_apply_grp<T, SC, 2>, (int)smem));                                  \
    prof_start(SC ? KC_APPLY_S : KC_APPLY_F, st);                                                             \
    ENG_CK(launch_pdl(k_local_apply_grp<T, SC, 2>, dim3(ngrp_), dim3(256), smem, st, g, mv_, Op, Frc_, v, R, \
                      active, Y_, tc, vscale));                                                               \
    prof_stop(SC ? KC_APPLY_S : KC_APPLY_F, st);                                                              \
  } while (0)
        if (precond) LG_CASE(true);
        else LG_CASE(false);
#undef LG_CASE
        ENG_LAUNCH();
        return SCHUR_OK;
      }
    }
    if (R == 1 && g.nD <= 128 && g.nq <= 16) {
      const size_t smem1 = ((size_t)sym_ld(g.nD) + (((size_t)g.nD + 1) & ~(size_t)1)) * sizeof(cx<T>);
      if (smem1 <= ((size_t)96 << 10)) {
        const int thr1 = ((g.nD + 31) / 32) * 32;
        cx<T>* tc = want_tc ? Tc_ : nullptr;
#define L1_CASE(SC)                                                                                            \
  do {                                                                                                         \
    ENG_CK(smem_attr((const void*)k_local_apply_1<T, SC>, (int)smem1));                                       \
    prof_start(SC ? KC_APPLY_S : KC_APPLY_F, st);                                                              \
    ENG_CK(launch_pdl(k_local_apply_1<T, SC>, dim3(g.nsd), dim3(thr1), smem1, st, g, mv_, Op, Frc_, v, active, \
                      Y_, tc, vscale));                                                                        \
    prof_stop(SC ? KC_APPLY_S : KC_APPLY_F, st);                                                               \
  } while (0)
        if (precond) L1_CASE(true);
        else L1_CASE(false);
#undef L1_CASE
        ENG_LAUNCH();
        return SCHUR_OK;
      }
    }
    int thr = std::min(512, ((g.nD + 31) / 32) * 32);
    const size_t xcnt = ((size_t)R * g.nD + 1) & ~(size_t)1;
    const size_t opb = (size_t)sym_ld(g.nD) * sizeof(cx<T>);
    const int stage = (xcnt * sizeof(cx<T>) + opb <= ((size_t)96 << 10)) ? 1 : 0;
    size_t smem = xcnt * sizeof(cx<T>) + (stage ? opb : 0);
    cx<T>* tc = want_tc ? Tc_ : nullptr;
#define LA_CASE(SC, MR)                                                                                 \
  do {                                                                                                  \
    ENG_CK(smem_attr((const void*)k_local_apply<T, SC, MR>,                                       \
                                (int)std::max<size_t>(smem, 1)));                                       \
    prof_start(SC ? KC_APPLY_S : KC_APPLY_F, st);                                                      \
    ENG_CK(launch_pdl(k_local_apply<T, SC, MR>, dim3(g.nsd), dim3(thr), smem, st, g, mv_, Op, Frc_, v, R, active, Y_, \
                      tc, stage, vscale));                                                                             \
    prof_stop(SC ? KC_APPLY_S : KC_APPLY_F, st);                                                       \
  } while (0)
    if (precond) {
      if (R == 1) LA_CASE(true, 1);
      else if (R <= 4) LA_CASE(true, 4);
      else if (R <= 8) LA_CASE(true, 8);
      else LA_CASE(true, 16);
    } else {
      if (R == 1) LA_CASE(false, 1);
      else if (R <= 4) LA_CASE(false, 4);
      else if (R <= 8) LA_CASE(false, 8);
      else LA_CASE(false, 16);
    }
#undef LA_CASE
    ENG_LAUNCH();
    return SCHUR_OK;
  }

  // out = P^{-1} (diag(vscale) v)  (Dirichlet preconditioner; vscale optional)
  int precond(const cx<T>* v, int R, const int* active, cx<T>* out, cudaStream_t st, std::string* msg,
              const double* vscale = nullptr) {
    int rc = local_apply(true, Sd_, v, R, active, false, st, msg, vscale);
    if (rc) return rc;
    long long tot = (long long)R * g_.nlam;
    prof_start(KC_SCATTER, st);
    ENG_CK(launch_pdl(k_scatter<T, true>, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st, g_, mv_, Y_,
                      (const cx<T>*)nullptr, (const cx<T>*)nullptr, R, active, out));
    prof_stop(KC_SCATTER, st);
    ENG_LAUNCH();
    return SCHUR_OK;
  }

  // out = F_DP v = F_rr v + Frc~ Kcc~^{-1} Frc~^T v
  // out = F_DP v; with oa set, the closing scatter also takes the first Gram-Schmidt dots of out
  // against the Krylov basis (k_scatter_orth_dots)
  int dual_apply(const cx<T>* v, int R, const int* active, cx<T>* out, cudaStream_t st, std::string* msg,
                 const OrthArgs* oa = nullptr) {
    const bool coarse = g_.nco > 0;
    int rc = local_apply(false, F_, v, R, active, coarse, st, msg);
    if (rc) return rc;
    if (coarse && split_) {
      // the level-0 steps of the coarse solve assemble g from the corner couplings themselves
      rc = coarse_apply(nullptr, R, active, wc_, st, msg, Tc_);
      if (rc) return rc;
    } else if (coarse) {
      int tot = R * g_.nco;
      prof_start(KC_CORNER, st);
      ENG_CK(launch_pdl(k_corner_gather<T>, dim3((tot + 255) / 256), dim3(256), 0, st, g_, mv_, Tc_, R,
                        (const cx<double>*)nullptr, 0, (const cx<T>*)nullptr, T(1), gc_));
      prof_stop(KC_CORNER, st);
      ENG_LAUNCH();
      rc = coarse_apply(gc_, R, active, wc_, st, msg);
      if (rc) return rc;
    }
    if (oa) {
      const int seg = (g_.nlam + oa->nblk - 1) / oa->nblk;
      prof_start(KC_GMRES_DOTS, st);
      ENG_CK(launch_pdl(k_scatter_orth_dots<T>, dim3(oa->nblk, R), dim3(256), (size_t)seg * sizeof(cx<T>), st, g_, mv_,
                        Y_, Frc_, coarse ? wc_ : nullptr, V_, out, R, *oa));
      prof_stop(KC_GMRES_DOTS, st);
      ENG_LAUNCH();
      return SCHUR_OK;
    }
    long long tot = (long long)R * g_.nlam;
    prof_start(KC_SCATTER, st);
    ENG_CK(launch_pdl(k_scatter<T, false>, dim3((unsigned)((tot + 255) / 256)), dim3(256), 0, st, g_, mv_, Y_, Frc_,
                      coarse ? wc_ : nullptr, R, active, out));
    prof_stop(KC_SCATTER, st);
    ENG_LAUNCH();
    return SCHUR_OK;
  }

  int gmres(int R, int m, double tol, cudaStream_t st, int* iters, int* conv, std::string* msg) {
    const Geom& g = g_;
    const int nlam = g.nlam, nblk = nblk_;
    const long long vstride = (long long)R * nlam;
    const size_t cxT = sizeof(cx<T>);
    const int gs = std::max(1, std::min((nlam + 255) / 256, 4 * nsm_));
    ENG_CK(cudaMemsetAsync(H_, 0, (size_t)R * m * (m + 1) * sizeof(cx<double>), st));
    ENG_CK(cudaMemsetAsync(bad_, 0, kMaxRdev * sizeof(int), st));
    prof_start(KC_GMRES_OTHER, st);
    k_norm2<T><<<dim3(nblk, R), 256, 0, st>>>(d_, nlam, R, nullptr, nblk, nrm_part_);
    prof_stop(KC_GMRES_OTHER, st);
    ENG_LAUNCH();
    ENG_CK(cudaMemcpyAsync(V_, d_, (size_t)R * nlam * cxT, cudaMemcpyDeviceToDevice, st));
    prof_start(KC_GMRES_OTHER, st);
    k_gmres_init<<<R, 32, 0, st>>>(R, nrm_part_, nblk, m, beta0_, gvec_, active_, kk_, inv_nrm_, resid_);
    prof_stop(KC_GMRES_OTHER, st);
    ENG_LAUNCH();
    prof_start(KC_GMRES_OTHER, st);
    k_scale_vec<T><<<dim3(gs, R), 256, 0, st>>>(V_, nlam, R, active_, inv_nrm_);
    prof_stop(KC_GMRES_OTHER, st);
    ENG_LAUNCH();
    const int seg = (nlam + nblk - 1) / nblk;
    const size_t dot_smem = (size_t)seg * cxT, upd_smem = (size_t)(seg + m + 1) * cxT;
    ENG_CK(smem_attr((const void*)k_scatter_orth_dots<T>, (int)dot_smem));
    ENG_CK(smem_attr((const void*)k_orth_update_dots<T>, (int)upd_smem));
    ENG_CK(smem_attr((const void*)k_orth_update_norm<T>, (int)upd_smem));
    OrthArgs oa;
    oa.vstride = vstride;
    oa.nlam = nlam;
    oa.m = m;
    oa.nblk = nblk;
    oa.active = active_;
    oa.part = part_;
    oa.nrm_part = nrm_part_;
    oa.cnt = cnt_;
    oa.H = H_;
    oa.hc = hc_;
    oa.cs_c = cs_c_;
    oa.cs_s = cs_s_;
    oa.gvec = gvec_;
    oa.beta0 = beta0_;
    oa.tol = tol;
    oa.active_w = active_;
    oa.kk = kk_;
    oa.inv_nrm = inv_nrm_;
    oa.resid = resid_;
    oa.bad = bad_;
    oa.lazy = 0;
    const int check_every = 4;
    int k = 0;
    for (; k < m; ++k) {
      cx<T>* vk = V_ + k * vstride;
      cx<T>* vk1 = V_ + (k + 1) * vstride;
      // v_k (k > 0) is normalised lazily: the preconditioner scales what it gathers, and the first
      // Gram-Schmidt pass scales v_k in place before reading it
      int rc = precond(vk, R, active_, zv_, st, msg, k > 0 ? inv_nrm_ : nullptr);
      if (rc) return rc;
      oa.k = k;
      oa.lazy = k > 0 ? 1 : 0;
      rc = dual_apply(zv_, R, active_, vk1, st, msg, &oa);  // with the first Gram-Schmidt dots
      if (rc) return rc;
      const dim3 og(nblk, R);
      prof_start(KC_GMRES_UPDATE, st);
      ENG_CK(launch_pdl(k_orth_update_dots<T>, og, dim3(256), upd_smem, st, V_, vk1, oa));
      prof_stop(KC_GMRES_UPDATE, st);
      ENG_LAUNCH();
      prof_start(KC_GMRES_OTHER, st);
      ENG_CK(launch_pdl(k_orth_update_norm<T>, og, dim3(256), upd_smem, st, V_, vk1, oa));
      prof_stop(KC_GMRES_OTHER, st);
      ENG_LAUNCH();
      if ((k + 1) % check_every == 0 || k + 1 == m) {
        ENG_CK(cudaMemcpyAsync(h_active_, active_, R * sizeof(int), cudaMemcpyDeviceToHost, st));
        ENG_CK(cudaStreamSynchronize(st));
        bool any = false;
        for (int r = 0; r < R; ++r) any = any || h_active_[r];
        if (!any) break;
      }
    }
    prof_start(KC_GMRES_OTHER, st);
    k_hess_solve<<<R, 256, 0, st>>>(m, H_, gvec_, kk_, y_);
    prof_stop(KC_GMRES_OTHER, st);
    ENG_LAUNCH();
    prof_start(KC_GMRES_OTHER, st);
    k_combine<T><<<dim3(gs, R), 256, (size_t)m * cxT, st>>>(V_, vstride, nlam, R, y_, kk_, d_);
    prof_stop(KC_GMRES_OTHER, st);
    ENG_LAUNCH();
    int rc = precond(d_, R, ones_, lam_, st, msg);
    if (rc) return rc;
    ENG_CK(cudaMemcpyAsync(h_active_, kk_, R * sizeof(int), cudaMemcpyDeviceToHost, st));
    ENG_CK(cudaMemcpyAsync(h_active_ + kMaxRdev, active_, R * sizeof(int), cudaMemcpyDeviceToHost, st));
    ENG_CK(cudaStreamSynchronize(st));
    double hres[kMaxRdev], hb0[kMaxRdev];
    ENG_CK(cudaMemcpy(hres, resid_, R * sizeof(double), cudaMemcpyDeviceToHost));
    ENG_CK(cudaMemcpy(hb0, beta0_, R * sizeof(double), cudaMemcpyDeviceToHost));
    int it = 0, ok = 1;
    for (int r = 0; r < R; ++r) {
      it = std::max(it, h_active_[r]);
      if (hb0[r] > 0 && hres[r] > tol * hb0[r]) ok = 0;
    }
    *iters = it;
    *conv = ok;
    return SCHUR_OK;
  }

  const HostMaps* hm_;
  const DevMaps* dm_;
  Geom g_;
  double gamma_;
  MapsView mv_;
  Stencil<T> st_;
  StencilProv<T> prr_, pii_;
  StoredProv<double> cprov_;
  int ncls_ = 0, ngrp_ = 0, nsm_ = 152, nblk_ = 1, coarse_cluster_ = 0, ldk_ = 0, nct_ = 0;
  long long op_bytes_ = 0;
  std::vector<void*> allocs_, ws_;
  int* err_ = nullptr;
  int* ones_ = nullptr;
  cx<T>*Dinv_ = nullptr, *F_ = nullptr, *Frc_ = nullptr, *Sd_ = nullptr, *Kinv_ = nullptr, *Kt_ = nullptr;
  // coarse solve: level 0 of the reduction kept as blocks around the reduced inverse (split_)
  bool split_ = false;
  int ncr_ = 0, nj0_ = 0, nr0_ = 0;  // unknowns of the stored inverse; layers eliminated / kept at level 0
  int *bcr_tgt_ = nullptr, *bcr_elim_ = nullptr, *bcr_rem_ = nullptr;
  cx<T>*D0_ = nullptr, *Lp0_ = nullptr, *Lq0_ = nullptr, *LpT0_ = nullptr, *LqT0_ = nullptr, *cfr_ = nullptr,
  *cxr_ = nullptr;
  cx<T>*cpu_ = nullptr, *cpv_ = nullptr;  // partial products of the packed coarse inverse
  cx<double>*Kcc_ = nullptr, *CA_ = nullptr, *CB_ = nullptr, *Dc_ = nullptr;
  int wsR_ = 0, wsM_ = 0;
  cx<T>*Xs_ = nullptr, *VD_ = nullptr, *Y_ = nullptr, *Tc_ = nullptr, *d_ = nullptr, *zv_ = nullptr, *lam_ = nullptr,
  *V_ = nullptr, *ftc_ = nullptr, *gc_ = nullptr, *wc_ = nullptr, *uc_ = nullptr;
  cx<double>*part_ = nullptr, *H_ = nullptr, *hc_ = nullptr, *gvec_ = nullptr, *cs_s_ = nullptr, *y_ = nullptr;
  double *cs_c_ = nullptr, *nrm_part_ = nullptr, *beta0_ = nullptr, *inv_nrm_ = nullptr, *resid_ = nullptr;
  int *active_ = nullptr, *kk_ = nullptr, *bad_ = nullptr, *cnt_ = nullptr;
  int* h_active_ = nullptr;
  cudaStream_t ast_ = nullptr;  // stream of the current setup / solve (stream-ordered allocations)
  cudaStream_t side_ = nullptr;  // second setup stream (interior branch)
  cudaEvent_t fork_ = nullptr, join_ = nullptr, corner_ev_ = nullptr;
};

}  // namespace schur
