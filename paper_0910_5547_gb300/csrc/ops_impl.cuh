// ops_impl.cuh -- Ops<T, NV>: launch configuration of every kernel for one
// (precision, physics) pair.  Included by the four ops_*.cu units only.
#pragma once
#include "kernels.cuh"
#include "ops.h"

namespace amr {

template <typename T, int NV>
struct Ops final : OpsBase {
  Phys<T> ph{};
  double gamma = 1.4;
  int occ = 0;   // 0: default build; kAlt: the alternate register budget
  bool weno = false;   // third-order WENO face states: the default build with WENO = true
  // default resident CTAs per SM of the stage kernel, and the alternate build
  // (FP32 Euler: 2 -> 3; FP32 MHD and FP64 Euler: 1 -> 2; FP64 MHD: none)
  static constexpr int kDef = (sizeof(T) == 4 && NV == 5) ? 2 : 1;
  static constexpr int kAlt = (sizeof(T) == 4 && NV == 5) ? 3 : 2;
  static constexpr bool kHasAlt = !(sizeof(T) == 8 && NV == 9);
  // 128-thread CTAs: 2 kDef per SM with the default registers; FP32 MHD also
  // has a 3-per-SM build (168 registers: 12 warps instead of 8)
  static constexpr int kAlt128 = (sizeof(T) == 4 && NV == 9) ? 3 : 0;
  int nt = kStageThreads;   // 256, or 128 (launched with twice the CTAs per SM, same register budget)

  explicit Ops(const PhysParams& p) {
    gamma = p.gamma;
    ph.gamma = (T)p.gamma;
    ph.gm1 = (T)(p.gamma - 1.0);
    ph.ggm1 = (T)(p.gamma * (p.gamma - 1.0));
    ph.theta = (T)p.theta;
    ph.llf = p.llf;
    ph.fluxrec = NV == 5 ? p.fluxrec : 0;
    weno = p.weno != 0;
    ph.weno = p.weno != 0 ? 1 : 0;
    ph.ch = ph.ch2 = ph.half_inv_ch = T(0);
    ph.efl = (T)(p.p_floor / (p.gamma - 1.0));
    ph.glm_alpha = (T)p.glm_alpha;
    set_smem<kDef, kStageThreads, false>();
    set_smem<2 * kDef, 128, false>();
    if constexpr (kAlt128 > 0) set_smem<kAlt128, 128, false>();
    set_smem<kDef, kStageThreads, true>();
    if constexpr (kHasAlt) set_smem<kAlt, kStageThreads, false>();
  }

  // dynamic shared memory limit of one build (both stages, blocks in one patch or spanning)
  template <int MINB, int NTT, bool WENO>
  static void set_smem() {
    const int sm = (int)stage_smem_bytes<T, NV, MINB, NTT>();
    constexpr auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaFuncSetAttribute(stage_kernel<T, NV, 1, MINB, NTT, WENO, false>, attr, sm);
    cudaFuncSetAttribute(stage_kernel<T, NV, 2, MINB, NTT, WENO, false>, attr, sm);
    cudaFuncSetAttribute(stage_kernel<T, NV, 1, MINB, NTT, WENO, true>, attr, sm);
    cudaFuncSetAttribute(stage_kernel<T, NV, 2, MINB, NTT, WENO, true>, attr, sm);
  }

  // launch of one build; span: the items include blocks that span patches
  template <int MINB, int NTT, bool WENO>
  static cudaError_t launch(int stage, bool span, int g, cudaStream_t s, const StageArgs<T>& a) {
    const size_t sm = stage_smem_bytes<T, NV, MINB, NTT>();
    if (span) {
      if (stage == 1) stage_kernel<T, NV, 1, MINB, NTT, WENO, true><<<g, NTT, sm, s>>>(a);
      else stage_kernel<T, NV, 2, MINB, NTT, WENO, true><<<g, NTT, sm, s>>>(a);
    } else {
      if (stage == 1) stage_kernel<T, NV, 1, MINB, NTT, WENO, false><<<g, NTT, sm, s>>>(a);
      else stage_kernel<T, NV, 2, MINB, NTT, WENO, false><<<g, NTT, sm, s>>>(a);
    }
    return cudaGetLastError();
  }

  void set_stage_threads(int n) override { nt = n == 128 ? 128 : kStageThreads; }
  int stage_occupancy() const override { return occ == kAlt ? kAlt : kDef; }
  int alt_occupancy() const override { return kHasAlt ? kAlt : 0; }
  void set_stage_occupancy(int c) override { occ = (kHasAlt && c == kAlt) ? kAlt : 0; }
  bool has_alt128() const override { return kAlt128 > 0; }
  int resident_ctas() const override {
    if (nt == 128) return (kAlt128 > 0 && occ == kAlt) ? kAlt128 : 2 * kDef;
    return occ == kAlt ? kAlt : kDef;
  }

  size_t elem_size() const override { return sizeof(T); }
  bool stage_stores_old() const override { return !(NV == 5 && ph.fluxrec); }

  cudaError_t stage(int stage, cudaStream_t s, const PatchDesc* desc, const StageItem* items, int nitems,
                    const ItemSpan* spans, const void* Uin, void* Uout, StepParams* prm, int level,
                    const double dx[3], const double dx0[3], int fuse_rate, int grid,
                    void* uold = nullptr) override {
    if (nitems <= 0) return cudaSuccess;
    StageArgs<T> a;
    a.desc = desc;
    a.items = items;
    a.nitems = nitems;
    a.spans = spans;
    a.Uin = static_cast<const T*>(Uin);
    a.Uout = static_cast<T*>(Uout);
    a.params = prm;
    a.dt_scale = 1.0 / (double)(1 << level);
    a.idx = (T)(1.0 / dx[0]);
    a.idy = (T)(1.0 / dx[1]);
    a.idz = (T)(1.0 / dx[2]);
    a.idx0 = 1.0 / dx0[0];
    a.idy0 = 1.0 / dx0[1];
    a.idz0 = 1.0 / dx0[2];
    a.fuse_rate = fuse_rate;
    a.Uold = stage == 1 ? static_cast<T*>(uold) : nullptr;
    a.ph = ph;
    // grid > 0: that many persistent CTAs, items handed out by a device counter
    a.dynamic = grid > 0 ? 1 : 0;
    const int g = grid > 0 ? (grid < nitems ? grid : nitems) : nitems;
    if constexpr (NV == 5) {
      if (ph.fluxrec) {
        if (stage == 1) fluxrec_stage_kernel<T, 1><<<g, kStageThreads, 0, s>>>(a);
        else fluxrec_stage_kernel<T, 2><<<g, kStageThreads, 0, s>>>(a);
        return cudaGetLastError();
      }
    }
    const bool span = spans != nullptr;
    if (weno) return launch<kDef, kStageThreads, true>(stage, span, g, s, a);   // any tiling's items fit 256 threads
    if constexpr (kAlt128 > 0) {
      if (nt == 128 && occ == kAlt) return launch<kAlt128, 128, false>(stage, span, g, s, a);
    }
    if (nt == 128) return launch<2 * kDef, 128, false>(stage, span, g, s, a);
    if constexpr (kHasAlt) {
      if (occ == kAlt) return launch<kAlt, kStageThreads, false>(stage, span, g, s, a);
    }
    return launch<kDef, kStageThreads, false>(stage, span, g, s, a);
  }

  static int grid_for(int n) { return n < 65535 ? n : 65535; }

  cudaError_t ghost_copy(cudaStream_t s, const CopySeg* segs, int nseg, const PatchDesc* desc, void* arena) override {
    if (nseg <= 0) return cudaSuccess;
    copy_kernel<T, NV, false><<<grid_for(nseg), 256, 0, s>>>(segs, nseg, desc, static_cast<T*>(arena),
                                                             static_cast<const T*>(arena), nullptr, T(0));
    return cudaGetLastError();
  }

  cudaError_t ghost_copy_flat(cudaStream_t s, const FlatCopy* boxes, const int* first, const int* chunk_box,
                              int nchunk, int total, void* arena) override {
    if (nchunk <= 0) return cudaSuccess;
    box_copy_kernel<T, NV, false><<<grid_for(nchunk), kBoxThreads, 0, s>>>(
        boxes, first, chunk_box, nchunk, total, static_cast<T*>(arena), static_cast<const T*>(arena), nullptr, T(0));
    return cudaGetLastError();
  }

  cudaError_t gather_flat(cudaStream_t s, const FlatCopy* boxes, const int* first, const int* chunk_box, int nchunk,
                          int total, void* tile, const void* U, const void* Uold, double alpha) override {
    if (nchunk <= 0) return cudaSuccess;
    box_copy_kernel<T, NV, true><<<grid_for(nchunk), kBoxThreads, 0, s>>>(
        boxes, first, chunk_box, nchunk, total, static_cast<T*>(tile), static_cast<const T*>(U),
        static_cast<const T*>(Uold), (T)alpha);
    return cudaGetLastError();
  }

  cudaError_t restrict_flat(cudaStream_t s, const FlatCopy* boxes, const int* first, const int* chunk_box, int nchunk,
                            int total, void* U) override {
    if (nchunk <= 0) return cudaSuccess;
    box_restrict_kernel<T, NV><<<grid_for(nchunk), kBoxThreads, 0, s>>>(boxes, first, chunk_box, nchunk, total,
                                                                         static_cast<T*>(U));
    return cudaGetLastError();
  }

  cudaError_t prolong_flat(cudaStream_t s, const FlatProlong* boxes, const int* first, const int* chunk_box,
                           int nchunk, int total, const void* tile, void* arena) override {
    if (nchunk <= 0) return cudaSuccess;
    box_prolong_kernel<T, NV><<<grid_for(nchunk), kBoxThreads, 0, s>>>(
        boxes, first, chunk_box, nchunk, total, static_cast<const T*>(tile), static_cast<T*>(arena));
    return cudaGetLastError();
  }

  cudaError_t gather(cudaStream_t s, const CopySeg* segs, int nseg, const PatchDesc* desc, void* tile,
                     const void* U, const void* Uold, double alpha) override {
    if (nseg <= 0) return cudaSuccess;
    copy_kernel<T, NV, true><<<grid_for(nseg), 128, 0, s>>>(segs, nseg, desc, static_cast<T*>(tile),
                                                            static_cast<const T*>(U), static_cast<const T*>(Uold),
                                                            (T)alpha);
    return cudaGetLastError();
  }

  cudaError_t prolong(cudaStream_t s, const ProlongBox* boxes, int nbox, const PatchDesc* desc, const void* tile,
                      void* arena) override {
    if (nbox <= 0) return cudaSuccess;
    prolong_kernel<T, NV><<<grid_for(nbox), 128, 0, s>>>(boxes, nbox, desc, static_cast<const T*>(tile),
                                                         static_cast<T*>(arena));
    return cudaGetLastError();
  }

  cudaError_t restrict_(cudaStream_t s, const RestrictSeg* segs, int nseg, const PatchDesc* desc, void* U) override {
    if (nseg <= 0) return cudaSuccess;
    restrict_kernel<T, NV><<<grid_for(nseg), 128, 0, s>>>(segs, nseg, desc, static_cast<T*>(U));
    return cudaGetLastError();
  }

  cudaError_t reg_coarse(cudaStream_t s, const RegRect* rects, const int* first, const int* chunk_box, int nrect,
                         int nreg,
                         const PatchDesc* desc, const void* Uin, double* R, StepParams* prm, int level,
                         int stage) override {
    if (nreg <= 0) return cudaSuccess;
    reg_coarse_kernel<T, NV><<<grid_for((nreg + kRegThreads - 1) / kRegThreads), kRegThreads, 0, s>>>(
        rects, first, chunk_box, nrect, nreg, desc, static_cast<const T*>(Uin), R, prm, 1.0 / (double)(1 << level), ph,
        stage);
    return cudaGetLastError();
  }

  cudaError_t reg_fine(cudaStream_t s, const RegRect* rects, const int* first, const int* chunk_box, int nrect,
                       int nreg,
                       const PatchDesc* desc, const void* Uin, double* R, StepParams* prm, int level) override {
    if (nreg <= 0) return cudaSuccess;
    // four lanes per register (one per fine sub-face)
    reg_fine_kernel<T, NV><<<grid_for((4 * nreg + kRegThreads - 1) / kRegThreads), kRegThreads, 0, s>>>(
        rects, first, chunk_box, nrect, nreg, desc, static_cast<const T*>(Uin), R, prm, 1.0 / (double)(1 << level),
        ph);
    return cudaGetLastError();
  }

  cudaError_t reflux(cudaStream_t s, const RegRect* rects, const int* first, const int* chunk_box, int nrect, int e0,
                     int e1,
                     int nreg, const PatchDesc* desc, const double* R, void* U, const double dxc[3],
                     int ordered) override {
    if (e1 <= e0) return cudaSuccess;
    reflux_kernel<T, NV><<<grid_for((e1 - e0 + kRegThreads - 1) / kRegThreads), kRegThreads, 0, s>>>(
        rects, first, chunk_box, nrect, e0, e1, nreg, desc, R, static_cast<T*>(U), dxc[0], dxc[1], dxc[2], ordered);
    return cudaGetLastError();
  }

  cudaError_t speed(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const void* U,
                    StepParams* prm, const double dx0[3]) override {
    speed_kernel<T, NV><<<grid_for(nchunk), 256, 0, s>>>(chunks, nchunk, desc, static_cast<const T*>(U), prm,
                                                         1.0 / dx0[0], 1.0 / dx0[1], 1.0 / dx0[2], ph);
    return cudaGetLastError();
  }

  cudaError_t totals(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const void* U,
                     const CoverBox* cover, const int* cover_first, const double* level_vol, double* partial,
                     double* out) override {
    totals_kernel<T, NV><<<grid_for(nchunk), 256, 0, s>>>(chunks, nchunk, desc, static_cast<const T*>(U), cover,
                                                          cover_first, level_vol, partial);
    totals_final_kernel<NV><<<1, 32, 0, s>>>(partial, nchunk, out);
    return cudaGetLastError();
  }

  cudaError_t divb(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const void* U,
                   const CoverBox* cover, const int* cover_first, const double dx0[3], double* partial,
                   double* out) override {
    if constexpr (NV == 9) {
      divb_kernel<T, NV><<<grid_for(nchunk), 256, 0, s>>>(chunks, nchunk, desc, static_cast<const T*>(U), cover,
                                                          cover_first, dx0[0], dx0[1], dx0[2], partial);
      divb_final_kernel<4><<<1, 32, 0, s>>>(partial, nchunk, out);
      return cudaGetLastError();
    } else {
      return cudaErrorInvalidValue;
    }
  }

  cudaError_t pack_in(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                      const int64_t* packed_off, const double* src, void* U, int prim, StepParams* prm) override {
    pack_in_kernel<T, NV><<<grid_for(nchunk), 256, 0, s>>>(chunks, nchunk, desc, packed_off, src,
                                                           static_cast<T*>(U), prim, gamma, prm);
    return cudaGetLastError();
  }

  cudaError_t flag(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                   const int64_t* packed_off, const void* U, double threshold, unsigned char* flags) override {
    flag_kernel<T, NV><<<grid_for(nchunk), 256, 0, s>>>(chunks, nchunk, desc, packed_off, static_cast<const T*>(U),
                                                        (T)threshold, flags);
    return cudaGetLastError();
  }

  cudaError_t tag(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const void* U,
                  double threshold, const TagArgs& a, unsigned int* words) override {
    tag_kernel<T, NV><<<grid_for(nchunk), 256, 0, s>>>(chunks, nchunk, desc, static_cast<const T*>(U), (T)threshold,
                                                       a, words);
    return cudaGetLastError();
  }

  cudaError_t xcopy(cudaStream_t s, const CopySeg* segs, int nseg, const PatchDesc* dst_desc,
                    const PatchDesc* src_desc, void* dst, const void* src) override {
    if (nseg <= 0) return cudaSuccess;
    xcopy_kernel<T, NV><<<grid_for(nseg), 256, 0, s>>>(segs, nseg, dst_desc, src_desc, static_cast<T*>(dst),
                                                       static_cast<const T*>(src));
    return cudaGetLastError();
  }

  cudaError_t pack_out(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                       const int64_t* packed_off, const void* U, double* dst) override {
    pack_out_kernel<T, NV><<<grid_for(nchunk), 256, 0, s>>>(chunks, nchunk, desc, packed_off,
                                                            static_cast<const T*>(U), dst);
    return cudaGetLastError();
  }
};

}  // namespace amr
