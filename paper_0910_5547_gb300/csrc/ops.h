// ops.h -- type-erased launchers of the kernels of one (precision, physics)
// instantiation.  The host orchestration (amr_api.cu) talks to the kernels only
// through this interface; each ops_*.cu translation unit instantiates one.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "amr_types.h"

namespace amr {

struct ChunkDesc;

struct PhysParams {  // host copy of the physics constants
  double gamma, theta, ch_fixed;
  int llf;
  double p_floor, glm_alpha;
  int fluxrec;
  int weno;   // third-order WENO face states (the default build only)
};

struct OpsBase {
  virtual ~OpsBase() {}
  virtual size_t elem_size() const = 0;
  // fused RK2 stage over items [0, nitems) of `items` (device pointer)
  virtual cudaError_t stage(int stage, cudaStream_t s, const PatchDesc* desc, const StageItem* items, int nitems,
                            const ItemSpan* spans, const void* Uin, void* Uout, StepParams* prm, int level,
                            const double dx[3], const double dx0[3], int fuse_rate, int grid,
                            void* uold = nullptr) = 0;
  // whether stage 1 stores its input into uold (every build but the flux-reconstruction kernel)
  virtual bool stage_stores_old() const = 0;
  // resident CTAs per SM the stage kernel is compiled for (register budget);
  // each variant except FP64 MHD has a second build, selected here
  virtual int stage_occupancy() const = 0;
  virtual int alt_occupancy() const = 0;   // the other compiled budget (0: none)
  virtual void set_stage_occupancy(int ctas_per_sm) = 0;
  // threads per stage CTA: 256 (default) or 128 (same registers per thread, twice the CTAs)
  virtual void set_stage_threads(int nt) = 0;
  // whether the 128-thread build also has an alternate (smaller) register budget
  virtual bool has_alt128() const = 0;
  // resident CTAs per SM of the build the next stage launch uses
  virtual int resident_ctas() const = 0;
  virtual cudaError_t ghost_copy(cudaStream_t s, const CopySeg* segs, int nseg, const PatchDesc* desc, void* arena) = 0;
  // batched forms over flattened boxes (same values as ghost_copy / gather / prolong)
  virtual cudaError_t ghost_copy_flat(cudaStream_t s, const FlatCopy* boxes, const int* first, const int* chunk_box,
                                      int nchunk, int total, void* arena) = 0;
  virtual cudaError_t gather_flat(cudaStream_t s, const FlatCopy* boxes, const int* first, const int* chunk_box,
                                  int nchunk, int total, void* tile, const void* U, const void* Uold,
                                  double alpha) = 0;
  virtual cudaError_t restrict_flat(cudaStream_t s, const FlatCopy* boxes, const int* first, const int* chunk_box,
                                    int nchunk, int total, void* U) = 0;
  virtual cudaError_t prolong_flat(cudaStream_t s, const FlatProlong* boxes, const int* first, const int* chunk_box,
                                   int nchunk, int total, const void* tile, void* arena) = 0;
  virtual cudaError_t gather(cudaStream_t s, const CopySeg* segs, int nseg, const PatchDesc* desc, void* tile,
                             const void* U, const void* Uold, double alpha) = 0;
  virtual cudaError_t prolong(cudaStream_t s, const ProlongBox* boxes, int nbox, const PatchDesc* desc,
                              const void* tile, void* arena) = 0;
  virtual cudaError_t restrict_(cudaStream_t s, const RestrictSeg* segs, int nseg, const PatchDesc* desc, void* U) = 0;
  // flux registers over register rectangles (first / chunk_box: flattened, chunks of kBoxThreads)
  virtual cudaError_t reg_coarse(cudaStream_t s, const RegRect* rects, const int* first, const int* chunk_box,
                                 int nrect, int nreg, const PatchDesc* desc, const void* Uin, double* R, StepParams* prm,
                                 int level, int stage) = 0;
  virtual cudaError_t reg_fine(cudaStream_t s, const RegRect* rects, const int* first, const int* chunk_box,
                               int nrect, int nreg, const PatchDesc* desc, const void* Uin, double* R, StepParams* prm,
                               int level) = 0;
  // reflux of the registers [e0, e1) of the rectangles whose `ordered` flag equals `ordered`
  virtual cudaError_t reflux(cudaStream_t s, const RegRect* rects, const int* first, const int* chunk_box, int nrect,
                             int e0,
                             int e1, int nreg, const PatchDesc* desc, const double* R, void* U, const double dxc[3],
                             int ordered) = 0;
  virtual cudaError_t speed(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                            const void* U, StepParams* prm, const double dx0[3]) = 0;
  virtual cudaError_t totals(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                             const void* U, const CoverBox* cover, const int* cover_first, const double* level_vol,
                             double* partial, double* out) = 0;
  // GLM-MHD only (cudaErrorInvalidValue otherwise): out[4] = div B norms over leaf cells
  virtual cudaError_t divb(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                           const void* U, const CoverBox* cover, const int* cover_first, const double dx0[3],
                           double* partial, double* out) = 0;
  virtual cudaError_t pack_in(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                              const int64_t* packed_off, const double* src, void* U, int prim, StepParams* prm) = 0;
  virtual cudaError_t flag(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                           const int64_t* packed_off, const void* U, double threshold, unsigned char* flags) = 0;
  virtual cudaError_t tag(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const void* U,
                          double threshold, const TagArgs& a, unsigned int* words) = 0;
  virtual cudaError_t xcopy(cudaStream_t s, const CopySeg* segs, int nseg, const PatchDesc* dst_desc,
                            const PatchDesc* src_desc, void* dst, const void* src) = 0;
  virtual cudaError_t pack_out(cudaStream_t s, const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                               const int64_t* packed_off, const void* U, double* dst) = 0;
};

// factories, one per translation unit
OpsBase* make_ops_f64_euler(const PhysParams&);
OpsBase* make_ops_f32_euler(const PhysParams&);
OpsBase* make_ops_f64_mhd(const PhysParams&);
OpsBase* make_ops_f32_mhd(const PhysParams&);

}  // namespace amr
