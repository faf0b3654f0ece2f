// amr_api.cu -- the C ABI of include/amr.h: handle lifecycle, device memory,
// table upload, and the host recursion of one coarse step (Sec. 3,
// Berger-Colella subcycling; Sec. 5.1 two Euler stages plus the average,
// fused on the GPU).  A coarse step is enqueued as a fixed launch sequence
// whose dt is read from device memory, so it can be captured once as a CUDA
// graph and replayed.
#include <cuda_runtime.h>

#include <chrono>

#include <nvtx3/nvToolsExt.h>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/amr.h"
#include "hierarchy.h"
#include "kernels.cuh"
#include "ops.h"

using namespace amr;

namespace {

// NVTX range for profilers (a no-op unless a tool is attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

}  // namespace

namespace {

thread_local std::string g_global_err;

__global__ void begin_speed_kernel(StepParams* params) {
  params->rate_bits = 0ull;
  params->speed_bits = 0ull;
}

// dt0 = cfl / max rate (CFL mode); GLM cleaning speed = fixed value or max signal speed.
// The maxima come from the standalone reduction (from_next = 0) or from the
// previous stage 2 of a single-level grid (from_next = 1); the stage-2
// accumulators are cleared for the step about to run.
__global__ void finalize_speed_kernel(StepParams* params, double cfl, double ch_fixed, int set_dt, int from_next,
                                      int use_rates, int clear_next) {
  if (use_rates) {
    const unsigned long long rb = from_next ? params->next_rate_bits : params->rate_bits;
    const unsigned long long sb = from_next ? params->next_speed_bits : params->speed_bits;
    const double rate = __longlong_as_double((long long)rb);
    const double speed = __longlong_as_double((long long)sb);
    if (set_dt) params->dt0 = cfl / rate;
    params->ch = ch_fixed > 0.0 ? ch_fixed : speed;
  }
  if (clear_next) {
    params->next_rate_bits = 0ull;
    params->next_speed_bits = 0ull;
  }
}

__global__ void set_dt_kernel(StepParams* params, double dt) { params->dt0 = dt; }

struct DevLevel {
  int nitems = 0, nghost = 0, nghost_stage = 0, nprolong = 0, ngather_ghost = 0, nrestrict = 0, nreg = 0, nrect = 0;
  const StageItem* items = nullptr;        // per-patch stage items (plain launches)
  const StageItem* bitems = nullptr;       // stage items of the batched launch
  int nbitems = 0;
  bool has_span = false;                   // some batched items span patches
  const CopySeg* ghost = nullptr;          // every face ghost segment (diagnostics, regrid flags)
  const CopySeg* ghost_stage = nullptr;    // the faces a stage does not read directly
  const ProlongBox* prolong = nullptr;
  const CopySeg* gather_ghost = nullptr;   // the tile cells the per-stage prolongation reads
  const RestrictSeg* restrict_segs = nullptr;
  const RegRect* regs = nullptr;           // register rectangles (flattened: reg_first, reg_chunk)
  const int* reg_first = nullptr;
  const int* reg_chunk = nullptr;
  int reg_pass[7] = {0, 0, 0, 0, 0, 0, 0};  // reflux passes: registers of fine faces (d, side) = p / 2, p % 2
  int reg_ordered[6] = {0, 0, 0, 0, 0, 0};  // pass p has rectangles sharing cells with others
  double* R = nullptr;  // registers: [2][nvar][nreg]
  // flattened boxes of the batched ghost copy, gather and prolongation launches
  struct Flat {
    const void* boxes = nullptr;
    const int* first = nullptr;
    const int* chunk_box = nullptr;
    int nchunk = 0, total = 0;
  } fghost, fghost_all, fgather, fprolong, frestrict;
  int64_t arena_begin = 0, arena_end = 0;  // element range of the level's patches
};

}  // namespace

struct amr_handle {
  amr_config cfg{};
  double regrid_sec[AMR_RG_NPHASE] = {};   // host phases of the regrids since the last query
  long long regrid_counts[2] = {0, 0};     // regrids that rebuilt the hierarchy / found it unchanged
  // last clustering per min_level: its inputs (kept levels, parameters, refinable
  // block bitmaps)
  // and its result; the clustering is a function of these alone
  struct ClusterMemo {
    bool valid = false;
    RegridParams rp;
    std::vector<HPatch> kept, result;
    std::vector<std::vector<uint64_t>> words;
  };
  ClusterMemo memo[kTagLevels];
  long long memo_hits = 0;
  // regrid schedule: after each step of a level l <= sched_level, rebuild the finer levels
  long long cell_updates = 0;   // interior cells advanced by amr_step, summed over level steps
  bool capturing = false;       // advance() is being captured into a graph (not executed)
  bool sched_on = false;
  int sched_level = -1;
  RegridParams sched_rp;
  amr_status sched_status = AMR_OK;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaMemPool_t pool = nullptr;   // stream-ordered device memory (no caller allocator)
  unsigned char* stage = nullptr; // pinned host staging of the table uploads
  size_t stage_cap = 0, stage_cap_seen = 0;
  // asynchronous state copies: one copy stream per direction, kSlots device
  // slots per direction (packed FP64), events that order slot reuse across streams
  static constexpr int kSlots = 3;
  cudaStream_t cs_in = nullptr, cs_out = nullptr;
  double* in_slot[kSlots] = {};
  double* out_slot[kSlots] = {};
  int64_t slot_elems = -1;
  cudaEvent_t ev_h2d[kSlots] = {}, ev_in_used[kSlots] = {}, ev_packout[kSlots] = {}, ev_d2h[kSlots] = {};
  long long n_in = 0, n_out = 0;
  OpsBase* ops = nullptr;
  std::string err;
  Plan plan;
  bool ready = false;
  // device memory
  void* U = nullptr;
  void* U1 = nullptr;
  void* Uold = nullptr;
  void* tile = nullptr;
  double* packed = nullptr;
  double* partial = nullptr;
  double* totals = nullptr;
  double* regs = nullptr;
  unsigned char* tables = nullptr;
  StepParams* params = nullptr;
  const PatchDesc* d_desc = nullptr;
  const ChunkDesc* d_chunks = nullptr;
  const CoverBox* d_cover = nullptr;
  const int* d_cover_first = nullptr;
  const int64_t* d_packed_off = nullptr;
  const double* d_level_vol = nullptr;
  int nchunk = 0;
  std::vector<ChunkDesc> chunks;
  std::vector<DevLevel> dl;
  double dx0[3] = {1, 1, 1};
  // graphs: index = cfl + 2 * standalone-reduction
  cudaGraphExec_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
  long long graph_launches[4] = {0, 0, 0, 0};
  bool rates_valid = false;   // stage 2 of the last step left next-step maxima (single level)
  long long launches = 0;
  long long counting = 0;   // launches counted while enqueueing
  // stage-kernel work items (own buffer: the autotuner swaps the tiling)
  StageItem* items_dev = nullptr;
  const ItemSpan* d_spans = nullptr;   // inside items_dev: the spanning batched items' patch lists
  TileParams tp;            // tile shape in use (autotuned or default)
  int sms = 0;              // SMs of the device (persistent stage grids)
  int persist_mode = -1;    // -1: the autotuner decides; 0 / 1: one CTA per item / persistent CTAs
  // second stream of a batched multi-level step: the parent-cell gather and
  // prolongation of a level's stage-2 ghost cells and the flux-register kernels
  // run on it beside the stage kernels (fork / join through events, captured
  // into the step graph as parallel branches)
  bool overlap = true;               // amr_set_overlap
  cudaStream_t side = nullptr;
  std::vector<cudaEvent_t> side_ev;  // ring of fork / join events
  size_t side_next = 0;
  bool side_dirty = false;           // the side stream holds work the main stream has not joined
  std::vector<cudaEvent_t> u1_ev;    // per level: recorded on the side stream after its last read of U1
  std::vector<char> u1_pend;         // per level: u1_ev recorded in this step and not yet waited for
  // optional per-class event timing (eager steps only)
  bool timing = false;
  int cur_class = 0;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_pairs[AMR_T_NCLASS];  // (start, stop) indices into ev_pool
  size_t ev_used = 0;
  double t_ms[AMR_T_NCLASS] = {0};
  long long t_cnt[AMR_T_NCLASS] = {0};
};

namespace {

amr_status fail(amr_handle* h, amr_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

#define CK(call)                                                                                  \
  do {                                                                                            \
    cudaError_t e_ = (call);                                                                      \
    if (e_ != cudaSuccess)                                                                        \
      return fail(h, AMR_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));           \
  } while (0)

cudaEvent_t next_event(amr_handle* h, int* idx) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  *idx = (int)h->ev_used;
  return h->ev_pool[h->ev_used++];
}

// Launch wrapper: counts the launch and, when timing is on, brackets it with
// an event pair on the handle's stream.
#define LK(call)                                                   \
  do {                                                             \
    int i0_ = -1, i1_ = -1;                                        \
    if (h->timing) cudaEventRecord(next_event(h, &i0_), h->stream); \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return e_;                              \
    if (h->timing) {                                               \
      cudaEventRecord(next_event(h, &i1_), h->stream);             \
      h->ev_pairs[h->cur_class].push_back({i0_, i1_});             \
    }                                                              \
    h->counting += 1;                                              \
  } while (0)

// Device memory of a handle: the caller's allocator (dev_alloc / dev_free) or
// stream-ordered allocations on the handle's stream from the handle's own memory
// pool.  The pool keeps freed memory mapped (release threshold: unlimited), so a
// regrid that swaps a multi-GB arena for a new one reuses the pages instead of
// mapping fresh ones; amr_destroy returns it all.
cudaError_t dmalloc(amr_handle* h, void** p, size_t bytes) {
  bytes = std::max<size_t>(bytes, 256);
  if (h->cfg.dev_alloc && h->cfg.dev_free) {
    *p = h->cfg.dev_alloc(bytes, h->stream, h->cfg.alloc_ctx);
    if (!*p) return cudaErrorMemoryAllocation;
    // the kernels' vector loads and asynchronous copies assume the alignment cudaMalloc gives
    if (reinterpret_cast<uintptr_t>(*p) % 256 != 0) {
      h->cfg.dev_free(*p, h->stream, h->cfg.alloc_ctx);
      *p = nullptr;
      return cudaErrorMisalignedAddress;
    }
    return cudaSuccess;
  }
  if (h->pool) return cudaMallocFromPoolAsync(p, bytes, h->pool, h->stream);
  return cudaMallocAsync(p, bytes, h->stream);
}

// ---- block bitmaps of the regrid on the GPU: bit i = block (x, y, z) with
// i = (z n1 + y) n0 + x, 32 bits per word from word `off` of a buffer; every
// kernel writes whole words (one thread per word), so no stale bit survives ----
struct BGrid {
  int n0, n1, n2;
  long long off;     // first word
  long long nw;      // words (two per 64 bits of the grid, the host's layout)
};

__device__ __forceinline__ bool bit_at(const unsigned* w, const BGrid& g, int x, int y, int z) {
  const long long i = ((long long)z * g.n1 + y) * g.n0 + x;
  return (w[g.off + (i >> 5)] >> (i & 31)) & 1u;
}

// parent block q of level l-1 is set when one of its 8 children is tagged on level l
__global__ void bm_downsample(const unsigned* fine, BGrid F, unsigned* out, BGrid G) {
  const long long total = (long long)G.n0 * G.n1 * G.n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < G.nw; t += (long long)gridDim.x * blockDim.x) {
    unsigned word = 0;
    for (int b = 0; b < 32; ++b) {
      const long long i = t * 32 + b;
      if (i >= total) break;
      const int x = (int)(i % G.n0), y = (int)((i / G.n0) % G.n1), z = (int)(i / ((long long)G.n0 * G.n1));
      bool v = false;
      for (int dz = 0; dz < 2 && !v; ++dz)
        for (int dy = 0; dy < 2 && !v; ++dy)
          for (int dx = 0; dx < 2 && !v; ++dx) {
            const int cx = 2 * x + dx, cy = 2 * y + dy, cz = 2 * z + dz;
            if (cx < F.n0 && cy < F.n1 && cz < F.n2) v = bit_at(fine, F, cx, cy, cz);
          }
      word |= (unsigned)v << b;
    }
    out[G.off + t] = word;
  }
}

// one axis of a 3-cell box filter: OR (dilate) or AND (erode) of the cell and its
// two neighbours along `axis`; a periodic axis wraps, otherwise a neighbour
// outside the grid is 0 for OR and 1 for AND (outside an outflow face counts as
// covered)
__global__ void bm_box_axis(const unsigned* src, BGrid S, unsigned* dst, BGrid D, int axis, int periodic,
                            int erode) {
  const long long total = (long long)S.n0 * S.n1 * S.n2;
  const int n[3] = {S.n0, S.n1, S.n2};
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < D.nw; t += (long long)gridDim.x * blockDim.x) {
    unsigned word = 0;
    for (int b = 0; b < 32; ++b) {
      const long long i = t * 32 + b;
      if (i >= total) break;
      const int c[3] = {(int)(i % S.n0), (int)((i / S.n0) % S.n1), (int)(i / ((long long)S.n0 * S.n1))};
      bool v = erode != 0;
      for (int s = -1; s <= 1; ++s) {
        int r[3] = {c[0], c[1], c[2]};
        r[axis] += s;
        if (r[axis] < 0 || r[axis] >= n[axis]) {
          if (!periodic) continue;
          r[axis] = ((r[axis] % n[axis]) + n[axis]) % n[axis];
        }
        const bool q = bit_at(src, S, r[0], r[1], r[2]);
        v = erode ? (v && q) : (v || q);
      }
      word |= (unsigned)v << b;
    }
    dst[D.off + t] = word;
  }
}

// cover of level l: block q is covered when its parent block (q / 2) is refinable
__global__ void bm_from_parent(const unsigned* parent, BGrid P, unsigned* out, BGrid G) {
  const long long total = (long long)G.n0 * G.n1 * G.n2;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < G.nw; t += (long long)gridDim.x * blockDim.x) {
    unsigned word = 0;
    for (int b = 0; b < 32; ++b) {
      const long long i = t * 32 + b;
      if (i >= total) break;
      const int x = (int)(i % G.n0), y = (int)((i / G.n0) % G.n1), z = (int)(i / ((long long)G.n0 * G.n1));
      word |= (unsigned)bit_at(parent, P, x >> 1, y >> 1, z >> 1) << b;
    }
    out[G.off + t] = word;
  }
}

// dst = a | b (op 0) or a & b (op 1), word by word
__global__ void bm_combine(unsigned* dst, long long dst_off, const unsigned* a, long long a_off, const unsigned* b,
                           long long b_off, long long nw, int op) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < nw; t += (long long)gridDim.x * blockDim.x)
    dst[dst_off + t] = op ? (a[a_off + t] & b[b_off + t]) : (a[a_off + t] | b[b_off + t]);
}

int bm_grid(long long nw) { return (int)std::min<long long>(std::max<long long>((nw + 255) / 256, 1), 65535); }

void dfree(amr_handle* h, void* p);

// Copy streams, events and device slots of the asynchronous state copies, sized
// for the installed hierarchy (remade after a regrid or a new patch set, once
// the copies in flight are done).
cudaError_t ensure_async(amr_handle* h) {
  cudaError_t e = cudaSuccess;
  if (!h->cs_in) {
    e = cudaStreamCreateWithFlags(&h->cs_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cs_out, cudaStreamNonBlocking);
    for (int k = 0; k < amr_handle::kSlots && e == cudaSuccess; ++k) {
      cudaEvent_t* evs[4] = {&h->ev_h2d[k], &h->ev_in_used[k], &h->ev_packout[k], &h->ev_d2h[k]};
      for (cudaEvent_t* ev : evs)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return e;
  }
  if (h->slot_elems == h->plan.packed_elems) return cudaSuccess;
  e = cudaStreamSynchronize(h->cs_in);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->cs_out);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < amr_handle::kSlots; ++k) {
    dfree(h, h->in_slot[k]);
    dfree(h, h->out_slot[k]);
    h->in_slot[k] = h->out_slot[k] = nullptr;
  }
  h->slot_elems = -1;
  const size_t bytes = std::max<int64_t>(h->plan.packed_elems, 1) * sizeof(double);
  for (int k = 0; k < amr_handle::kSlots && e == cudaSuccess; ++k) {
    void* p = nullptr;
    e = dmalloc(h, &p, bytes);
    h->in_slot[k] = static_cast<double*>(p);
    if (e == cudaSuccess) e = dmalloc(h, &p, bytes);
    h->out_slot[k] = static_cast<double*>(p);
  }
  // the slots are allocated in the order of the handle's stream; the copy streams
  // use them next
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e == cudaSuccess) h->slot_elems = h->plan.packed_elems;
  return e;
}

void release_async(amr_handle* h) {
  if (h->cs_in) cudaStreamSynchronize(h->cs_in);
  if (h->cs_out) cudaStreamSynchronize(h->cs_out);
  for (int k = 0; k < amr_handle::kSlots; ++k) {
    dfree(h, h->in_slot[k]);
    dfree(h, h->out_slot[k]);
    h->in_slot[k] = h->out_slot[k] = nullptr;
    cudaEvent_t evs[4] = {h->ev_h2d[k], h->ev_in_used[k], h->ev_packout[k], h->ev_d2h[k]};
    for (cudaEvent_t ev : evs)
      if (ev) cudaEventDestroy(ev);
  }
  if (h->cs_in) cudaStreamDestroy(h->cs_in);
  if (h->cs_out) cudaStreamDestroy(h->cs_out);
  h->cs_in = h->cs_out = nullptr;
}

// The packed FP64 staging buffer of the host copies (set/get state) is made on
// first use after each install: regrids never need it.
cudaError_t ensure_packed(amr_handle* h) {
  if (h->packed) return cudaSuccess;
  void* p = nullptr;
  cudaError_t e = dmalloc(h, &p, std::max<int64_t>(h->plan.packed_elems, 1) * sizeof(double));
  if (e == cudaSuccess) h->packed = static_cast<double*>(p);
  return e;
}

void dfree(amr_handle* h, void* p) {
  if (!p) return;
  if (h->cfg.dev_alloc && h->cfg.dev_free) h->cfg.dev_free(p, h->stream, h->cfg.alloc_ctx);
  else cudaFreeAsync(p, h->stream);
}

void free_device(amr_handle* h) {
  for (int g = 0; g < 4; ++g) {
    if (h->graph[g]) cudaGraphExecDestroy(h->graph[g]);
    h->graph[g] = nullptr;
  }
  h->rates_valid = false;
  void* ptrs[] = {h->U, h->U1, h->Uold, h->tile, h->packed, h->partial, h->totals, h->regs, h->tables,
                  h->items_dev};
  for (void* p : ptrs) dfree(h, p);
  h->items_dev = nullptr;
  h->U = h->U1 = h->Uold = h->tile = nullptr;
  h->packed = h->partial = h->totals = h->regs = nullptr;
  h->tables = nullptr;
  h->dl.clear();
  h->ready = false;
}

OpsBase* make_ops(const amr_config& c) {
  PhysParams p{c.gamma, c.theta, c.ch, c.riemann == AMR_LLF ? 1 : 0, c.p_floor, c.glm_alpha,
               c.riemann == AMR_FLUXREC ? 1 : 0, c.recon == AMR_WENO3 ? 1 : 0};
  if (c.nvar == 5) return c.precision == AMR_FP32 ? make_ops_f32_euler(p) : make_ops_f64_euler(p);
  return c.precision == AMR_FP32 ? make_ops_f32_mhd(p) : make_ops_f64_mhd(p);
}

double level_dx(const amr_handle* h, int l, int d) { return h->dx0[d] / (double)(1 << l); }

// ---- one coarse step -------------------------------------------------------

// Face ghosts of level l in arr: parent data at fraction alpha of the parent step
// prolonged into coarse-fine faces, then same-level copies.  all = false: only
// the faces the stage kernel does not read straight from their source
// (PatchDesc::face); all = true: every face (for kernels that read ghost cells
// themselves: regrid flags, div B).
cudaError_t fill_parent(amr_handle* h, int l, void* arr, double alpha, cudaStream_t st, void* tile) {
  const DevLevel& L = h->dl[l];
  if (l == 0) return cudaSuccess;
  h->cur_class = AMR_T_PARENT;
  if (h->cfg.batched) {
    const DevLevel::Flat& G = L.fgather;
    const DevLevel::Flat& P = L.fprolong;
    LK(h->ops->gather_flat(st, static_cast<const FlatCopy*>(G.boxes), G.first, G.chunk_box, G.nchunk, G.total, tile,
                           h->U, h->Uold, alpha));
    LK(h->ops->prolong_flat(st, static_cast<const FlatProlong*>(P.boxes), P.first, P.chunk_box, P.nchunk, P.total,
                            tile, arr));
  } else {
    LK(h->ops->gather(st, L.gather_ghost, L.ngather_ghost, h->d_desc, tile, h->U, h->Uold, alpha));
    LK(h->ops->prolong(st, L.prolong, L.nprolong, h->d_desc, tile, arr));
  }
  return cudaSuccess;
}

cudaError_t fill_same(amr_handle* h, int l, void* arr, bool all) {
  const DevLevel& L = h->dl[l];
  const LevelPlan& LP = h->plan.levels[l];
  h->cur_class = AMR_T_GHOST;
  if (all && h->cfg.batched) {   // every face, over flattened boxes
    const DevLevel::Flat& G = L.fghost_all;
    LK(h->ops->ghost_copy_flat(h->stream, static_cast<const FlatCopy*>(G.boxes), G.first, G.chunk_box, G.nchunk,
                               G.total, arr));
  } else if (all) {
    LK(h->ops->ghost_copy(h->stream, L.ghost, L.nghost, h->d_desc, arr));
  } else if (h->cfg.batched) {
    const DevLevel::Flat& G = L.fghost;
    LK(h->ops->ghost_copy_flat(h->stream, static_cast<const FlatCopy*>(G.boxes), G.first, G.chunk_box, G.nchunk,
                               G.total, arr));
  } else if (L.nghost_stage == 0) {
    LK(h->ops->ghost_copy(h->stream, L.ghost_stage, L.nghost_stage, h->d_desc, arr));
  } else {
    for (int p = 0; p < LP.count; ++p) {
      int a = LP.ghost_stage_first[p], b = LP.ghost_stage_first[p + 1];
      if (b > a) LK(h->ops->ghost_copy(h->stream, L.ghost_stage + a, b - a, h->d_desc, arr));
    }
  }
  return cudaSuccess;
}

cudaError_t fill_ghosts(amr_handle* h, int l, void* arr, double alpha, bool all = false) {
  cudaError_t e = fill_parent(h, l, arr, alpha, h->stream, h->tile);
  return e == cudaSuccess ? fill_same(h, l, arr, all) : e;
}

// ---- the side stream of a step ----
// Order (main | side), level l, one step:
//   main: stage-1 ghosts of U | fork | stage 1 (U -> U1, and U^n -> Uold for a level with
//         children) | join | same-level ghosts of U1 | stage 2 (U1 -> U) | fork | children | join |
//         restriction, reflux
//   side: after the first fork: stage-2 parent gather (second tile) and prolongation into U1,
//         stage-1 registers (read U); after the second fork: stage-2 registers (read U1)
// Stage 1 of a level waits for the side stream's last read of that level's U1
// (u1_ev); the joins cover every other hazard (ghost cells of U1 before stage 2;
// U of the level, which the registers and the children's gathers read, before
// stage 2 and the restriction write it; its Uold, which the children's gathers
// read, before the next stage 1 writes it; the registers before the reflux).
bool overlap_on(const amr_handle* h) {
  return h->overlap && h->side && h->cfg.batched && !h->timing && h->dl.size() > 1;
}

int side_event(amr_handle* h) {
  if (h->side_ev.empty()) {
    h->side_ev.resize(64);
    for (cudaEvent_t& e : h->side_ev) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
  }
  const int k = (int)(h->side_next++ % h->side_ev.size());
  return k;
}

// The side stream waits for everything enqueued on the main stream so far.
cudaError_t fork_side(amr_handle* h) {
  const int k = side_event(h);
  cudaError_t e = cudaEventRecord(h->side_ev[k], h->stream);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->side, h->side_ev[k], 0);
  return e;
}

// The main stream waits for everything enqueued on the side stream so far.
cudaError_t join_side(amr_handle* h) {
  if (!h->side_dirty) return cudaSuccess;
  const int k = side_event(h);
  cudaError_t e = cudaEventRecord(h->side_ev[k], h->side);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(h->stream, h->side_ev[k], 0);
  if (e == cudaSuccess) h->side_dirty = false;
  return e;
}

cudaError_t stage(amr_handle* h, int l, int s, const void* in, void* out, void* uold = nullptr) {
  const DevLevel& L = h->dl[l];
  const LevelPlan& LP = h->plan.levels[l];
  double dx[3] = {level_dx(h, l, 0), level_dx(h, l, 1), level_dx(h, l, 2)};
  h->cur_class = s == 1 ? AMR_T_STAGE1 : AMR_T_STAGE2;
  const int fuse = (s == 2 && h->dl.size() == 1) ? 1 : 0;
  if (h->cfg.batched) {
    // persistent: one wave of resident CTAs takes the level's items from a device counter
    const int grid = h->tp.persistent ? h->sms * h->ops->resident_ctas() : 0;
    LK(h->ops->stage(s, h->stream, h->d_desc, L.bitems, L.nbitems, L.has_span ? h->d_spans : nullptr, in, out,
                     h->params, l, dx, h->dx0, fuse, grid, uold));
  } else {
    for (int p = 0; p < LP.count; ++p) {
      int a = LP.item_first[p], b = LP.item_first[p + 1];
      if (b > a)
        LK(h->ops->stage(s, h->stream, h->d_desc, L.items + a, b - a, nullptr, in, out, h->params, l, dx, h->dx0,
                         fuse, 0, uold));
    }
  }
  return cudaSuccess;
}

amr_status regrid_impl(amr_handle* h, const RegridParams& rp, int mid_level, double alpha);

cudaError_t u1_wait(amr_handle* h, int l) {
  if (l >= (int)h->u1_pend.size() || !h->u1_pend[l]) return cudaSuccess;
  h->u1_pend[l] = 0;
  return cudaStreamWaitEvent(h->stream, h->u1_ev[l], 0);
}

cudaError_t u1_mark(amr_handle* h, int l) {
  if ((int)h->u1_ev.size() <= l) {
    const size_t n0 = h->u1_ev.size();
    h->u1_ev.resize(l + 1, nullptr);
    h->u1_pend.resize(l + 1, 0);
    for (size_t k = n0; k < h->u1_ev.size(); ++k) {
      cudaError_t e = cudaEventCreateWithFlags(&h->u1_ev[k], cudaEventDisableTiming);
      if (e != cudaSuccess) return e;
    }
  }
  cudaError_t e = cudaEventRecord(h->u1_ev[l], h->side);
  if (e == cudaSuccess) h->u1_pend[l] = 1;
  return e;
}

// The two flux-register kernels after stage s of level l on stream st: the
// coarse side of the registers of level l+1 and the fine side of level l's.
cudaError_t registers(amr_handle* h, int l, int s, const void* in, cudaStream_t st) {
  const bool kids = l + 1 < (int)h->dl.size();
  h->cur_class = AMR_T_REG;
  if (kids) {
    DevLevel& K = h->dl[l + 1];
    if (K.nreg)
      LK(h->ops->reg_coarse(st, K.regs, K.reg_first, K.reg_chunk, K.nrect, K.nreg, h->d_desc, in, K.R, h->params, l,
                            s));
  }
  DevLevel& L = h->dl[l];
  if (l > 0 && L.nreg)
    LK(h->ops->reg_fine(st, L.regs, L.reg_first, L.reg_chunk, L.nrect, L.nreg, h->d_desc, in, L.R, h->params, l));
  return cudaSuccess;
}

cudaError_t advance(amr_handle* h, int l, double alpha0) {
  static const char* names[] = {"level 0 step", "level 1 step", "level 2 step", "level 3 step", "level 4 step",
                                "level 5 step", "level 6 step", "level 7+ step"};
  Range range(names[l < 7 ? l : 7]);
  if (!h->capturing) h->cell_updates += h->plan.levels[l].cells;
  const int nlev = (int)h->dl.size();
  const bool kids = l + 1 < nlev;
  const bool ov = overlap_on(h);
  DevLevel& L = h->dl[l];
  const size_t es = h->ops->elem_size();
  // the level's state at the start of its step (U^n), which its children
  // interpolate in time: stored by stage 1 beside its own output (every interior
  // cell is updated exactly once), or copied
  void* uold = (kids && h->ops->stage_stores_old()) ? h->Uold : nullptr;
  if (kids && !uold) {
    cudaError_t e = cudaMemcpyAsync((char*)h->Uold + L.arena_begin * es, (char*)h->U + L.arena_begin * es,
                                    (L.arena_end - L.arena_begin) * es, cudaMemcpyDeviceToDevice, h->stream);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e;
  if ((e = fill_ghosts(h, l, h->U, alpha0)) != cudaSuccess) return e;
  if (ov) {
    // stage 2's parent cells into the second tile and prolonged into U1's ghost
    // cells, and stage 1's registers, beside stage 1
    if ((e = fork_side(h)) != cudaSuccess) return e;
    void* tile2 = h->tile ? (char*)h->tile + std::max<int64_t>(h->plan.tile_elems, 1) * es : nullptr;
    if ((e = fill_parent(h, l, h->U1, alpha0 + 0.5, h->side, tile2)) != cudaSuccess) return e;
    if ((e = registers(h, l, 1, h->U, h->side)) != cudaSuccess) return e;
    h->side_dirty = true;
    if ((e = u1_wait(h, l)) != cudaSuccess) return e;
    if ((e = stage(h, l, 1, h->U, h->U1, uold)) != cudaSuccess) return e;
    if ((e = join_side(h)) != cudaSuccess) return e;
    if ((e = fill_same(h, l, h->U1, false)) != cudaSuccess) return e;
    if ((e = stage(h, l, 2, h->U1, h->U)) != cudaSuccess) return e;
    if ((e = fork_side(h)) != cudaSuccess) return e;
    if ((e = registers(h, l, 2, h->U1, h->side)) != cudaSuccess) return e;
    if ((e = u1_mark(h, l)) != cudaSuccess) return e;
    h->side_dirty = true;
  } else {
    if ((e = stage(h, l, 1, h->U, h->U1, uold)) != cudaSuccess) return e;
    if ((e = registers(h, l, 1, h->U, h->stream)) != cudaSuccess) return e;
    if ((e = fill_ghosts(h, l, h->U1, alpha0 + 0.5)) != cudaSuccess) return e;
    if ((e = stage(h, l, 2, h->U1, h->U)) != cudaSuccess) return e;
    if ((e = registers(h, l, 2, h->U1, h->stream)) != cudaSuccess) return e;
  }
  if (kids) {
    if ((e = advance(h, l + 1, 0.0)) != cudaSuccess) return e;
    if ((e = advance(h, l + 1, 0.5)) != cudaSuccess) return e;
    if ((e = join_side(h)) != cudaSuccess) return e;
    DevLevel& K = h->dl[l + 1];
    h->cur_class = AMR_T_SYNC;
    if (h->cfg.batched) {
      const DevLevel::Flat& R = K.frestrict;
      LK(h->ops->restrict_flat(h->stream, static_cast<const FlatCopy*>(R.boxes), R.first, R.chunk_box, R.nchunk,
                               R.total, h->U));
    } else {
      LK(h->ops->restrict_(h->stream, K.restrict_segs, K.nrestrict, h->d_desc, h->U));
    }
    // reflux: the cells with one register in one launch; cells with several
    // registers in (d, side) passes, so each gets its corrections in that order
    const double dxc[3] = {level_dx(h, l, 0), level_dx(h, l, 1), level_dx(h, l, 2)};
    if (K.nreg)
      LK(h->ops->reflux(h->stream, K.regs, K.reg_first, K.reg_chunk, K.nrect, 0, K.nreg, K.nreg, h->d_desc, K.R, h->U,
                        dxc, 0));
    for (int pass = 0; pass < 6; ++pass)
      if (K.reg_ordered[pass] && K.reg_pass[pass + 1] > K.reg_pass[pass])
        LK(h->ops->reflux(h->stream, K.regs, K.reg_first, K.reg_chunk, K.nrect, K.reg_pass[pass],
                          K.reg_pass[pass + 1], K.nreg, h->d_desc, K.R, h->U, dxc, 1));
  }
  // scheduled regrid: rebuild the levels finer than l now that l has completed a
  // step (its parent has reached fraction alpha0 + 1/2 of its own step)
  if (h->sched_on && l <= h->sched_level && l < h->cfg.max_level) {
    if ((e = join_side(h)) != cudaSuccess) return e;
    const amr_status st = regrid_impl(h, h->sched_rp, l, l == 0 ? 1.0 : alpha0 + 0.5);
    for (char& p : h->u1_pend) p = 0;   // the side stream was joined
    if (st != AMR_OK) {
      h->sched_status = st;
      return cudaErrorUnknown;
    }
  }
  if (l == 0) {   // a step ends with nothing left on the side stream
    if ((e = join_side(h)) != cudaSuccess) return e;
    for (char& p : h->u1_pend) p = 0;
  }
  return cudaSuccess;
}

cudaError_t launch_begin_speed(amr_handle* h) {
  begin_speed_kernel<<<1, 1, 0, h->stream>>>(h->params);
  return cudaGetLastError();
}

cudaError_t launch_finalize_speed(amr_handle* h, int set_dt, int from_next, int use_rates, int clear_next) {
  finalize_speed_kernel<<<1, 1, 0, h->stream>>>(h->params, h->cfg.cfl, h->cfg.nvar == 9 ? h->cfg.ch : 1.0, set_dt,
                                                from_next, use_rates, clear_next);
  return cudaGetLastError();
}

// Standalone reduction over the state; clear_next = 1 when a step follows.
cudaError_t enqueue_speed(amr_handle* h, int set_dt, int clear_next) {
  h->cur_class = AMR_T_SPEED;
  LK(launch_begin_speed(h));
  LK(h->ops->speed(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->U, h->params, h->dx0));
  LK(launch_finalize_speed(h, set_dt, 0, 1, clear_next));
  return cudaSuccess;
}

bool fused_rates(const amr_handle* h) { return h->dl.size() == 1; }

// Which step variant runs: 1 bit "CFL dt", 2 bit "standalone reduction over the state".
int step_variant(const amr_handle* h, bool cfl) {
  const bool need = cfl || h->cfg.nvar == 9;
  const bool standalone = need && !(fused_rates(h) && h->rates_valid);
  return (cfl ? 1 : 0) + (standalone ? 2 : 0);
}

cudaError_t enqueue_step(amr_handle* h, int variant) {
  const bool cfl = variant & 1, standalone = variant & 2;
  const bool need = cfl || h->cfg.nvar == 9;
  if (standalone) {
    cudaError_t e = enqueue_speed(h, cfl ? 1 : 0, 1);
    if (e != cudaSuccess) return e;
  } else if (fused_rates(h)) {
    h->cur_class = AMR_T_SPEED;
    LK(launch_finalize_speed(h, cfl ? 1 : 0, 1, need ? 1 : 0, 1));
  }
  return advance(h, 0, 0.0);
}

amr_status run_step(amr_handle* h, bool cfl) {
  const int g = step_variant(h, cfl);
  if (h->cfg.use_graph && !h->timing && !h->sched_on) {
    if (!h->graph[g]) {
      cudaGraph_t graph;
      CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
      h->counting = 0;
      h->capturing = true;
      cudaError_t e = enqueue_step(h, g);
      h->capturing = false;
      cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
      if (e != cudaSuccess) return fail(h, AMR_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e));
      CK(e2);
      CK(cudaGraphInstantiate(&h->graph[g], graph, 0));
      cudaGraphDestroy(graph);
      h->graph_launches[g] = h->counting;
    }
    CK(cudaGraphLaunch(h->graph[g], h->stream));
    h->launches += h->graph_launches[g];
    for (size_t l = 0; l < h->plan.levels.size(); ++l) h->cell_updates += h->plan.levels[l].cells << l;
  } else {
    h->counting = 0;
    h->sched_status = AMR_OK;
    const cudaError_t e = enqueue_step(h, g);
    h->launches += h->counting;
    if (h->sched_status != AMR_OK) return h->sched_status;   // message set by the regrid
    CK(e);
  }
  if (fused_rates(h)) h->rates_valid = true;
  return AMR_OK;
}

amr_status read_bad(amr_handle* h) {
  unsigned int bad = 0;
  CK(cudaMemcpyAsync(&bad, &h->params->bad, sizeof bad, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (bad) {
    CK(cudaMemsetAsync(&h->params->bad, 0, sizeof(unsigned int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return fail(h, AMR_ERR_NONPHYSICAL, "non-physical state (rho <= 0, p <= 0 or NaN) detected on the device");
  }
  return AMR_OK;
}

// Layout of many host tables in one upload buffer (256-byte aligned offsets),
// assigned first and copied afterwards in parallel pieces, so no buffer grows
// or is zero-filled on the way.  The source vectors must outlive copy_to().
struct TablePack {
  struct Item { const unsigned char* src; size_t bytes, off; };
  std::vector<Item> items;
  size_t size = 1;
  template <typename X, typename A>
  size_t add(const std::vector<X, A>& v) {
    const size_t off = (size + 255) / 256 * 256;
    items.push_back({reinterpret_cast<const unsigned char*>(v.data()), v.size() * sizeof(X), off});
    size = off + v.size() * sizeof(X) + 1;
    return off;
  }
  void copy_to(unsigned char* dst) const {
    constexpr size_t kPiece = size_t(1) << 20;
    std::vector<Item> pieces;
    for (const Item& it : items)
      for (size_t b = 0; b < it.bytes; b += kPiece)
        pieces.push_back({it.src + b, std::min(kPiece, it.bytes - b), it.off + b});
    parallel_run((int)pieces.size(), [&](int i) { std::memcpy(dst + pieces[i].off, pieces[i].src, pieces[i].bytes); });
  }
};

// Pinned host staging of at least `bytes` (kept across installs, doubled when
// short).  Waits for the stream first: the previous upload may still read it.
cudaError_t host_stage(amr_handle* h, size_t bytes) {
  cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess || bytes <= h->stage_cap) return e;
  if (h->stage) cudaFreeHost(h->stage);
  h->stage = nullptr;
  h->stage_cap = 0;
  const size_t cap = std::max(bytes, 2 * h->stage_cap_seen);
  e = cudaMallocHost(reinterpret_cast<void**>(&h->stage), cap);
  if (e != cudaSuccess) {
    h->stage = nullptr;
    return e;
  }
  h->stage_cap = h->stage_cap_seen = cap;
  return cudaSuccess;
}

// Upload the stage work items of every level into their own device buffer.
amr_status upload_items(amr_handle* h) {
  // one buffer: every level's per-patch items, then its batched items, then the spans
  std::vector<StageItem> all;
  std::vector<size_t> first, bfirst;
  for (const LevelPlan& L : h->plan.levels) {
    first.push_back(all.size());
    all.insert(all.end(), L.items.begin(), L.items.end());
    bfirst.push_back(all.size());
    all.insert(all.end(), L.bitems.begin(), L.bitems.end());
  }
  const size_t span_off = (all.size() * sizeof(StageItem) + 255) / 256 * 256;
  const size_t bytes = span_off + h->plan.spans.size() * sizeof(ItemSpan);
  dfree(h, h->items_dev);
  h->items_dev = nullptr;
  void* p = nullptr;
  CK(dmalloc(h, &p, std::max<size_t>(bytes, 256)));
  h->items_dev = static_cast<StageItem*>(p);
  CK(cudaMemcpyAsync(h->items_dev, all.data(), all.size() * sizeof(StageItem), cudaMemcpyHostToDevice, h->stream));
  h->d_spans = reinterpret_cast<const ItemSpan*>(static_cast<unsigned char*>(p) + span_off);
  if (!h->plan.spans.empty())
    CK(cudaMemcpyAsync(static_cast<unsigned char*>(p) + span_off, h->plan.spans.data(),
                       h->plan.spans.size() * sizeof(ItemSpan), cudaMemcpyHostToDevice, h->stream));
  for (size_t l = 0; l < h->dl.size(); ++l) {
    h->dl[l].items = h->items_dev + first[l];
    h->dl[l].nitems = (int)h->plan.levels[l].items.size();
    h->dl[l].bitems = h->items_dev + bfirst[l];
    h->dl[l].nbitems = (int)h->plan.levels[l].bitems.size();
    h->dl[l].has_span = false;
    for (const StageItem& it : h->plan.levels[l].bitems) h->dl[l].has_span = h->dl[l].has_span || it.span >= 0;
  }
  return AMR_OK;
}

// Device buffers of one installed plan.
struct DeviceBufs {
  void* U = nullptr;
  void* U1 = nullptr;
  void* Uold = nullptr;
  void* tile = nullptr;
  double* packed = nullptr;
  double* partial = nullptr;
  double* totals = nullptr;
  double* regs = nullptr;
  unsigned char* tables = nullptr;
  StageItem* items = nullptr;
};

// Take the buffers out of the handle (graphs are dropped: they refer to them).
DeviceBufs detach(amr_handle* h) {
  for (int g = 0; g < 4; ++g) {
    if (h->graph[g]) cudaGraphExecDestroy(h->graph[g]);
    h->graph[g] = nullptr;
  }
  DeviceBufs b;
  b.U = h->U; b.U1 = h->U1; b.Uold = h->Uold; b.tile = h->tile;
  b.packed = h->packed; b.partial = h->partial; b.totals = h->totals; b.regs = h->regs; b.tables = h->tables;
  b.items = h->items_dev;
  h->items_dev = nullptr;
  h->U = h->U1 = h->Uold = h->tile = nullptr;
  h->packed = h->partial = h->totals = h->regs = nullptr;
  h->tables = nullptr;
  h->dl.clear();
  h->ready = false;
  h->rates_valid = false;
  return b;
}

void free_bufs(amr_handle* h, DeviceBufs& b) {
  void* ptrs[] = {b.U, b.U1, b.Uold, b.tile, b.packed, b.partial, b.totals, b.regs, b.tables, b.items};
  for (void* p : ptrs) dfree(h, p);
  b = DeviceBufs();
}

// Allocate the device state of `plan` and upload its tables (state left zero).
amr_status install_plan(amr_handle* h, Plan&& plan) {
  h->plan = std::move(plan);
  Plan& pl = h->plan;
  const int nv = pl.nvar;
  const size_t es = h->ops->elem_size();
  const int nlev = (int)pl.levels.size();
  const int npatch = (int)pl.patches.size();
  // chunks of <= 16384 interior cells
  h->chunks.clear();
  for (int i = 0; i < npatch; ++i) {
    int nc = pl.patches[i].n[0] * pl.patches[i].n[1] * pl.patches[i].n[2];
    for (int b = 0; b < nc; b += 16384) h->chunks.push_back({i, b, std::min(16384, nc - b)});
  }
  h->nchunk = (int)h->chunks.size();
  std::vector<size_t> reg_off(nlev, 0);
  size_t nregd = 0;
  for (int l = 1; l < nlev; ++l) {
    reg_off[l] = nregd;
    nregd += 2 * (size_t)nv * pl.levels[l].regs.total;
  }
  TablePack buf;
  size_t o_desc = buf.add(pl.desc);
  size_t o_chunks = buf.add(h->chunks);
  size_t o_cover = buf.add(pl.cover);
  size_t o_cover_first = buf.add(pl.cover_first);
  size_t o_packed_off = buf.add(pl.packed_off);
  std::vector<double> lvol(nlev);
  for (int l = 0; l < nlev; ++l) lvol[l] = level_dx(h, l, 0) * level_dx(h, l, 1) * level_dx(h, l, 2);
  size_t o_lvol = buf.add(lvol);
  struct FlatOffs { size_t boxes, first, chunk; };
  struct Offs { size_t items, ghost, ghost_stage, prolong, gather_ghost, restr; FlatOffs fg, fga, fa, fp, fr, rg; };
  std::vector<Offs> lo(nlev);
  auto put_flat = [&](const auto& f) { return FlatOffs{buf.add(f.boxes), buf.add(f.first), buf.add(f.chunk_box)}; };
  for (int l = 0; l < nlev; ++l) {
    LevelPlan& L = pl.levels[l];
    lo[l].fg = put_flat(L.fghost);
    lo[l].fga = put_flat(L.fghost_all);
    lo[l].fa = put_flat(L.fgather);
    lo[l].fp = put_flat(L.fprolong);
    lo[l].fr = put_flat(L.frestrict);
    lo[l].ghost = buf.add(L.ghost);
    lo[l].ghost_stage = buf.add(L.ghost_stage);
    lo[l].prolong = buf.add(L.prolong);
    lo[l].gather_ghost = buf.add(L.gather_ghost);
    lo[l].restr = buf.add(L.restrict_segs);
    lo[l].rg = put_flat(L.regs);
  }
  void* p = nullptr;
  CK(dmalloc(h, &p, buf.size));
  h->tables = static_cast<unsigned char*>(p);
  CK(host_stage(h, buf.size));
  buf.copy_to(h->stage);
  CK(cudaMemcpyAsync(h->tables, h->stage, buf.size, cudaMemcpyHostToDevice, h->stream));
  h->d_desc = reinterpret_cast<const PatchDesc*>(h->tables + o_desc);
  h->d_chunks = reinterpret_cast<const ChunkDesc*>(h->tables + o_chunks);
  h->d_cover = reinterpret_cast<const CoverBox*>(h->tables + o_cover);
  h->d_cover_first = reinterpret_cast<const int*>(h->tables + o_cover_first);
  h->d_packed_off = reinterpret_cast<const int64_t*>(h->tables + o_packed_off);
  h->d_level_vol = reinterpret_cast<const double*>(h->tables + o_lvol);
  CK(dmalloc(h, &h->U, pl.arena_elems * es));
  CK(dmalloc(h, &h->U1, pl.arena_elems * es));
  CK(cudaMemsetAsync(h->U, 0, pl.arena_elems * es, h->stream));
  CK(cudaMemsetAsync(h->U1, 0, pl.arena_elems * es, h->stream));
  if (nlev > 1) {
    CK(dmalloc(h, &h->Uold, pl.arena_elems * es));
    CK(cudaMemsetAsync(h->Uold, 0, pl.arena_elems * es, h->stream));
    // two parent tiles: stage 1's and (gathered on the side stream meanwhile) stage 2's
    CK(dmalloc(h, &h->tile, 2 * std::max<int64_t>(pl.tile_elems, 1) * es));
  }
  CK(dmalloc(h, &p, (size_t)h->nchunk * nv * sizeof(double)));
  h->partial = static_cast<double*>(p);
  CK(dmalloc(h, &p, 16 * sizeof(double)));
  h->totals = static_cast<double*>(p);
  if (nregd) {
    CK(dmalloc(h, &p, nregd * sizeof(double)));
    h->regs = static_cast<double*>(p);
    CK(cudaMemsetAsync(h->regs, 0, nregd * sizeof(double), h->stream));
  }
  h->dl.assign(nlev, DevLevel());
  for (int l = 0; l < nlev; ++l) {
    LevelPlan& L = pl.levels[l];
    DevLevel& D = h->dl[l];
    D.nghost = (int)L.ghost.size();
    D.nghost_stage = (int)L.ghost_stage.size();
    D.nprolong = (int)L.prolong.size();
    D.ngather_ghost = (int)L.gather_ghost.size();
    D.nrestrict = (int)L.restrict_segs.size();
    D.nreg = L.regs.total;
    D.nrect = (int)L.regs.boxes.size();
    for (int p = 0; p < 7; ++p) D.reg_pass[p] = L.reg_pass[p];
    for (int p = 0; p < 6; ++p) D.reg_ordered[p] = L.reg_ordered[p];
    D.ghost = reinterpret_cast<const CopySeg*>(h->tables + lo[l].ghost);
    D.ghost_stage = reinterpret_cast<const CopySeg*>(h->tables + lo[l].ghost_stage);
    D.prolong = reinterpret_cast<const ProlongBox*>(h->tables + lo[l].prolong);
    D.gather_ghost = reinterpret_cast<const CopySeg*>(h->tables + lo[l].gather_ghost);
    D.restrict_segs = reinterpret_cast<const RestrictSeg*>(h->tables + lo[l].restr);
    D.regs = reinterpret_cast<const RegRect*>(h->tables + lo[l].rg.boxes);
    D.reg_first = reinterpret_cast<const int*>(h->tables + lo[l].rg.first);
    D.reg_chunk = reinterpret_cast<const int*>(h->tables + lo[l].rg.chunk);
    D.R = h->regs ? h->regs + reg_off[l] : nullptr;
    auto set_flat = [&](DevLevel::Flat& F, const auto& f, const FlatOffs& o) {
      F.boxes = h->tables + o.boxes;
      F.first = reinterpret_cast<const int*>(h->tables + o.first);
      F.chunk_box = reinterpret_cast<const int*>(h->tables + o.chunk);
      F.nchunk = (int)f.chunk_box.size();
      F.total = f.total;
    };
    set_flat(D.fghost, L.fghost, lo[l].fg);
    set_flat(D.fghost_all, L.fghost_all, lo[l].fga);
    set_flat(D.fgather, L.fgather, lo[l].fa);
    set_flat(D.fprolong, L.fprolong, lo[l].fp);
    set_flat(D.frestrict, L.frestrict, lo[l].fr);
    const PatchDesc& a = pl.desc[L.first];
    const PatchDesc& b = pl.desc[L.first + L.count - 1];
    D.arena_begin = a.off;
    D.arena_end = b.off + b.vstride * nv;
  }
  return upload_items(h);
}

// Flag, cluster, plan and refill.  mid_level < 0: between coarse steps (levels
// above rp.min_level rebuilt, parent data at the current time).  mid_level >= 0:
// in the middle of a coarse step, right after a step of level mid_level whose
// parent has reached fraction alpha of its step: the levels above mid_level are
// rebuilt, ghosts of mid_level come from its parent at alpha, and the old-time
// states and flux registers of the kept levels carry over so the step goes on.
amr_status regrid_impl(amr_handle* h, const RegridParams& rp_in, int mid_level, double alpha) {
  Range range(mid_level >= 0 ? "regrid (inside a step)" : "regrid");
  // the work already queued on the stream (e.g. the level steps) is not regrid time
  CK(cudaStreamSynchronize(h->stream));
  using clk = std::chrono::steady_clock;
  auto t_mark = clk::now();
  auto lap = [&](int phase) {
    const auto t = clk::now();
    h->regrid_sec[phase] += std::chrono::duration<double>(t - t_mark).count();
    t_mark = t;
  };
  RegridParams rp = rp_in;
  const bool mid = mid_level >= 0;
  if (mid) rp.min_level = mid_level;
  const int nlev = (int)h->dl.size();
  const size_t es = h->ops->elem_size();
  Plan& op = h->plan;
  const int nv = op.nvar;
  std::string msg;
  {
    amr_status pst = check_regrid_params(h->cfg, rp, msg);
    if (pst != AMR_OK) return fail(h, pst, msg);
  }
  // 1. face ghosts of the flagged levels at the current time
  if (mid) {
    // the saved old-time states are still needed by the step: parent data of the
    // stepped level at fraction alpha, of the finer levels at fraction 1
    CK(fill_ghosts(h, mid_level, h->U, mid_level == 0 ? 1.0 : alpha, true));
    for (int l = mid_level + 1; l < nlev; ++l) CK(fill_ghosts(h, l, h->U, 1.0, true));
  } else {
    if (nlev > 1)
      CK(cudaMemcpyAsync(h->Uold, h->U, op.arena_elems * es, cudaMemcpyDeviceToDevice, h->stream));
    h->counting = 0;
    for (int l = 0; l < nlev; ++l) CK(fill_ghosts(h, l, h->U, 1.0, true));
  }
  // 2. density-gradient criterion.  Block tags and refinable blocks made on the
  //    GPU when every flagged level's block grid fits a bitmap (only the
  //    refinable bitmaps come back); otherwise one byte per interior cell, and
  //    the host clusters.
  const int L = h->cfg.max_level;
  TagArgs ta{};
  ta.l0 = rp.min_level;
  ta.L = L;
  ta.block = rp.block;
  ta.buffer = rp.buffer;
  bool dev_tags = L < kTagLevels;
  long long nwords = 0;
  for (int d = 0; d < 3; ++d) ta.per[d] = h->cfg.bc[2 * d] == AMR_BC_PERIODIC;
  for (int l = rp.min_level; l < L && dev_tags; ++l) {
    const int64_t nbt = regrid_tag_blocks(h->cfg, rp, l, ta.nb[l]);
    for (int d = 0; d < 3; ++d) ta.N[l][d] = h->cfg.base_n[d] << l;
    ta.off[l] = nwords;
    nwords += 2 * ((nbt + 63) / 64);
    dev_tags = nbt <= kTagDenseMax;
  }
  std::vector<HPatch> newp;
  amr_status st = AMR_OK;
  if (dev_tags) {
    // block tags, then (all on the GPU) the parent rings of finer tags, finest
    // level first, and the refinable blocks of every level, coarsest first: tagged
    // and with all 26 neighbours covered (the first level by its own patches, a
    // finer one by the refinable blocks of its parent level); only those bitmaps
    // come back, and the host keeps the greedy box merge
    auto grid = [&](int l, long long off) {
      const long long nbt = (long long)ta.nb[l][0] * ta.nb[l][1] * ta.nb[l][2];
      return BGrid{ta.nb[l][0], ta.nb[l][1], ta.nb[l][2], off, 2 * ((nbt + 63) / 64)};
    };
    long long maxnw = 2;
    for (int l = rp.min_level; l < L; ++l) maxnw = std::max(maxnw, grid(l, 0).nw);
    unsigned int *d_words = nullptr, *d_ref = nullptr, *d_tmp = nullptr;
    const size_t wbytes = std::max<long long>(nwords, 2) * sizeof(unsigned int);
    cudaError_t fe = dmalloc(h, reinterpret_cast<void**>(&d_words), wbytes);
    if (fe == cudaSuccess) fe = dmalloc(h, reinterpret_cast<void**>(&d_ref), wbytes);
    if (fe == cudaSuccess) fe = dmalloc(h, reinterpret_cast<void**>(&d_tmp), 2 * maxnw * sizeof(unsigned int));
    std::vector<uint32_t> hw((size_t)nwords);
    int nlaunch = 0;
    if (fe == cudaSuccess) fe = cudaMemsetAsync(d_words, 0, wbytes, h->stream);
    if (fe == cudaSuccess && nwords > 0) {
      fe = h->ops->tag(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->U, rp.threshold, ta, d_words);
      ++nlaunch;
    }
    unsigned int *tA = d_tmp, *tB = d_tmp + maxnw;
    auto box3 = [&](BGrid g, int erode) {   // tA -> (x) tB -> (y) tA -> (z) tB
      const BGrid a{g.n0, g.n1, g.n2, 0, g.nw};
      bm_box_axis<<<bm_grid(g.nw), 256, 0, h->stream>>>(tA, a, tB, a, 0, ta.per[0], erode);
      bm_box_axis<<<bm_grid(g.nw), 256, 0, h->stream>>>(tB, a, tA, a, 1, ta.per[1], erode);
      bm_box_axis<<<bm_grid(g.nw), 256, 0, h->stream>>>(tA, a, tB, a, 2, ta.per[2], erode);
      nlaunch += 3;
    };
    for (int l = L - 1; l > rp.min_level && fe == cudaSuccess && nwords > 0; --l) {
      const BGrid f = grid(l, ta.off[l]), g = grid(l - 1, ta.off[l - 1]);
      bm_downsample<<<bm_grid(g.nw), 256, 0, h->stream>>>(d_words, f, tA, BGrid{g.n0, g.n1, g.n2, 0, g.nw});
      box3(g, 0);
      bm_combine<<<bm_grid(g.nw), 256, 0, h->stream>>>(d_words, g.off, d_words, g.off, tB, 0, g.nw, 0);
      nlaunch += 2;
      fe = cudaGetLastError();
    }
    if (fe == cudaSuccess && nwords > 0) {
      const std::vector<uint64_t> base = regrid_base_cover(h->cfg, op.patches, rp);
      std::vector<uint32_t> b32(2 * base.size());
      for (size_t k = 0; k < base.size(); ++k) {
        b32[2 * k] = (uint32_t)(base[k] & 0xffffffffu);
        b32[2 * k + 1] = (uint32_t)(base[k] >> 32);
      }
      fe = cudaMemcpyAsync(tA, b32.data(), b32.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, h->stream);
      for (int l = rp.min_level; l < L && fe == cudaSuccess; ++l) {
        const BGrid g = grid(l, ta.off[l]);
        if (l > rp.min_level)
          bm_from_parent<<<bm_grid(g.nw), 256, 0, h->stream>>>(d_ref, grid(l - 1, ta.off[l - 1]), tA,
                                                                BGrid{g.n0, g.n1, g.n2, 0, g.nw});
        box3(g, 1);
        bm_combine<<<bm_grid(g.nw), 256, 0, h->stream>>>(d_ref, g.off, d_words, g.off, tB, 0, g.nw, 1);
        nlaunch += 1 + (l > rp.min_level ? 1 : 0);
        fe = cudaGetLastError();
      }
      if (fe == cudaSuccess)
        fe = cudaMemcpyAsync(hw.data(), d_ref, nwords * sizeof(unsigned int), cudaMemcpyDeviceToHost, h->stream);
      if (fe == cudaSuccess) fe = cudaStreamSynchronize(h->stream);
    } else if (fe == cudaSuccess) {
      fe = cudaStreamSynchronize(h->stream);
    }
    dfree(h, d_words);
    dfree(h, d_ref);
    dfree(h, d_tmp);
    CK(fe);
    if (!mid) h->launches += h->counting + nlaunch;
    else h->counting += nlaunch;
    std::vector<std::vector<uint64_t>> words(L);
    for (int l = rp.min_level; l < L; ++l) {
      const size_t n64 = (size_t)((l + 1 < L ? ta.off[l + 1] : nwords) - ta.off[l]) / 2;
      words[l].resize(n64);
      const uint32_t* w = hw.data() + ta.off[l];
      parallel_run((int)((n64 + 4095) / 4096), [&](int b) {
        for (size_t k = (size_t)b * 4096; k < std::min(n64, (size_t)(b + 1) * 4096); ++k)
          words[l][k] = (uint64_t)w[2 * k] | ((uint64_t)w[2 * k + 1] << 32);
      });
    }
    lap(AMR_RG_FLAG);
    // 3. merge the refinable blocks into patches on the host (or reuse the last
    //    clustering of this min_level when all of its inputs are the same)
    std::vector<HPatch> kept;
    for (const HPatch& p : op.patches)
      if (p.level <= rp.min_level) kept.push_back(p);
    auto same_patches = [](const std::vector<HPatch>& a, const std::vector<HPatch>& b) {
      if (a.size() != b.size()) return false;
      for (size_t i = 0; i < a.size(); ++i)
        if (std::memcmp(&a[i], &b[i], sizeof(HPatch)) != 0) return false;
      return true;
    };
    auto& M = h->memo[rp.min_level];
    const bool hit = M.valid && M.rp.threshold == rp.threshold && M.rp.buffer == rp.buffer &&
                     M.rp.block == rp.block && M.rp.max_patch == rp.max_patch && same_patches(M.kept, kept) &&
                     M.words == words;
    if (hit) {
      newp = M.result;
      h->memo_hits += 1;
    } else {
      M.valid = false;
      M.words = words;   // cluster_patches_refinable consumes its copy
      st = cluster_patches_refinable(h->cfg, op.patches, words, rp, newp, msg);
      if (st == AMR_OK) {
        M.rp = rp;
        M.kept = kept;
        M.result = newp;
        M.valid = true;
      }
    }
  } else {
    const size_t ncell = (size_t)(op.packed_elems / nv);
    unsigned char* d_flags = nullptr;
    CK(dmalloc(h, reinterpret_cast<void**>(&d_flags), std::max<size_t>(ncell, 1)));
    cudaError_t fe = h->ops->flag(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->d_packed_off, h->U,
                                  rp.threshold, d_flags);
    std::vector<unsigned char> hflags(ncell);
    if (fe == cudaSuccess)
      fe = cudaMemcpyAsync(hflags.data(), d_flags, ncell, cudaMemcpyDeviceToHost, h->stream);
    if (fe == cudaSuccess) fe = cudaStreamSynchronize(h->stream);
    dfree(h, d_flags);
    CK(fe);
    if (!mid) h->launches += h->counting + 1;
    else h->counting += 1;
    std::vector<std::vector<uint8_t>> flags(op.patches.size());
    for (size_t i = 0; i < op.patches.size(); ++i) {
      const HPatch& p = op.patches[i];
      if (p.level >= L) continue;
      const size_t n = (size_t)p.n[0] * p.n[1] * p.n[2];
      const size_t o = (size_t)(op.packed_off[i] / nv);
      flags[i].assign(hflags.begin() + o, hflags.begin() + o + n);
    }
    lap(AMR_RG_FLAG);
    // 3. cluster on the host, build the new hierarchy
    st = cluster_patches(h->cfg, op.patches, flags, rp, newp, msg);
  }
  if (st != AMR_OK) return fail(h, st, msg);
  lap(AMR_RG_CLUSTER);
  // the same hierarchy again: the refill would copy every cell onto itself
  bool same = newp.size() == op.patches.size();
  for (size_t i = 0; same && i < newp.size(); ++i) {
    const HPatch &a = newp[i], &b = op.patches[i];
    same = a.level == b.level && a.lo[0] == b.lo[0] && a.lo[1] == b.lo[1] && a.lo[2] == b.lo[2] &&
           a.n[0] == b.n[0] && a.n[1] == b.n[1] && a.n[2] == b.n[2];
  }
  if (same) {
    h->regrid_counts[1] += 1;
    return AMR_OK;
  }
  h->regrid_counts[0] += 1;
  Plan np;
  st = build_plan(h->cfg, newp, np, msg, h->tp);
  if (st != AMR_OK) return fail(h, st, "regrid produced an invalid hierarchy: " + msg);
  lap(AMR_RG_PLAN);
  RegridFill fill;
  build_regrid_fill(op.patches, newp, rp.min_level, fill);
  std::vector<std::vector<CopySeg>> fill_gather;   // parent cells of the fresh boxes' prolongation
  build_fill_gathers(h->cfg, np, fill.fresh, fill_gather, msg);
  if (!msg.empty()) return fail(h, AMR_ERR_NESTING, "regrid fill: " + msg);
  lap(AMR_RG_FILLTAB);
  // 4. new device state, filled from the old one
  const PatchDesc* old_desc = h->d_desc;
  const std::vector<HPatch> oldp = op.patches;
  int64_t keep_end = 0;    // arena range of the kept levels (same patches, same layout)
  for (size_t i = 0; i < oldp.size(); ++i)
    if (oldp[i].level <= rp.min_level) keep_end = op.desc[i].off + op.desc[i].vstride * nv;
  // flux registers of the kept levels (same faces, same order, same layout)
  size_t keep_regs = 0;
  if (mid) {
    for (int l = 1; l <= rp.min_level && l < (int)op.levels.size(); ++l) {
      if (l >= (int)np.levels.size() || np.levels[l].regs.total != op.levels[l].regs.total)
        return fail(h, AMR_ERR_STATE, "regrid: the kept levels changed");
      keep_regs += 2 * (size_t)nv * op.levels[l].regs.total;
    }
  }
  DeviceBufs old = detach(h);
  st = install_plan(h, std::move(np));
  if (st != AMR_OK) {
    free_bufs(h, old);
    return st;
  }
  TablePack buf;
  std::vector<size_t> o_copy(fill.copy.size()), o_fresh(fill.fresh.size()), o_fg(fill.fresh.size());
  cudaError_t ei = cudaStreamSynchronize(h->stream);   // uploads of the new tables done
  if (ei != cudaSuccess) {
    free_bufs(h, old);
    CK(ei);
  }
  lap(AMR_RG_INSTALL);
  for (size_t l = 0; l < fill.copy.size(); ++l) {
    o_copy[l] = buf.add(fill.copy[l]);
    o_fresh[l] = buf.add(fill.fresh[l]);
    o_fg[l] = buf.add(fill_gather[l]);
  }
  unsigned char* d_fill = nullptr;
  cudaError_t e = dmalloc(h, reinterpret_cast<void**>(&d_fill), buf.size);
  if (e == cudaSuccess) e = host_stage(h, buf.size);
  if (e == cudaSuccess) {
    buf.copy_to(h->stage);
    e = cudaMemcpyAsync(d_fill, h->stage, buf.size, cudaMemcpyHostToDevice, h->stream);
  }
  if (e == cudaSuccess && keep_end > 0)
    e = cudaMemcpyAsync(h->U, old.U, keep_end * es, cudaMemcpyDeviceToDevice, h->stream);
  const int nl_new = (int)h->dl.size();
  if (e == cudaSuccess && nl_new > 1 && keep_end > 0)
    e = cudaMemcpyAsync(h->Uold, (mid && old.Uold) ? old.Uold : h->U, keep_end * es, cudaMemcpyDeviceToDevice,
                        h->stream);   // (no old-time state yet when the kept levels had no children)
  if (e == cudaSuccess && keep_regs > 0)
    e = cudaMemcpyAsync(h->regs, old.regs, keep_regs * sizeof(double), cudaMemcpyDeviceToDevice, h->stream);
  for (int l = rp.min_level + 1; l < nl_new && e == cudaSuccess; ++l) {
    const DevLevel& L = h->dl[l];
    // interior cells no old patch covers: conservative prolongation from the (new) parent level
    if (l < (int)fill.fresh.size())
      e = h->ops->gather(h->stream, reinterpret_cast<const CopySeg*>(d_fill + o_fg[l]), (int)fill_gather[l].size(),
                         h->d_desc, h->tile, h->U, h->U, 1.0);
    if (e == cudaSuccess && l < (int)fill.fresh.size())
      e = h->ops->prolong(h->stream, reinterpret_cast<const ProlongBox*>(d_fill + o_fresh[l]),
                          (int)fill.fresh[l].size(), h->d_desc, h->tile, h->U);
    if (e == cudaSuccess && l < (int)fill.copy.size())
      e = h->ops->xcopy(h->stream, reinterpret_cast<const CopySeg*>(d_fill + o_copy[l]), (int)fill.copy[l].size(),
                        h->d_desc, old_desc, h->U, old.U);
    if (mid) h->counting += 3;
    else h->launches += 3;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dfree(h, d_fill);
  free_bufs(h, old);
  CK(e);
  lap(AMR_RG_FILL);
  h->ready = true;
  return AMR_OK;
}


}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

extern "C" {

void amr_default_config(amr_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof *c);
  c->nvar = 5;
  c->precision = AMR_FP64;
  c->riemann = AMR_HLL;
  c->gamma = 1.4;
  c->theta = 1.5;
  c->cfl = 0.4;
  for (int d = 0; d < 3; ++d) {
    c->base_n[d] = 32;
    c->domain_lo[d] = 0.0;
    c->domain_hi[d] = 1.0;
  }
  for (int f = 0; f < 6; ++f) c->bc[f] = AMR_BC_OUTFLOW;
  c->max_level = 0;
  c->ref_ratio = 2;
  c->ch = 0.0;
  c->batched = 1;
  c->use_graph = 1;
  c->cuda_stream = nullptr;
  c->recon = AMR_PLM;
}

const char* amr_global_error(void) { return g_global_err.c_str(); }

amr_status amr_create(const amr_config* cfg, amr_handle** out) {
  if (!out) { g_global_err = "out is NULL"; return AMR_ERR_ARG; }
  *out = nullptr;
  if (!cfg) { g_global_err = "cfg is NULL"; return AMR_ERR_ARG; }
  std::string msg;
  amr_status st = validate_config(*cfg, msg);
  if (st != AMR_OK) { g_global_err = msg; return st; }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    g_global_err = "no CUDA device";
    return AMR_ERR_CUDA;
  }
  amr_handle* h = new amr_handle();
  h->cfg = *cfg;
  for (int d = 0; d < 3; ++d) h->dx0[d] = (cfg->domain_hi[d] - cfg->domain_lo[d]) / cfg->base_n[d];
  if (cfg->cuda_stream) {
    h->stream = static_cast<cudaStream_t>(cfg->cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      g_global_err = "cudaStreamCreate failed";
      delete h;
      return AMR_ERR_CUDA;
    }
    h->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess) {
    g_global_err = "cudaStreamCreate failed";
    if (h->own_stream) cudaStreamDestroy(h->stream);
    delete h;
    return AMR_ERR_CUDA;
  }
  h->ops = make_ops(*cfg);
  {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
      cudaGetLastError();
      g_global_err = "device query failed";
      amr_destroy(h);
      return AMR_ERR_CUDA;
    }
  }
  if (!(cfg->dev_alloc && cfg->dev_free)) {
    int dev = 0;
    cudaError_t pe = cudaGetDevice(&dev);
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    uint64_t keep = UINT64_MAX;
    if (pe == cudaSuccess) pe = cudaMemPoolCreate(&h->pool, &props);
    if (pe == cudaSuccess) pe = cudaMemPoolSetAttribute(h->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (pe != cudaSuccess) {
      cudaGetLastError();
      g_global_err = "creation of the device memory pool failed";
      amr_destroy(h);
      return AMR_ERR_CUDA;
    }
  }
  void* p = nullptr;
  if (dmalloc(h, &p, sizeof(StepParams)) != cudaSuccess) {
    g_global_err = "allocation of the step parameters failed";
    amr_destroy(h);
    return AMR_ERR_CUDA;
  }
  h->params = static_cast<StepParams*>(p);
  cudaMemsetAsync(h->params, 0, sizeof(StepParams), h->stream);
  if (cudaGetLastError() != cudaSuccess) {
    g_global_err = "CUDA error at create";
    amr_destroy(h);
    return AMR_ERR_CUDA;
  }
  *out = h;
  return AMR_OK;
}

amr_status amr_partition_patches(const amr_config* cfg, int npatch, const amr_patch* patches, int nranks,
                                 int* owner) {
  if (!cfg || npatch <= 0 || !patches || nranks < 1 || !owner) return AMR_ERR_ARG;
  std::vector<HPatch> P(npatch);
  for (int i = 0; i < npatch; ++i) {
    P[i].level = patches[i].level;
    for (int d = 0; d < 3; ++d) {
      P[i].lo[d] = patches[i].lo[d];
      P[i].n[d] = patches[i].n[d];
      if (P[i].lo[d] < 0 || P[i].n[d] < 1 || P[i].level < 0 || P[i].level > 12) return AMR_ERR_ARG;
    }
  }
  const std::vector<int> o = morton_partition(*cfg, P, nranks);
  std::memcpy(owner, o.data(), npatch * sizeof(int));
  return AMR_OK;
}

amr_status amr_validate_patches(const amr_config* cfg, int npatch, const amr_patch* patches, char* msg,
                                int msg_len) {
  std::string m;
  amr_status st;
  if (!cfg || npatch <= 0 || !patches) {
    m = "null config, no patches or null patch array";
    st = AMR_ERR_ARG;
  } else {
    std::vector<HPatch> P(npatch);
    for (int i = 0; i < npatch; ++i) {
      P[i].level = patches[i].level;
      for (int d = 0; d < 3; ++d) { P[i].lo[d] = patches[i].lo[d]; P[i].n[d] = patches[i].n[d]; }
    }
    st = validate_patches(*cfg, P, m);
  }
  g_global_err = m;
  if (msg && msg_len > 0) {
    std::strncpy(msg, m.c_str(), (size_t)msg_len - 1);
    msg[msg_len - 1] = 0;
  }
  return st;
}

amr_status amr_set_patches(amr_handle* h, int npatch, const amr_patch* patches, const double* const* state,
                           int state_kind) {
  if (!h) return AMR_ERR_ARG;
  if (npatch <= 0 || !patches || !state) return fail(h, AMR_ERR_ARG, "null patches or state");
  if (state_kind != AMR_STATE_CONSERVED && state_kind != AMR_STATE_PRIMITIVE)
    return fail(h, AMR_ERR_ARG, "state_kind must be AMR_STATE_CONSERVED or AMR_STATE_PRIMITIVE");
  for (int i = 0; i < npatch; ++i)
    if (!state[i]) return fail(h, AMR_ERR_ARG, "null state pointer");
  std::vector<HPatch> P(npatch);
  for (int i = 0; i < npatch; ++i) {
    P[i].level = patches[i].level;
    for (int d = 0; d < 3; ++d) { P[i].lo[d] = patches[i].lo[d]; P[i].n[d] = patches[i].n[d]; }
  }
  Plan plan;
  std::string msg;
  amr_status st = build_plan(h->cfg, P, plan, msg, h->tp);
  if (st != AMR_OK) return fail(h, st, msg);
  CK(cudaStreamSynchronize(h->stream));
  DeviceBufs old = detach(h);
  free_bufs(h, old);
  st = install_plan(h, std::move(plan));
  if (st != AMR_OK) return st;
  Plan& pl = h->plan;
  const int nv = pl.nvar;
  // initial state: pack on the host, one copy, convert on the device
  std::vector<double> host(pl.packed_elems);
  for (int i = 0; i < npatch; ++i) {
    size_t n = (size_t)P[i].n[0] * P[i].n[1] * P[i].n[2] * nv;
    std::memcpy(host.data() + pl.packed_off[i], state[i], n * sizeof(double));
  }
  CK(ensure_packed(h));
  CK(cudaMemcpyAsync(h->packed, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(cudaMemsetAsync(&h->params->bad, 0, sizeof(unsigned int), h->stream));
  CK(h->ops->pack_in(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->d_packed_off, h->packed, h->U,
                     state_kind == AMR_STATE_PRIMITIVE, h->params));
  h->launches += 1;
  CK(cudaStreamSynchronize(h->stream));
  h->ready = true;
  return read_bad(h);
}

amr_status amr_get_regrid_timing(amr_handle* h, double* sec, int n) {
  if (!h || !sec || n < 1 || n > AMR_RG_NPHASE) return AMR_ERR_ARG;
  for (int i = 0; i < n; ++i) sec[i] = h->regrid_sec[i];
  for (double& x : h->regrid_sec) x = 0.0;
  return AMR_OK;
}

amr_status amr_regrid(amr_handle* h, const amr_regrid_params* prm, int* npatch_out) {
  if (!h) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  RegridParams rp;
  if (prm) {
    rp.threshold = prm->threshold;
    rp.buffer = prm->buffer;
    rp.block = prm->block;
    rp.max_patch = prm->max_patch;
    rp.min_level = prm->min_level;
  }
  if (!(rp.threshold > 0.0)) return fail(h, AMR_ERR_ARG, "regrid threshold must be > 0");
  const amr_status st = regrid_impl(h, rp, -1, 1.0);
  if (st != AMR_OK) return st;
  if (npatch_out) *npatch_out = (int)h->plan.patches.size();
  return AMR_OK;
}

amr_status amr_set_regrid_schedule(amr_handle* h, const amr_regrid_params* prm, int max_level) {
  if (!h) return AMR_ERR_ARG;
  if (max_level < 0) {
    h->sched_on = false;
    h->sched_level = -1;
    return AMR_OK;
  }
  RegridParams rp;
  if (prm) {
    rp.threshold = prm->threshold;
    rp.buffer = prm->buffer;
    rp.block = prm->block;
    rp.max_patch = prm->max_patch;
  }
  if (!(rp.threshold > 0.0)) return fail(h, AMR_ERR_ARG, "regrid threshold must be > 0");
  if (rp.block < 2 || (rp.block & 1) || rp.buffer < 0 || rp.buffer > rp.block || rp.max_patch < 2 * rp.block ||
      rp.max_patch % (2 * rp.block))
    return fail(h, AMR_ERR_ARG, "bad regrid parameters (block even >= 2, 0 <= buffer <= block, "
                                "max_patch a multiple of 2 block)");
  h->sched_rp = rp;
  h->sched_level = max_level;
  h->sched_on = true;
  for (int g = 0; g < 4; ++g) {   // scheduled steps run eagerly
    if (h->graph[g]) cudaGraphExecDestroy(h->graph[g]);
    h->graph[g] = nullptr;
  }
  return AMR_OK;
}

amr_status amr_set_tiling(amr_handle* h, int max_wx, int max_cols, int zchunk, int ctas_per_sm) {
  if (!h) return AMR_ERR_ARG;
  if (max_wx < 0 || max_wx > kMaxTileX) return fail(h, AMR_ERR_ARG, "max_wx must be in 0..32");
  if (max_cols != 0 && max_cols != 128 && max_cols != kStageThreads)
    return fail(h, AMR_ERR_ARG, "max_cols must be 0, 128 or 256");
  if (zchunk < 0) return fail(h, AMR_ERR_ARG, "zchunk must be >= 0");
  if (ctas_per_sm < 0) return fail(h, AMR_ERR_ARG, "ctas_per_sm must be >= 0");
  const int keep_occ = h->ops->stage_occupancy();
  h->ops->set_stage_threads(max_cols == 128 ? 128 : kStageThreads);
  int occ = -1;
  for (int o : {0, h->ops->alt_occupancy()}) {
    h->ops->set_stage_occupancy(o);
    if (ctas_per_sm == 0 ? o == 0 : h->ops->resident_ctas() == ctas_per_sm) {
      occ = o;
      break;
    }
  }
  if (occ < 0) {
    h->ops->set_stage_occupancy(keep_occ);
    h->ops->set_stage_threads(h->tp.max_cols);
    return fail(h, AMR_ERR_ARG, "no stage-kernel build with that many CTAs per SM for this column count");
  }
  h->tp.max_wx = max_wx;
  h->tp.max_cols = max_cols;
  h->tp.zchunk = zchunk;
  h->tp.persistent = h->persist_mode == 1 ? 1 : 0;
  for (int g = 0; g < 4; ++g) {
    if (h->graph[g]) cudaGraphExecDestroy(h->graph[g]);
    h->graph[g] = nullptr;
  }
  if (!h->ready) return AMR_OK;
  build_items(h->plan, h->tp);
  return upload_items(h);
}

amr_status amr_set_overlap(amr_handle* h, int on) {
  if (!h) return AMR_ERR_ARG;
  if (on != 0 && on != 1) return fail(h, AMR_ERR_ARG, "on must be 0 or 1");
  if (h->overlap != (on == 1)) {
    h->overlap = on == 1;
    for (int g = 0; g < 4; ++g) {
      if (h->graph[g]) cudaGraphExecDestroy(h->graph[g]);
      h->graph[g] = nullptr;
    }
  }
  return AMR_OK;
}

amr_status amr_set_persistent(amr_handle* h, int mode) {
  if (!h) return AMR_ERR_ARG;
  if (mode < -1 || mode > 1) return fail(h, AMR_ERR_ARG, "mode must be -1, 0 or 1");
  h->persist_mode = mode;
  if (mode >= 0 && h->tp.persistent != mode) {
    h->tp.persistent = mode;
    for (int g = 0; g < 4; ++g) {
      if (h->graph[g]) cudaGraphExecDestroy(h->graph[g]);
      h->graph[g] = nullptr;
    }
  }
  return AMR_OK;
}

amr_status amr_autotune(amr_handle* h, char* report, int report_len) {
  if (!h) return AMR_ERR_ARG;
  Range range("amr_autotune");
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  struct Cand { TileParams tp; int occ; };
  std::vector<Cand> cands;
  const int occs[2] = {0, h->ops->alt_occupancy()};
  const int shapes[7][3] = {{32, 256, 32}, {32, 256, 16}, {16, 256, 16}, {32, 256, 64},
                            {16, 128, 8}, {16, 128, 16}, {16, 128, 32}};
  // the WENO3 stage runs one build (256 threads, default register budget) for every
  // tiling, so only the work-item shapes are tuned
  const bool one_build = h->cfg.recon == AMR_WENO3;
  // launch forms: one CTA per work item, and persistent CTAs fed by a device
  // counter (default build only), unless amr_set_persistent fixed one
  for (int pers = 0; pers < 2; ++pers) {
    if (h->persist_mode >= 0 && pers != h->persist_mode) continue;
    for (int o = 0; o < 2; ++o) {
      if (o == 1 && (occs[1] == 0 || one_build || pers == 1)) continue;
      for (auto& sh : shapes) {
        if (o == 1 && sh[1] == 128 && !h->ops->has_alt128()) continue;   // no second 128-thread budget
        Cand c;
        c.tp.max_wx = sh[0]; c.tp.max_cols = sh[1]; c.tp.zchunk = sh[2];
        c.tp.persistent = pers;
        c.occ = occs[o];
        cands.push_back(c);
      }
    }
  }
  // valid ghosts everywhere (stage 1 reads them; U1 is scratch, U is not modified)
  const int nlev = (int)h->dl.size();
  const size_t es = h->ops->elem_size();
  if (nlev > 1) CK(cudaMemcpyAsync(h->Uold, h->U, h->plan.arena_elems * es, cudaMemcpyDeviceToDevice, h->stream));
  h->counting = 0;
  for (int l = 0; l < nlev; ++l) CK(fill_ghosts(h, l, h->U, 1.0));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  const TileParams keep_tp = h->tp;
  const int keep_occ = h->ops->stage_occupancy();
  double best = 1e300;
  int best_i = -1;
  std::string rep;
  for (size_t ci = 0; ci < cands.size(); ++ci) {
    h->tp = cands[ci].tp;
    h->ops->set_stage_occupancy(cands[ci].occ);
    h->ops->set_stage_threads(h->tp.max_cols);
    build_items(h->plan, h->tp);
    amr_status st = upload_items(h);
    if (st != AMR_OK) break;
    double t_best = 1e300;
    for (int rep_i = 0; rep_i < 4; ++rep_i) {
      CK(cudaEventRecord(e0, h->stream));
      for (int l = 0; l < nlev; ++l) CK(stage(h, l, 1, h->U, h->U1));
      CK(cudaEventRecord(e1, h->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep_i > 0) t_best = std::min(t_best, (double)ms);   // first run warms up
    }
    char line[160];
    std::snprintf(line, sizeof line, "tile wx<=%d cols<=%d z=%d ctas/SM=%d%s: %.4f ms%s\n", h->tp.max_wx,
                  h->tp.max_cols, h->tp.zchunk, h->ops->resident_ctas(), h->tp.persistent ? " persistent" : "",
                  t_best, one_build ? " (WENO3: default 256-thread build)" : "");
    rep += line;
    if (t_best < best) { best = t_best; best_i = (int)ci; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_i < 0) {
    h->tp = keep_tp;
    h->ops->set_stage_occupancy(keep_occ);
    h->ops->set_stage_threads(h->tp.max_cols);
  } else {
    h->tp = cands[best_i].tp;
    h->ops->set_stage_occupancy(cands[best_i].occ);
    h->ops->set_stage_threads(h->tp.max_cols);
    char line[96];
    std::snprintf(line, sizeof line, "chosen: candidate %d\n", best_i);
    rep += line;
  }
  build_items(h->plan, h->tp);
  amr_status st = upload_items(h);
  for (int g = 0; g < 4; ++g) {
    if (h->graph[g]) cudaGraphExecDestroy(h->graph[g]);
    h->graph[g] = nullptr;
  }
  CK(cudaMemsetAsync(&h->params->bad, 0, sizeof(unsigned int), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  h->launches += h->counting;
  if (report && report_len > 0) {
    std::strncpy(report, rep.c_str(), (size_t)report_len - 1);
    report[report_len - 1] = 0;
  }
  return st;
}

int amr_get_patches(const amr_handle* h, amr_patch* out, int capacity) {
  if (!h || !h->ready) return -1;
  const int n = (int)h->plan.patches.size();
  if (out)
    for (int i = 0; i < n && i < capacity; ++i) {
      out[i].level = h->plan.patches[i].level;
      for (int d = 0; d < 3; ++d) {
        out[i].lo[d] = h->plan.patches[i].lo[d];
        out[i].n[d] = h->plan.patches[i].n[d];
      }
    }
  return n;
}

long long amr_state_size(const amr_handle* h) { return (h && h->ready) ? h->plan.packed_elems : 0; }

amr_status amr_set_state(amr_handle* h, const double* packed, int state_kind) {
  if (!h) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  if (!packed) return fail(h, AMR_ERR_ARG, "null state buffer");
  if (state_kind != AMR_STATE_CONSERVED && state_kind != AMR_STATE_PRIMITIVE)
    return fail(h, AMR_ERR_ARG, "bad state_kind");
  CK(ensure_packed(h));
  CK(cudaMemcpyAsync(h->packed, packed, h->plan.packed_elems * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  CK(h->ops->pack_in(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->d_packed_off, h->packed, h->U,
                     state_kind == AMR_STATE_PRIMITIVE, h->params));
  h->launches += 1;
  h->rates_valid = false;
  return AMR_OK;
}

amr_status amr_step(amr_handle* h, double dt, double* dt_used) {
  if (!h) return AMR_ERR_ARG;
  Range range("amr_step");
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  if (!std::isfinite(dt)) return fail(h, AMR_ERR_ARG, "dt must be finite");
  const bool cfl = !(dt > 0.0);
  if (!cfl) {
    set_dt_kernel<<<1, 1, 0, h->stream>>>(h->params, dt);
    CK(cudaGetLastError());
    h->launches += 1;
  }
  amr_status st = run_step(h, cfl);
  if (st != AMR_OK) return st;
  if (dt_used) {
    CK(cudaMemcpyAsync(dt_used, &h->params->dt0, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    return read_bad(h);
  }
  return AMR_OK;
}

amr_status amr_cfl_dt(amr_handle* h, double* dt) {
  if (!h || !dt) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  h->counting = 0;
  h->cur_class = AMR_T_SPEED;
  if (fused_rates(h) && h->rates_valid) {
    // maxima of the current state were left by the last stage 2: no pass over the state
    CK(launch_finalize_speed(h, 1, 1, 1, 0));
    h->counting += 1;
  } else {
    CK(enqueue_speed(h, 1, 0));
  }
  h->launches += h->counting;
  CK(cudaMemcpyAsync(dt, &h->params->dt0, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

amr_status amr_get_state_all(amr_handle* h, double* packed) {
  if (!h || !packed) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  CK(ensure_packed(h));
  CK(h->ops->pack_out(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->d_packed_off, h->U, h->packed));
  h->launches += 1;
  CK(cudaMemcpyAsync(packed, h->packed, h->plan.packed_elems * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

amr_status amr_set_state_async(amr_handle* h, const double* packed, int state_kind) {
  if (!h) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  if (!packed) return fail(h, AMR_ERR_ARG, "null state buffer");
  if (state_kind != AMR_STATE_CONSERVED && state_kind != AMR_STATE_PRIMITIVE)
    return fail(h, AMR_ERR_ARG, "bad state_kind");
  CK(ensure_async(h));
  const int k = (int)(h->n_in % amr_handle::kSlots);
  CK(cudaStreamWaitEvent(h->cs_in, h->ev_in_used[k], 0));   // the slot's previous conversion is done
  CK(cudaMemcpyAsync(h->in_slot[k], packed, h->plan.packed_elems * sizeof(double), cudaMemcpyHostToDevice,
                     h->cs_in));
  CK(cudaEventRecord(h->ev_h2d[k], h->cs_in));
  CK(cudaStreamWaitEvent(h->stream, h->ev_h2d[k], 0));
  CK(h->ops->pack_in(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->d_packed_off, h->in_slot[k], h->U,
                     state_kind == AMR_STATE_PRIMITIVE, h->params));
  CK(cudaEventRecord(h->ev_in_used[k], h->stream));
  h->launches += 1;
  h->rates_valid = false;
  h->n_in += 1;
  return AMR_OK;
}

amr_status amr_get_state_all_async(amr_handle* h, double* packed, long long* ticket) {
  if (!h || !packed || !ticket) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  CK(ensure_async(h));
  const int k = (int)(h->n_out % amr_handle::kSlots);
  CK(cudaStreamWaitEvent(h->stream, h->ev_d2h[k], 0));   // the slot's previous download is done
  CK(h->ops->pack_out(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->d_packed_off, h->U, h->out_slot[k]));
  CK(cudaEventRecord(h->ev_packout[k], h->stream));
  CK(cudaStreamWaitEvent(h->cs_out, h->ev_packout[k], 0));
  CK(cudaMemcpyAsync(packed, h->out_slot[k], h->plan.packed_elems * sizeof(double), cudaMemcpyDeviceToHost,
                     h->cs_out));
  CK(cudaEventRecord(h->ev_d2h[k], h->cs_out));
  h->launches += 1;
  *ticket = h->n_out++;
  return AMR_OK;
}

amr_status amr_wait_state(amr_handle* h, long long ticket) {
  if (!h) return AMR_ERR_ARG;
  if (ticket < 0 || ticket >= h->n_out) return fail(h, AMR_ERR_ARG, "unknown ticket");
  // a later download from the same slot completes after this one (one copy stream)
  CK(cudaEventSynchronize(h->ev_d2h[ticket % amr_handle::kSlots]));
  return AMR_OK;
}

amr_status amr_get_state(amr_handle* h, int patch, double* out) {
  if (!h || !out) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  if (patch < 0 || patch >= (int)h->plan.patches.size()) return fail(h, AMR_ERR_ARG, "patch index out of range");
  CK(ensure_packed(h));
  CK(h->ops->pack_out(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->d_packed_off, h->U, h->packed));
  h->launches += 1;
  const HPatch& P = h->plan.patches[patch];
  size_t n = (size_t)P.n[0] * P.n[1] * P.n[2] * h->plan.nvar;
  CK(cudaMemcpyAsync(out, h->packed + h->plan.packed_off[patch], n * sizeof(double), cudaMemcpyDeviceToHost,
                     h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

amr_status amr_conserved_totals(amr_handle* h, double* out) {
  if (!h || !out) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  CK(h->ops->totals(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->U, h->d_cover, h->d_cover_first,
                    h->d_level_vol, h->partial, h->totals));
  h->launches += 2;
  CK(cudaMemcpyAsync(out, h->totals, h->plan.nvar * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

amr_status amr_divb_norms(amr_handle* h, double* out) {
  if (!h || !out) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  if (h->plan.nvar != 9) return fail(h, AMR_ERR_ARG, "div B needs nvar = 9 (GLM-MHD)");
  Range range("div B");
  const int nlev = (int)h->dl.size();
  const size_t es = h->ops->elem_size();
  if (nlev > 1)
    CK(cudaMemcpyAsync(h->Uold, h->U, h->plan.arena_elems * es, cudaMemcpyDeviceToDevice, h->stream));
  h->counting = 0;
  for (int l = 0; l < nlev; ++l) CK(fill_ghosts(h, l, h->U, 1.0, true));
  CK(h->ops->divb(h->stream, h->d_chunks, h->nchunk, h->d_desc, h->U, h->d_cover, h->d_cover_first, h->dx0,
                  h->partial, h->totals));
  h->launches += h->counting + 2;
  CK(cudaMemcpyAsync(out, h->totals, 4 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

amr_status amr_get_regrid_counts(amr_handle* h, long long* counts) {
  if (!h || !counts) return AMR_ERR_ARG;
  counts[0] = h->regrid_counts[0];
  counts[1] = h->regrid_counts[1];
  counts[2] = h->memo_hits;
  return AMR_OK;
}

amr_status amr_floor_count(amr_handle* h, long long* count) {
  if (!h || !count) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  unsigned long long v = 0;
  CK(cudaMemcpyAsync(&v, &h->params->floor_hits, sizeof v, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaMemsetAsync(&h->params->floor_hits, 0, sizeof v, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *count = (long long)v;
  return AMR_OK;
}

amr_status amr_check(amr_handle* h) {
  if (!h) return AMR_ERR_ARG;
  if (!h->ready) return fail(h, AMR_ERR_STATE, "amr_set_patches has not been called");
  return read_bad(h);
}

amr_status amr_set_timing(amr_handle* h, int on) {
  if (!h) return AMR_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  h->timing = on != 0;
  h->ev_used = 0;
  for (int c = 0; c < AMR_T_NCLASS; ++c) {
    h->ev_pairs[c].clear();
    h->t_ms[c] = 0.0;
    h->t_cnt[c] = 0;
  }
  return AMR_OK;
}

amr_status amr_get_timing(amr_handle* h, double* ms, long long* count, int nclass) {
  if (!h || !ms || !count || nclass < 1) return AMR_ERR_ARG;
  CK(cudaStreamSynchronize(h->stream));
  for (int c = 0; c < AMR_T_NCLASS; ++c) {
    for (auto& pr : h->ev_pairs[c]) {
      float t = 0.f;
      CK(cudaEventElapsedTime(&t, h->ev_pool[pr.first], h->ev_pool[pr.second]));
      h->t_ms[c] += t;
      h->t_cnt[c] += 1;
    }
    h->ev_pairs[c].clear();
  }
  h->ev_used = 0;
  for (int c = 0; c < nclass && c < AMR_T_NCLASS; ++c) {
    ms[c] = h->t_ms[c];
    count[c] = h->t_cnt[c];
    h->t_ms[c] = 0.0;
    h->t_cnt[c] = 0;
  }
  return AMR_OK;
}

long long amr_kernel_launches(const amr_handle* h) { return h ? h->launches : 0; }

long long amr_cell_updates(const amr_handle* h) { return h ? h->cell_updates : 0; }

const char* amr_last_error(const amr_handle* h) { return h ? h->err.c_str() : "null handle"; }

void amr_destroy(amr_handle* h) {
  if (!h) return;
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->stream) cudaStreamSynchronize(h->stream);
  release_async(h);
  free_device(h);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : h->side_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : h->u1_ev)
    if (e) cudaEventDestroy(e);
  if (h->side) cudaStreamDestroy(h->side);
  dfree(h, h->params);
  if (h->stream) cudaStreamSynchronize(h->stream);   // stream-ordered frees done
  if (h->pool) cudaMemPoolDestroy(h->pool);
  if (h->stage) cudaFreeHost(h->stage);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h->ops;
  delete h;
}

}  // extern "C"
