// hierarchy.h -- host-side planning of one patch hierarchy: validation and
// every launch table the kernels consume (stage work items, ghost copies,
// prolongation boxes, parent-tile gathers, restriction, flux registers,
// coverage).  Pure C++, no CUDA calls: usable on a host without a GPU.
#pragma once
#include <cstdint>
#include <functional>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "../../include/amr.h"
#include "amr_types.h"

namespace amr {

struct HPatch {
  int level;
  int lo[3];
  int n[3];
};

// Flattened boxes of one batched launch: prefix sums of their cell counts and,
// per chunk of `chunk` cells, the box holding the chunk's first cell.
template <class B>
struct FlatList {
  std::vector<B> boxes;
  std::vector<int> first;      // size boxes + 1
  std::vector<int> chunk_box;  // size ceil(total / chunk)
  int total = 0;
};

// std::allocator that default-initialises (no zero fill of trivial types), for
// large tables that are written in parallel right after allocation.
template <typename T>
struct NoInitAlloc : std::allocator<T> {
  template <typename U>
  struct rebind { using other = NoInitAlloc<U>; };
  NoInitAlloc() = default;
  template <typename U>
  NoInitAlloc(const NoInitAlloc<U>&) noexcept {}
  template <typename U, typename... A>
  void construct(U* p, A&&... a) {
    if constexpr (sizeof...(A) == 0) ::new (static_cast<void*>(p)) U;
    else ::new (static_cast<void*>(p)) U(std::forward<A>(a)...);
  }
};

struct LevelPlan {
  int first = 0, count = 0;                  // patch range [first, first + count)
  std::vector<StageItem> items;              // stage work items, grouped by patch (plain launches)
  std::vector<int> item_first;               // per patch of the level: first item (size count + 1)
  std::vector<StageItem> bitems;             // items of the batched launch (blocks may span the patches
                                             //   of a z-layer that tiles a rectangle)
  std::vector<CopySeg> ghost;                // sibling copies + outflow boundary, grouped by dst patch
  std::vector<int> ghost_first;              // per patch (size count + 1)
  std::vector<CopySeg> ghost_stage;          // the ghost segments of the faces a stage does not read
  std::vector<int> ghost_stage_first;        //   directly (desc.face), per patch (size count + 1)
  std::vector<ProlongBox> prolong;           // fine ghosts from the parent tile (level >= 1)
  std::vector<int> prolong_first;
  std::vector<CopySeg> gather_ghost;         // parent-cell gathers (level >= 1): the tile cells the per-stage
                                             //   prolongation reads, grouped by fine patch
  std::vector<RestrictSeg> restrict_segs;    // this level -> parent (level >= 1)
  // coarse-fine faces of this level (level >= 1) as rectangles, in (d, side, fine patch) order;
  // flattened: register e belongs to the rectangle b with first[b] <= e < first[b + 1]
  FlatList<RegRect> regs;
  int reg_pass[7] = {0, 0, 0, 0, 0, 0, 0};   // registers of the fine faces (d, side) = p / 2, p % 2: [pass[p], pass[p+1])
  int reg_ordered[6] = {0, 0, 0, 0, 0, 0};   // pass p holds rectangles whose cells have several registers
  FlatList<FlatCopy> fghost, fgather;        // the ghost and gather boxes, flattened (batched launches)
  FlatList<FlatCopy> fghost_all;             // every face's ghost segments, flattened (refills of all faces)
  FlatList<FlatProlong> fprolong;            // the prolongation boxes, flattened
  FlatList<FlatCopy> frestrict;              // the restriction boxes (this level -> parent), flattened
  int64_t cells = 0;
};

struct Plan {
  amr_config cfg{};
  int nvar = 5;
  std::vector<HPatch> patches;
  std::vector<PatchDesc> desc;
  std::vector<LevelPlan> levels;
  std::vector<ItemSpan> spans;               // the spanning batched items of all levels
  std::vector<CoverBox> cover;               // covered boxes, grouped by patch
  std::vector<int> cover_first;              // size npatch + 1
  int64_t arena_elems = 0;                   // elements of one state array (U, U1, Uold)
  int64_t tile_elems = 0;                    // elements of the parent-tile buffer
  int64_t packed_elems = 0;                  // doubles of the packed interior state
  std::vector<int64_t> packed_off;           // per patch offset (doubles) in the packed state
};

// Validation only (no allocation of plan tables).  Returns AMR_OK or an error
// status with a message.
amr_status validate_config(const amr_config& cfg, std::string& msg);
amr_status validate_patches(const amr_config& cfg, const std::vector<HPatch>& P, std::string& msg);

// Shape of the stage kernel's work items: x width cap, columns per CTA (<= 256)
// and z chunk length.  Zero fields take the defaults (32, 256, 32).
struct TileParams {
  int max_wx = 0;
  int max_cols = 0;
  int zchunk = 0;
  int persistent = 0;   // batched stages: persistent CTAs taking items from a device counter
  int span = 1;         // batched stages: blocks over the z-layers of a level that tile a rectangle
};

// Regridding: cluster cells flagged on levels min_level .. max_level-1 into the
// patches of levels min_level+1 .. max_level (levels <= min_level are kept).
struct RegridParams {
  double threshold = 0.3;  // flag where max_d |rho_{i+1} - rho_{i-1}| / (2 rho_i) > threshold
  int buffer = 2;          // flagged cells are grown by `buffer` cells of their level
  int block = 4;           // clustering block edge in cells of the flagged level (even)
  int max_patch = 32;      // largest edge of a new patch in its own cells (multiple of 2*block)
  int min_level = 0;
};

amr_status check_regrid_params(const amr_config& cfg, const RegridParams& rp, std::string& msg);

// flags[i]: one byte per interior cell of old patch i ([z][y][x]); empty for
// patches whose level is not flagged.
amr_status cluster_patches(const amr_config& cfg, const std::vector<HPatch>& old,
                           const std::vector<std::vector<uint8_t>>& flags, const RegridParams& rp,
                           std::vector<HPatch>& out, std::string& msg);

// Block grid of a flagged level (blocks of rp.block cells per axis): fills nb,
// returns the block count.  A level whose count is at most kTagDenseMax can be
// tagged as a bitmap.
constexpr int64_t kTagDenseMax = (int64_t)1 << 28;
int64_t regrid_tag_blocks(const amr_config& cfg, const RegridParams& rp, int level, int nb[3]);

// Blocks of level min_level fully inside one of its patches (a partial block at
// the domain's end counts when the patch reaches the end): the cover of the
// clustering's first level, as a dense bitmap laid out as the block tags.
std::vector<uint64_t> regrid_base_cover(const amr_config& cfg, const std::vector<HPatch>& old,
                                        const RegridParams& rp);

// The clustering's last step (the greedy box merge) from the refinable blocks of
// levels min_level .. max_level-1 made elsewhere (the GPU), dense bitmaps laid
// out as the block tags: a block is refinable when it is tagged (after the
// parent rings of finer tags) and all 26 neighbours inside the domain are
// covered (level min_level: regrid_base_cover; finer levels: the parent block is
// refinable).  Gives the same patches as cluster_patches.  refinable is consumed.
amr_status cluster_patches_refinable(const amr_config& cfg, const std::vector<HPatch>& old,
                                     std::vector<std::vector<uint64_t>>& refinable, const RegridParams& rp,
                                     std::vector<HPatch>& out, std::string& msg);

// Tables that fill a new hierarchy from an old one: per new level l > keep_level,
// same-level box copies (dst = new patch, src = old patch, local coordinates)
// and the interior boxes of new patches that no old patch covers (prolonged
// from the new parent level).
struct RegridFill {
  std::vector<std::vector<CopySeg>> copy;       // per level
  std::vector<std::vector<ProlongBox>> fresh;   // per level
};
// Gathers into the parent tiles of the fresh (prolonged) boxes of a regrid fill,
// per level; msg is set if a parent cell is missing.
void build_fill_gathers(const amr_config& cfg, const Plan& plan, const std::vector<std::vector<ProlongBox>>& fresh,
                        std::vector<std::vector<CopySeg>>& out, std::string& msg);

void build_regrid_fill(const std::vector<HPatch>& oldp, const std::vector<HPatch>& newp, int keep_level,
                       RegridFill& fill);

// Flattened box lists of every level (FlatList) from its ghost, gather and
// prolongation boxes; build_plan calls it.
void build_flat(Plan& plan);

// Rebuild only the stage work items of `plan` with another tile shape.
void build_items(Plan& plan, const TileParams& tp);

// Validate and build every table.  `align` = element alignment of patch
// offsets (e.g. 64 for 256-byte alignment of FP32 arrays).
amr_status build_plan(const amr_config& cfg, const std::vector<HPatch>& P, Plan& plan,
                      std::string& msg, const TileParams& tp = TileParams());

// Owner rank of every patch for a run over nranks GPUs: each level's patches in
// Morton order of their centres (on the finest level's cells), cut into
// contiguous ranges of nearly equal cell counts.  nranks <= 1: all 0.
std::vector<int> morton_partition(const amr_config& cfg, const std::vector<HPatch>& P, int nranks);

// f(0) .. f(n-1) on the host cores (the planner's thread pool policy).
void parallel_run(int n, const std::function<void(int)>& f);

}  // namespace amr
