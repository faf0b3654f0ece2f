// amr_types.h -- plain structs shared by the host planner (hierarchy.cpp) and
// the sm_103a kernels.  Everything here is POD so tables can be copied to the
// device with one cudaMemcpyAsync each.
#pragma once
#include <cstdint>

#ifndef AMR_HD
#ifdef __CUDACC__
#define AMR_HD __host__ __device__
#else
#define AMR_HD
#endif
#endif

namespace amr {

constexpr int kGhost = 2;      // two ghost cells: the PLM face stencil reaches two cells out (Sec. 4)
constexpr int kMaxVar = 9;
constexpr int kStageThreads = 256;  // threads of one stage-kernel CTA (one per x-y column)
constexpr int kMaxTileX = 32;
constexpr int kPlaneMax = 432;    // max (wx + 4) * (wy + 4) of a stage tile
// 128-thread stage CTAs: wx * wy <= 128 and wx + wy <= 32 give (wx + 4)(wy + 4) <= 272
constexpr int kPlaneMax128 = 272;
AMR_HD constexpr int stage_plane_max(int nt) { return nt == 128 ? kPlaneMax128 : kPlaneMax; }

// Where the stage kernel reads the two ghost layers of one face of a patch: the
// ghost cell at local (i, j, k) of that face holds variable v at element
//   base + i * sx + j * sy + k * sz + v * vs
// of the state arena.  Three kinds, chosen by the planner per face:
//   own ghost cells (filled by the ghost-copy and prolongation kernels before
//     each stage): the patch's own layout;
//   a same-level neighbour (or the patch itself across a periodic boundary)
//     whose interior holds the whole two-layer face: its layout, translated;
//   an outflow boundary: the patch's own boundary cells (stride 0 along the
//     face normal: zero-gradient extension).
struct FaceSrc {
  int64_t base;
  int sx, sy, sz;
  int vs;
};

// Device view of one patch.  Arrays U, U1 and Uold share the same layout and
// offsets: var v, ghosted local cell (i, j, k) with -2 <= i < n0 + 2 sits at
//   off + v * vstride + ((k + 2) * m1 + (j + 2)) * pitch + (i + 2)
struct PatchDesc {
  int64_t off;       // element offset of the patch in the state arena
  int64_t vstride;   // elements between variables
  int n[3];          // interior cells
  int pitch;         // elements per x row (>= n0 + 4)
  int m1;            // rows per z plane (n1 + 4)
  int level;
  int lo[3];         // level index of interior cell (0,0,0)
  int tile_off;      // parent-tile offset (elements) for level >= 1, else -1
  int tn[3];         // parent tile extent (n/2 + 4), level >= 1
  FaceSrc face[6];   // ghost source of the faces x-lo, x-hi, y-lo, y-hi, z-lo, z-hi
};

AMR_HD inline int64_t cell_index(const PatchDesc& p, int i, int j, int k) {
  return ((int64_t)(k + kGhost) * p.m1 + (j + kGhost)) * p.pitch + (i + kGhost);
}

// One CTA of the fused stage kernel: a wx * wy column block marching through
// wz planes.  span < 0: a block of patch `patch` starting at its local cell
// (x0, y0, z0).  span >= 0: a block of one z-layer of a level (patches with
// the same z range that tile a rectangle), described by spans[span]; its
// columns may lie in different patches of the layer.
struct StageItem {
  int patch;
  int16_t x0, y0, z0, wx, wy, wz;
  int span;
};

// A stage work item spanning patches: the level index of its first cell
// (ox, oy, oz) and the patches of its z-layer that meet the block grown by the
// two halo cells in x and y (each column, and each halo cell inside the layer,
// lies in one of them).
constexpr int kSpanMax = 24;
struct ItemSpan {
  int ox, oy, oz;
  int n;
  int patch[kSpanMax];
};

// Box copy used by ghost fill and parent-tile gather.  dst cell (a, b, c) of
// the box maps to src local coordinate per axis: mode 0 -> a + sh, mode 1 -> sh.
struct CopySeg {
  int dst_patch;     // patch (ghost fill) or fine patch owning the tile (gather)
  int src_patch;
  int16_t dlo[3];    // dst box start in dst-local coordinates (ghosted / tile)
  int16_t dn[3];     // dst box extent
  int16_t sh[3];     // src mapping parameter per axis
  uint8_t mode[3];   // 0 translate, 1 constant
  uint8_t pad;
};

// Batched box launches (ghost copies, parent-tile gathers, prolongation) run
// over flattened boxes with precomputed strides: a CTA of kBoxThreads takes a
// chunk of consecutive cells of the launch (several cells per thread), which
// may span several boxes, so that small boxes do not leave CTAs idle.
constexpr int kBoxThreads = 256;
constexpr int kCopyPerThread = 4;
constexpr int kCopyChunk = kBoxThreads * kCopyPerThread;
constexpr int kProlongPerThread = 1;   // parent cells (eight fine cells each)
constexpr int kProlongChunk = kBoxThreads * kProlongPerThread;
constexpr int kRestrictPerThread = 2;
constexpr int kRestrictChunk = kBoxThreads * kRestrictPerThread;

// Copy box: cell (a, b, c) of the box goes from src0 + a ssx + b ssy + c ssz
// (variable stride svs; ssx/ssy/ssz = 0 on an axis held constant) to
// dst0 + a + b dsy + c dsz (variable stride dvs).  A restriction box uses the
// same record: coarse cell (a, b, c) at dst0 + a + b dsy + c dsz averages the
// fine cells src0 + (2a + i) + (2b + j) ssy + (2c + k) ssz, i, j, k in {0, 1}.
struct alignas(16) FlatCopy {
  int64_t dst0, src0;
  int dvs, svs;
  int dsy, dsz;
  int ssx, ssy, ssz;
  int n0, n1;
  int pad;
};

// Prolongation box, walked by parent cell: parent (pa, pb, pc) of the box is
// the tile cell tp0 + pa + pb tsy + pc tsz (variable stride tvol) and has the
// children a = 2 pa + i - odd_x, b = 2 pb + j - odd_y, c = 2 pc + k - odd_z
// (i, j, k in {0, 1}) in the fine box [0, n) at dst0 + a + b dsy + c dsz
// (variable stride dvs); children outside the box are skipped.  odd_d is the
// parity of the box's first fine cell along d, np0 x np1 the parents per plane.
struct alignas(16) FlatProlong {
  int64_t dst0, tp0;
  int dvs, dsy, dsz;
  int tvol, tsy, tsz;
  int n[3];
  int np0, np1;
  int odd;   // bit d: odd_d
};

// Box of fine ghost cells filled by prolongation from the parent tile.
struct ProlongBox {
  int patch;
  int16_t lo[3];     // fine local coordinates (may be negative: ghost region)
  int16_t n[3];
};

// Restriction of a fine patch into (part of) one coarse patch.
struct RestrictSeg {
  int fine, coarse;
  int16_t clo[3];    // coarse-local box start
  int16_t cn[3];     // box extent
};

// Coarse-fine faces of one fine-patch face against one coarse patch: a
// rectangle of uncovered coarse cells C with a fixed coordinate along the face
// normal d and na x nb cells along t1 = (d+1)%3, t2 = (d+2)%3.  Its flux
// registers are na * nb consecutive entries, the in-plane x axis fastest (b,
// along t2 = x, for d = 1; a, along t1, otherwise); the face of entry (a, b)
// sits between C = clo + a e_t1 + b e_t2 and the covered cell on C's side
// cside, and its four fine sub-faces start at flo + 2a e_t1 + 2b e_t2.
struct RegRect {
  int fpatch, cpatch;
  int16_t clo[3];    // coarse local index of the first cell C
  int16_t flo[3];    // fine local face index of the first (0,0) sub-face (face i sits at the low side of cell i)
  int16_t na, nb;
  int8_t d, side;    // axis, side of the fine patch (0 lo, 1 hi)
  int8_t cside;      // +1: the face is C's high face, -1: C's low face
  int8_t ordered;    // 1: some cell C also has a register of another rectangle (reflux in (d, side) order)
};

// Regrid block tagging on the device: levels [l0, L) of a hierarchy with at
// most kTagLevels levels, each with a dense bitmap of its block grid (bit i =
// block (x, y, z), i = (z nb1 + y) nb0 + x) starting at 32-bit word off[l] of
// one buffer (off[l] even, so the host reads 64-bit words).
constexpr int kTagLevels = 13;
struct TagArgs {
  int l0, L;
  int block, buffer;
  int per[3];                 // periodic axes
  int N[kTagLevels][3];       // cells per axis of each level
  int nb[kTagLevels][3];      // blocks per axis of each level
  long long off[kTagLevels];  // first word of each level's bitmap
};

// Box of a coarse patch covered by a finer level (excluded from totals).
struct CoverBox {
  int16_t lo[3], n[3];
};

// Step parameters read by the kernels from device memory, so a captured step
// graph stays valid for any dt.
struct StepParams {
  double dt0;          // coarse-level dt
  double ch;           // GLM cleaning speed in use
  unsigned long long rate_bits;   // max CFL rate (double bits, atomicMax)
  unsigned long long speed_bits;  // max signal speed (double bits, atomicMax)
  unsigned int bad;    // non-physical state detected
  unsigned int pad;
  // maxima of the state written by the last stage 2 (single-level grids): the
  // next step's CFL rate and signal speed without another pass over the state
  unsigned long long next_rate_bits;
  unsigned long long next_speed_bits;
  unsigned long long floor_hits;   // interior primitive recoveries raised by the pressure floor
  // persistent stage launches: next work item to hand out and CTAs finished
  // (zero between launches: the last CTA of a launch resets them)
  unsigned int work_next;
  unsigned int work_done;
};

}  // namespace amr
