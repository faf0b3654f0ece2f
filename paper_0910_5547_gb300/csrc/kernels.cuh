// kernels.cuh -- the sm_103a kernels of one coarse step, templated on the bulk
// precision T (float / double) and the variable count NV (5 Euler, 9 GLM-MHD).
//
//   stage_kernel     fused RK2 stage: primitive recovery, PLM on every face,
//                    HLL/LLF flux, flux difference L(U) and the stage update
//                    U1 = U + dt L(U) (stage 1) or U = U/2 + (U1 + dt L(U1))/2
//                    (stage 2, Sec. 5.1), one CTA per x-y column block
//                    marching through z: two barrier-separated phases per
//                    plane (plane j skewed against j-1), x/y states and fluxes
//                    through shared memory, z faces in registers, FP32 Euler
//                    inputs staged by cp.async rings.
//   box_copy_kernel  batched ghost fill (siblings, periodic images, outflow)
//                    and parent-tile gathers with linear time interpolation,
//                    over flattened boxes in fixed chunks of cells per CTA;
//                    copy_kernel is the one-CTA-per-box form (plain launches).
//   box_prolong_kernel / prolong_kernel
//                    conservative minmod prolongation into fine ghost cells.
//   reg_*_kernel     FP64 flux registers at coarse-fine faces.
//   reflux_kernel    register correction of uncovered coarse cells.
//   box_restrict_kernel / restrict_kernel
//                    mean of the 8 children (pairwise sums).
//   flag_kernel, tag_kernel, xcopy_kernel
//                    regrid: density-gradient flags; copies from the old
//                    hierarchy into the new one.
//   speed_kernel     CFL rate / max signal speed reduction (warp shuffles).
//   fluxrec_stage_kernel  the RK2 stage with direct flux reconstruction (Euler).
//   totals_kernel    FP64 conserved totals over leaf cells (fixed order).
//   divb_kernel      GLM-MHD: FP64 norms of the centred div B over leaf cells.
//   pack kernels     FP64 host layout <-> ghosted device arena.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "amr_types.h"
#include "physics.cuh"

namespace amr {

// Shared memory of a stage CTA of NT threads, per variable: the primitive
// plane with its face halo, (wy + 4) x (wx + 4) <= plane cells; four face-state
// arrays (left/right states of x faces, (wx + 2) wy <= state, and of y faces,
// (wy + 2) wx <= state); and the x face fluxes, wy (wx + 1) <= facex, and y
// face fluxes, (wy + 1) wx <= facey.  The planner keeps wx * wy <= NT, wx <= 32,
// 4 (wx + wy) <= NT and (wx + 4)(wy + 4) <= plane; for NT = 256 that bounds
// wy <= 63, for NT = 128 wx, wy <= 31.  Fixed strides keep every shared-memory
// address an immediate offset.
template <int NT>
struct StageDims {
  static constexpr int plane = NT == 128 ? kPlaneMax128 : kPlaneMax;
  static constexpr int state = NT == 128 ? NT + 64 : NT + 128;
  static constexpr int facex = NT + 64;
  static constexpr int facey = NT + 32;
  static constexpr int face = facex + facey;
};

// FP32 Euler stage kernels also stage their conserved inputs through shared
// memory, filled by cp.async: a ring of four planes of the stage input (own
// columns and halo cells) and, in stage 2, a ring of two planes of U^n (own
// columns).  The other variants load them into registers (their shared memory
// has no room for the rings at the occupancy they run at).
constexpr int kRing = 4;
constexpr int kRingN = 2;

template <typename T, int NV, int NT = kStageThreads>
__host__ __device__ constexpr size_t stage_smem_base() {
  using D = StageDims<NT>;
  return sizeof(T) * NV * (D::plane + 4 * D::state + D::face);
}
template <typename T, int NV, int NT = kStageThreads>
__host__ __device__ constexpr size_t stage_smem_rings() {
  return sizeof(T) * NV * (kRing * StageDims<NT>::plane + kRingN * NT);
}
// The rings are used where the CTAs per SM a variant asks for (MINB) still fit
// in the SM's 228 KB of shared memory (1 KB reserved per CTA).
template <typename T, int NV, int MINB, int NT = kStageThreads>
__host__ __device__ constexpr bool stage_async() {
  return NV == 5 && sizeof(T) == 4 &&
         (size_t)MINB * (stage_smem_base<T, NV, NT>() + stage_smem_rings<T, NV, NT>() + 1024) <=
             (size_t)228 * 1024;
}
template <typename T, int NV, int MINB = 2, int NT = kStageThreads>
constexpr size_t stage_smem_bytes() {
  return stage_smem_base<T, NV, NT>() + (stage_async<T, NV, MINB, NT>() ? stage_smem_rings<T, NV, NT>() : 0);
}

// Asynchronous global -> shared copy of one element (sm_80+ cp.async).
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* sdst, const T* gsrc) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(sdst);
  if (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Shared-memory arrays of the stage kernel hold NV variables of S cells.
// GLM-MHD groups them by G = 16 / sizeof(T) variables: variable v < NG*G of
// cell c at (v / G) * S * G + c * G + v % G, the remaining NV % G variables one
// array of S cells each after the groups.  A cell's nine variables then load
// and store as 16-byte vectors (2 vectors + 1 scalar in FP32), and a
// quarter-warp of consecutive cells covers all 32 banks even when a warp spans
// two tile rows.  Euler keeps one array per variable (G = 1; measured no
// faster grouped).
template <typename T, int NV>
__host__ __device__ constexpr int sgroup() {
  return NV == 9 ? 16 / (int)sizeof(T) : 1;
}
template <typename T, int NV, int S>
__host__ __device__ constexpr int sidx(int v, int c) {
  constexpr int G = sgroup<T, NV>(), NG = NV / G;
  return v < NG * G ? (v / G) * S * G + c * G + v % G : NG * G * S + (v - NG * G) * S + c;
}
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

template <typename T, int NV, int S>
__device__ __forceinline__ void sload(const T* base, int c, T* out) {
  constexpr int G = sgroup<T, NV>(), NG = NV / G;
  if constexpr (G == 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) out[v] = base[v * S + c];
  } else {
    using V = typename Vec16<T>::type;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      const V x = *reinterpret_cast<const V*>(base + g * S * G + c * G);
      if constexpr (G == 4) {
        out[4 * g] = x.x; out[4 * g + 1] = x.y; out[4 * g + 2] = x.z; out[4 * g + 3] = x.w;
      } else {
        out[2 * g] = x.x; out[2 * g + 1] = x.y;
      }
    }
#pragma unroll
    for (int v = NG * G; v < NV; ++v) out[v] = base[NG * G * S + (v - NG * G) * S + c];
  }
}

template <typename T, int NV, int S>
__device__ __forceinline__ void sstore(T* base, int c, const T* in) {
  constexpr int G = sgroup<T, NV>(), NG = NV / G;
  if constexpr (G == 1) {
#pragma unroll
    for (int v = 0; v < NV; ++v) base[v * S + c] = in[v];
  } else {
    using V = typename Vec16<T>::type;
#pragma unroll
    for (int g = 0; g < NG; ++g) {
      V x;
      if constexpr (G == 4) {
        x.x = in[4 * g]; x.y = in[4 * g + 1]; x.z = in[4 * g + 2]; x.w = in[4 * g + 3];
      } else {
        x.x = in[2 * g]; x.y = in[2 * g + 1];
      }
      *reinterpret_cast<V*>(base + g * S * G + c * G) = x;
    }
#pragma unroll
    for (int v = NG * G; v < NV; ++v) base[NG * G * S + (v - NG * G) * S + c] = in[v];
  }
}

struct ChunkDesc {  // a contiguous range of interior cells of one patch
  int patch;
  int begin;
  int count;
};

template <typename T>
struct StageArgs {
  const PatchDesc* desc;
  const StageItem* items;
  int nitems;
  const T* Uin;      // stage input (ghosts filled)
  T* Uout;           // stage output (U1 for stage 1, U in place for stage 2)
  StepParams* params;
  double dt_scale;   // 2^-level
  T idx, idy, idz;   // 1 / dx of the level
  double idx0, idy0, idz0;  // 1 / dx of level 0 (CFL rate)
  int fuse_rate;     // stage 2: accumulate the CFL rate of the new state
  int dynamic;       // persistent CTAs take items from params->work_next (stage_kernel)
  const ItemSpan* spans;   // the spanning blocks' patch lists (items with span >= 0)
  T* Uold;           // stage 1: also store the stage input (U^n) of every updated cell here, or nullptr
  Phys<T> ph;
};

template <typename T, int NV>
__device__ __forceinline__ void load_cons(const T* base, int vstride, int c, T* u) {
#pragma unroll
  for (int v = 0; v < NV; ++v) u[v] = base[v * vstride + c];
}

template <typename T, int NV>
__device__ __forceinline__ void load_cons(const T* base, int64_t vstride, int64_t c, T* u) {
#pragma unroll
  for (int v = 0; v < NV; ++v) u[v] = base[v * vstride + c];
}

template <typename T, int NV>
__device__ __forceinline__ Phys<T> phys_with_ch(Phys<T> ph, const StepParams* prm) {
  if (NV == 9) {
    T ch = (T)prm->ch;
    ph.ch = ch;
    ph.ch2 = ch * ch;
    ph.half_inv_ch = T(0.5) / ch;
  }
  return ph;
}

// CFL rate sum_d (|v_d| + c_d) / dx0_d and max signal speed of a conserved state.
template <typename T, int NV>
__device__ __forceinline__ void cell_rate(const T* u, const Phys<T>& ph, T idx0, T idy0, T idz0, T& rate,
                                          T& speed) {
  T w[NV];
  cons_to_prim<T, NV>(u, w, ph.efl);
  T c0, c1, c2;
  if (NV == 5) {
    c0 = c1 = c2 = dsqrt(ph.ggm1 * w[4]);
  } else {
    const T r = drcp(w[0]);
    const T a2 = ph.ggm1 * w[4];
    const T b2 = (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]) * r;
    const T s = a2 + b2;
    const T s2 = s * s;
    const T f = T(4) * a2 * r;
    c0 = dsqrt(T(0.5) * (s + dsqrt(dmax(s2 - f * w[5] * w[5], T(0)))));
    c1 = dsqrt(T(0.5) * (s + dsqrt(dmax(s2 - f * w[6] * w[6], T(0)))));
    c2 = dsqrt(T(0.5) * (s + dsqrt(dmax(s2 - f * w[7] * w[7], T(0)))));
  }
  const T s0 = dabs(w[1]) + c0, s1 = dabs(w[2]) + c1, s2 = dabs(w[3]) + c2;
  rate = s0 * idx0 + s1 * idy0 + s2 * idz0;
  speed = dmax(s0, dmax(s1, s2));
}

__device__ __forceinline__ void atomic_max_pos_double(unsigned long long* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Fused RK2 stage over work items (patch, wx x wy column block, z range).
// Each thread owns one column and marches in z: primitives of two planes, one
// z slope and the last z-face flux live in registers and the next plane's
// global loads are issued one iteration ahead.  Shared memory holds, per plane,
// the primitives with a two-cell face halo, every cell's x and y face states
// w +- s (each limited slope computed once) and every x and y face flux
// (each solved once); the update differences the fluxes of the cell's six
// faces.  The work of plane j is skewed against that of plane j-1 so that
// one plane costs two barriers.
template <typename T, int NV, int STAGE, int MINB = (sizeof(T) == 4 && NV == 5) ? 2 : 1, int NT = kStageThreads,
          bool WENO = false, bool SPAN = false>
__global__ void __launch_bounds__(NT, MINB) stage_kernel(StageArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int kPlane = StageDims<NT>::plane, kState = StageDims<NT>::state;
  constexpr int kFaceX = StageDims<NT>::facex, kFaceY = StageDims<NT>::facey;
  T* W = reinterpret_cast<T*>(smem_raw);
  T* XL = W + NV * kPlane;
  T* XR = XL + NV * kState;
  T* YL = XR + NV * kState;
  T* YR = YL + NV * kState;
  T* FX = YR + NV * kState;
  constexpr bool kAsync = stage_async<T, NV, MINB, NT>();
  // 128-thread builds at 3+ CTAs per SM (FP32 MHD, 168 registers) read the stage
  // input and U^n of the updated cell in phase B, and the halo cell when it is
  // converted, instead of carrying register prefetches through phase A (8-16 B
  // of spills left); the latency is covered by 12 warps per SM
  constexpr bool kLean = !kAsync && NT == 128 && MINB >= 3;
  // ring of stage-input planes: plane p of the item lives in slot p & 3, [slot][var][plane cell];
  // ring of U^n planes (stage 2): plane p in slot p & 1, [slot][var][thread].  Each thread
  // reads back only the cells it copied itself (own column, own halo cell).
  T* CR = FX + NV * StageDims<NT>::face;
  T* CN = CR + kRing * NV * kPlane;

  const Phys<T> ph = phys_with_ch<T, NV>(a.ph, a.params);
  const T dt = (T)(a.params->dt0 * a.dt_scale);
  const T dtx = dt * a.idx, dty = dt * a.idy, dtz = dt * a.idz;
  const T sc = slope_scale<T>();   // face state = w +- sc * limited_slope
  const int t = threadIdx.x;
  bool bad = false;
  int floor_hits = 0;
  T rate_max = T(0), speed_max = T(0);
  // GLM damping after the stage-2 average: psi *= exp(-alpha c_h dt_l / min_d dx_l);
  // dt_l / dx_l is the same on every level (dt0 / dx0)
  T damp = T(1);
  if (NV == 9 && STAGE == 2 && a.ph.glm_alpha > T(0)) {
    const double idmax = fmax(a.idx0, fmax(a.idy0, a.idz0));
    damp = (T)exp(-(double)a.ph.glm_alpha * a.params->ch * a.params->dt0 * idmax);
  }

  // work items: one per CTA, or (a.dynamic) persistent CTAs that take the next
  // item from a device counter until none is left
  __shared__ int s_next;
  int itn = blockIdx.x;
  if (a.dynamic) {
    if (t == 0) s_next = (int)atomicAdd(&a.params->work_next, 1u);
    __syncthreads();
    itn = s_next;
  }
  for (; itn < a.nitems;) {
    const StageItem it = a.items[itn];
    const int wx = it.wx, wy = it.wy, wz = it.wz;
    const int sw = wx + 4;
    const int ncol = wx * wy;
    T* FY = FX + NV * kFaceX;
    const bool active = t < ncol;
    const int tx = active ? t % wx : 0, ty = active ? t / wx : 0;
    // the patch among the block's patches (its own patch, or the patches of its
    // z-layer for a spanning block) that holds level cell (gx, gy) of the layer; -1: none
    auto find = [&](int gx, int gy) -> int {
      if (!SPAN || it.span < 0) {
        const PatchDesc& Q = a.desc[it.patch];
        return (gx >= Q.lo[0] && gx < Q.lo[0] + Q.n[0] && gy >= Q.lo[1] && gy < Q.lo[1] + Q.n[1]) ? it.patch : -1;
      }
      const ItemSpan& S = a.spans[it.span];
      for (int k = 0; k < S.n; ++k) {
        const int q = S.patch[k];
        const PatchDesc& Q = a.desc[q];
        if (gx >= Q.lo[0] && gx < Q.lo[0] + Q.n[0] && gy >= Q.lo[1] && gy < Q.lo[1] + Q.n[1]) return q;
      }
      return -1;
    };
    // level index of the block's first cell
    int ox, oy, oz;
    if (SPAN && it.span >= 0) {
      const ItemSpan& S = a.spans[it.span];
      ox = S.ox; oy = S.oy; oz = S.oz;
    } else {
      const PatchDesc& Q = a.desc[it.patch];
      ox = Q.lo[0] + it.x0; oy = Q.lo[1] + it.y0; oz = Q.lo[2] + it.z0;
    }
    // this thread's column: its patch qc and local cell (lx, ly, lz0) at the block's first plane
    // (SPAN = false: a launch whose blocks all lie in one patch each)
    int qc = it.patch;
    if constexpr (SPAN) {
      if (it.span >= 0) qc = find(ox + tx, oy + ty);
      if (qc < 0) {   // not reached: the planner puts every column of a block in one of its patches
        qc = it.patch;
        bad = true;
      }
    }
    const PatchDesc P = a.desc[qc];
    const int lx = ox + tx - P.lo[0], ly = oy + ty - P.lo[1], lz0 = oz - P.lo[2];
    const T* Ub = a.Uin + P.off;
    T* Ob = a.Uout + P.off;
    T* Oo = a.Uold == nullptr ? nullptr : a.Uold + P.off;   // stage 1's copy of U^n, if asked
    const int vs = (int)P.vstride;
    const int plane = P.pitch * P.m1;
    const int col = ((lz0 + kGhost) * P.m1 + (ly + kGhost)) * P.pitch + (lx + kGhost);
    const int me = (ty + 2) * sw + (tx + 2);
    const int xs = ty * (wx + 2) + (tx + 1);     // x-state slot of the own cell
    const int ys = (ty + 1) * wx + tx;           // y-state slot of the own cell
    // this thread's halo cell (one per thread, 4 (wx + wy) <= blockDim)
    const int nhalo = 4 * (wx + wy);
    const bool has_halo = t < nhalo;
    // this thread's halo cell at the block's first plane, planes hpl and variables
    // hvs elements apart: an interior cell of one of the block's patches, or a
    // ghost cell of an x/y face read where the face's source lies (own ghost
    // cells, a neighbour's interior, outflow boundary cells)
    const T* hsrc = Ub;
    int hpl = plane, hvs = vs, hpos = 0;
    if (has_halo) {
      int hx, hy;
      if (t < 4 * wy) {
        const int r = t >> 2, c = t & 3;
        hy = r;
        hx = c < 2 ? c - 2 : wx + (c - 2);
      } else {
        const int h2 = t - 4 * wy;
        const int r = h2 / wx, c = h2 - r * wx;
        hx = c;
        hy = r < 2 ? r - 2 : wy + (r - 2);
      }
      const int hgx = ox + hx, hgy = oy + hy;
      const int qh = find(hgx, hgy);
      if (qh >= 0) {
        const PatchDesc& Q = a.desc[qh];
        hsrc = a.Uin + Q.off + ((oz - Q.lo[2] + kGhost) * Q.m1 + (hgy - Q.lo[1] + kGhost)) * Q.pitch +
               (hgx - Q.lo[0] + kGhost);
        hpl = Q.pitch * Q.m1;
        hvs = (int)Q.vstride;
      } else {   // beyond the block's patches: a ghost cell of the face of the patch next to it
        const bool xh = hx < 0 || hx >= wx;
        int qi = find(xh ? (hx < 0 ? ox : ox + wx - 1) : hgx, xh ? hgy : (hy < 0 ? oy : oy + wy - 1));
        if (qi < 0) {   // not reached (the block's own cells lie in its patches)
          qi = qc;
          bad = true;
        }
        const PatchDesc& Q = a.desc[qi];
        const FaceSrc fs = Q.face[xh ? (hx < 0 ? 0 : 1) : (hy < 0 ? 2 : 3)];
        hsrc = a.Uin + (fs.base + (int64_t)(hgx - Q.lo[0]) * fs.sx + (int64_t)(hgy - Q.lo[1]) * fs.sy +
                        (int64_t)(oz - Q.lo[2]) * fs.sz);
        hpl = fs.sz;
        hvs = fs.vs;
      }
      hpos = (hy + 2) * sw + (hx + 2);
    }
    // this thread's boundary slope (the halo cell next to the block edge), if any
    const int eb = (int)blockDim.x - 1 - t;
    int bkind = -1, bpos = 0, bslot = 0, bstep = 0;
    if (eb < 2 * (wx + wy)) {
      if (eb < wy) { bkind = 0; bpos = (eb + 2) * sw + 1; bslot = eb * (wx + 2); bstep = 1; }            // XL, x = -1
      else if (eb < 2 * wy) {
        const int r = eb - wy;
        bkind = 1; bpos = (r + 2) * sw + wx + 2; bslot = r * (wx + 2) + wx + 1; bstep = 1;                // XR, x = wx
      } else if (eb < 2 * wy + wx) {
        const int c = eb - 2 * wy;
        bkind = 2; bpos = 1 * sw + c + 2; bslot = c; bstep = sw;                                          // YL, y = -1
      } else {
        const int c = eb - 2 * wy - wx;
        bkind = 3; bpos = (wy + 2) * sw + c + 2; bslot = (wy + 1) * wx + c; bstep = sw;                   // YR, y = wy
      }
    }

    // source of this column's plane z0 + p and its variable stride: the patch's own
    // array inside it; below and above it the z faces' sources (warp-uniform branch)
    auto col_src = [&](int p, int& svs) -> const T* {
      const int lz = lz0 + p;
      if (lz >= 0 && lz < P.n[2]) {
        svs = vs;
        return Ub + col + p * plane;
      }
      const FaceSrc fs = a.desc[qc].face[lz < 0 ? 4 : 5];
      svs = fs.vs;
      return a.Uin + (fs.base + (int64_t)lx * fs.sx + (int64_t)ly * fs.sy + (int64_t)lz * fs.sz);
    };

    // z-march registers at the start of iteration j: wA = w(j-1), wB = w(j),
    // sA = slope(j-1), uD = conserved plane j+1 (in flight); Fzm = flux of face
    // j-3/2 (from the previous iteration).
    T uD[NV], wA[NV], wB[NV], sA[NV], Fzm[NV], hN[NV], unN[NV];
    if (active) {  // prologue: planes z0-2 .. z0+1
      T u0[NV], w0[NV];
      int svs;
      const T* s0 = col_src(-2, svs);
      load_cons<T, NV>(s0, svs, 0, u0);
      s0 = col_src(-1, svs);
      load_cons<T, NV>(s0, svs, 0, uD);
      cons_to_prim<T, NV>(u0, w0, ph.efl);
      cons_to_prim<T, NV>(uD, wA, ph.efl);
      load_cons<T, NV>(Ub, vs, col, uD);
      bad |= !cons_to_prim<T, NV>(uD, wB, ph.efl, &floor_hits);   // plane 0: an interior plane
      s0 = col_src(1, svs);
      if (kAsync) {
#pragma unroll
        for (int v = 0; v < NV; ++v)   // plane 1, slot 1
          cp_async_elem(&CR[NV * kPlane + sidx<T, NV, kPlane>(v, me)], s0 + v * svs);
        sstore<T, NV, kPlane>(CR, me, uD);   // plane 0, slot 0
      } else {
        load_cons<T, NV>(s0, svs, 0, uD);
      }
      if (STAGE == 2 && !kAsync && !kLean) load_cons<T, NV>(Ob, vs, col, unN);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if constexpr (WENO) {
          T dm;
          weno3_offsets(w0[v], wA[v], wB[v], sA[v], dm);   // sA: offset of the upper face
        } else {
          sA[v] = limited_slope(w0[v], wA[v], wB[v], ph.theta);
        }
      }
    }
    if (kAsync) {
      if (has_halo) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          cp_async_elem(&CR[sidx<T, NV, kPlane>(v, hpos)], hsrc + v * hvs);
          if (wz > 1) cp_async_elem(&CR[NV * kPlane + sidx<T, NV, kPlane>(v, hpos)], hsrc + v * hvs + hpl);
        }
      }
      cp_async_commit();
    } else if (has_halo) {
      if (!kLean) load_cons<T, NV>(hsrc, hvs, 0, hN);
    }

    // Iteration j runs two phases separated by barriers:
    //   A: z face j-1/2 and the primitives of plane j into shared memory;
    //      x and y face fluxes of plane j-1
    //   B: update of plane j-1; x and y limited slopes of plane j
    // Each shared buffer is written in one phase and read in the other.  For
    // MHD (kMerge) the arithmetic of a phase runs as one straight-line block so
    // that the three Riemann solves of phase A can interleave: at j = 0 the x/y
    // fluxes are solved from stale face states and at j = wz the slopes from a
    // stale plane, and the results are overwritten before anything reads them;
    // only the global stores of the update and the CFL maxima are predicated.
    // Euler skips that work (measured faster).
    constexpr bool kMerge = NV == 9;
    // the own cell's low-side face states (x and y), kept in registers from the
    // slopes of plane j to the fluxes of plane j in the next iteration; only
    // the tile-boundary cells' states go through shared memory
    T xrOwn[NV], yrOwn[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) xrOwn[v] = yrOwn[v] = T(0);
    // FP32 Euler blocks of one patch with 128 registers per thread (512 threads
    // per SM) unroll the march by two planes (measured: three or four planes are
    // slower; the other builds would spill at their register budgets)
    constexpr int kMarchUnroll = (NV == 5 && sizeof(T) == 4 && !SPAN && MINB * NT <= 512) ? 2 : 1;
#pragma unroll kMarchUnroll
    for (int j = 0; j <= wz; ++j) {
      const bool cur = j < wz, prev = j > 0;
      T Fzp[NV], Fx0[NV], Fy0[NV], own[NV], un[NV], uin[NV];
      // ---- phase A ----
      if (kAsync) {  // copies of plane j+2 (ghost planes end at wz+1), then wait for plane j+1
        const int jn = j + 2;
        T* slot = CR + (jn & (kRing - 1)) * NV * kPlane;
        if (active && jn <= wz + 1) {
          int svs;
          const T* src = col_src(jn, svs);
#pragma unroll
          for (int v = 0; v < NV; ++v) cp_async_elem(&slot[sidx<T, NV, kPlane>(v, me)], src + v * svs);
        }
        if (has_halo && jn < wz) {
#pragma unroll
          for (int v = 0; v < NV; ++v)
            cp_async_elem(&slot[sidx<T, NV, kPlane>(v, hpos)], hsrc + v * hvs + jn * hpl);
        }
        if (STAGE == 2 && active && cur) {  // U^n of plane j, used by the update of plane j
          T* sn = CN + (j & (kRingN - 1)) * NV * NT;
#pragma unroll
          for (int v = 0; v < NV; ++v) cp_async_elem(&sn[sidx<T, NV, NT>(v, t)], Ob + v * vs + col + j * plane);
        }
        cp_async_commit();
        cp_async_wait1();
      }
      if (has_halo && cur) {
        T w[NV];
        if (kAsync) {
          sload<T, NV, kPlane>(CR + (j & (kRing - 1)) * NV * kPlane, hpos, hN);
        }
        if (kLean) load_cons<T, NV>(hsrc, hvs, j * hpl, hN);
        cons_to_prim<T, NV>(hN, w, ph.efl);
        if (!kAsync && !kLean) load_cons<T, NV>(hsrc, hvs, (j + 1 < wz ? j + 1 : j) * hpl, hN);
        sstore<T, NV, kPlane>(W, hpos, w);
      }
      if (active) {
        // stage input of the own cell, plane j-1 (read earlier: a cache hit; plane -1 is a ghost plane)
        if (!kAsync && !kLean) load_cons<T, NV>(Ub, vs, col + (j - 1) * plane, uin);
        T wC[NV], sB[NV], wl[NV], wr[NV], xl[NV], xr[NV], yl[NV], yr[NV];
        if (kAsync) {
          sload<T, NV, kPlane>(CR + ((j + 1) & (kRing - 1)) * NV * kPlane, me, uD);
        }
        int hit = 0;
        const bool ok = cons_to_prim<T, NV>(uD, wC, ph.efl, &hit);   // plane j+1
        if (j + 1 < wz) {   // interior planes are checked and counted once each
          bad |= !ok;
          floor_hits += hit;
        }
        if (!kAsync) {
          const int jn = j + 2 <= wz + 1 ? j + 2 : wz + 1;   // ghost planes end at wz+1
          int svs;
          const T* src = col_src(jn, svs);
          load_cons<T, NV>(src, svs, 0, uD);                   // prefetch plane j+2
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if constexpr (WENO) {
            T dm;
            weno3_offsets(wA[v], wB[v], wC[v], sB[v], dm);
            wl[v] = wA[v] + sA[v];
            wr[v] = wB[v] - dm;
          } else {
            sB[v] = limited_slope(wA[v], wB[v], wC[v], ph.theta);
            wl[v] = wA[v] + sc * sA[v];
            wr[v] = wB[v] - sc * sB[v];
          }
          own[v] = wB[v];
        }
        sstore<T, NV, kPlane>(W, me, wB);
        {   // own x/y face states of plane j-1 (read at j = 0 too: in bounds, unused)
          sload<T, NV, kState>(XL, xs - 1, xl);
          sload<T, NV, kState>(YL, ys - wx, yl);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            xr[v] = xrOwn[v];
            yr[v] = yrOwn[v];
          }
        }
        if (STAGE == 2 && !kAsync && !kLean) {
#pragma unroll
          for (int v = 0; v < NV; ++v) un[v] = unN[v];
          load_cons<T, NV>(Ob, vs, col + (cur ? j : j - 1) * plane, unN);
        }
        riemann<T, NV, 2>(wl, wr, ph, Fzp);                  // face j-1/2
        if (kMerge || prev) {
          riemann<T, NV, 0>(xl, xr, ph, Fx0);                // x face of plane j-1
          riemann<T, NV, 1>(yl, yr, ph, Fy0);                // y face of plane j-1
          sstore<T, NV, kFaceX>(FX, ty * (wx + 1) + tx, Fx0);
          sstore<T, NV, kFaceY>(FY, ty * wx + tx, Fy0);
        }
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          sA[v] = sB[v];
          wA[v] = wB[v];
          wB[v] = wC[v];
        }
      }
      if (!(kMerge || prev)) {
        // no x/y fluxes at j = 0
      } else if (eb < wy) {  // x face at the right edge of row eb
        T wl[NV], wr[NV], F[NV];
        const int sl = eb * (wx + 2) + wx;
        sload<T, NV, kState>(XL, sl, wl);
        sload<T, NV, kState>(XR, sl + 1, wr);
        riemann<T, NV, 0>(wl, wr, ph, F);
        sstore<T, NV, kFaceX>(FX, eb * (wx + 1) + wx, F);
      } else if (eb < wy + wx) {  // y face at the top edge of column eb - wy
        const int c = eb - wy;
        T wl[NV], wr[NV], F[NV];
        const int sl = wy * wx + c;
        sload<T, NV, kState>(YL, sl, wl);
        sload<T, NV, kState>(YR, sl + wx, wr);
        riemann<T, NV, 1>(wl, wr, ph, F);
        sstore<T, NV, kFaceY>(FY, wy * wx + c, F);
      }
      __syncthreads();
      // ---- phase B ----
      if (active && (kMerge || prev)) {  // U1 = U + dt L(U)  |  U = U^n / 2 + (U1 + dt L(U1)) / 2, plane j-1
        const int c = col + (j - 1) * plane;
        if (kLean) {
          load_cons<T, NV>(Ub, vs, c, uin);
          if (STAGE == 2) load_cons<T, NV>(Ob, vs, c, un);
        }
        if (kAsync) {
          sload<T, NV, kPlane>(CR + ((j - 1) & (kRing - 1)) * NV * kPlane, me, uin);
          if (STAGE == 2) sload<T, NV, NT>(CN + ((j - 1) & (kRingN - 1)) * NV * NT, t, un);
        }
        T fxp[NV], fyp[NV];
        sload<T, NV, kFaceX>(FX, ty * (wx + 1) + tx + 1, fxp);
        sload<T, NV, kFaceY>(FY, (ty + 1) * wx + tx, fyp);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          // u + dt L(u), L = -sum_d (F_{d,+} - F_{d,-}) / dx_d
          const T u2 = uin[v] - dtx * (fxp[v] - Fx0[v]) - dty * (fyp[v] - Fy0[v]) - dtz * (Fzp[v] - Fzm[v]);
          if (STAGE == 1) {
            if (prev) Ob[v * vs + c] = u2;
            if (Oo != nullptr && prev) Oo[v * vs + c] = uin[v];   // U^n for the finer levels' time interpolation
          } else {
            un[v] = T(0.5) * un[v] + T(0.5) * u2;
            if (NV == 9 && v == 8) un[v] *= damp;
            if (prev) Ob[v * vs + c] = un[v];
          }
        }
        if (STAGE == 2 && a.fuse_rate) {
          T r, sp;
          cell_rate<T, NV>(un, ph, (T)a.idx0, (T)a.idy0, (T)a.idz0, r, sp);
          if (prev) {
            rate_max = dmax(rate_max, r);
            speed_max = dmax(speed_max, sp);
          }
        }
      }
      if (active) {
#pragma unroll
        for (int v = 0; v < NV; ++v) Fzm[v] = Fzp[v];
      }
      if (active && (kMerge || cur)) {
        T wm[NV], wp[NV], xs_l[NV], ys_l[NV];
        sload<T, NV, kPlane>(W, me - 1, wm);
        sload<T, NV, kPlane>(W, me + 1, wp);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if constexpr (WENO) {
            T dp, dm;
            weno3_offsets(wm[v], own[v], wp[v], dp, dm);
            xs_l[v] = own[v] + dp;
            xrOwn[v] = own[v] - dm;
          } else {
            const T sx = limited_slope(wm[v], own[v], wp[v], ph.theta);
            xs_l[v] = own[v] + sc * sx;
            xrOwn[v] = own[v] - sc * sx;
          }
        }
        sstore<T, NV, kState>(XL, xs, xs_l);
        sload<T, NV, kPlane>(W, me - sw, wm);
        sload<T, NV, kPlane>(W, me + sw, wp);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if constexpr (WENO) {
            T dp, dm;
            weno3_offsets(wm[v], own[v], wp[v], dp, dm);
            ys_l[v] = own[v] + dp;
            yrOwn[v] = own[v] - dm;
          } else {
            const T sy = limited_slope(wm[v], own[v], wp[v], ph.theta);
            ys_l[v] = own[v] + sc * sy;
            yrOwn[v] = own[v] - sc * sy;
          }
        }
        sstore<T, NV, kState>(YL, ys, ys_l);
      }
      if (bkind >= 0 && (kMerge || cur)) {
        T* dst = bkind == 0 ? XL : (bkind == 1 ? XR : (bkind == 2 ? YL : YR));
        const T sgn = (bkind == 0 || bkind == 2) ? sc : -sc;
        T wm[NV], w0[NV], wp[NV];
        sload<T, NV, kPlane>(W, bpos - bstep, wm);
        sload<T, NV, kPlane>(W, bpos, w0);
        sload<T, NV, kPlane>(W, bpos + bstep, wp);
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if constexpr (WENO) {   // XL / YL: the face toward wp; XR / YR: toward wm
            T dp, dm;
            weno3_offsets(wm[v], w0[v], wp[v], dp, dm);
            w0[v] = (bkind == 0 || bkind == 2) ? w0[v] + dp : w0[v] - dm;
          } else {
            w0[v] = w0[v] + sgn * limited_slope(wm[v], w0[v], wp[v], ph.theta);
          }
        }
        sstore<T, NV, kState>(dst, bslot, w0);
      }
      __syncthreads();
    }
    if (a.dynamic) {   // every thread has read s_next (barriers since); fetch the next item
      if (t == 0) s_next = (int)atomicAdd(&a.params->work_next, 1u);
      __syncthreads();
      itn = s_next;
    } else {
      itn += gridDim.x;
    }
  }
  if (a.dynamic && t == 0) {
    // the last CTA to finish (all CTAs have made their final fetch) resets the
    // counters for the next launch on the stream
    __threadfence();
    if (atomicAdd(&a.params->work_done, 1u) == gridDim.x - 1) {
      a.params->work_next = 0u;
      a.params->work_done = 0u;
    }
  }
  if (bad) atomicOr(&a.params->bad, 1u);
  if (floor_hits) atomicAdd(&a.params->floor_hits, (unsigned long long)floor_hits);
  if (STAGE == 2 && a.fuse_rate) {
    double r = (double)rate_max, sp = (double)speed_max;
    for (int o = 16; o > 0; o >>= 1) {
      r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
      sp = fmax(sp, __shfl_xor_sync(0xffffffffu, sp, o));
    }
    if ((t & 31) == 0) {
      atomic_max_pos_double(&a.params->next_rate_bits, r);
      atomic_max_pos_double(&a.params->next_speed_bits, sp);
    }
  }
}

// RK2 stage with direct flux reconstruction (Euler, the AMR_FLUXREC variant)
// over the same work items: each thread owns one column of the item and marches
// in z; the x and y face fluxes of its cell are formed from the four-cell
// conserved stencils (L1-cached global loads), the z flux of the face below is
// carried from the previous plane.  No shared memory and no barriers.
template <typename T, int STAGE>
__global__ void __launch_bounds__(kStageThreads) fluxrec_stage_kernel(StageArgs<T> a) {
  const Phys<T> ph = phys_with_ch<T, 5>(a.ph, a.params);
  const T dt = (T)(a.params->dt0 * a.dt_scale);
  const T dtx = dt * a.idx, dty = dt * a.idy, dtz = dt * a.idz;
  bool ok = true;
  int floor_hits = 0;
  T rate_max = T(0), speed_max = T(0);
  auto face = [&](const T* in, int64_t vs, int64_t c1, int64_t step, int d, T* F) {
    T u[4][5];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int v = 0; v < 5; ++v) u[q][v] = in[v * vs + c1 + (q - 2) * step];
    if (d == 0) fluxrec_face<T, 0>(u, ph, F, ok, nullptr);
    else if (d == 1) fluxrec_face<T, 1>(u, ph, F, ok, nullptr);
    else fluxrec_face<T, 2>(u, ph, F, ok, nullptr);
  };
  for (int it = blockIdx.x; it < a.nitems; it += gridDim.x) {
    const StageItem w = a.items[it];
    const PatchDesc P = a.desc[w.patch];
    const int ncol = w.wx * w.wy;
    if ((int)threadIdx.x >= ncol) continue;
    const int i = w.x0 + (int)threadIdx.x % w.wx, j = w.y0 + (int)threadIdx.x / w.wx;
    const T* in = a.Uin + P.off;
    T* out = a.Uout + P.off;
    const int64_t vs = P.vstride, sy = P.pitch, sz = (int64_t)P.pitch * P.m1;
    T Fzm[5], Fzp[5], Fx0[5], Fx1[5], Fy0[5], Fy1[5];
    face(in, vs, cell_index(P, i, j, w.z0), sz, 2, Fzm);
    for (int k = w.z0; k < w.z0 + w.wz; ++k) {
      const int64_t c = cell_index(P, i, j, k);
      T uin[5], un[5], wc[5];
      if (STAGE == 2) {   // U^n, loaded ahead of the face work that hides its latency
#pragma unroll
        for (int v = 0; v < 5; ++v) un[v] = out[v * vs + c];
      }
      face(in, vs, c, 1, 0, Fx0);
      face(in, vs, c + 1, 1, 0, Fx1);
      face(in, vs, c, sy, 1, Fy0);
      face(in, vs, c + sy, sy, 1, Fy1);
      face(in, vs, c + sz, sz, 2, Fzp);
#pragma unroll
      for (int v = 0; v < 5; ++v) uin[v] = in[v * vs + c];
      ok &= cons_to_prim<T, 5>(uin, wc, ph.efl, &floor_hits);
#pragma unroll
      for (int v = 0; v < 5; ++v) {
        // u + dt L(u), L = -sum_d (F_{d,+} - F_{d,-}) / dx_d
        const T u2 = uin[v] - dtx * (Fx1[v] - Fx0[v]) - dty * (Fy1[v] - Fy0[v]) - dtz * (Fzp[v] - Fzm[v]);
        if (STAGE == 1) {
          out[v * vs + c] = u2;
        } else {
          un[v] = T(0.5) * un[v] + T(0.5) * u2;
          out[v * vs + c] = un[v];
        }
        Fzm[v] = Fzp[v];
      }
      if (STAGE == 2 && a.fuse_rate) {
        T r, sp;
        cell_rate<T, 5>(un, ph, (T)a.idx0, (T)a.idy0, (T)a.idz0, r, sp);
        rate_max = dmax(rate_max, r);
        speed_max = dmax(speed_max, sp);
      }
    }
  }
  if (!ok) atomicOr(&a.params->bad, 1u);
  if (floor_hits) atomicAdd(&a.params->floor_hits, (unsigned long long)floor_hits);
  if (STAGE == 2 && a.fuse_rate) {
    double r = (double)rate_max, sp = (double)speed_max;
    for (int o = 16; o > 0; o >>= 1) {
      r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
      sp = fmax(sp, __shfl_xor_sync(0xffffffffu, sp, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomic_max_pos_double(&a.params->next_rate_bits, r);
      atomic_max_pos_double(&a.params->next_speed_bits, sp);
    }
  }
}

// ---------------------------------------------------------------------------
// ghost fill and parent-tile gather
// ---------------------------------------------------------------------------

// Parent data at fraction alpha of the parent step: (1 - alpha) U_old + alpha U,
// with one fixed rounding order for every kernel that forms it.
template <typename T>
__device__ __forceinline__ T time_lerp(T u_old, T u, T alpha) {
  return fma(alpha, u, (T(1) - alpha) * u_old);
}

// One CTA per box: dst cell (a, b, c) = dlo + (i, j, k) takes the src cell whose
// local coordinate per axis is (dst + sh) (translate) or sh (constant).
template <typename T, int NV, bool GATHER>
__global__ void copy_kernel(const CopySeg* segs, int nseg, const PatchDesc* desc, T* dst_arena,
                            const T* src_arena, const T* src_old, T alpha) {
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const CopySeg g = segs[s];
    const PatchDesc D = desc[g.dst_patch];
    const PatchDesc S = desc[g.src_patch];
    const int n0 = g.dn[0], n1 = g.dn[1], n2 = g.dn[2];
    const int total = n0 * n1 * n2;
    const int svs = (int)S.vstride;
    const int sp = S.pitch, sm1 = S.m1;
    const T* Sb = src_arena + S.off;
    const T* Ob = GATHER ? src_old + S.off : nullptr;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int r = e / n0, a = e - r * n0;
      const int c = r / n1, b = r - c * n1;
      const int da = g.dlo[0] + a, db = g.dlo[1] + b, dc = g.dlo[2] + c;
      const int sa = g.mode[0] ? g.sh[0] : da + g.sh[0];
      const int sb = g.mode[1] ? g.sh[1] : db + g.sh[1];
      const int sc = g.mode[2] ? g.sh[2] : dc + g.sh[2];
      const int si = ((sc + kGhost) * sm1 + (sb + kGhost)) * sp + (sa + kGhost);
      if (GATHER) {
        const int tvol = D.tn[0] * D.tn[1] * D.tn[2];
        T* Tb = dst_arena + D.tile_off + (dc * D.tn[1] + db) * D.tn[0] + da;
#pragma unroll
        for (int v = 0; v < NV; ++v) Tb[v * tvol] = time_lerp(Ob[si + v * svs], Sb[si + v * svs], alpha);
      } else {
        T* Db = dst_arena + D.off + ((dc + kGhost) * D.m1 + (db + kGhost)) * D.pitch + (da + kGhost);
        const int dvs = (int)D.vstride;
        T val[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) val[v] = Sb[si + v * svs];
#pragma unroll
        for (int v = 0; v < NV; ++v) Db[v * dvs] = val[v];
      }
    }
  }
}

template <typename T>
__device__ __forceinline__ T minmod2(T a, T b) {
  return (a * b > T(0)) ? (dabs(a) < dabs(b) ? a : b) : T(0);
}

// Conservative prolongation: child = parent + sum_d (+-1/4) minmod(U_{C+1} - U_C, U_C - U_{C-1}),
// parent values taken from the time-interpolated tile (footprint grown by 2 parent cells).
template <typename T, int NV>
__global__ void prolong_kernel(const ProlongBox* boxes, int nbox, const PatchDesc* desc, const T* tile,
                               T* dst_arena) {
  for (int s = blockIdx.x; s < nbox; s += gridDim.x) {
    const ProlongBox b = boxes[s];
    const PatchDesc D = desc[b.patch];
    const int n0 = b.n[0], n1 = b.n[1], n2 = b.n[2];
    const int total = n0 * n1 * n2;
    const int64_t tvol = (int64_t)D.tn[0] * D.tn[1] * D.tn[2];
    const T* Tb = tile + D.tile_off;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int li = b.lo[0] + e % n0, lj = b.lo[1] + (e / n0) % n1, lk = b.lo[2] + e / (n0 * n1);
      const int g0 = D.lo[0] + li, g1 = D.lo[1] + lj, g2 = D.lo[2] + lk;
      // tile-local parent index: (g >> 1) - (lo >> 1) + 2
      const int c0 = (g0 >> 1) - (D.lo[0] >> 1) + 2;
      const int c1 = (g1 >> 1) - (D.lo[1] >> 1) + 2;
      const int c2 = (g2 >> 1) - (D.lo[2] >> 1) + 2;
      const int64_t ci = ((int64_t)c2 * D.tn[1] + c1) * D.tn[0] + c0;
      const int64_t st[3] = {1, (int64_t)D.tn[0], (int64_t)D.tn[0] * D.tn[1]};
      const T sg[3] = {(g0 & 1) ? T(0.25) : T(-0.25), (g1 & 1) ? T(0.25) : T(-0.25),
                       (g2 & 1) ? T(0.25) : T(-0.25)};
      const int64_t di = D.off + cell_index(D, li, lj, lk);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T* tv = Tb + v * tvol;
        const T uc = tv[ci];
        T val = uc;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T up = tv[ci + st[d]], um = tv[ci - st[d]];
          val = fma(sg[d], minmod2(up - uc, uc - um), val);
        }
        dst_arena[di + v * D.vstride] = val;
      }
    }
  }
}

// Batched ghost copy (GATHER = false) or parent-tile gather with time
// interpolation (GATHER = true) over flattened boxes: CTA k takes cells
// [k kCopyChunk, (k+1) kCopyChunk) of the launch, kCopyPerThread per thread,
// all loads issued before the stores.  Same values as copy_kernel.
template <typename T, int NV, bool GATHER>
__global__ void __launch_bounds__(kBoxThreads) box_copy_kernel(const FlatCopy* boxes, const int* first,
                                                               const int* chunk_box, int nchunk, int total, T* dst,
                                                               const T* src, const T* old, T alpha) {
  for (int k = blockIdx.x; k < nchunk; k += gridDim.x) {
    int b = chunk_box[k];
    T val[kCopyPerThread][NV];
    int64_t di[kCopyPerThread];
    int dvs[kCopyPerThread];
#pragma unroll
    for (int i = 0; i < kCopyPerThread; ++i) {
      const int e = k * kCopyChunk + i * kBoxThreads + (int)threadIdx.x;
      di[i] = -1;
      if (e < total) {
        while (first[b + 1] <= e) ++b;
        const FlatCopy g = boxes[b];
        const int q = e - first[b];
        const int r = q / g.n0, a = q - r * g.n0;
        const int c = r / g.n1, y = r - c * g.n1;
        const int64_t so = g.src0 + (int64_t)a * g.ssx + (int64_t)y * g.ssy + (int64_t)c * g.ssz;
        di[i] = g.dst0 + a + (int64_t)y * g.dsy + (int64_t)c * g.dsz;
        dvs[i] = g.dvs;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const int64_t sv = so + (int64_t)v * g.svs;
          val[i][v] = GATHER ? time_lerp(old[sv], src[sv], alpha) : src[sv];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kCopyPerThread; ++i) {
      if (di[i] >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) dst[di[i] + (int64_t)v * dvs[i]] = val[i][v];
      }
    }
  }
}

// Batched prolongation over flattened boxes, one parent cell per thread: the
// three limited slopes of a parent are formed once and its (up to) eight
// children in the box are written from them, each child by the same
// operations in the same order as prolong_kernel (same values).
template <typename T, int NV>
__global__ void __launch_bounds__(kBoxThreads) box_prolong_kernel(const FlatProlong* boxes, const int* first,
                                                                  const int* chunk_box, int nchunk, int total,
                                                                  const T* tile, T* dst) {
  for (int k = blockIdx.x; k < nchunk; k += gridDim.x) {
    const int e = k * kProlongChunk + (int)threadIdx.x;
    if (e >= total) continue;
    int b = chunk_box[k];
    while (first[b + 1] <= e) ++b;
    const FlatProlong g = boxes[b];
    const int q = e - first[b];
    const int r = q / g.np0, pa = q - r * g.np0;
    const int pc = r / g.np1, pb = r - pc * g.np1;
    const T* tc = tile + g.tp0 + pa + (int64_t)pb * g.tsy + (int64_t)pc * g.tsz;
    // children's fine coordinates in the box: 2 p + i - odd, i in {0, 1}
    const int a0 = 2 * pa - (g.odd & 1), b0 = 2 * pb - ((g.odd >> 1) & 1), c0 = 2 * pc - ((g.odd >> 2) & 1);
    const int64_t d0 = g.dst0 + a0 + (int64_t)b0 * g.dsy + (int64_t)c0 * g.dsz;
    bool in[3][2];
    in[0][0] = a0 >= 0; in[0][1] = a0 + 1 < g.n[0];
    in[1][0] = b0 >= 0; in[1][1] = b0 + 1 < g.n[1];
    in[2][0] = c0 >= 0; in[2][1] = c0 + 1 < g.n[2];
    const int st[3] = {1, g.tsy, g.tsz};
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const T* tv = tc + (int64_t)v * g.tvol;
      const T uc = tv[0];
      T sl[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const T up = tv[st[d]], um = tv[-st[d]];
        sl[d] = minmod2(up - uc, uc - um);
      }
      T* dv = dst + d0 + (int64_t)v * g.dvs;
#pragma unroll
      for (int kz = 0; kz < 2; ++kz)
#pragma unroll
        for (int jy = 0; jy < 2; ++jy)
#pragma unroll
          for (int ix = 0; ix < 2; ++ix) {
            if (!(in[0][ix] && in[1][jy] && in[2][kz])) continue;
            T u = fma(ix ? T(0.25) : T(-0.25), sl[0], uc);
            u = fma(jy ? T(0.25) : T(-0.25), sl[1], u);
            u = fma(kz ? T(0.25) : T(-0.25), sl[2], u);
            dv[ix + (int64_t)jy * g.dsy + (int64_t)kz * g.dsz] = u;
          }
    }
  }
}

// ---------------------------------------------------------------------------
// restriction, flux registers, reflux
// ---------------------------------------------------------------------------

template <typename T, int NV>
__global__ void restrict_kernel(const RestrictSeg* segs, int nseg, const PatchDesc* desc, T* U) {
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const RestrictSeg r = segs[s];
    const PatchDesc C = desc[r.coarse];
    const PatchDesc F = desc[r.fine];
    const int n0 = r.cn[0], n1 = r.cn[1], n2 = r.cn[2];
    const int total = n0 * n1 * n2;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int a = r.clo[0] + e % n0, b = r.clo[1] + (e / n0) % n1, c = r.clo[2] + e / (n0 * n1);
      const int f0 = 2 * (C.lo[0] + a) - F.lo[0];
      const int f1 = 2 * (C.lo[1] + b) - F.lo[1];
      const int f2 = 2 * (C.lo[2] + c) - F.lo[2];
      const int64_t ci = C.off + cell_index(C, a, b, c);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T* Y = U + F.off + v * F.vstride;
        T zs[2];
#pragma unroll
        for (int dz = 0; dz < 2; ++dz) {
          T ys[2];
#pragma unroll
          for (int dy = 0; dy < 2; ++dy)
            ys[dy] = Y[cell_index(F, f0, f1 + dy, f2 + dz)] + Y[cell_index(F, f0 + 1, f1 + dy, f2 + dz)];
          zs[dz] = ys[0] + ys[1];
        }
        U[ci + v * C.vstride] = T(0.125) * (zs[0] + zs[1]);
      }
    }
  }
}

template <typename T> struct Pair2Of;
template <> struct Pair2Of<float> { using type = float2; };
template <> struct Pair2Of<double> { using type = double2; };
template <typename T> using Pair2 = typename Pair2Of<T>::type;

// Batched restriction over flattened boxes (chunks of kRestrictChunk coarse
// cells); same pairwise sums as restrict_kernel.
template <typename T, int NV>
__global__ void __launch_bounds__(kBoxThreads) box_restrict_kernel(const FlatCopy* boxes, const int* first,
                                                                   const int* chunk_box, int nchunk, int total, T* U) {
  for (int k = blockIdx.x; k < nchunk; k += gridDim.x) {
    int b = chunk_box[k];
    T val[kRestrictPerThread][NV];
    int64_t di[kRestrictPerThread];
    int dvs[kRestrictPerThread];
#pragma unroll
    for (int i = 0; i < kRestrictPerThread; ++i) {
      const int e = k * kRestrictChunk + i * kBoxThreads + (int)threadIdx.x;
      di[i] = -1;
      if (e < total) {
        while (first[b + 1] <= e) ++b;
        const FlatCopy g = boxes[b];
        const int q = e - first[b];
        const int r = q / g.n0, a = q - r * g.n0;
        const int c = r / g.n1, y = r - c * g.n1;
        const int64_t f = g.src0 + 2 * a + (int64_t)(2 * y) * g.ssy + (int64_t)(2 * c) * g.ssz;
        di[i] = g.dst0 + a + (int64_t)y * g.dsy + (int64_t)c * g.dsz;
        dvs[i] = g.dvs;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T* Y = U + f + (int64_t)v * g.svs;
          T zs[2];
#pragma unroll
          for (int dz = 0; dz < 2; ++dz) {
            T ys[2];
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
              // the fine pair (2a, 2a+1) starts at an even element of an even-pitched,
              // 32-element-aligned patch block: one aligned two-element load
              const Pair2<T> row = *reinterpret_cast<const Pair2<T>*>(Y + (int64_t)dy * g.ssy + (int64_t)dz * g.ssz);
              ys[dy] = row.x + row.y;
            }
            zs[dz] = ys[0] + ys[1];
          }
          val[i][v] = T(0.125) * (zs[0] + zs[1]);
        }
      }
    }
#pragma unroll
    for (int i = 0; i < kRestrictPerThread; ++i) {
      if (di[i] >= 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) U[di[i] + (int64_t)v * dvs[i]] = val[i][v];
      }
    }
  }
}

template <typename T, int NV>
__device__ __forceinline__ void face_flux_dir(const T* base, const PatchDesc& P, int i, int j, int k, int d,
                                              const Phys<T>& ph, T* F) {
  const int64_t c1 = cell_index(P, i, j, k);
  if (d == 0) face_flux_from_array<T, NV, 0>(base, P.vstride, c1, 1, ph, F);
  else if (d == 1) face_flux_from_array<T, NV, 1>(base, P.vstride, c1, P.pitch, ph, F);
  else face_flux_from_array<T, NV, 2>(base, P.vstride, c1, (int64_t)P.pitch * P.m1, ph, F);
}

// Flux registers are stored per rectangle of coarse-fine faces (RegRect):
// register e of a level belongs to rectangle b with first[b] <= e < first[b+1];
// chunk_box[e / kBoxThreads] is the rectangle holding the first register of
// e's chunk.  Entry (a, b) of a rectangle: coarse cell C = clo + a e_t1 + b e_t2.
// Threads per CTA of the register kernels: small CTAs spread the few thousand
// registers of a small level over all SMs (each register is several flux solves).
constexpr int kRegThreads = 64;

// Entry q of a rectangle as (a, b) along (t1, t2): the in-plane axis that is x
// (t2 for d = 1) runs fastest, so neighbouring threads touch neighbouring cells.
__device__ __forceinline__ void reg_entry(const RegRect& r, int q, int& a, int& b) {
  if (r.d == 1) { a = q / r.nb; b = q - a * r.nb; }
  else { b = q / r.na; a = q - b * r.na; }
}

__device__ __forceinline__ int reg_rect_of(const int* first, const int* chunk_box, int nrect, int nreg, int e) {
  const int k = e / kBoxThreads;
  int lo = chunk_box[k];                                                 // first[lo] <= e
  int hi = (k + 1) * kBoxThreads < nreg ? chunk_box[k + 1] : nrect - 1;  // e < first[hi + 1]
  while (lo < hi) {   // the last rectangle starting at or before e (rectangles are never empty)
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Coarse side: R_c (+)= dt/2 * F_coarse at the face of C (stage 1 also clears R_f).
template <typename T, int NV>
__global__ void __launch_bounds__(kRegThreads) reg_coarse_kernel(const RegRect* rects, const int* first,
                                                                 const int* chunk_box, int nrect, int nreg,
                                                                 const PatchDesc* desc, const T* Uin, double* R,
                                                                 StepParams* params, double dt_scale, Phys<T> ph0,
                                                                 int stage) {
  const Phys<T> ph = phys_with_ch<T, NV>(ph0, params);
  const double dt = (double)(T)(params->dt0 * dt_scale);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nreg; e += gridDim.x * blockDim.x) {
    const int b0 = reg_rect_of(first, chunk_box, nrect, nreg, e);
    const RegRect r = rects[b0];
    const int q = e - first[b0];
    const int d = r.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int a, bb;
    reg_entry(r, q, a, bb);
    const PatchDesc C = desc[r.cpatch];
    int f[3] = {r.clo[0], r.clo[1], r.clo[2]};
    f[t1] += a;
    f[t2] += bb;
    if (r.cside > 0) f[d] += 1;
    T F[NV];
    face_flux_dir<T, NV>(Uin + C.off, C, f[0], f[1], f[2], d, ph, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double* Rc = R + (size_t)v * nreg + e;
      double* Rf = R + (size_t)(NV + v) * nreg + e;
      const double add = 0.5 * dt * (double)F[v];
      if (stage == 1) { *Rc = 0.0 + add; *Rf = 0.0; }
      else *Rc += add;
    }
  }
}

// Fine side: R_f += dt_f/2 * (1/4) * sum of the 4 fine sub-face fluxes.  Four
// neighbouring lanes take the four sub-faces (a, b) of one register, lane
// a + 2 b of the group, and add them with two butterfly shuffles:
// (F_00 + F_01) + (F_10 + F_11) (additions commute exactly, so every lane of
// the group holds the same sum).
template <typename T, int NV>
__global__ void __launch_bounds__(kRegThreads) reg_fine_kernel(const RegRect* rects, const int* first,
                                                               const int* chunk_box, int nrect, int nreg,
                                                               const PatchDesc* desc,
                                                               const T* Uin, double* R, StepParams* params,
                                                               double dt_scale, Phys<T> ph0) {
  const Phys<T> ph = phys_with_ch<T, NV>(ph0, params);
  const double dt = (double)(T)(params->dt0 * dt_scale);
  const int lane = (int)threadIdx.x & 31;
  const int64_t nsub = 4 * (int64_t)nreg;
  // warp-uniform trip count: the shuffles see all 32 lanes
  for (int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; t0 < nsub;
       t0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = t0 + lane;
    const bool act = t < nsub;
    const int e = act ? (int)(t >> 2) : nreg - 1;
    const int sub = (int)(t & 3);
    const int b0 = reg_rect_of(first, chunk_box, nrect, nreg, e);
    const RegRect r = rects[b0];
    const int q = e - first[b0];
    const int d = r.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    const PatchDesc Pf = desc[r.fpatch];
    int ea, eb;
    reg_entry(r, q, ea, eb);
    int f[3] = {r.flo[0], r.flo[1], r.flo[2]};
    f[t1] += 2 * ea + (sub & 1);
    f[t2] += 2 * eb + (sub >> 1);
    T F[NV];
    face_flux_dir<T, NV>(Uin + Pf.off, Pf, f[0], f[1], f[2], d, ph, F);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double x = (double)F[v];
      x = x + __shfl_xor_sync(0xffffffffu, x, 1);
      x = x + __shfl_xor_sync(0xffffffffu, x, 2);
      if (act && sub == 0) R[(size_t)(NV + v) * nreg + e] += 0.5 * dt * (0.25 * x);
    }
  }
}

// Reflux: U_C -= cside (R_f - R_c) / dx_d for the registers [e0, e1), in FP64.
// ordered = 0: the registers of rectangles whose cells have no other register
// (any order; one launch over all of them); ordered = 1: one pass over the
// registers of one fine-face orientation (d, side) that share cells with
// other rectangles.  The ordered passes run in (d, side) order, and within a
// pass a coarse cell has at most one register (a coarse face borders one fine
// patch), so a cell's corrections apply in that order without races.
template <typename T, int NV>
__global__ void __launch_bounds__(kRegThreads) reflux_kernel(const RegRect* rects, const int* first,
                                                             const int* chunk_box, int nrect, int e0, int e1, int nreg,
                                                             const PatchDesc* desc, const double* R, T* U,
                                                             double dx0, double dx1, double dx2, int ordered) {
  for (int e = e0 + blockIdx.x * blockDim.x + threadIdx.x; e < e1; e += gridDim.x * blockDim.x) {
    const int b0 = reg_rect_of(first, chunk_box, nrect, nreg, e);
    const RegRect r = rects[b0];
    if (r.ordered != ordered) continue;
    const double dxd = r.d == 0 ? dx0 : (r.d == 1 ? dx1 : dx2);
    const int q = e - first[b0];
    const int d = r.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    int ea, eb;
    reg_entry(r, q, ea, eb);
    int c[3] = {r.clo[0], r.clo[1], r.clo[2]};
    c[t1] += ea;
    c[t2] += eb;
    const PatchDesc C = desc[r.cpatch];
    const int64_t ci = C.off + cell_index(C, c[0], c[1], c[2]);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double delta = R[(size_t)(NV + v) * nreg + e] - R[(size_t)v * nreg + e];
      const double val = (double)U[ci + v * C.vstride] - (double)r.cside * delta / dxd;
      U[ci + v * C.vstride] = (T)val;
    }
  }
}

// ---------------------------------------------------------------------------
// reductions and host-layout conversion
// ---------------------------------------------------------------------------

// Per-cell CFL rate sum_d (|v_d| + c_d) / dx0_d and max signal speed max_d (|v_d| + c_d),
// reduced with warp shuffles and one atomic per warp.
template <typename T, int NV>
__global__ void speed_kernel(const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const T* U,
                             StepParams* params, double idx0, double idy0, double idz0, Phys<T> ph) {
  T rate = T(0), speed = T(0);
  const T i0 = (T)idx0, i1 = (T)idy0, i2 = (T)idz0;
  for (int s = blockIdx.x; s < nchunk; s += gridDim.x) {
    const ChunkDesc ch = chunks[s];
    const PatchDesc P = desc[ch.patch];
    const T* Ub = U + P.off;
    const int vs = (int)P.vstride;
    const int nx = P.n[0], nxy = P.n[0] * P.n[1];
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
      const int idx = ch.begin + e;
      const int k = idx / nxy, r2 = idx - k * nxy, j = r2 / nx, i = r2 - j * nx;
      T u[NV];
      load_cons<T, NV>(Ub, vs, ((k + kGhost) * P.m1 + (j + kGhost)) * P.pitch + (i + kGhost), u);
      T r, sp;
      cell_rate<T, NV>(u, ph, i0, i1, i2, r, sp);
      rate = dmax(rate, r);
      speed = dmax(speed, sp);
    }
  }
  double rd = (double)rate, sd = (double)speed;
  for (int o = 16; o > 0; o >>= 1) {
    rd = fmax(rd, __shfl_xor_sync(0xffffffffu, rd, o));
    sd = fmax(sd, __shfl_xor_sync(0xffffffffu, sd, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_pos_double(&params->rate_bits, rd);
    atomic_max_pos_double(&params->speed_bits, sd);
  }
}

// Sum over leaf cells of each chunk (FP64, fixed in-block order) times the cell volume.
template <typename T, int NV>
__global__ void totals_kernel(const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const T* U,
                              const CoverBox* cover, const int* cover_first, const double* level_vol,
                              double* partial) {
  __shared__ double red[NV][256];
  for (int s = blockIdx.x; s < nchunk; s += gridDim.x) {
    const ChunkDesc ch = chunks[s];
    const PatchDesc P = desc[ch.patch];
    const int cb0 = cover_first[ch.patch], cb1 = cover_first[ch.patch + 1];
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
      const int idx = ch.begin + e;
      const int i = idx % P.n[0], j = (idx / P.n[0]) % P.n[1], k = idx / (P.n[0] * P.n[1]);
      bool covered = false;
      for (int b = cb0; b < cb1 && !covered; ++b) {
        const CoverBox cb = cover[b];
        covered = i >= cb.lo[0] && i < cb.lo[0] + cb.n[0] && j >= cb.lo[1] && j < cb.lo[1] + cb.n[1] &&
                  k >= cb.lo[2] && k < cb.lo[2] + cb.n[2];
      }
      if (covered) continue;
      const int64_t c = P.off + cell_index(P, i, j, k);
#pragma unroll
      for (int v = 0; v < NV; ++v) acc[v] += (double)U[c + v * P.vstride];
    }
#pragma unroll
    for (int v = 0; v < NV; ++v) red[v][threadIdx.x] = acc[v];
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) {
#pragma unroll
        for (int v = 0; v < NV; ++v) red[v][threadIdx.x] += red[v][threadIdx.x + o];
      }
      __syncthreads();
    }
    if (threadIdx.x < NV) partial[(size_t)s * NV + threadIdx.x] = red[threadIdx.x][0] * level_vol[P.level];
    __syncthreads();
  }
}

template <int NV>
__global__ void totals_final_kernel(const double* partial, int nchunk, double* out) {
  const int v = threadIdx.x;
  if (v < NV) {
    double s = 0.0;
    for (int c = 0; c < nchunk; ++c) s += partial[(size_t)c * NV + v];
    out[v] = s;
  }
}

// div B over the leaf cells of each chunk (GLM-MHD, face ghosts filled): per chunk
// {sum |D| dV, max |D|, sum |B|/dx_min dV, max |B|/dx_min} with
// D = sum_d (B_d(i + e_d) - B_d(i - e_d)) / (2 dx_d), in FP64 without contraction.
template <typename T, int NV>
__global__ void divb_kernel(const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const T* U,
                            const CoverBox* cover, const int* cover_first, double dx0, double dy0, double dz0,
                            double* partial) {
  static_assert(NV == 9, "div B needs the magnetic field");
  __shared__ double red[4][256];
  for (int s = blockIdx.x; s < nchunk; s += gridDim.x) {
    const ChunkDesc ch = chunks[s];
    const PatchDesc P = desc[ch.patch];
    const int cb0 = cover_first[ch.patch], cb1 = cover_first[ch.patch + 1];
    const double sc = 1.0 / (double)(1 << P.level);
    const double hx = dx0 * sc, hy = dy0 * sc, hz = dz0 * sc;
    const double vol = __dmul_rn(__dmul_rn(hx, hy), hz);
    const double hmin = fmin(hx, fmin(hy, hz));
    const T* Bx = U + P.off + 5 * P.vstride;
    const T* By = U + P.off + 6 * P.vstride;
    const T* Bz = U + P.off + 7 * P.vstride;
    const int plane = P.pitch * P.m1;
    double l1 = 0.0, dmx = 0.0, bs = 0.0, bmx = 0.0;
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
      const int idx = ch.begin + e;
      const int i = idx % P.n[0], j = (idx / P.n[0]) % P.n[1], k = idx / (P.n[0] * P.n[1]);
      bool covered = false;
      for (int b = cb0; b < cb1 && !covered; ++b) {
        const CoverBox cb = cover[b];
        covered = i >= cb.lo[0] && i < cb.lo[0] + cb.n[0] && j >= cb.lo[1] && j < cb.lo[1] + cb.n[1] &&
                  k >= cb.lo[2] && k < cb.lo[2] + cb.n[2];
      }
      if (covered) continue;
      const int64_t c = cell_index(P, i, j, k);
      const double ddx = ((double)Bx[c + 1] - (double)Bx[c - 1]) / (2.0 * hx);
      const double ddy = ((double)By[c + P.pitch] - (double)By[c - P.pitch]) / (2.0 * hy);
      const double ddz = ((double)Bz[c + plane] - (double)Bz[c - plane]) / (2.0 * hz);
      const double dv = fabs(__dadd_rn(__dadd_rn(ddx, ddy), ddz));
      const double bx = Bx[c], by = By[c], bz = Bz[c];
      const double bm =
          sqrt(__dadd_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)), __dmul_rn(bz, bz))) / hmin;
      l1 += __dmul_rn(dv, vol);
      bs += __dmul_rn(bm, vol);
      dmx = fmax(dmx, dv);
      bmx = fmax(bmx, bm);
    }
    red[0][threadIdx.x] = l1;
    red[1][threadIdx.x] = dmx;
    red[2][threadIdx.x] = bs;
    red[3][threadIdx.x] = bmx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if ((int)threadIdx.x < o) {
        red[0][threadIdx.x] += red[0][threadIdx.x + o];
        red[1][threadIdx.x] = fmax(red[1][threadIdx.x], red[1][threadIdx.x + o]);
        red[2][threadIdx.x] += red[2][threadIdx.x + o];
        red[3][threadIdx.x] = fmax(red[3][threadIdx.x], red[3][threadIdx.x + o]);
      }
      __syncthreads();
    }
    if (threadIdx.x < 4) partial[(size_t)s * 4 + threadIdx.x] = red[threadIdx.x][0];
    __syncthreads();
  }
}

template <int NQ>   // NQ = 4 norms per chunk: even ones summed, odd ones maxed
__global__ void divb_final_kernel(const double* partial, int nchunk, double* out) {
  const int v = threadIdx.x;
  if (v < NQ) {
    double a = 0.0;
    for (int c = 0; c < nchunk; ++c) {
      const double x = partial[(size_t)c * NQ + v];
      a = (v & 1) ? fmax(a, x) : a + x;
    }
    out[v] = a;
  }
}

// Packed FP64 host layout (per patch [nvar][n2][n1][n0]) -> ghosted arena,
// converting primitive input to conserved variables when `prim` is set.
template <typename T, int NV>
__global__ void pack_in_kernel(const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                               const int64_t* packed_off, const double* src, T* U, int prim, double gamma,
                               StepParams* params) {
  bool bad = false;
  for (int s = blockIdx.x; s < nchunk; s += gridDim.x) {
    const ChunkDesc ch = chunks[s];
    const PatchDesc P = desc[ch.patch];
    const int64_t ncell = (int64_t)P.n[0] * P.n[1] * P.n[2];
    const double* sp = src + packed_off[ch.patch];
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
      const int idx = ch.begin + e;
      const int i = idx % P.n[0], j = (idx / P.n[0]) % P.n[1], k = idx / (P.n[0] * P.n[1]);
      double w[NV], u[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) w[v] = sp[v * ncell + idx];
      if (prim) {
        // e = p / ((gamma - 1) rho), rho E = rho (v^2 / 2 + e) (+ B^2 / 2)
        const double eint = w[4] / ((gamma - 1.0) * w[0]);
        const double v2 = w[1] * w[1] + w[2] * w[2] + w[3] * w[3];
        u[0] = w[0]; u[1] = w[0] * w[1]; u[2] = w[0] * w[2]; u[3] = w[0] * w[3];
        u[4] = w[0] * (v2 / 2.0 + eint);
        if (NV == 9) {
          u[4] += (w[5] * w[5] + w[6] * w[6] + w[7] * w[7]) / 2.0;
          u[5] = w[5]; u[6] = w[6]; u[7] = w[7]; u[8] = w[8];
        }
        bad |= !(w[0] > 0.0) || !(w[4] > 0.0);
      } else {
#pragma unroll
        for (int v = 0; v < NV; ++v) u[v] = w[v];
        const double r = 1.0 / u[0];
        double ek = u[4] - 0.5 * (u[1] * u[1] + u[2] * u[2] + u[3] * u[3]) * r;
        if (NV == 9) ek -= 0.5 * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
        bad |= !(u[0] > 0.0) || !(ek > 0.0);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        bad |= !(u[v] - u[v] == 0.0);  // not finite
        U[P.off + v * P.vstride + cell_index(P, i, j, k)] = (T)u[v];
      }
    }
  }
  if (bad) atomicOr(&params->bad, 2u);
}

template <typename T, int NV>
__global__ void pack_out_kernel(const ChunkDesc* chunks, int nchunk, const PatchDesc* desc,
                                const int64_t* packed_off, const T* U, double* dst) {
  for (int s = blockIdx.x; s < nchunk; s += gridDim.x) {
    const ChunkDesc ch = chunks[s];
    const PatchDesc P = desc[ch.patch];
    const int64_t ncell = (int64_t)P.n[0] * P.n[1] * P.n[2];
    double* dp = dst + packed_off[ch.patch];
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
      const int idx = ch.begin + e;
      const int i = idx % P.n[0], j = (idx / P.n[0]) % P.n[1], k = idx / (P.n[0] * P.n[1]);
#pragma unroll
      for (int v = 0; v < NV; ++v) dp[v * ncell + idx] = (double)U[P.off + v * P.vstride + cell_index(P, i, j, k)];
    }
  }
}

// ---------------------------------------------------------------------------
// regridding
// ---------------------------------------------------------------------------

// Density-gradient criterion of one interior cell (face ghosts filled):
// max_d |rho(i + e_d) - rho(i - e_d)| / (2 rho(i)) > threshold, in the bulk precision.
template <typename T>
__device__ __forceinline__ bool density_flag(const PatchDesc& P, const T* R, int c, T threshold) {
  const int plane = P.pitch * P.m1;
  const T rho = R[c];
  const T gx = dabs(R[c + 1] - R[c - 1]);
  const T gy = dabs(R[c + P.pitch] - R[c - P.pitch]);
  const T gz = dabs(R[c + plane] - R[c - plane]);
  const T g = dmax(gx, dmax(gy, gz)) / (T(2) * rho);
  return g > threshold;
}

// One byte per interior cell: 1 where the density-gradient criterion holds.
template <typename T, int NV>
__global__ void flag_kernel(const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const int64_t* packed_off,
                            const T* U, T threshold, unsigned char* flags) {
  for (int s = blockIdx.x; s < nchunk; s += gridDim.x) {
    const ChunkDesc ch = chunks[s];
    const PatchDesc P = desc[ch.patch];
    const T* R = U + P.off;   // density is variable 0
    const int nx = P.n[0], nxy = P.n[0] * P.n[1];
    unsigned char* fp = flags + packed_off[ch.patch] / NV;
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
      const int idx = ch.begin + e;
      const int k = idx / nxy, r2 = idx - k * nxy, j = r2 / nx, i = r2 - j * nx;
      const int c = ((k + kGhost) * P.m1 + (j + kGhost)) * P.pitch + (i + kGhost);
      fp[idx] = density_flag(P, R, c, threshold) ? 1 : 0;
    }
  }
}

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// Regrid tagging: every flagged cell of a level in [l0, L), grown by `buffer`
// cells (clipped at outflow faces), marks the blocks it touches in its level's
// bitmap (periodic block coordinates wrapped), as the host clustering does from
// the byte flags.
template <typename T, int NV>
__global__ void tag_kernel(const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const T* U, T threshold,
                           TagArgs a, unsigned int* words) {
  for (int s = blockIdx.x; s < nchunk; s += gridDim.x) {
    const ChunkDesc ch = chunks[s];
    const PatchDesc P = desc[ch.patch];
    const int l = P.level;
    if (l < a.l0 || l >= a.L) continue;
    const T* R = U + P.off;
    const int nx = P.n[0], nxy = P.n[0] * P.n[1];
    unsigned int* w = words + a.off[l];
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
      const int idx = ch.begin + e;
      const int k = idx / nxy, r2 = idx - k * nxy, j = r2 / nx, i = r2 - j * nx;
      const int c = ((k + kGhost) * P.m1 + (j + kGhost)) * P.pitch + (i + kGhost);
      if (!density_flag(P, R, c, threshold)) continue;
      const int cell[3] = {P.lo[0] + i, P.lo[1] + j, P.lo[2] + k};
      int b0[3], b1[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        int lo = cell[d] - a.buffer, hi = cell[d] + a.buffer;
        if (!a.per[d]) {
          lo = max(lo, 0);
          hi = min(hi, a.N[l][d] - 1);
        }
        b0[d] = floor_div(lo, a.block);
        b1[d] = floor_div(hi, a.block);
      }
      for (int z = b0[2]; z <= b1[2]; ++z)
        for (int y = b0[1]; y <= b1[1]; ++y)
          for (int x = b0[0]; x <= b1[0]; ++x) {
            int q[3] = {x, y, z};
#pragma unroll
            for (int d = 0; d < 3; ++d)
              if (a.per[d]) q[d] = ((q[d] % a.nb[l][d]) + a.nb[l][d]) % a.nb[l][d];
            const long long bi = ((long long)q[2] * a.nb[l][1] + q[1]) * a.nb[l][0] + q[0];
            atomicOr(w + (bi >> 5), 1u << (bi & 31));
          }
    }
  }
}

// Box copies between two hierarchies (interior cells of new patches from old patches).
template <typename T, int NV>
__global__ void xcopy_kernel(const CopySeg* segs, int nseg, const PatchDesc* dst_desc, const PatchDesc* src_desc,
                             T* dst_arena, const T* src_arena) {
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const CopySeg g = segs[s];
    const PatchDesc D = dst_desc[g.dst_patch];
    const PatchDesc S = src_desc[g.src_patch];
    const int n0 = g.dn[0], n1 = g.dn[1], n2 = g.dn[2];
    const int total = n0 * n1 * n2;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int r = e / n0, a = e - r * n0;
      const int c = r / n1, b = r - c * n1;
      const int da = g.dlo[0] + a, db = g.dlo[1] + b, dc = g.dlo[2] + c;
      const int si = ((dc + g.sh[2] + kGhost) * S.m1 + (db + g.sh[1] + kGhost)) * S.pitch + (da + g.sh[0] + kGhost);
      const int di = ((dc + kGhost) * D.m1 + (db + kGhost)) * D.pitch + (da + kGhost);
#pragma unroll
      for (int v = 0; v < NV; ++v) dst_arena[D.off + (int64_t)v * D.vstride + di] = src_arena[S.off + (int64_t)v * S.vstride + si];
    }
  }
}

}  // namespace amr
