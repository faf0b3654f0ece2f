// kernels.cuh -- the sm_103a kernels of one coarse step, templated on the bulk
// precision T (float / double) and the variable count NV (5 Euler, 9 GLM-MHD).
//
//   stage_kernel     fused RK2 stage: primitive recovery, PLM on every face,
//                    HLL/LLF flux, flux difference L(U) and the stage update
//                    U1 = U + dt L(U) (stage 1) or U = U/2 + (U1 + dt L(U1))/2
//                    (stage 2, Sec. 5.1), one CTA per x-y column block
//                    marching through z with a double-buffered shared-memory
//                    plane and z-fluxes carried in registers.
//   copy_kernel      ghost fill by box copies (siblings, periodic images,
//                    outflow) and parent-tile gathers with linear time
//                    interpolation.
//   prolong_kernel   conservative minmod prolongation into fine ghost cells.
//   reg_*_kernel     FP64 flux registers at coarse-fine faces.
//   reflux_kernel    register correction of uncovered coarse cells.
//   restrict_kernel  mean of the 8 children (pairwise sums).
//   speed_kernel     CFL rate / max signal speed reduction (warp shuffles).
//   totals_kernel    FP64 conserved totals over leaf cells (fixed order).
//   pack kernels     FP64 host layout <-> ghosted device arena.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "amr_types.h"
#include "physics.cuh"

namespace amr {

// Shared-memory plane of a stage CTA: (wy + 4) x (wx + 4) cells; the planner
// keeps wx * wy <= 256, wx <= 32 and (wx + 4)(wy + 4) <= kPlaneMax.
// Face count wy (wx + 1) + (wy + 1) wx = 2 wx wy + wx + wy <= 512 + 70.
constexpr int kFaceMax = 2 * kStageThreads + 88;

template <typename T, int NV>
constexpr size_t stage_smem_bytes() {
  return sizeof(T) * NV * (2 * kPlaneMax + kFaceMax);
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
  Phys<T> ph;
};

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

template <typename T, int NV, int STAGE>
__global__ void __launch_bounds__(kStageThreads) stage_kernel(StageArgs<T> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Wb0 = reinterpret_cast<T*>(smem_raw);
  T* Wb1 = Wb0 + NV * kPlaneMax;
  T* FX = Wb1 + NV * kPlaneMax;

  const Phys<T> ph = phys_with_ch<T, NV>(a.ph, a.params);
  const T dt = (T)(a.params->dt0 * a.dt_scale);
  const int t = threadIdx.x;
  bool bad = false;

  for (int itn = blockIdx.x; itn < a.nitems; itn += gridDim.x) {
    const StageItem it = a.items[itn];
    const PatchDesc P = a.desc[it.patch];
    const int wx = it.wx, wy = it.wy, wz = it.wz;
    const int sw = wx + 4;
    const int ncol = wx * wy;
    const int nfx = wy * (wx + 1);
    T* FY = FX + NV * nfx;
    const bool active = t < ncol;
    const int tx = active ? t % wx : 0, ty = active ? t / wx : 0;
    const int gi = it.x0 + tx, gj = it.y0 + ty;
    const T* Ub = a.Uin + P.off;
    const int64_t plane = (int64_t)P.pitch * P.m1;
    const int64_t col = cell_index(P, gi, gj, 0);   // (k = 0) of own column
    const int me = (ty + 2) * sw + (tx + 2);

    T wA[NV], wB[NV], sA[NV], Fm[NV];
    if (active) {  // prologue: planes z0-2 .. z0+1
      T u[NV], w0[NV], w1[NV];
      const int k0 = it.z0;
      load_cons<T, NV>(Ub, P.vstride, col + (int64_t)(k0 - 2) * plane, u);
      cons_to_prim<T, NV>(u, w0);
      load_cons<T, NV>(Ub, P.vstride, col + (int64_t)(k0 - 1) * plane, u);
      cons_to_prim<T, NV>(u, w1);
      load_cons<T, NV>(Ub, P.vstride, col + (int64_t)k0 * plane, u);
      bad |= !cons_to_prim<T, NV>(u, wA);
      load_cons<T, NV>(Ub, P.vstride, col + (int64_t)(k0 + 1) * plane, u);
      bad |= !cons_to_prim<T, NV>(u, wB) && wz > 1;
      T wl[NV], wr[NV];
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        T s_m1 = half_slope(w0[v], w1[v], wA[v], ph.theta);
        sA[v] = half_slope(w1[v], wA[v], wB[v], ph.theta);
        wl[v] = w1[v] + s_m1;
        wr[v] = wA[v] - sA[v];
      }
      riemann<T, NV, 2>(wl, wr, ph, Fm);
    }

    const int nhalo = 4 * (wx + wy);
    for (int kk = 0; kk < wz; ++kk) {
      const int k = it.z0 + kk;
      T* W = (kk & 1) ? Wb1 : Wb0;
      T Fp[NV];
      if (active) {
        T u[NV], wC[NV], sB[NV], wl[NV], wr[NV];
        load_cons<T, NV>(Ub, P.vstride, col + (int64_t)(k + 2) * plane, u);
        bool ok = cons_to_prim<T, NV>(u, wC);
        if (kk + 2 < wz) bad |= !ok;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          sB[v] = half_slope(wA[v], wB[v], wC[v], ph.theta);
          wl[v] = wA[v] + sA[v];
          wr[v] = wB[v] - sB[v];
          W[v * kPlaneMax + me] = wA[v];
        }
        riemann<T, NV, 2>(wl, wr, ph, Fp);
#pragma unroll
        for (int v = 0; v < NV; ++v) { sA[v] = sB[v]; }
        // shift happens after the update (wA is needed there only through W)
#pragma unroll
        for (int v = 0; v < NV; ++v) { wA[v] = wB[v]; wB[v] = wC[v]; }
      }
      // face halo of plane k: x-halo (4 cells per row) and y-halo (4 rows per column)
      for (int h = t; h < nhalo; h += blockDim.x) {
        int hx, hy;
        if (h < 4 * wy) {
          int r = h >> 2, c = h & 3;
          hy = r;
          hx = c < 2 ? c - 2 : wx + (c - 2);
        } else {
          int h2 = h - 4 * wy;
          int r = h2 / wx, c = h2 - r * wx;
          hx = c;
          hy = r < 2 ? r - 2 : wy + (r - 2);
        }
        T u[NV], w[NV];
        load_cons<T, NV>(Ub, P.vstride, cell_index(P, it.x0 + hx, it.y0 + hy, k), u);
        cons_to_prim<T, NV>(u, w);
        const int pos = (hy + 2) * sw + (hx + 2);
#pragma unroll
        for (int v = 0; v < NV; ++v) W[v * kPlaneMax + pos] = w[v];
      }
      __syncthreads();
      // x and y faces at the low side of every column, then the high edge faces
      if (active) {
        T wl[NV], wr[NV], F[NV];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T* Wv = W + v * kPlaneMax + me;
          wl[v] = Wv[-1] + half_slope(Wv[-2], Wv[-1], Wv[0], ph.theta);
          wr[v] = Wv[0] - half_slope(Wv[-1], Wv[0], Wv[1], ph.theta);
        }
        riemann<T, NV, 0>(wl, wr, ph, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) FX[v * nfx + ty * (wx + 1) + tx] = F[v];
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T* Wv = W + v * kPlaneMax + me;
          wl[v] = Wv[-sw] + half_slope(Wv[-2 * sw], Wv[-sw], Wv[0], ph.theta);
          wr[v] = Wv[0] - half_slope(Wv[-sw], Wv[0], Wv[sw], ph.theta);
        }
        riemann<T, NV, 1>(wl, wr, ph, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) FY[v * (wx * (wy + 1)) + ty * wx + tx] = F[v];
      }
      {
        const int e = (int)blockDim.x - 1 - t;
        if (e < wy) {  // x face at the right edge of row e
          T wl[NV], wr[NV], F[NV];
          const int pos = (e + 2) * sw + (wx + 2);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const T* Wv = W + v * kPlaneMax + pos;
            wl[v] = Wv[-1] + half_slope(Wv[-2], Wv[-1], Wv[0], ph.theta);
            wr[v] = Wv[0] - half_slope(Wv[-1], Wv[0], Wv[1], ph.theta);
          }
          riemann<T, NV, 0>(wl, wr, ph, F);
#pragma unroll
          for (int v = 0; v < NV; ++v) FX[v * nfx + e * (wx + 1) + wx] = F[v];
        } else if (e < wy + wx) {  // y face at the top edge of column e - wy
          const int c = e - wy;
          T wl[NV], wr[NV], F[NV];
          const int pos = (wy + 2) * sw + (c + 2);
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            const T* Wv = W + v * kPlaneMax + pos;
            wl[v] = Wv[-sw] + half_slope(Wv[-2 * sw], Wv[-sw], Wv[0], ph.theta);
            wr[v] = Wv[0] - half_slope(Wv[-sw], Wv[0], Wv[sw], ph.theta);
          }
          riemann<T, NV, 1>(wl, wr, ph, F);
#pragma unroll
          for (int v = 0; v < NV; ++v) FY[v * (wx * (wy + 1)) + wy * wx + c] = F[v];
        }
      }
      __syncthreads();
      if (active) {
        const int64_t c = col + (int64_t)k * plane;
        const int nfy = wx * (wy + 1);
        T* Ob = a.Uout + P.off;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          const T Lx = (FX[v * nfx + ty * (wx + 1) + tx + 1] - FX[v * nfx + ty * (wx + 1) + tx]) * a.idx;
          const T Ly = (FY[v * nfy + (ty + 1) * wx + tx] - FY[v * nfy + ty * wx + tx]) * a.idy;
          const T Lz = (Fp[v] - Fm[v]) * a.idz;
          const T L = -(Lx + Ly + Lz);
          const T uin = Ub[v * P.vstride + c];
          if (STAGE == 1) {
            Ob[v * P.vstride + c] = uin + dt * L;
          } else {
            const T un = Ob[v * P.vstride + c];
            const T u2 = uin + dt * L;
            Ob[v * P.vstride + c] = T(0.5) * un + T(0.5) * u2;
          }
          Fm[v] = Fp[v];
        }
      }
    }
    __syncthreads();  // the next item reuses the shared buffers
  }
  if (bad) atomicOr(&a.params->bad, 1u);
}

// ---------------------------------------------------------------------------
// ghost fill and parent-tile gather
// ---------------------------------------------------------------------------

template <typename T, int NV, bool GATHER>
__global__ void copy_kernel(const CopySeg* segs, int nseg, const PatchDesc* desc, T* dst_arena,
                            const T* src_arena, const T* src_old, T alpha) {
  for (int s = blockIdx.x; s < nseg; s += gridDim.x) {
    const CopySeg g = segs[s];
    const PatchDesc D = desc[g.dst_patch];
    const PatchDesc S = desc[g.src_patch];
    const int n0 = g.dn[0], n1 = g.dn[1], n2 = g.dn[2];
    const int total = n0 * n1 * n2;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
      const int a = e % n0, b = (e / n0) % n1, c = e / (n0 * n1);
      const int da = g.dlo[0] + a, db = g.dlo[1] + b, dc = g.dlo[2] + c;
      const int sa = g.mode[0] ? g.sh[0] : da + g.sh[0];
      const int sb = g.mode[1] ? g.sh[1] : db + g.sh[1];
      const int sc = g.mode[2] ? g.sh[2] : dc + g.sh[2];
      const int64_t si = S.off + cell_index(S, sa, sb, sc);
      if (GATHER) {
        const int64_t di = (int64_t)D.tile_off + ((int64_t)dc * D.tn[1] + db) * D.tn[0] + da;
        const int64_t tvol = (int64_t)D.tn[0] * D.tn[1] * D.tn[2];
#pragma unroll
        for (int v = 0; v < NV; ++v)
          dst_arena[di + v * tvol] = (T(1) - alpha) * src_old[si + v * S.vstride] + alpha * src_arena[si + v * S.vstride];
      } else {
        const int64_t di = D.off + cell_index(D, da, db, dc);
#pragma unroll
        for (int v = 0; v < NV; ++v) dst_arena[di + v * D.vstride] = src_arena[si + v * S.vstride];
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
      const T sg[3] = {(g0 & 1) ? T(1) : T(-1), (g1 & 1) ? T(1) : T(-1), (g2 & 1) ? T(1) : T(-1)};
      const int64_t di = D.off + cell_index(D, li, lj, lk);
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const T* tv = Tb + v * tvol;
        const T uc = tv[ci];
        T val = uc;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const T up = tv[ci + st[d]], um = tv[ci - st[d]];
          const T sl = minmod2(up - uc, uc - um);
          val = val + sg[d] * T(0.25) * sl;
        }
        dst_arena[di + v * D.vstride] = val;
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

template <typename T, int NV>
__device__ __forceinline__ void face_flux_dir(const T* base, const PatchDesc& P, int i, int j, int k, int d,
                                              const Phys<T>& ph, T* F) {
  const int64_t c1 = cell_index(P, i, j, k);
  if (d == 0) face_flux_from_array<T, NV, 0>(base, P.vstride, c1, 1, ph, F);
  else if (d == 1) face_flux_from_array<T, NV, 1>(base, P.vstride, c1, P.pitch, ph, F);
  else face_flux_from_array<T, NV, 2>(base, P.vstride, c1, (int64_t)P.pitch * P.m1, ph, F);
}

// Coarse side: R_c (+)= dt/2 * F_coarse at the face of C (stage 1 also clears R_f).
template <typename T, int NV>
__global__ void reg_coarse_kernel(const RegFace* regs, int nreg, const PatchDesc* desc, const T* Uin,
                                  double* R, StepParams* params, double dt_scale, Phys<T> ph0, int stage) {
  const Phys<T> ph = phys_with_ch<T, NV>(ph0, params);
  const double dt = (double)(T)(params->dt0 * dt_scale);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nreg; e += gridDim.x * blockDim.x) {
    const RegFace r = regs[e];
    const PatchDesc C = desc[r.cpatch];
    int f[3] = {r.cidx[0], r.cidx[1], r.cidx[2]};
    if (r.cside > 0) f[r.d] += 1;
    T F[NV];
    face_flux_dir<T, NV>(Uin + C.off, C, f[0], f[1], f[2], r.d, ph, F);
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

// Fine side: R_f += dt_f/2 * (1/4) * sum of the 4 fine sub-face fluxes.
template <typename T, int NV>
__global__ void reg_fine_kernel(const RegFace* regs, int nreg, const PatchDesc* desc, const T* Uin, double* R,
                                StepParams* params, double dt_scale, Phys<T> ph0) {
  const Phys<T> ph = phys_with_ch<T, NV>(ph0, params);
  const double dt = (double)(T)(params->dt0 * dt_scale);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < nreg; e += gridDim.x * blockDim.x) {
    const RegFace r = regs[e];
    const PatchDesc Pf = desc[r.fpatch];
    const int d = r.d, t1 = (d + 1) % 3, t2 = (d + 2) % 3;
    double q[2][2][NV];
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        int f[3] = {r.fface[0], r.fface[1], r.fface[2]};
        f[t1] += a;
        f[t2] += b;
        T F[NV];
        face_flux_dir<T, NV>(Uin + Pf.off, Pf, f[0], f[1], f[2], d, ph, F);
#pragma unroll
        for (int v = 0; v < NV; ++v) q[b][a][v] = (double)F[v];
      }
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const double sum = (q[0][0][v] + q[0][1][v]) + (q[1][0][v] + q[1][1][v]);
      R[(size_t)(NV + v) * nreg + e] += 0.5 * dt * (0.25 * sum);
    }
  }
}

// U_C -= side * (R_f - R_c) / dx_c, every register of one coarse cell in (axis, side) order.
template <typename T, int NV>
__global__ void reflux_kernel(const RegFace* regs, const int* first, int nuniq, int nreg, const PatchDesc* desc,
                              const double* R, T* U, double dx0, double dx1, double dx2) {
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < nuniq; u += gridDim.x * blockDim.x) {
    const int e0 = first[u], e1 = first[u + 1];
    const RegFace r0 = regs[e0];
    const PatchDesc C = desc[r0.cpatch];
    const int64_t ci = C.off + cell_index(C, r0.cidx[0], r0.cidx[1], r0.cidx[2]);
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      double val = (double)U[ci + v * C.vstride];
      for (int e = e0; e < e1; ++e) {
        const RegFace r = regs[e];
        const double dxc = r.d == 0 ? dx0 : (r.d == 1 ? dx1 : dx2);
        const double delta = R[(size_t)(NV + v) * nreg + e] - R[(size_t)v * nreg + e];
        val = val - (double)r.cside * delta / dxc;
      }
      U[ci + v * C.vstride] = (T)val;
    }
  }
}

// ---------------------------------------------------------------------------
// reductions and host-layout conversion
// ---------------------------------------------------------------------------

__device__ __forceinline__ void atomic_max_pos_double(unsigned long long* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

// Per-cell CFL rate sum_d (|v_d| + c_d) / dx0_d and max signal speed max_d (|v_d| + c_d).
template <typename T, int NV>
__global__ void speed_kernel(const ChunkDesc* chunks, int nchunk, const PatchDesc* desc, const T* U,
                             StepParams* params, double idx0, double idy0, double idz0, Phys<T> ph) {
  double rate = 0.0, speed = 0.0;
  for (int s = blockIdx.x; s < nchunk; s += gridDim.x) {
    const ChunkDesc ch = chunks[s];
    const PatchDesc P = desc[ch.patch];
    for (int e = threadIdx.x; e < ch.count; e += blockDim.x) {
      const int idx = ch.begin + e;
      const int i = idx % P.n[0], j = (idx / P.n[0]) % P.n[1], k = idx / (P.n[0] * P.n[1]);
      T u[NV], w[NV];
      load_cons<T, NV>(U + P.off, P.vstride, cell_index(P, i, j, k), u);
      cons_to_prim<T, NV>(u, w);
      T Ud[NV], Fd[NV], c0, c1, c2;
      state_flux<T, NV, 0>(w, ph, Ud, Fd, c0);
      state_flux<T, NV, 1>(w, ph, Ud, Fd, c1);
      state_flux<T, NV, 2>(w, ph, Ud, Fd, c2);
      const double s0 = (double)(dabs(w[1]) + c0), s1 = (double)(dabs(w[2]) + c1), s2 = (double)(dabs(w[3]) + c2);
      const double r = s0 * idx0 + s1 * idy0 + s2 * idz0;
      rate = fmax(rate, r);
      speed = fmax(speed, fmax(s0, fmax(s1, s2)));
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    rate = fmax(rate, __shfl_xor_sync(0xffffffffu, rate, o));
    speed = fmax(speed, __shfl_xor_sync(0xffffffffu, speed, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomic_max_pos_double(&params->rate_bits, rate);
    atomic_max_pos_double(&params->speed_bits, speed);
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

}  // namespace amr
