// physics.cuh -- per-cell and per-face device arithmetic of the method:
// primitive recovery, generalised-minmod PLM (Sec. 4), physical fluxes of the
// Euler (Sec. 4) and GLM-MHD (Sec. 7.1) systems, and the HLL / LLF interface
// flux.  Reconstructed variables W = (rho, vx, vy, vz, e [, Bx, By, Bz, psi]),
// e the specific internal energy, p = (gamma - 1) rho e.
#pragma once
#include <cuda_runtime.h>

#include "amr_types.h"

namespace amr {

template <typename T>
struct Phys {
  T gamma;     // adiabatic index
  T gm1;       // gamma - 1
  T ggm1;      // gamma * (gamma - 1): c_s^2 = gamma p / rho = ggm1 * e
  T theta;     // generalised minmod parameter
  T ch;        // GLM cleaning speed (MHD)
  T ch2;       // ch^2
  T half_inv_ch;  // 1 / (2 ch)
  int llf;     // 1: the printed Sec. 4 flux with lambda_0; 0: two-wave HLL
  int fluxrec; // 1: direct flux reconstruction (Euler; replaces the Riemann solve)
  T efl;       // p_floor / (gamma - 1): the specific internal energy floor is efl / rho
  T glm_alpha; // GLM damping parameter (0 = off)
  int weno;    // 1: third-order WENO face states (flux-register faces; the stage kernel has its own build)
};

template <typename T> __device__ __forceinline__ T dmin(T a, T b) { return a < b ? a : b; }
template <typename T> __device__ __forceinline__ T dmax(T a, T b) { return a > b ? a : b; }
// FP32: the approximate PTX square root and reciprocal with subnormals flushed
// (no FP32 quantity of the method is subnormal), one instruction each.
__device__ __forceinline__ float dsqrt(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double dsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float dabs(float x) { return fabsf(x); }
__device__ __forceinline__ double dabs(double x) { return fabs(x); }
__device__ __forceinline__ float drcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double drcp(double x) { return 1.0 / x; }

// Half of the limited slope of cell i from (w_{i-1}, w_i, w_{i+1}):
// 1/2 minmod(theta (w_i - w_{i-1}), theta (w_{i+1} - w_i), (w_{i+1} - w_{i-1}) / 2),
// where minmod keeps the smallest magnitude if all three share a sign, else 0.
template <typename T>
__device__ __forceinline__ T half_slope(T wm, T w0, T wp, T theta) {
  T a = w0 - wm, b = wp - w0;
  T c = (wp - wm) * T(0.5);
  T m = dmin(dmin(dabs(a * theta), dabs(b * theta)), dabs(c));
  T s = (a * b > T(0)) ? (a > T(0) ? m : -m) : T(0);
  return T(0.5) * s;
}

// Limited slope in the scale the stage kernel carries: a face state is
// w +- kSlopeScale<T> * limited_slope(...).  FP64 carries the half slope itself.
// FP32 carries four times the half slope, minmod(2 theta a, 2 theta b, w_{i+1} - w_{i-1}),
// and folds the exact factor 1/4 into the fused multiply-add that forms the
// face state (the rounding is that of w + s with s the half slope).  It uses
// min.xorsign.abs (sm_100 family): min(|x|, |y|) with the sign of x*y, so
// max(min.xorsign.abs(a, b), 0) is min(|a|, |b|) when a and b share a sign and
// 0 otherwise; the result takes the sign of a.
template <typename T> struct SlopeScale { static constexpr double v = 1.0; };
template <> struct SlopeScale<float> { static constexpr double v = 0.25; };
template <typename T> __device__ __forceinline__ T slope_scale() { return T(SlopeScale<T>::v); }

template <typename T>
__device__ __forceinline__ T limited_slope(T wm, T w0, T wp, T theta) { return half_slope(wm, w0, wp, theta); }

__device__ __forceinline__ float limited_slope(float wm, float w0, float wp, float theta) {
  const float a = w0 - wm, b = wp - w0;
  float t;
  asm("min.xorsign.abs.f32 %0, %1, %2;" : "=f"(t) : "f"(a), "f"(b));
  return copysignf(fminf(fmaxf(t, 0.0f) * (2.0f * theta), fabsf(wp - wm)), a);
}

__device__ __forceinline__ float half_slope(float wm, float w0, float wp, float theta) {
  return 0.25f * limited_slope(wm, w0, wp, theta);
}

__device__ __forceinline__ float min3(float a, float b, float c) {
  float r;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ float max3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}
__device__ __forceinline__ double min3(double a, double b, double c) { return dmin(dmin(a, b), c); }
__device__ __forceinline__ double max3(double a, double b, double c) { return dmax(dmax(a, b), c); }

// Conserved -> reconstructed variables; returns false for rho <= 0, e <= 0 or NaN.
// The specific internal energy is raised to the floor efl / rho (efl = 0: no
// floor for a physical state); *hits (if given) counts where it acted.
template <typename T, int NV>
__device__ __forceinline__ bool cons_to_prim(const T* u, T* w, T efl, int* hits = nullptr) {
  T rho = u[0];
  T r = drcp(rho);
  T vx = u[1] * r, vy = u[2] * r, vz = u[3] * r;
  T E = u[4];
  if (NV == 9) E = E - T(0.5) * (u[5] * u[5] + u[6] * u[6] + u[7] * u[7]);
  T e = E * r - T(0.5) * (vx * vx + vy * vy + vz * vz);
  const T ef = efl * r;
  const bool low = e < ef;
  if (hits) *hits += low ? 1 : 0;
  e = low ? ef : e;
  w[0] = rho; w[1] = vx; w[2] = vy; w[3] = vz; w[4] = e;
  if (NV == 9) { w[5] = u[5]; w[6] = u[6]; w[7] = u[7]; w[8] = u[8]; }
  return (rho > T(0)) && (e > T(0));
}

// Conserved vector, physical flux along D, normal velocity and signal speed of
// a reconstructed state (Sec. 4 U, F^x/F^y/F^z; Sec. 7.1 for NV == 9 with the
// induction entries F^d_{B_k} = v_d B_k - v_k B_d).  For MHD the caller has
// already replaced B_D by the resolved normal field; F[5+D] and F[8] are left
// for the caller (Dedner pair).
template <typename T, int NV, int D>
__device__ __forceinline__ void state_flux(const T* w, const Phys<T>& ph, T* U, T* F, T& c) {
  const T rho = w[0], vx = w[1], vy = w[2], vz = w[3], e = w[4];
  const T vn = w[1 + D];
  const T p = ph.gm1 * rho * e;
  const T v2 = vx * vx + vy * vy + vz * vz;
  U[0] = rho;
  U[1] = rho * vx; U[2] = rho * vy; U[3] = rho * vz;
  U[4] = rho * (T(0.5) * v2 + e);
  if (NV == 5) {
    c = dsqrt(ph.ggm1 * e);
    F[0] = U[1 + D];
    F[1] = U[1] * vn; F[2] = U[2] * vn; F[3] = U[3] * vn;
    F[1 + D] += p;
    F[4] = (U[4] + p) * vn;
  } else {
    const T Bx = w[5], By = w[6], Bz = w[7];
    const T Bn = w[5 + D];
    const T B2 = Bx * Bx + By * By + Bz * Bz;
    const T pt = p + T(0.5) * B2;
    U[4] += T(0.5) * B2;
    U[5] = Bx; U[6] = By; U[7] = Bz; U[8] = w[8];
    // fast magnetosonic speed along D
    const T r = drcp(rho);
    const T a2 = ph.ggm1 * e;
    const T b2 = B2 * r;
    const T bn2 = Bn * Bn * r;
    const T s = a2 + b2;
    const T disc = dmax(s * s - T(4) * a2 * bn2, T(0));
    c = dsqrt(T(0.5) * (s + dsqrt(disc)));
    const T Bv = Bx * vx + By * vy + Bz * vz;
    F[0] = U[1 + D];
    F[1] = U[1] * vn - Bx * Bn; F[2] = U[2] * vn - By * Bn; F[3] = U[3] * vn - Bz * Bn;
    F[1 + D] += pt;
    F[4] = (U[4] + pt) * vn - Bn * Bv;
    F[5] = vn * Bx - vx * Bn; F[6] = vn * By - vy * Bn; F[7] = vn * Bz - vz * Bn;
    F[8] = T(0);
  }
}

// Third-order WENO face states (Jiang and Shu, r = 2; the higher-order scheme
// the abstract says the framework extends to) on the PLM stencil of a cell w0
// with neighbours wm, wp: the face toward wp is w0 + dp, the face toward wm is
// w0 - dm.  Each blends the half differences dl = w0 - wm and dr = wp - w0
// with linear weights 1/3 (the difference away from the face) and 2/3 (toward
// it), turned into nonlinear weights by (eps + d^2)^-2, eps = 1e-6.  The weight
// is formed from the ratio of the two indicators, so large jumps send it to its
// limit instead of overflowing.
template <typename T>
__device__ __forceinline__ void weno3_offsets(T wm, T w0, T wp, T& dp, T& dm) {
  const T eps = T(1e-6);
  const T dl = w0 - wm, dr = wp - w0;
  const T gl = eps + dl * dl, gr = eps + dr * dr;
  const T ql = gr * drcp(gl), qr = gl * drcp(gr);
  const T wr_p = T(2) * drcp(T(2) + ql * ql);   // weight of dr at the face toward wp
  const T wl_m = T(2) * drcp(T(2) + qr * qr);   // weight of dl at the face toward wm
  dp = T(0.5) * (dl + wr_p * (dr - dl));
  dm = T(0.5) * (dr + wl_m * (dl - dr));
}

// Interface flux along D from reconstructed left/right states (copied: the MHD
// branch overwrites the normal field with the Dedner-resolved value).
// Euler HLL without forming the two physical fluxes: with F = U v_n + P,
// P = (0, p e_D, p v_n), the two-wave flux
//   (S_R F_l - S_L F_r + S_L S_R (U_r - U_l)) / (S_R - S_L)
// equals alpha U_l + beta U_r + a P_l - b P_r with a = S_R / (S_R - S_L),
// b = S_L / (S_R - S_L), alpha = a (v_l - S_L), beta = b (S_R - v_r).  Since
// U = rho (1, v, v^2/2 + e), alpha U_l + beta U_r is formed from alpha rho_l and
// beta rho_r and the primitive states without the conserved vectors.
// FP32: the left and right halves of the solve as packed pairs (one
// instruction for two FMUL / FADD / FFMA lanes on sm_100 and later).
template <int D>
__device__ __forceinline__ void hll_euler_f32x2(const float* wl, const float* wr, const Phys<float>& ph, float* F) {
  const float2 rho = make_float2(wl[0], wr[0]);
  const float2 e = make_float2(wl[4], wr[4]);
  const float2 v = make_float2(wl[1 + D], wr[1 + D]);
  const float2 c2 = __fmul2_rn(make_float2(ph.ggm1, ph.ggm1), e);
  const float2 c = make_float2(dsqrt(c2.x), dsqrt(c2.y));
  const float2 lo = __fadd2_rn(v, make_float2(-c.x, -c.y));   // v - c
  const float2 hi = __fadd2_rn(v, c);                            // v + c
  const float SL = min3(0.0f, lo.x, lo.y);
  const float SR = max3(0.0f, hi.x, hi.y);
  const float inv = drcp(SR - SL);
  const float2 ab = __fmul2_rn(make_float2(SR, SL), make_float2(inv, inv));            // (a, b)
  const float2 d = __fadd2_rn(make_float2(v.x, SR), make_float2(-SL, -v.y));           // (v_l - S_L, S_R - v_r)
  const float2 abr = __fmul2_rn(__fmul2_rn(ab, d), rho);                                // (alpha rho_l, beta rho_r)
  float2 s2 = __fmul2_rn(make_float2(wl[1], wr[1]), make_float2(wl[1], wr[1]));
  s2 = __ffma2_rn(make_float2(wl[2], wr[2]), make_float2(wl[2], wr[2]), s2);
  s2 = __ffma2_rn(make_float2(wl[3], wr[3]), make_float2(wl[3], wr[3]), s2);
  const float2 h = __ffma2_rn(make_float2(0.5f, 0.5f), s2, e);                        // v^2/2 + e
  const float2 ar2 = make_float2(abr.x, abr.x), br2 = make_float2(abr.y, abr.y);
  const float2 f12 = __ffma2_rn(br2, make_float2(wr[1], wr[2]), __fmul2_rn(ar2, make_float2(wl[1], wl[2])));
  const float2 f34 = __ffma2_rn(br2, make_float2(wr[3], h.y), __fmul2_rn(ar2, make_float2(wl[3], h.x)));
  F[0] = abr.x + abr.y;
  F[1] = f12.x; F[2] = f12.y; F[3] = f34.x; F[4] = f34.y;
  // a p_l and b p_r, p = (gamma - 1) rho e
  const float2 q = __fmul2_rn(ab, __fmul2_rn(make_float2(ph.gm1, ph.gm1), __fmul2_rn(rho, e)));
  F[1 + D] += q.x - q.y;
  F[4] += q.x * v.x - q.y * v.y;
}

template <typename T, int D>
__device__ __forceinline__ void hll_euler(const T* wl, const T* wr, const Phys<T>& ph, T* F) {
  if constexpr (sizeof(T) == 4) {
    hll_euler_f32x2<D>(wl, wr, ph, F);
    return;
  }
  const T rl = wl[0], rr = wr[0], el = wl[4], er = wr[4];
  const T vl = wl[1 + D], vr = wr[1 + D];
  const T cl = dsqrt(ph.ggm1 * el), cr = dsqrt(ph.ggm1 * er);
  const T SL = min3(T(0), vl - cl, vr - cr);
  const T SR = max3(T(0), vl + cl, vr + cr);
  const T inv = drcp(SR - SL);
  const T a = SR * inv, b = SL * inv;
  const T ar = a * (vl - SL) * rl;   // alpha rho_l
  const T br = b * (SR - vr) * rr;   // beta rho_r
  const T hl = T(0.5) * (wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3]) + el;
  const T hr = T(0.5) * (wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3]) + er;
  F[0] = ar + br;
#pragma unroll
  for (int k = 1; k < 4; ++k) F[k] = ar * wl[k] + br * wr[k];
  F[4] = ar * hl + br * hr;
  const T ql = a * (ph.gm1 * (rl * el)), qr = b * (ph.gm1 * (rr * er));   // a p_l, b p_r
  F[1 + D] += ql - qr;
  F[4] += ql * vl - qr * vr;
}

// GLM-MHD HLL in the same form as hll_euler: with F = U v_n + P,
// P = (0, pt e_D - B B_n, pt v_n - B_n (B.v), -v B_n, 0), the two-wave flux is
// alpha U_l + beta U_r + a P_l - b P_r, so neither side's conserved vector nor
// physical flux is formed.  wl/wr carry the Dedner-resolved normal field Bm.
template <typename T, int D>
__device__ __forceinline__ void hll_mhd(const T* wl, const T* wr, const Phys<T>& ph, T Bm, T* F) {
  T pt[2], c[2], B2[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    const T* w = s ? wr : wl;
    const T b2 = w[5] * w[5] + w[6] * w[6] + w[7] * w[7];
    const T a2 = ph.ggm1 * w[4];
    const T r = drcp(w[0]);
    const T q = a2 + b2 * r;
    const T disc = dmax(q * q - T(4) * a2 * (Bm * Bm * r), T(0));
    c[s] = dsqrt(T(0.5) * (q + dsqrt(disc)));
    pt[s] = ph.gm1 * w[0] * w[4] + T(0.5) * b2;
    B2[s] = b2;
  }
  const T vl = wl[1 + D], vr = wr[1 + D];
  const T SL = min3(T(0), vl - c[0], vr - c[1]);
  const T SR = max3(T(0), vl + c[0], vr + c[1]);
  const T inv = drcp(SR - SL);
  const T a = SR * inv, b = SL * inv;
  const T al = a * (vl - SL), be = b * (SR - vr);
  const T ar = al * wl[0], br = be * wr[0];
  F[0] = ar + br;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    F[1 + k] = ar * wl[1 + k] + br * wr[1 + k] - Bm * (a * wl[5 + k] - b * wr[5 + k]);
    if (k != D) F[5 + k] = al * wl[5 + k] + be * wr[5 + k] - Bm * (a * wl[1 + k] - b * wr[1 + k]);
  }
  F[1 + D] += a * pt[0] - b * pt[1];
  const T hl = T(0.5) * (wl[1] * wl[1] + wl[2] * wl[2] + wl[3] * wl[3]) + wl[4];
  const T hr = T(0.5) * (wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3]) + wr[4];
  const T bvl = wl[5] * wl[1] + wl[6] * wl[2] + wl[7] * wl[3];
  const T bvr = wr[5] * wr[1] + wr[6] * wr[2] + wr[7] * wr[3];
  F[4] = ar * hl + br * hr + T(0.5) * (al * B2[0] + be * B2[1]) + a * (pt[0] * vl - Bm * bvl) -
         b * (pt[1] * vr - Bm * bvr);
}

template <typename T, int NV, int D>
__device__ __forceinline__ void riemann(T* wl, T* wr, const Phys<T>& ph, T* F) {
  if (NV == 5) {
    if (!ph.llf) {
      hll_euler<T, D>(wl, wr, ph, F);
      return;
    }
  }
  T Bm = T(0), psim = T(0);
  if (NV == 9) {
    const T Bl = wl[5 + D], Br = wr[5 + D];
    Bm = T(0.5) * (Bl + Br) - (wr[8] - wl[8]) * ph.half_inv_ch;
    psim = T(0.5) * (wl[8] + wr[8]) - T(0.5) * ph.ch * (Br - Bl);
    wl[5 + D] = Bm;
    wr[5 + D] = Bm;
    if (!ph.llf) {
      hll_mhd<T, D>(wl, wr, ph, Bm, F);
      F[5 + D] = psim;
      F[8] = ph.ch2 * Bm;
      return;
    }
  }
  T Ul[NV], Ur[NV], Fl[NV], Fr[NV], cl, cr;
  state_flux<T, NV, D>(wl, ph, Ul, Fl, cl);
  state_flux<T, NV, D>(wr, ph, Ur, Fr, cr);
  const T vl = wl[1 + D], vr = wr[1 + D];
  if (ph.llf) {
    const T a = dmax(dmax(dmax(T(0), vl + cl), vr + cr), dmax(cl - vl, cr - vr));
#pragma unroll
    for (int k = 0; k < NV; ++k) F[k] = T(0.5) * (Fl[k] + Fr[k] - a * (Ur[k] - Ul[k]));
  } else {
    // S_R - S_L > 0 for every state with c > 0 (the kernels flag e <= 0 as non-physical)
    const T SL = min3(T(0), vl - cl, vr - cr);
    const T SR = max3(T(0), vl + cl, vr + cr);
    const T inv = drcp(SR - SL);
    const T slsr = SL * SR;
#pragma unroll
    for (int k = 0; k < NV; ++k) F[k] = (SR * Fl[k] - SL * Fr[k] + slsr * (Ur[k] - Ul[k])) * inv;
  }
  if (NV == 9) {
    F[5 + D] = psim;
    F[8] = ph.ch2 * Bm;
  }
}

// Direct flux reconstruction (Euler) at the face between cells 1 and 2 of the
// conserved stencil u[0..3] along D: Lax-Friedrichs splitting
// F+- = (F(U) +- alpha U) / 2 with alpha = max over the four cells of |v_D| + c,
// F+ reconstructed from the left, F- from the right, each with the Sec. 4
// half-slope PLM; F = F+ + F-.
template <typename T, int D>
__device__ __forceinline__ void fluxrec_face(const T (&u)[4][5], const Phys<T>& ph, T* F, bool& ok, int* hits) {
  T f[4][5];
  T alpha = T(0);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T w[5];
    ok &= cons_to_prim<T, 5>(u[q], w, ph.efl, hits);
    const T p = ph.gm1 * (w[0] * w[4]);
    const T vd = w[1 + D];
    alpha = dmax(alpha, dabs(vd) + dsqrt(ph.ggm1 * w[4]));
    f[q][0] = u[q][1 + D];
#pragma unroll
    for (int k = 0; k < 3; ++k) f[q][1 + k] = u[q][1 + k] * vd + (k == D ? p : T(0));
    f[q][4] = (u[q][4] + p) * vd;
  }
#pragma unroll
  for (int v = 0; v < 5; ++v) {
    T fp[4], fm[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      fp[q] = T(0.5) * (f[q][v] + alpha * u[q][v]);
      fm[q] = T(0.5) * (f[q][v] - alpha * u[q][v]);
    }
    F[v] = (fp[1] + half_slope(fp[0], fp[1], fp[2], ph.theta)) +
           (fm[2] - half_slope(fm[1], fm[2], fm[3], ph.theta));
  }
}

// Interface flux along D at the face between cells (c1 - e_D) and c1 of an
// array holding conserved variables, stencil c1-2 .. c1+1 (used by the flux
// register kernels: same arithmetic as the stage kernel's faces).
template <typename T, int NV, int D>
__device__ __forceinline__ void face_flux_from_array(const T* base, int64_t vstride, int64_t c1, int64_t step,
                                                     const Phys<T>& ph, T* F) {
  if constexpr (NV == 5) {
    if (ph.fluxrec) {
      T u[4][5];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int v = 0; v < 5; ++v) u[q][v] = base[v * vstride + c1 + (q - 2) * step];
      bool ok = true;
      fluxrec_face<T, D>(u, ph, F, ok, nullptr);
      return;
    }
  }
  T w[4][NV];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T u[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) u[v] = base[v * vstride + c1 + (q - 2) * step];
    cons_to_prim<T, NV>(u, w[q], ph.efl);
  }
  T wl[NV], wr[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    if (ph.weno) {
      T dp, dm;
      weno3_offsets(w[0][v], w[1][v], w[2][v], dp, dm);
      wl[v] = w[1][v] + dp;
      weno3_offsets(w[1][v], w[2][v], w[3][v], dp, dm);
      wr[v] = w[2][v] - dm;
    } else {
      wl[v] = w[1][v] + half_slope(w[0][v], w[1][v], w[2][v], ph.theta);
      wr[v] = w[2][v] - half_slope(w[1][v], w[2][v], w[3][v], ph.theta);
    }
  }
  riemann<T, NV, D>(wl, wr, ph, F);
}

}  // namespace amr
