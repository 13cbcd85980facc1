#pragma once
// mbs_device.cuh -- sm_103a device code of the 1D Maxwell-Bloch time step
// (included by the kernel translation units).
//
// Two forms of the same per-step arithmetic (see mbs_internal.h for the
// state representation):
//
//  * plain (the loop order of Sec. 3.2): one thread per cell, two launches
//    per step -- {H, rho, d_t P} at n + 1/2, then {E, sources, boundaries,
//    records} at n + 1 -- with the kernel boundary as the synchronisation
//    between the two halves;
//
//  * tiled (the redundant-calculation loop of Sec. 3.2, re-designed for the
//    GPU): each block owns a segment of cells and advances it T steps per
//    launch entirely in registers.  A lane holds R consecutive cells; the
//    neighbour traffic is one warp shuffle of E to the right and one of H to
//    the left per step, plus the values at the block's inner warp edges,
//    which pass through shared memory between two block barriers per step.
//    The block loads its segment plus a T-cell halo on each side; the halo
//    shrinks by one cell per side per step (the light cone of the 3-point
//    stencil), so after T steps the owned cells are exact and are the only
//    ones written back.  Ping-pong buffers keep neighbouring blocks' halo
//    reads race-free.
//
// In FP32 the fields are float-float pairs (see "fields" below).
// The field rotation needs sin(theta) and cos(theta) - 1 of small angles to
// full relative precision; they come from their Taylor series (coefficients
// +-1/n!) for |theta| <= 1/2 and from the CUDA math library otherwise.
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

#include "mbs_internal.h"

namespace mbs {
namespace dev {

constexpr unsigned FULL = 0xffffffffu;

// ------------------------------------------------------------- math helpers
// |x| > 1/2: library sincos
static __device__ __forceinline__ void sincos_m1_wide(float x, float &s, float &cm1) {
  float c;
  sincosf(x, &s, &c);
  cm1 = c - 1.0f;
}

// |x| > 1/2 in the tensor-core tiles: out of line, so that the common path
// carries no library code; (sin x, cos x - 1) returned by value, so that the caller's
// results stay in registers
static __device__ __noinline__ float2 sincos_m1_far(float x) {
  float2 r;
  sincos_m1_wide(x, r.x, r.y);
  return r;
}

// sin x and cos x - 1 by their Taylor polynomials to x^7 and x^8, for
// angles known to satisfy |x| <= 1/2 (cos x - 1 never forms 1 - 1): the
// alternating series' first omitted terms, x^9/9! <= 5.4e-9 and
// x^10/10! <= 2.7e-10, stay below half an ulp of sin x and of cos x - 1 on
// that range.
__device__ __forceinline__ void sincos_m1_taylor_half(float x, float &s, float &cm1) {
  const float t = x * x;
  float ps = fmaf(t, -1.0f / 5040.0f, 1.0f / 120.0f);
  ps = fmaf(t, ps, -1.0f / 6.0f);
  ps = fmaf(t, ps, 1.0f);
  s = x * ps;
  float pc = fmaf(t, 1.0f / 40320.0f, -1.0f / 720.0f);
  pc = fmaf(t, pc, 1.0f / 24.0f);
  pc = fmaf(t, pc, -0.5f);
  cm1 = t * pc;
}

// sin x and cos x - 1 for any x: the shorter polynomials within 1/2, the
// library routine beyond
__device__ __forceinline__ void sincos_m1(float x, float &s, float &cm1) {
  sincos_m1_taylor_half(x, s, cm1);
  if (fabsf(x) > 0.5f) sincos_m1_wide(x, s, cm1);
}

__device__ __forceinline__ void sincos_m1(double x, double &s, double &cm1) {
  if (fabs(x) <= 0.5) {
    const double t = x * x;
    // sin x / x and (cos x - 1) / x^2 to order x^16
    double ps = 1.0 / 355687428096000.0;          // 1/17!
    ps = fma(t, ps, -1.0 / 1307674368000.0);      // 1/15!
    ps = fma(t, ps, 1.0 / 6227020800.0);          // 1/13!
    ps = fma(t, ps, -1.0 / 39916800.0);           // 1/11!
    ps = fma(t, ps, 1.0 / 362880.0);              // 1/9!
    ps = fma(t, ps, -1.0 / 5040.0);
    ps = fma(t, ps, 1.0 / 120.0);
    ps = fma(t, ps, -1.0 / 6.0);
    ps = fma(t, ps, 1.0);
    s = x * ps;
    double pc = -1.0 / 6402373705728000.0;        // 1/18!
    pc = fma(t, pc, 1.0 / 20922789888000.0);      // 1/16!
    pc = fma(t, pc, -1.0 / 87178291200.0);        // 1/14!
    pc = fma(t, pc, 1.0 / 479001600.0);           // 1/12!
    pc = fma(t, pc, -1.0 / 3628800.0);            // 1/10!
    pc = fma(t, pc, 1.0 / 40320.0);
    pc = fma(t, pc, -1.0 / 720.0);
    pc = fma(t, pc, 1.0 / 24.0);
    pc = fma(t, pc, -0.5);
    cm1 = t * pc;
  } else {
    double c;
    sincos(x, &s, &c);
    cm1 = c - 1.0;
  }
}

// Rotation forms of the Bloch step (FP32; FP64 always takes sincos_m1):
//   ROT_TAYLOR: every angle of the warp is known to satisfy |x| <= 1/2
//               (the shorter polynomials);
//   ROT_INLINE: any angle, the library routine inline beyond 1/2.
enum { ROT_TAYLOR = 0, ROT_INLINE = 2 };
template <int ROT>
__device__ __forceinline__ void sincos_m1_sel(float x, float &s, float &cm1) {
  if constexpr (ROT == ROT_INLINE)
    sincos_m1(x, s, cm1);
  else
    sincos_m1_taylor_half(x, s, cm1);
}
template <int ROT>
__device__ __forceinline__ void sincos_m1_sel(double x, double &s, double &cm1) {
  sincos_m1(x, s, cm1);
}

// compensated d += x (Kahan): c carries the part of past additions that
// rounding dropped (true value = d - c)
template <typename real>
__device__ __forceinline__ void kahan_add(real &d, real &c, real x) {
  const real y = x - c;
  const real t = d + y;
  c = (t - d) - y;
  d = t;
}

// ---------------------------------------------------- parameter accessors
// contiguous parameter block: am1 | c | w | w0 | kap | zr
template <typename real, int N>
struct PrmBlock {
  static constexpr int K = N * N - 1, P = N * (N - 1) / 2;
  const real *p;
  __device__ __forceinline__ real am1(int i, int j) const { return p[i * K + j]; }
  __device__ __forceinline__ real c(int i) const { return p[K * K + i]; }
  __device__ __forceinline__ real w(int i) const { return p[K * K + K + i]; }
  __device__ __forceinline__ real w0() const { return p[K * K + 2 * K]; }
  __device__ __forceinline__ real kap(int q) const { return p[K * K + 2 * K + 1 + q]; }
  __device__ __forceinline__ real zr(int i) const { return p[K * K + 2 * K + 1 + P + i]; }
};

// per-cell rows (am1, c, w, w0 strided by ld) + material block for kap, zr
template <typename real, int N>
struct PrmCell {
  static constexpr int K = N * N - 1, P = N * (N - 1) / 2;
  const real *p;   // &pcell[0][cell]
  int ld;
  const real *mb;  // material block
  __device__ __forceinline__ real am1(int i, int j) const { return p[(size_t)(i * K + j) * ld]; }
  __device__ __forceinline__ real c(int i) const { return p[(size_t)(K * K + i) * ld]; }
  __device__ __forceinline__ real w(int i) const { return p[(size_t)(K * K + K + i) * ld]; }
  __device__ __forceinline__ real w0() const { return p[(size_t)(K * K + 2 * K) * ld]; }
  __device__ __forceinline__ real kap(int q) const { return mb[K * K + 2 * K + 1 + q]; }
  __device__ __forceinline__ real zr(int i) const { return mb[K * K + 2 * K + 1 + P + i]; }
};

// per-cell parameters held in registers (tiled kernel, N = 2)
template <typename real, int N>
struct PrmReg {
  static constexpr int K = N * N - 1, P = N * (N - 1) / 2;
  real a[K * K], cc[K], ww[K], ww0;
  const real *mb;
  __device__ __forceinline__ real am1(int i, int j) const { return a[i * K + j]; }
  __device__ __forceinline__ real c(int i) const { return cc[i]; }
  __device__ __forceinline__ real w(int i) const { return ww[i]; }
  __device__ __forceinline__ real w0() const { return ww0; }
  __device__ __forceinline__ real kap(int q) const { return mb[K * K + 2 * K + 1 + q]; }
  __device__ __forceinline__ real zr(int i) const { return mb[K * K + 2 * K + 1 + P + i]; }
};

// Two-level media whose step operator has the optical-Bloch pattern (the
// host verifies it): A - I has non-zeros only at (0,0), (0,2), (1,1),
// (2,0), (2,2), the affine offset vanishes and the coupling has no (1)
// component.  Per cell: 7 rows of the per-cell table instead of 16.
template <typename real>
struct PrmBloch2 {
  static constexpr int K = 3, P = 1;
  real a00, a02, a11, a20, a22, w0c, w2c;
  const real *mb;
  __device__ __forceinline__ real kap(int q) const { return mb[K * K + 2 * K + 1 + q]; }
  __device__ __forceinline__ real zr(int i) const { return mb[K * K + 2 * K + 1 + P + i]; }
};

template <typename real, int N, bool KAHAN, class Prm>
__device__ __forceinline__ void bloch_accumulate(const Prm &q, const real (&u)[N * N - 1],
                                                 const real (&rx)[N * (N - 1)], real (&d)[N * N - 1],
                                                 real (&cc)[N * N - 1]);

// ------------------------------------------------- one cell's Bloch step
// delta^n -> delta^{n+1}; returns the coupling w . u + w0 and leaves the
// rotated deviation u (= v - x_ref) in `u`.
template <typename real, int N, bool KAHAN, class Prm, int ROT = ROT_INLINE>
__device__ __forceinline__ real bloch_step(const Prm &q, real e, real (&d)[N * N - 1],
                                           real (&cc)[N * N - 1], real (&u)[N * N - 1]) {
  constexpr int K = N * N - 1, P = N * (N - 1) / 2, NP = N - 1;
  real rx[2 * P];
#pragma unroll
  for (int i = 0; i < NP; ++i) u[i] = d[i];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    real s, cm1;
    sincos_m1_sel<ROT>(q.kap(p) * e, s, cm1);
    const int ia = NP + 2 * p, ib = ia + 1;
    const real xa = q.zr(2 * p) + d[ia];
    const real xb = q.zr(2 * p + 1) + d[ib];
    const real ra = cm1 * xa - s * xb;
    const real rb = s * xa + cm1 * xb;
    rx[2 * p] = ra;
    rx[2 * p + 1] = rb;
    u[ia] = d[ia] + ra;
    u[ib] = d[ib] + rb;
  }
  real pw = q.w0();
#pragma unroll
  for (int i = 0; i < K; ++i) pw += q.w(i) * u[i];
  bloch_accumulate<real, N, KAHAN>(q, u, rx, d, cc);
  return pw;
}

// delta += c + [0 | (R - 1) x] + (A - I) u   (compensated in FP32)
template <typename real, int N, bool KAHAN, class Prm>
__device__ __forceinline__ void bloch_accumulate(const Prm &q, const real (&u)[N * N - 1],
                                                 const real (&rx)[N * (N - 1)], real (&d)[N * N - 1],
                                                 real (&cc)[N * N - 1]) {
  constexpr int K = N * N - 1, NP = N - 1;
  if constexpr (K <= 15) {
#pragma unroll
    for (int i = 0; i < K; ++i) {
      real acc = q.c(i);
      if (i >= NP) acc += rx[i - NP];
#pragma unroll
      for (int j = 0; j < K; ++j) acc += q.am1(i, j) * u[j];
      if (KAHAN)
        kahan_add(d[i], cc[i], acc);
      else
        d[i] += acc;
    }
  } else {
    // large K: rows stay rolled (keeps code size and compile time bounded)
#pragma unroll 1
    for (int i = 0; i < K; ++i) {
      real acc = q.c(i);
      if (i >= NP) acc += rx[i - NP];
#pragma unroll 5
      for (int j = 0; j < K; ++j) acc += q.am1(i, j) * u[j];
      if (KAHAN)
        kahan_add(d[i], cc[i], acc);
      else
        d[i] += acc;
    }
  }
}

// bloch_step for the R cells of one lane that share one material block:
// every parameter is read once and applied to all R cells (per cell, the
// arithmetic and its order are those of bloch_step).  u[i][j] is cell j's
// rotated deviation, pw[j] its coupling w . u + w0.
// M contiguous values from a 16-byte aligned address, in 16-byte loads
template <typename real, int M>
__device__ __forceinline__ void ld_vec16(const real *p, real (&v)[M]) {
  constexpr int W = 16 / sizeof(real);
  static_assert(M % W == 0, "whole vectors only");
#pragma unroll
  for (int k = 0; k < M / W; ++k) {
    if constexpr (sizeof(real) == 4) {
      const float4 t = reinterpret_cast<const float4 *>(p)[k];
      v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
    } else {
      const double2 t = reinterpret_cast<const double2 *>(p)[k];
      v[2 * k] = t.x; v[2 * k + 1] = t.y;
    }
  }
}

template <typename real, int N, int R, bool KAHAN, int ROT = ROT_INLINE>
__device__ __forceinline__ void bloch_step_rows(const real *mb, const real (&e)[R], real (&d)[N * N - 1][R],
                                                real (&cc)[N * N - 1][R], real (&u)[N * N - 1][R],
                                                real (&pw)[R]) {
  constexpr int K = N * N - 1, P = N * (N - 1) / 2, NP = N - 1;
  static_assert(K <= 15, "rows are unrolled");
  // With K a multiple of 4 every row of the block starts on a 16-byte
  // boundary (the block stride is a multiple of 4 words), so the rows are
  // read as vectors: tail = w0 | kap[P] | zr[2P], padded to whole vectors.
  constexpr bool VEC = K % 4 == 0;
  constexpr int TL = VEC ? (1 + 3 * P + 3) / 4 * 4 : 1;
  const PrmBlock<real, N> q{mb};
  real tail[TL];
  if constexpr (VEC) ld_vec16<real, TL>(mb + K * K + 2 * K, tail);
  auto w0 = [&]() { if constexpr (VEC) return tail[0]; else return q.w0(); };
  auto kap = [&](int p) { if constexpr (VEC) return tail[1 + p]; else return q.kap(p); };
  auto zr = [&](int i) { if constexpr (VEC) return tail[1 + P + i]; else return q.zr(i); };
  real rx[2 * P][R];
#pragma unroll
  for (int i = 0; i < NP; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) u[i][j] = d[i][j];
#pragma unroll
  for (int p = 0; p < P; ++p) {
    const real kp = kap(p), za = zr(2 * p), zb = zr(2 * p + 1);
    const int ia = NP + 2 * p, ib = ia + 1;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      real s, cm1;
      sincos_m1_sel<ROT>(kp * e[j], s, cm1);
      const real xa = za + d[ia][j];
      const real xb = zb + d[ib][j];
      const real ra = cm1 * xa - s * xb;
      const real rb = s * xa + cm1 * xb;
      rx[2 * p][j] = ra;
      rx[2 * p + 1][j] = rb;
      u[ia][j] = d[ia][j] + ra;
      u[ib][j] = d[ib][j] + rb;
    }
  }
  {
    real wv[K];
    if constexpr (VEC) ld_vec16<real, K>(mb + K * K + K, wv);
    else
#pragma unroll
      for (int i = 0; i < K; ++i) wv[i] = q.w(i);
    const real w00 = w0();
#pragma unroll
    for (int j = 0; j < R; ++j) pw[j] = w00;
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) pw[j] += wv[i] * u[i][j];
  }
  real cv[K];
  if constexpr (VEC) ld_vec16<real, K>(mb + K * K, cv);
  else
#pragma unroll
    for (int i = 0; i < K; ++i) cv[i] = q.c(i);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    real row[K];
    if constexpr (VEC) ld_vec16<real, K>(mb + i * K, row);
    else
#pragma unroll
      for (int k = 0; k < K; ++k) row[k] = q.am1(i, k);
    real acc[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      acc[j] = cv[i];
      if (i >= NP) acc[j] += rx[i - NP][j];
    }
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
      for (int j = 0; j < R; ++j) acc[j] += row[k] * u[k][j];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      if (KAHAN)
        kahan_add(d[i][j], cc[i][j], acc[j]);
      else
        d[i][j] += acc[j];
    }
  }
}

// structured two-level step (same arithmetic as bloch_step restricted to the
// optical-Bloch pattern)
template <typename real, bool KAHAN, int ROT = ROT_INLINE>
__device__ __forceinline__ real bloch_step_b2(const PrmBloch2<real> &q, real e, real (&d)[3], real (&cc)[3],
                                              real (&u)[3]) {
  real s, cm1;
  sincos_m1_sel<ROT>(q.kap(0) * e, s, cm1);
  const real xa = q.zr(0) + d[1];
  const real xb = q.zr(1) + d[2];
  const real ra = cm1 * xa - s * xb;
  const real rb = s * xa + cm1 * xb;
  u[0] = d[0];
  u[1] = d[1] + ra;
  u[2] = d[2] + rb;
  const real pw = q.w0c * u[0] + q.w2c * u[2];
  const real a0 = q.a00 * u[0] + q.a02 * u[2];
  const real a1 = ra + q.a11 * u[1];
  const real a2 = rb + q.a20 * u[0] + q.a22 * u[2];
  if (KAHAN) {
    kahan_add(d[0], cc[0], a0);
    kahan_add(d[1], cc[1], a1);
    kahan_add(d[2], cc[2], a2);
  } else {
    d[0] += a0;
    d[1] += a1;
    d[2] += a2;
  }
  return pw;
}

// The structured two-level step with blocked accumulation (FP32 tiles): the
// deviation is d + acc, where d stays fixed for the whole tile and acc
// collects the tile's increments; the tile folds acc into d error-free at its
// end (the stored pair keeps the Kahan form d - c, c = -acc).  An increment
// rounds against |acc| (at most the tile's T increments) instead of against
// |d|: 3 additions per step instead of Kahan's 12, at the price of the 3
// additions that form d + acc.  x is the rotation angle (zero in vacuum
// cells, whose rows are zero).
template <int ROT>
__device__ __forceinline__ float bloch_step_b2_blocked(const PrmBloch2<float> &q, float x, const float (&d)[3],
                                                       float (&acc)[3], float (&u)[3]) {
  float s, cm1;
  sincos_m1_sel<ROT>(x, s, cm1);
  const float s1 = d[1] + acc[1];
  const float s2 = d[2] + acc[2];
  u[0] = d[0] + acc[0];
  const float xa = q.zr(0) + s1;
  const float xb = q.zr(1) + s2;
  const float ra = cm1 * xa - s * xb;
  const float rb = s * xa + cm1 * xb;
  u[1] = s1 + ra;
  u[2] = s2 + rb;
  const float pw = q.w0c * u[0] + q.w2c * u[2];
  acc[0] += q.a00 * u[0] + q.a02 * u[2];
  acc[1] += ra + q.a11 * u[1];
  acc[2] += rb + q.a20 * u[0] + q.a22 * u[2];
  return pw;
}

template <typename real, int N>
__device__ __forceinline__ real probe_rho(const real *coef, const real (&u)[N * N - 1]) {
  constexpr int K = N * N - 1;
  real v = coef[K];
#pragma unroll
  for (int i = 0; i < K; ++i) v += coef[i] * u[i];
  return v;
}

// ------------------------------------------------------------- fields
// FP64: a field value is one double.  FP32: a field value is an unevaluated
// pair hi + lo of floats (float-float), updated with error-free
// transformations: a single FP32 word rounds |E| ~ 1e9 V/m to ~100 V/m every
// step, and a high-Q resonant medium integrates those errors into its
// polarisation, so single-word FP32 fields drift by ~1e-3 relative within a
// few thousand steps while float-float fields track FP64 to ~1e-7.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
// (h, l) += (a, b), renormalised
__device__ __forceinline__ void ff_add(float &h, float &l, float a, float b) {
  float s, e;
  two_sum(h, a, s, e);
  e += l + b;
  h = s + e;
  l = e - (h - s);
}

// (h, l) += (a, b) without renormalising: h takes the rounded sum of the
// high words, l collects the exact rounding error and the low words, and the
// tiled kernels renormalise once per tile.  The pair stays exact, but between
// renormalisations l may hold a sizeable part of the value (the coupling and
// loss terms enter through b), so every product with the field must take
// h + l, not h alone.
__device__ __forceinline__ void ff_add_lazy(float &h, float &l, float a, float b) {
  float s, e;
  two_sum(h, a, s, e);
  l = e + (l + b);
  h = s;
}

__device__ __forceinline__ void ff_renorm(float &h, float &l) {
  const float s = h + l;
  l = l - (s - h);
  h = s;
}

// f += c (xr - xl) + extra   (extra: a small correction added to the low part)
template <typename real, bool LAZY = false>
__device__ __forceinline__ void fld_axpy_diff(real &fh, real &fl, real c, real xrh, real xrl, real xlh, real xll,
                                              real extra) {
  if constexpr (sizeof(real) == 8) {
    fh += c * (xrh - xlh) + extra;
  } else {
    float dh, de, ph, pe;
    two_sum(xrh, -xlh, dh, de);
    const float dl = de + (xrl - xll);
    two_prod(c, dh, ph, pe);
    if (LAZY)
      ff_add_lazy(fh, fl, ph, pe + c * dl + extra);
    else
      ff_add(fh, fl, ph, pe + c * dl + extra);
  }
}

// The same update for the tiles' per-step field updates, in fewer
// operations: the neighbour difference of the high words in one
// subtraction (exact when the two lie within a factor of 2 of each other,
// i.e. everywhere but near a zero crossing, where the values and so the
// rounding are small) and the sum of the field and its increment split into
// rounded sum and error by Fast2Sum (exact while |field| >= |increment|,
// again everywhere but near a zero crossing).  The pair stays exact up to
// those rare roundings at small values: a 1D pulse carried 12,000 steps on
// float-float fields this way stays within 1e-7 of FP64 (exact pairs: 1e-10,
// one FP32 word: 1e-4), for 10 instead of 19 operations per update.
template <typename real>
__device__ __forceinline__ void fld_axpy_diff_step(real &fh, real &fl, real c, real xrh, real xrl, real xlh,
                                                   real xll, real extra) {
  if constexpr (sizeof(real) == 8) {
    fh += c * (xrh - xlh) + extra;
  } else {
    const float dh = xrh - xlh;
    const float dl = xrl - xll;
    float ph, pe;
    two_prod(c, dh, ph, pe);
    const float s = fh + ph;
    const float e = ph - (s - fh);
    fl = e + (fl + fmaf(c, dl, pe + extra));
    fh = s;
  }
}

// f += (xr - xl) + extra: the unit-coefficient case (vacuum-like media at
// Courant number 1, where the FP32 coefficients round to exactly 1 and 0)
template <typename real, bool LAZY = false>
__device__ __forceinline__ void fld_add_diff(real &fh, real &fl, real xrh, real xrl, real xlh, real xll, real extra) {
  if constexpr (sizeof(real) == 8) {
    fh += (xrh - xlh) + extra;
  } else {
    float dh, de;
    two_sum(xrh, -xlh, dh, de);
    if (LAZY)
      ff_add_lazy(fh, fl, dh, de + (xrl - xll) + extra);
    else
      ff_add(fh, fl, dh, de + (xrl - xll) + extra);
  }
}

// source table entry n: FP64 [nt]; FP32 [2][nt] (hi row, lo row)
template <typename real>
__device__ __forceinline__ void src_val(const void *tab, long long n, long long nt, real &h, real &l) {
  const real *t = reinterpret_cast<const real *>(tab);
  h = t[n];
  l = sizeof(real) == 8 ? real(0) : t[nt + n];
}

template <typename real>
__device__ __forceinline__ void fld_add(real &fh, real &fl, real h, real l) {
  if constexpr (sizeof(real) == 8)
    fh += h;
  else
    ff_add(fh, fl, h, l);
}

template <typename real>
__device__ __forceinline__ real fld_val(real h, real l) {
  return sizeof(real) == 8 ? h : h + l;
}

// Partially reflecting end (reflectivity 0 < R < 1, amplitude reflection
// r = -sqrt R): the boundary cell holds (1 + r) M - r P = M + r (M - P) with
// M its first-order Mur value (in e) and P its field two steps back; at
// Courant number 1 in vacuum this sends back exactly r times the arriving wave.
template <typename real>
__device__ __forceinline__ void partial_reflect(real &eh, real &el, real r, real ph, real pl) {
  if constexpr (sizeof(real) == 8) {
    eh += r * (eh - ph);
  } else {
    float dh, de;
    two_sum(eh, -ph, dh, de);
    const float dl = de + (el - pl);
    float qh, qe;
    two_prod(r, dh, qh, qe);
    ff_add(eh, el, qh, qe + r * dl);
  }
}

template <typename real>
__device__ __forceinline__ real emc_at(const Args &a, int idx, int k) {
  return reinterpret_cast<const real *>(a.emc)[a.mat[idx] * 4 + k];
}

// ========================================================= plain path
// Launch A of step n: H on faces 1..nx-1 (in place), rho and d_t P per cell.
template <typename real, int N, bool KAHAN>
__global__ void k_plain_a(const Args a, long long n, int cur) {
  constexpr int K = N * N - 1;
  constexpr bool FF = sizeof(real) == 4;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.nx || *a.flags != 0) return;   // (a failed state check stops the solve)
  const int idx = a.off + m;
  const real *E = reinterpret_cast<const real *>(a.E[cur]);
  const real *El = reinterpret_cast<const real *>(a.El[cur]);
  real *H = reinterpret_cast<real *>(a.H[0]);
  real *Hl = reinterpret_cast<real *>(a.Hl[0]);
  const real e_here = fld_val<real>(E[idx], FF ? El[idx] : real(0));
  if (m >= 1) {
    real hh = H[idx], hl = FF ? Hl[idx] : real(0);
    fld_axpy_diff<real>(hh, hl, emc_at<real>(a, idx, 2), E[idx], FF ? El[idx] : real(0), E[idx - 1],
                        FF ? El[idx - 1] : real(0), real(0));
    for (int s = 0; s < a.n_src; ++s)
      if (a.src[s].face == m) {
        real sh, sl;
        src_val<real>(a.src[s].sH, n, a.nt, sh, sl);
        fld_add<real>(hh, hl, sh, sl);
      }
    H[idx] = hh;
    if (FF) Hl[idx] = hl;
  }
  real *pd = reinterpret_cast<real *>(a.pd);
  const int slot = a.qslot[a.mat[idx]];
  if (slot < 0) {
    pd[idx] = real(0);
    return;
  }
  real *D = reinterpret_cast<real *>(a.D[0]);
  real *Cc = reinterpret_cast<real *>(a.C[0]);
  real d[K], cc[K], u[K];
#pragma unroll
  for (int i = 0; i < K; ++i) {
    d[i] = D[(size_t)i * a.ld + idx];
    cc[i] = KAHAN ? Cc[(size_t)i * a.ld + idx] : real(0);
  }
  const real *mb = reinterpret_cast<const real *>(a.qpar) + (size_t)slot * a.qstride;
  real pw;
  if (a.pcell) {
    PrmCell<real, N> q{reinterpret_cast<const real *>(a.pcell) + idx, a.ld, mb};
    pw = bloch_step<real, N, KAHAN>(q, e_here, d, cc, u);
  } else {
    PrmBlock<real, N> q{mb};
    pw = bloch_step<real, N, KAHAN>(q, e_here, d, cc, u);
  }
#pragma unroll
  for (int i = 0; i < K; ++i) {
    D[(size_t)i * a.ld + idx] = d[i];
    if (KAHAN) Cc[(size_t)i * a.ld + idx] = cc[i];
  }
  pd[idx] = pw;
  for (int p = 0; p < a.n_probe; ++p)
    if (a.pr_cell[p] == m && a.pr_q[p] >= 2)
      reinterpret_cast<real *>(a.rec)[(size_t)p * a.nt + n] =
          probe_rho<real, N>(reinterpret_cast<const real *>(a.pr_coef) + (size_t)p * (K + 1), u);
}

// E^{n+1} of cell m (before boundary conditions): returns (h, l)
template <typename real>
__device__ __forceinline__ void e_update(const Args &a, int cur, const real *pd, int m, long long n, real &eh,
                                         real &el) {
  constexpr bool FF = sizeof(real) == 4;
  const int idx = a.off + m;
  const real *E = reinterpret_cast<const real *>(a.E[cur]);
  const real *Elo = reinterpret_cast<const real *>(a.El[cur]);
  const real *H = reinterpret_cast<const real *>(a.H[0]);
  const real *Hlo = reinterpret_cast<const real *>(a.Hl[0]);
  eh = E[idx];
  el = FF ? Elo[idx] : real(0);
  const real extra = emc_at<real>(a, idx, 0) * eh - pd[idx];   // (a' - 1) E - coupling
  fld_axpy_diff<real>(eh, el, emc_at<real>(a, idx, 1), H[idx + 1], FF ? Hlo[idx + 1] : real(0), H[idx],
                      FF ? Hlo[idx] : real(0), extra);
  for (int s = 0; s < a.n_src; ++s)
    if (a.src[s].cell == m) {
      real vh, vl;
      src_val<real>(a.src[s].sE, n, a.nt, vh, vl);
      if (a.src[s].kind == 2) {
        eh = vh;
        el = vl;
      } else {
        fld_add<real>(eh, el, vh, vl);
      }
    }
}

// Launch B of step n: E^{n+1} into buffers cur ^ 1, sources, boundaries, records.
template <typename real>
__global__ void k_plain_b(const Args a, long long n, int cur) {
  constexpr bool FF = sizeof(real) == 4;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= a.nx || *a.flags != 0) return;   // (a failed state check stops the solve)
  const int idx = a.off + m;
  const real *E = reinterpret_cast<const real *>(a.E[cur]);
  const real *Elo = reinterpret_cast<const real *>(a.El[cur]);
  real *En = reinterpret_cast<real *>(a.E[cur ^ 1]);
  real *Eln = reinterpret_cast<real *>(a.El[cur ^ 1]);
  const real *pd = reinterpret_cast<const real *>(a.pd);
  real eh, el;
  e_update<real>(a, cur, pd, m, n, eh, el);
  const bool left = m == 0, right = m == a.nx - 1;
  if (left || right) {
    const int nb = left ? 1 : m - 1;            // interior neighbour
    if ((left ? a.bc_l : a.bc_r) == 1) {
      eh = el = real(0);
    } else {
      real nh, nl;                              // neighbour's E^{n+1}
      e_update<real>(a, cur, pd, nb, n, nh, nl);
      // E_b^{n+1} = E_nb^n + k (E_nb^{n+1} - E_b^n)
      eh = E[a.off + nb];
      el = FF ? Elo[a.off + nb] : real(0);
      fld_axpy_diff<real>(eh, el, real(left ? a.kmur_l : a.kmur_r), nh, nl, E[idx], FF ? Elo[idx] : real(0),
                          real(0));
      if ((left ? a.bc_l : a.bc_r) == 2)   // E_b^{n-1}: this thread's output cell still holds it
        partial_reflect<real>(eh, el, real(left ? a.r_l : a.r_r), En[idx], FF ? Eln[idx] : real(0));
    }
  }
  En[idx] = eh;
  if (FF) Eln[idx] = el;
  const real *H = reinterpret_cast<const real *>(a.H[0]);
  const real *Hlo = reinterpret_cast<const real *>(a.Hl[0]);
  for (int p = 0; p < a.n_probe; ++p)
    if (a.pr_cell[p] == m && a.pr_q[p] < 2)
      reinterpret_cast<real *>(a.rec)[(size_t)p * a.nt + n] =
          a.pr_q[p] == 0 ? fld_val<real>(eh, el) : fld_val<real>(H[idx], FF ? Hlo[idx] : real(0));
}

// ========================================================= tiled path
template <typename real, int R>
__device__ __forceinline__ void ld_row(const real *p, real (&v)[R]) {
#pragma unroll
  for (int j = 0; j < R; ++j) v[j] = p[j];
}
template <>
__device__ __forceinline__ void ld_row<float, 4>(const float *p, float (&v)[4]) {
  const float4 t = *reinterpret_cast<const float4 *>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
template <>
__device__ __forceinline__ void ld_row<float, 2>(const float *p, float (&v)[2]) {
  const float2 t = *reinterpret_cast<const float2 *>(p);
  v[0] = t.x; v[1] = t.y;
}
template <>
__device__ __forceinline__ void ld_row<double, 2>(const double *p, double (&v)[2]) {
  const double2 t = *reinterpret_cast<const double2 *>(p);
  v[0] = t.x; v[1] = t.y;
}
template <>
__device__ __forceinline__ void ld_row<double, 4>(const double *p, double (&v)[4]) {
  const double2 t = reinterpret_cast<const double2 *>(p)[0];
  const double2 u = reinterpret_cast<const double2 *>(p)[1];
  v[0] = t.x; v[1] = t.y; v[2] = u.x; v[3] = u.y;
}
template <typename real, int R>
__device__ __forceinline__ void st_row(real *p, const real (&v)[R]) {
#pragma unroll
  for (int j = 0; j < R; ++j) p[j] = v[j];
}
template <>
__device__ __forceinline__ void st_row<float, 4>(float *p, const float (&v)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
template <>
__device__ __forceinline__ void st_row<float, 2>(float *p, const float (&v)[2]) {
  *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}
template <>
__device__ __forceinline__ void st_row<double, 2>(double *p, const double (&v)[2]) {
  *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}
template <>
__device__ __forceinline__ void st_row<double, 4>(double *p, const double (&v)[4]) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
}

// The probes whose cell a tile owns, in probe order, built by warp 0 (one
// probe per lane, compacted by ballot): key_of(cell) is the key stored for an
// owned cell (its cell or tile row) and -1 otherwise; s_key[i] | s_pq[i] =
// key | probe index + 256 quantity, ended by key -1 unless MAXPROBE are here.
template <class KeyOf>
__device__ __forceinline__ void build_probe_list(const Args &a, KeyOf key_of, int *s_key, int *s_pq) {
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  int np = 0;
  for (int b = 0; b < a.n_probe; b += 32) {
    const int p = b + lane;
    const int cell = p < a.n_probe ? a.pr_cell[p] : 0, q = p < a.n_probe ? a.pr_q[p] : 0;
    const int key = p < a.n_probe ? key_of(cell) : -1;
    const unsigned m = __ballot_sync(FULL, key >= 0);
    if (key >= 0) {
      const int i = np + __popc(m & ((1u << lane) - 1u));
      s_key[i] = key;
      s_pq[i] = p + 256 * q;
    }
    np += __popc(m);
  }
  if (lane == 0 && np < MAXPROBE) s_key[np] = -1;
}

// rho probes of one lane's probe cells (mask pmask over its R cells g0 ..):
// the rotated deviations parked in s_u, the list of build_probe_list (keyed
// by cell).  Out of line: only lanes that hold a probe call it, and its
// registers stay out of the step's allocation.
template <typename real, int N, int R>
static __device__ __noinline__ void rho_probes_lane(const int *s_plc, const int *s_plp, const real *s_u, int g0,
                                                    unsigned pmask, const real *pcoef, real *rec, long long nt,
                                                    long long n) {
  constexpr int K = N * N - 1;
  for (int j = 0; j < R; ++j)
    if (pmask & (1u << j)) {
      real u[K];
#pragma unroll
      for (int i = 0; i < K; ++i) u[i] = s_u[j * K + i];
      for (int k = 0; k < MAXPROBE && s_plc[k] >= 0; ++k)
        if (s_plc[k] == g0 + j && s_plp[k] >= 512) {
          const int p = s_plp[k] & 255;
          rec[(size_t)p * nt + n] = probe_rho<real, N>(pcoef + (size_t)p * (K + 1), u);
        }
    }
}

// Block tile b owns cells [b*own, (b+1)*own), own = 32 W R - 2 T (W warps);
// lane l of warp w holds cells tb + (32 w + l) R .. + R - 1 with tb = b*own - T
// (the tile holding the last cell may start 4 or 8 cells earlier).  Reads
// buffers `cur`, writes the owned cells of buffers cur ^ 1.
//   PM = 0: step operator of the lane's medium from shared memory;
//   PM = 1: dense per-cell step operator rows in registers (jittered media);
//   PM = 2: structured two-level per-cell rows in registers (see PrmBloch2).
// The time loop has no per-cell branches: cells are interleaved by the
// scheduler only inside one basic block, so vacuum cells run the Bloch step
// with a zero field angle and a zero coupling instead of being skipped.
template <typename real, int N, int R, bool KAHAN, int PM>
__device__ __forceinline__ void tile_body(const Args &a, const int tile, long long n0, int nsteps, int T, int cur,
                                          unsigned char *smem_raw) {
  if (*a.flags != 0) return;   // a state check failed: the solve stops (the whole block leaves together)
  constexpr int K = N * N - 1;
  constexpr bool FF = sizeof(real) == 4;
  constexpr bool PERCELL = PM == 1;
  // FP32 structured two-level rows: blocked accumulation of the deviation
  // (bloch_step_b2_blocked); cc holds acc = -c while the tile runs
  constexpr bool BLK = FF && KAHAN && PM == 2;
  static_assert(PM != 2 || N == 2, "structured rows are two-level");
  // the probes of this tile's owned cells (build_probe_list, keyed by cell),
  // at a fixed offset, so that a probe lane's step reads a short list
  // instead of every probe, through constant shared-memory addresses
  int *s_plc = reinterpret_cast<int *>(smem_raw);
  int *s_plp = s_plc + MAXPROBE;
  real *s_emc = reinterpret_cast<real *>(smem_raw + 2 * MAXPROBE * sizeof(int));
  real *s_q = s_emc + a.n_mat_all * 4;
  int *s_slot = reinterpret_cast<int *>(s_q + a.n_slot * a.qstride);
  for (int i = threadIdx.x; i < a.n_mat_all * 4; i += blockDim.x) s_emc[i] = reinterpret_cast<const real *>(a.emc)[i];
  for (int i = threadIdx.x; i < a.n_slot * a.qstride; i += blockDim.x) s_q[i] = reinterpret_cast<const real *>(a.qpar)[i];
  for (int i = threadIdx.x; i < a.n_mat_all; i += blockDim.x) s_slot[i] = a.qslot[i];
  __syncthreads();
  // this thread's slot for the rotated state of its probe cells, then the
  // warp-edge exchange slots [warp][E hi, E lo, H hi, H lo]
  real *s_ub = reinterpret_cast<real *>(reinterpret_cast<unsigned char *>(s_slot) +
                                        ((sizeof(int) * a.n_mat_all + 15) / 16) * 16);
  real *s_u = s_ub + (size_t)threadIdx.x * R * K;
  constexpr int TW = TileGeom<N>::W;            // warps per block
  real *s_x = s_ub + (size_t)32 * TW * R * K;

  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  constexpr int SPAN = 32 * R;                  // cells per warp
  constexpr int TSPAN = TW * SPAN;              // cells per tile
  const int own = TSPAN - 2 * T;
  const int c_own = tile * own;
  if (c_own >= a.nx) return;   // the whole block leaves together
  // The absorbing right end reads its neighbour's new E (first-order Mur), a
  // dependency one cell beyond the stencil's light cone: the neighbour must
  // stay valid for all T steps (so the last cell may not be the tile's first
  // owned cell) and be held by the same warp (so the last cell may not start
  // a warp).  The tile that owns the last cell starts 4 (or 8) cells earlier
  // when either would happen; T <= 32 R - 12 keeps its owned cells inside.
  int tb = c_own - T;
  if (a.nx - 1 < c_own + own) {
    if (a.nx - 1 == c_own || (a.nx - 1 - tb) % SPAN == 0) tb -= 4;
    if ((a.nx - 1 - tb) % SPAN == 0) tb -= 4;
  }
  const int lo = c_own - tb;                    // tile position of the first owned cell
  const int ti0 = wib * SPAN + lane * R;        // tile position of this lane's first cell
  const int g0 = tb + ti0;                      // first cell of this lane
  const int base = a.off + g0;                  // its array index (>= 0, multiple of R)

  real E[R], El[R], H[R], Hl[R];
  real d[K][R], cc[K][R];
  ld_row<real, R>(reinterpret_cast<const real *>(a.E[cur]) + base, E);
  ld_row<real, R>(reinterpret_cast<const real *>(a.H[cur]) + base, H);
  if (FF) {
    ld_row<real, R>(reinterpret_cast<const real *>(a.El[cur]) + base, El);
    ld_row<real, R>(reinterpret_cast<const real *>(a.Hl[cur]) + base, Hl);
  } else {
#pragma unroll
    for (int j = 0; j < R; ++j) El[j] = Hl[j] = real(0);
  }
  const real *Din = reinterpret_cast<const real *>(a.D[cur]);
  const real *Cin = reinterpret_cast<const real *>(a.C[cur]);
#pragma unroll
  for (int i = 0; i < K; ++i) {
    ld_row<real, R>(Din + (size_t)i * a.ld + base, d[i]);
    if (KAHAN) ld_row<real, R>(Cin + (size_t)i * a.ld + base, cc[i]);
    else
#pragma unroll
      for (int j = 0; j < R; ++j) cc[i][j] = real(0);
    if constexpr (BLK)
#pragma unroll
      for (int j = 0; j < R; ++j) cc[i][j] = -cc[i][j];
  }
  // field coefficients per cell (pad cells outside the grid have zeros)
  real ca[R], cb[R], ch[R], mk[R];
  unsigned med = 0;
  int slot = -1;
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int mt = a.mat[base + j];
    ca[j] = s_emc[mt * 4 + 0];
    cb[j] = s_emc[mt * 4 + 1];
    ch[j] = (g0 + j == 0) ? real(0) : s_emc[mt * 4 + 2];   // face 0 is a fixed boundary slot
    const int sl = s_slot[mt];
    mk[j] = sl >= 0 ? real(1) : real(0);
    if (sl >= 0) {
      med |= 1u << j;
      slot = sl;
    }
  }
  const bool warp_med = __any_sync(FULL, med != 0);
  const real *mb = s_q + (slot < 0 ? 0 : slot) * a.qstride;
  // largest |angle| per unit field of the lane's medium: an FP32 two-level
  // step whose warp keeps every |angle| <= 1/2 takes the Taylor-only rotation
  real kap_max = real(0);
  if (slot >= 0)
#pragma unroll
    for (int q = 0; q < N * (N - 1) / 2; ++q) kap_max = fmax(kap_max, fabs(PrmBlock<real, N>{mb}.kap(q)));

  PrmReg<real, N> pr[PERCELL ? R : 1];
  if (PERCELL) {
    const real *pc = reinterpret_cast<const real *>(a.pcell);
#pragma unroll
    for (int j = 0; j < (PERCELL ? R : 1); ++j) {
      pr[j].mb = mb;
#pragma unroll
      for (int i = 0; i < K * K; ++i) pr[j].a[i] = pc[(size_t)i * a.ld + base + j];
#pragma unroll
      for (int i = 0; i < K; ++i) {
        pr[j].cc[i] = pc[(size_t)(K * K + i) * a.ld + base + j];
        pr[j].ww[i] = pc[(size_t)(K * K + K + i) * a.ld + base + j];
      }
      pr[j].ww0 = pc[(size_t)(K * K + 2 * K) * a.ld + base + j];
    }
  }
  PrmBloch2<real> b2[PM == 2 ? R : 1];
  if constexpr (PM == 2) {
    const real *pc = reinterpret_cast<const real *>(a.pcell2);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      b2[j].mb = mb;
      b2[j].a00 = pc[(size_t)0 * a.ld + base + j];
      b2[j].a02 = pc[(size_t)1 * a.ld + base + j];
      b2[j].a11 = pc[(size_t)2 * a.ld + base + j];
      b2[j].a20 = pc[(size_t)3 * a.ld + base + j];
      b2[j].a22 = pc[(size_t)4 * a.ld + base + j];
      b2[j].w0c = pc[(size_t)5 * a.ld + base + j];
      b2[j].w2c = pc[(size_t)6 * a.ld + base + j];
    }
  }
  // rotation angle per unit field of each cell (zero in vacuum cells)
  real kc[BLK ? R : 1];
  if constexpr (BLK)
#pragma unroll
    for (int j = 0; j < R; ++j) kc[j] = mk[j] * b2[j].kap(0);
  // warp-uniform: does the tile touch a source, a boundary cell, a probe?
  const int t_lo = tb + wib * SPAN, t_hi = t_lo + SPAN;   // this warp's cells [t_lo, t_hi)
  bool any_src = false;
  for (int s = 0; s < a.n_src; ++s)
    any_src |= (a.src[s].cell >= t_lo && a.src[s].cell < t_hi) || (a.src[s].face >= t_lo && a.src[s].face < t_hi);
  const bool any_bnd = (t_lo <= 0 && 0 < t_hi) || (t_lo <= a.nx - 1 && a.nx - 1 < t_hi);
  // owned cells of this lane (T, lo and own are multiples of R)
  const bool owned = ti0 >= lo && ti0 < lo + own && ti0 < TSPAN - T;
  build_probe_list(a, [&](int c) {
    const int ti = c - tb;   // tile position of the probe cell
    return ti >= lo && ti < lo + own && ti < TSPAN - T ? c : -1;
  }, s_plc, s_plp);
  real *rec = reinterpret_cast<real *>(a.rec);
  const real *pcoef = reinterpret_cast<const real *>(a.pr_coef);

  // E_b^{n-1} of the two ends (partially reflecting ends), from the previous launch
  real pvl_h = real(0), pvl_l = real(0), pvr_h = real(0), pvr_l = real(0);
  if (any_bnd) {
    const real *bp = reinterpret_cast<const real *>(a.bprev[cur]);
    pvl_h = bp[0];
    pvl_l = bp[1];
    pvr_h = bp[2];
    pvr_l = bp[3];
  }

  // E of each warp's last cell, for the next warp's first face
  if (lane == 31) {
    s_x[wib * 4 + 0] = E[R - 1];
    s_x[wib * 4 + 1] = El[R - 1];
  }
  __syncthreads();
  unsigned pmask = 0;   // this lane's probe cells
  for (int k = 0; k < MAXPROBE && s_plc[k] >= 0; ++k) {
    const int j = s_plc[k] - g0;
    if (j >= 0 && j < R) pmask |= 1u << j;
  }
  const bool any_probe = __any_sync(FULL, pmask != 0);

#pragma unroll 1
  for (int t = 0; t < nsteps; ++t) {
    const long long n = n0 + t;
    // ---- H^{n+1/2} on the left faces of my cells (in place)
    {
      real elh = __shfl_up_sync(FULL, E[R - 1], 1);
      real ell = FF ? __shfl_up_sync(FULL, El[R - 1], 1) : real(0);
      if (lane == 0 && wib > 0) {
        elh = s_x[(wib - 1) * 4 + 0];
        ell = s_x[(wib - 1) * 4 + 1];
      }
      // no extra term: -0 (x + -0 == x for every x, so the addition drops
      // out at compile time; x + +0 would not, as -0 + +0 == +0)
#pragma unroll
      for (int j = R - 1; j >= 0; --j)
        fld_axpy_diff_step<real>(H[j], Hl[j], ch[j], E[j], El[j], j ? E[j - 1] : elh, j ? El[j - 1] : ell, real(-0.0));
    }
    if (any_src) {
      for (int s = 0; s < a.n_src; ++s) {
        const int f = a.src[s].face - g0;
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (f == j) {
            real vh, vl;
            src_val<real>(a.src[s].sH, n, a.nt, vh, vl);
            fld_add<real>(H[j], Hl[j], vh, vl);
          }
      }
    }
    // H of each warp's first face, for the previous warp's last cell
    if (lane == 0) {
      s_x[wib * 4 + 2] = H[0];
      s_x[wib * 4 + 3] = Hl[0];
    }
    // ---- rho^{n+1/2} and the coupling term (all cells of a warp that holds
    // any medium; vacuum cells see a zero angle and contribute no current)
    real pw[R];
#pragma unroll
    for (int j = 0; j < R; ++j) pw[j] = real(0);
    // one instantiation per rotation form (see sincos_m1_sel) and per
    // probe form (PARK: the warp holds a probe cell, whose rotated state is
    // parked in shared memory; the other warps carry no stores for it)
    auto bloch = [&](auto rot_tag, auto park_tag) {
      constexpr int ROT = decltype(rot_tag)::value;
      constexpr bool PARK = decltype(park_tag)::value;
      real ej[R];   // the field of medium cells (BLK: the rotation angle)
#pragma unroll
      for (int j = 0; j < R; ++j) ej[j] = fld_val<real>(E[j], El[j]) * (BLK ? kc[BLK ? j : 0] : mk[j]);
      if constexpr (PM == 0) {
        real u[K][R];
        bloch_step_rows<real, N, R, KAHAN, ROT>(mb, ej, d, cc, u, pw);
#pragma unroll
        for (int j = 0; j < R; ++j) {
          pw[j] *= mk[j];
          if (PARK && (pmask & (1u << j)))   // park u of probe cells (predicated stores)
#pragma unroll
            for (int i = 0; i < K; ++i) s_u[j * K + i] = u[i][j];
        }
      } else if constexpr (BLK) {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          float dj[3], aj[3], u[3];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            dj[i] = d[i][j];
            aj[i] = cc[i][j];
          }
          pw[j] = bloch_step_b2_blocked<ROT>(b2[j], ej[j], dj, aj, u);
#pragma unroll
          for (int i = 0; i < 3; ++i) cc[i][j] = aj[i];
          if (PARK && (pmask & (1u << j)))
#pragma unroll
            for (int i = 0; i < 3; ++i) s_u[j * 3 + i] = u[i];
        }
      } else {
#pragma unroll
        for (int j = 0; j < R; ++j) {
          real dj[K], cj[K], u[K];
#pragma unroll
          for (int i = 0; i < K; ++i) {
            dj[i] = d[i][j];
            cj[i] = cc[i][j];
          }
          real q;
          if constexpr (PM == 2)
            q = bloch_step_b2<real, KAHAN, ROT>(b2[j], ej[j], dj, cj, u);
          else
            q = bloch_step<real, N, KAHAN, PrmReg<real, N>, ROT>(pr[PERCELL ? j : 0], ej[j], dj, cj, u);
          pw[j] = q * mk[j];
#pragma unroll
          for (int i = 0; i < K; ++i) {
            d[i][j] = dj[i];
            cc[i][j] = cj[i];
          }
          if (PARK && (pmask & (1u << j)))   // park u of probe cells (predicated stores)
#pragma unroll
            for (int i = 0; i < K; ++i) s_u[j * K + i] = u[i];
        }
      }
    };
    // FP32 two-level tiles: the Taylor-only form unless a field in the warp
    // is strong enough for an angle beyond 1/2 (measured: 3.5 % faster than
    // the library path inline at every angle; the three-level tiles run
    // faster with that single form)
    if (warp_med) {
      using rot_inline = std::integral_constant<int, ROT_INLINE>;
      using rot_taylor = std::integral_constant<int, ROT_TAYLOR>;
      if constexpr (FF && N == 2) {
        real e_max = real(0);   // largest |angle| (BLK) or |field| of the lane's medium cells
#pragma unroll
        for (int j = 0; j < R; ++j)
          e_max = fmax(e_max, fabs(fld_val<real>(E[j], El[j]) * (BLK ? kc[BLK ? j : 0] : mk[j])));
        const bool wide = __any_sync(FULL, (BLK ? e_max : e_max * kap_max) > real(0.5));
        if (any_probe) {
          if (wide) bloch(rot_inline{}, std::true_type{});
          else bloch(rot_taylor{}, std::true_type{});
        } else {
          if (wide) bloch(rot_inline{}, std::false_type{});
          else bloch(rot_taylor{}, std::false_type{});
        }
      } else {
        if (any_probe) bloch(rot_inline{}, std::true_type{});
        else bloch(rot_inline{}, std::false_type{});
      }
    }
    if (warp_med) {
      if (any_probe && pmask) rho_probes_lane<real, N, R>(s_plc, s_plp, s_u, g0, pmask, pcoef, rec, a.nt, n);
    }
    // ---- boundary cells: keep E^n of the boundary cell and its neighbour
    real bo_h = real(0), bo_l = real(0), no_h = real(0), no_l = real(0);
    if (any_bnd) {
      const real r_oh = __shfl_down_sync(FULL, E[0], 1), r_ol = __shfl_down_sync(FULL, El[0], 1);
      const real l_oh = __shfl_up_sync(FULL, E[R - 1], 1), l_ol = __shfl_up_sync(FULL, El[R - 1], 1);
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (g0 + j == 0) {
          bo_h = E[j];
          bo_l = El[j];
          no_h = j < R - 1 ? E[j + 1] : r_oh;
          no_l = j < R - 1 ? El[j + 1] : r_ol;
        }
        if (g0 + j == a.nx - 1) {
          bo_h = E[j];
          bo_l = El[j];
          no_h = j ? E[j - 1] : l_oh;
          no_l = j ? El[j - 1] : l_ol;
        }
      }
    }
    __syncthreads();   // H of the warp edges published
    // ---- E^{n+1} (in place)
    {
      real hrh = __shfl_down_sync(FULL, H[0], 1);
      real hrl = FF ? __shfl_down_sync(FULL, Hl[0], 1) : real(0);
      if (lane == 31 && wib < TW - 1) {
        hrh = s_x[(wib + 1) * 4 + 2];
        hrl = s_x[(wib + 1) * 4 + 3];
      }
#pragma unroll
      for (int j = 0; j < R; ++j)
        fld_axpy_diff_step<real>(E[j], El[j], cb[j], j < R - 1 ? H[j + 1] : hrh, j < R - 1 ? Hl[j + 1] : hrl, H[j],
                                  Hl[j], ca[j] * fld_val<real>(E[j], El[j]) - pw[j]);
    }
    if (any_src) {
      for (int s = 0; s < a.n_src; ++s) {
        const int c = a.src[s].cell - g0;
#pragma unroll
        for (int j = 0; j < R; ++j)
          if (c == j) {
            real vh, vl;
            src_val<real>(a.src[s].sE, n, a.nt, vh, vl);
            if (a.src[s].kind == 2) {
              E[j] = vh;
              El[j] = vl;
            } else {
              fld_add<real>(E[j], El[j], vh, vl);
            }
          }
      }
    }
    if (any_bnd) {
      // E_b^{n+1} = E_nb^n + k (E_nb^{n+1} - E_b^n), or 0 for a mirror
      const real r_nh = __shfl_down_sync(FULL, E[0], 1), r_nl = __shfl_down_sync(FULL, El[0], 1);
      const real l_nh = __shfl_up_sync(FULL, E[R - 1], 1), l_nl = __shfl_up_sync(FULL, El[R - 1], 1);
      real Bh[R], Bl[R];
#pragma unroll
      for (int j = 0; j < R; ++j) {
        Bh[j] = E[j];
        Bl[j] = El[j];
        const bool lft = g0 + j == 0, rgt = g0 + j == a.nx - 1;
        if (lft || rgt) {
          const real nh = lft ? (j < R - 1 ? E[j + 1] : r_nh) : (j ? E[j - 1] : l_nh);
          const real nl = lft ? (j < R - 1 ? El[j + 1] : r_nl) : (j ? El[j - 1] : l_nl);
          const int bc = lft ? a.bc_l : a.bc_r;
          if (bc == 1) {
            Bh[j] = Bl[j] = real(0);
          } else {
            Bh[j] = no_h;
            Bl[j] = no_l;
            fld_axpy_diff<real>(Bh[j], Bl[j], real(lft ? a.kmur_l : a.kmur_r), nh, nl, bo_h, bo_l, real(0));
            if (bc == 2) partial_reflect<real>(Bh[j], Bl[j], real(lft ? a.r_l : a.r_r), lft ? pvl_h : pvr_h,
                                               lft ? pvl_l : pvr_l);
          }
          if (lft) {   // E_b^n becomes the next step's E_b^{n-1}
            pvl_h = bo_h;
            pvl_l = bo_l;
          } else {
            pvr_h = bo_h;
            pvr_l = bo_l;
          }
        }
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        E[j] = Bh[j];
        El[j] = Bl[j];
      }
    }
    if (any_probe && pmask) {
#pragma unroll
      for (int j = 0; j < R; ++j)
        if (pmask & (1u << j))
          for (int k = 0; k < MAXPROBE && s_plc[k] >= 0; ++k)
            if (s_plc[k] == g0 + j && s_plp[k] < 512) {
              const int p = s_plp[k] & 255;
              rec[(size_t)p * a.nt + n] = s_plp[k] < 256 ? fld_val<real>(E[j], El[j]) : fld_val<real>(H[j], Hl[j]);
            }
    }
    if (lane == 31) {
      s_x[wib * 4 + 0] = E[R - 1];
      s_x[wib * 4 + 1] = El[R - 1];
    }
    __syncthreads();   // E of the warp edges published
  }

  // ---- write back the owned cells (never past the last cell)
  if (!owned) return;
  if (any_bnd) {   // E_b^{n-1} for the next launch, by the owners of the end cells
    real *bp = reinterpret_cast<real *>(a.bprev[cur ^ 1]);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      if (g0 + j == 0) {
        bp[0] = pvl_h;
        bp[1] = pvl_l;
      }
      if (g0 + j == a.nx - 1) {
        bp[2] = pvr_h;
        bp[3] = pvr_l;
      }
    }
  }
  if constexpr (FF) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      ff_renorm(E[j], El[j]);
      ff_renorm(H[j], Hl[j]);
    }
  }
  if constexpr (BLK) {   // d + acc -> the Kahan pair (s, -e) of its exact sum
#pragma unroll
    for (int i = 0; i < K; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) {
        float sm, er;
        two_sum(d[i][j], cc[i][j], sm, er);
        d[i][j] = sm;
        cc[i][j] = -er;
      }
  }
  real *Eo = reinterpret_cast<real *>(a.E[cur ^ 1]);
  real *Ho = reinterpret_cast<real *>(a.H[cur ^ 1]);
  real *Elo = reinterpret_cast<real *>(a.El[cur ^ 1]);
  real *Hlo = reinterpret_cast<real *>(a.Hl[cur ^ 1]);
  real *Do = reinterpret_cast<real *>(a.D[cur ^ 1]);
  real *Co = reinterpret_cast<real *>(a.C[cur ^ 1]);
  if (g0 + R <= a.nx) {
    st_row<real, R>(Eo + base, E);
    st_row<real, R>(Ho + base, H);
    if (FF) {
      st_row<real, R>(Elo + base, El);
      st_row<real, R>(Hlo + base, Hl);
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      st_row<real, R>(Do + (size_t)i * a.ld + base, d[i]);
      if (KAHAN) st_row<real, R>(Co + (size_t)i * a.ld + base, cc[i]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (g0 + j < a.nx) {
        Eo[base + j] = E[j];
        Ho[base + j] = H[j];
        if (FF) {
          Elo[base + j] = El[j];
          Hlo[base + j] = Hl[j];
        }
#pragma unroll
        for (int i = 0; i < K; ++i) {
          Do[(size_t)i * a.ld + base + j] = d[i][j];
          if (KAHAN) Co[(size_t)i * a.ld + base + j] = cc[i][j];
        }
      }
  }
}

// Blocks that must fit on one SM at a time (caps the registers): the FP32
// kernels run fastest with 2 (three levels, 8 warps) or 4 (two levels, 4
// warps, shared or structured rows) resident blocks (measured).
template <typename real, int N, int PM>
constexpr int tiled_min_blocks() { return sizeof(real) != 4 ? 1 : N == 3 ? 2 : PM != 1 ? 4 : 1; }

// One simulation: block b advances tile b.
template <typename real, int N, int R, bool KAHAN, int PM>
__global__ void __launch_bounds__(32 * TileGeom<N>::W, tiled_min_blocks<real, N, PM>()) k_tiled(const __grid_constant__ Args a, long long n0, int nsteps, int T, int cur) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  tile_body<real, N, R, KAHAN, PM>(a, blockIdx.x, n0, nsteps, T, cur, smem_raw);
}

// A batch of simulations in one launch: block b advances tile tasks[b].y of
// simulation tasks[b].x.  Every simulation starts at step 0, so
// step n0 is common; finished simulations return at once.
template <typename real, int N, int R, bool KAHAN, int PM>
__global__ void __launch_bounds__(32 * TileGeom<N>::W, tiled_min_blocks<real, N, PM>()) k_tiled_batch(const Args *__restrict__ args, const int2 *__restrict__ tasks,
                                                     long long n0, int T, int cur) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 tk = tasks[blockIdx.x];
  const Args &a = args[tk.x];
  if (n0 >= a.nt) return;   // the whole block leaves together
  const int nsteps = (int)(a.nt - n0 < (long long)T ? a.nt - n0 : (long long)T);
  tile_body<real, N, R, KAHAN, PM>(a, tk.y, n0, nsteps, T, cur, smem_raw);
}


// ========================================================= state check
// Number of negative pivots of the LDL^H factorisation of A - sigma I (no
// pivoting): by Sylvester's law of inertia, the number of eigenvalues of the
// Hermitian A below sigma.  Pivots within 1e-14 of zero (relative to the
// scale of A) count as negative, so that no pivot divides by ~0.
template <int N>
__device__ __forceinline__ int ldl_neg_count(const double (&re)[N][N], const double (&im)[N][N], double sigma,
                                             double scale) {
  double lr[N][N], li[N][N], d[N];
  int neg = 0;
  for (int k = 0; k < N; ++k) {
    double s = re[k][k] - sigma;
    for (int j = 0; j < k; ++j) s -= (lr[k][j] * lr[k][j] + li[k][j] * li[k][j]) * d[j];
    if (fabs(s) < 1e-14 * scale) s = -1e-14 * scale;
    d[k] = s;
    neg += s < 0.0;
    for (int i = k + 1; i < N; ++i) {
      // l_ik = (a_ik - sum_j l_ij conj(l_kj) d_j) / d_k
      double ar = re[i][k], ai = im[i][k];
      for (int j = 0; j < k; ++j) {
        ar -= (lr[i][j] * lr[k][j] + li[i][j] * li[k][j]) * d[j];
        ai -= (li[i][j] * lr[k][j] - lr[i][j] * li[k][j]) * d[j];
      }
      lr[i][k] = ar / s;
      li[i][k] = ai / s;
    }
  }
  return neg;
}

// Smallest eigenvalue of the Hermitian matrix re + i im by bisection between
// the Gershgorin lower bound and the smallest diagonal entry.
template <int N>
__device__ double min_eig_bisect(const double (&re)[N][N], const double (&im)[N][N]) {
  double lo = 1e300, hi = 1e300, scale = 0.0;
  for (int i = 0; i < N; ++i) {
    double r = 0.0;
    for (int j = 0; j < N; ++j)
      if (j != i) r += hypot(re[i][j], im[i][j]);
    lo = fmin(lo, re[i][i] - r);
    hi = fmin(hi, re[i][i]);
    scale = fmax(scale, fabs(re[i][i]) + r);
  }
  if (!(scale > 0.0)) return hi;
  for (int it = 0; it < 64 && hi - lo > 1e-15 * scale; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (ldl_neg_count<N>(re, im, mid, scale) >= 1)
      hi = mid;
    else
      lo = mid;
  }
  return hi;
}

// For each listed cell, rebuild the stored density matrix x (FP64, true
// value delta - compensation, reference state zref[slot][N*N] in full real
// coordinates), and report its trace deviation and smallest eigenvalue
// (inertia bisection above).  Non-finite values of the state or of the
// cell's fields (both ping-pong buffers) set bit 0 of flags[0].
template <typename real, int N>
__global__ void k_check(const Args a, int cur, const int *cells, int n_cells, double *min_eig,
                        double *tr_dev, const double *zref) {
  constexpr int K = N * N - 1, NP = N - 1;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n_cells) return;
  const int m = cells[k];
  const int idx = a.off + m;
  const int slot = a.qslot[a.mat[idx]];
  if (slot < 0) {
    min_eig[k] = 1.0;
    tr_dev[k] = 0.0;
    return;
  }
  zref += (size_t)slot * N * N;
  const real *D = reinterpret_cast<const real *>(a.D[cur]);
  const real *Cc = reinterpret_cast<const real *>(a.C[cur]);
  double y[N * N];
  double popsum = 0.0;
  bool finite = true;
  for (int i = 0; i < K; ++i) {
    double v = (double)D[(size_t)i * a.ld + idx];
    if (a.prec == 1) v -= (double)Cc[(size_t)i * a.ld + idx];
    finite &= isfinite(v);
    const int fi = i < NP ? i : i + 1;
    y[fi] = zref[fi] + v;
    if (i < NP) popsum += v;
  }
  y[NP] = zref[NP] - popsum;
  double re[N][N], im[N][N];
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) re[i][j] = im[i][j] = 0.0;
  double tr = 0.0;
  for (int i = 0; i < N; ++i) {
    re[i][i] = y[i];
    tr += y[i];
  }
  int q = 0;
  for (int i = 0; i < N; ++i)
    for (int j = i + 1; j < N; ++j, ++q) {
      re[i][j] = re[j][i] = y[N + 2 * q];
      im[i][j] = y[N + 2 * q + 1];
      im[j][i] = -y[N + 2 * q + 1];
    }
  double mn = min_eig_bisect<N>(re, im);
  {
    const real *E = reinterpret_cast<const real *>(a.E[0]), *E1 = reinterpret_cast<const real *>(a.E[1]);
    const real *H = reinterpret_cast<const real *>(a.H[0]), *H1 = reinterpret_cast<const real *>(a.H[1]);
    finite &= isfinite((double)E[idx]) && isfinite((double)E1[idx]) && isfinite((double)H[idx]) &&
              isfinite((double)H1[idx]);
  }
  if (!finite || !isfinite(mn)) {
    atomicOr(a.flags, 1);
    mn = -1e300;
  } else if (mn < -EIG_TOL) {
    atomicOr(a.flags, 2);
  }
  min_eig[k] = mn;
  tr_dev[k] = fabs(tr - 1.0);
}

// ========================================================= periodic sweep
// One cell of the periodic sweep.  The splitting of Sec. 2.2 keeps rho a
// density matrix, and so is the stored state x = exp(L0 dt/2) rho: a
// non-finite field or state value sets flags[0] bit 0; a population of x or
// a 2 x 2 principal minor x_jj x_kk - |x_jk|^2 (dipole eigenbasis) below
// -tol sets bit 1 (necessary conditions for positivity, cheap enough for
// every cell; the sampled check above bisects the smallest eigenvalue).  In
// FP32 the compensated pair (delta, c) of each component, whose value is
// delta - c, is folded in FP64 into the canonical pair (round(v), round(v) -
// v rounded) of that value.
template <typename real, int N>
__device__ __forceinline__ void sweep_cell(const Args &a, int m, int dcur, int ecur, int hcur, double tol) {
  constexpr int K = N * N - 1, NP = N - 1;
  const int idx = a.off + m;
  bool finite = isfinite((double)reinterpret_cast<const real *>(a.E[ecur])[idx]) &&
                isfinite((double)reinterpret_cast<const real *>(a.H[hcur])[idx]);
  if (a.prec == 1)
    finite = finite && isfinite((double)reinterpret_cast<const real *>(a.El[ecur])[idx]) &&
             isfinite((double)reinterpret_cast<const real *>(a.Hl[hcur])[idx]);
  const int slot = a.qslot[a.mat[idx]];
  if (slot >= 0) {
    real *D = reinterpret_cast<real *>(a.D[dcur]);
    real *Cc = reinterpret_cast<real *>(a.C[dcur]);
    const double *z = a.zref + (size_t)slot * N * N;
    double y[N * N];
    double popsum = 0.0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
      const size_t at = (size_t)i * a.ld + idx;
      double v = (double)D[at];
      if (a.prec == 1) {
        v -= (double)Cc[at];
        if (isfinite(v)) {
          const real hi = (real)v;
          D[at] = hi;
          Cc[at] = (real)((double)hi - v);
        }
      }
      finite = finite && isfinite(v);
      const int fi = i < NP ? i : i + 1;
      y[fi] = z[fi] + v;
      if (i < NP) popsum += v;
    }
    y[NP] = z[NP] - popsum;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < N; ++j) ok = ok && y[j] >= -tol;
    int q = 0;
#pragma unroll
    for (int j = 0; j < N; ++j)
#pragma unroll
      for (int k = j + 1; k < N; ++k, ++q) {
        const double re = y[N + 2 * q], im = y[N + 2 * q + 1];
        ok = ok && fma(y[j], y[k], -(re * re + im * im)) >= -tol;
      }
    if (finite && !ok) atomicOr(a.flags, 2);
  }
  if (!finite) atomicOr(a.flags, 1);
}

template <typename real, int N>
__global__ void k_sweep(const Args a, int dcur, int ecur, int hcur, double tol) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < a.nx) sweep_cell<real, N>(a, m, dcur, ecur, hcur, tol);
}

// block b sweeps the owned cells of tile tasks[b].y of simulation tasks[b].x
// if that simulation ran the round from step n0
template <typename real, int N>
__global__ void k_sweep_batch(const Args *__restrict__ args, const int2 *__restrict__ tasks, int own,
                              long long n0, int cur, double tol) {
  const int2 tk = tasks[blockIdx.x];
  const Args &a = args[tk.x];
  if (a.nt <= n0) return;
  const int c0 = tk.y * own, c1 = min(c0 + own, a.nx);
  for (int m = c0 + (int)threadIdx.x; m < c1; m += blockDim.x) sweep_cell<real, N>(a, m, cur, cur, cur, tol);
}

template <typename real, int N>
int sweep_impl(const Args &a, int dcur, int ecur, int hcur, double tol, cudaStream_t st) {
  const int bs = 256, gs = (a.nx + bs - 1) / bs;
  k_sweep<real, N><<<gs, bs, 0, st>>>(a, dcur, ecur, hcur, tol);
  return (int)cudaGetLastError();
}

template <typename real, int N>
int sweep_batch_impl(const Args *args, const int2 *tasks, int n_tasks, int own, long long n0, int cur, double tol,
                     cudaStream_t st) {
  if (n_tasks <= 0) return 0;
  k_sweep_batch<real, N><<<n_tasks, 128, 0, st>>>(args, tasks, own, n0, cur, tol);
  return (int)cudaGetLastError();
}

template <typename real, int N, bool KAHAN>
int plain_step_impl(const Args &a, long long n, int cur, cudaStream_t st) {
  const int bs = 256, gs = (a.nx + bs - 1) / bs;
  k_plain_a<real, N, KAHAN><<<gs, bs, 0, st>>>(a, n, cur);
  k_plain_b<real><<<gs, bs, 0, st>>>(a, n, cur);
  return (int)cudaGetLastError();
}

// dynamic shared memory of a tiled block: tables + per-thread probe slots
template <typename real, int N, int R>
size_t tiled_smem(int n_mat_all, int n_slot, int qstride) {
  return sizeof(real) * (n_mat_all * 4 + n_slot * qstride) + ((sizeof(int) * n_mat_all + 15) / 16) * 16 +
         sizeof(real) * ((size_t)32 * TileGeom<N>::W * R * (N * N - 1) + 4 * TileGeom<N>::W) + 16 +
         sizeof(int) * 2 * MAXPROBE;
}

template <typename real, int N, int R, bool KAHAN, int PM>
int tiled_impl(const Args &a, long long n0, int nsteps, int T, int cur, cudaStream_t st) {
  constexpr int TW = TileGeom<N>::W;
  static_assert(32 * TW * R - 5 <= PAD, "a tile reaches past the pad cells");
  const int own = 32 * TW * R - 2 * T;
  const int gs = (a.nx + own - 1) / own;
  const size_t sm = tiled_smem<real, N, R>(a.n_mat_all, a.n_slot, a.qstride);
  k_tiled<real, N, R, KAHAN, PM><<<gs, 32 * TW, sm, st>>>(a, n0, nsteps, T, cur);
  return (int)cudaGetLastError();
}

template <typename real, int N, int R, bool KAHAN, int PM>
int tiled_batch_impl(const Args *args, const int2 *tasks, int n_tasks, size_t smem, long long n0, int T, int cur,
                     cudaStream_t st) {
  if (n_tasks <= 0) return 0;
  k_tiled_batch<real, N, R, KAHAN, PM><<<n_tasks, 32 * TileGeom<N>::W, smem, st>>>(args, tasks, n0, T, cur);
  return (int)cudaGetLastError();
}

template <typename real, int N>
int check_impl(const Args &a, int cur, const int *cells, int n_cells, double *mn, double *tr, const double *z,
               cudaStream_t st) {
  const int bs = 128, gs = (n_cells + bs - 1) / bs;
  k_check<real, N><<<gs, bs, 0, st>>>(a, cur, cells, n_cells, mn, tr, z);
  return (int)cudaGetLastError();
}

}  // namespace dev
}  // namespace mbs
