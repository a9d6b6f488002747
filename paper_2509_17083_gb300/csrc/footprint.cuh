// Opacity-aware footprint of a projected Gaussian: the tiles of its
// rectangle that it can show in. Eq. 1 skips a pixel where
// alpha = o exp(-q / 2) < 1/255, q = d^T Sigma'^-1 d, so nothing of the
// Gaussian shows where q > 2 ln(255 o). Per tile row of the rectangle, the
// binning keeps the tile columns whose pixel-centre box meets the ellipse
// q <= t, t = 1.02 x 2 ln(255 o) + 0.05 (the margin sits far above FP32
// rounding, so every tile dropped has alpha well below 1/255 at each of its
// pixels: the image is that of the whole rectangle).
//
// The projection counts these tiles (ntiles) and the instance expansion
// emits them; both call the functions below, which use correctly rounded
// FP32 operations in a fixed order (the _rn intrinsics are never fused into
// multiply-adds, whatever the unit's compile flags), so their decisions
// agree with each other and with the oracle's FP32 replay bit for bit.
#pragma once
#include "common.cuh"

namespace hyrf {

// t for opacity o; -1 when o < 1/255 (no footprint). ln x = e ln 2 + ln m
// for x = m 2^e, m in [1, 2), and ln m = 2 atanh(s), s = (m - 1) / (m + 1),
// by its series to s^9 (Abramowitz & Stegun 4.1.27; truncation < 2e-6).
__device__ __forceinline__ float fp_qlimit(float o) {
  if (!(o >= 1.0f / 255.0f)) return -1.0f;
  const float x = __fmul_rn(255.0f, o);  // >= 1
  const uint32_t u = __float_as_uint(x);
  const int e = (int)((u >> 23) & 0xffu) - 127;
  const float m = __uint_as_float((u & 0x7fffffu) | 0x3f800000u);
  const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float pz = 1.0f / 9.0f;
  pz = __fadd_rn(__fmul_rn(pz, s2), 1.0f / 7.0f);
  pz = __fadd_rn(__fmul_rn(pz, s2), 1.0f / 5.0f);
  pz = __fadd_rn(__fmul_rn(pz, s2), 1.0f / 3.0f);
  pz = __fadd_rn(__fmul_rn(pz, s2), 1.0f);
  const float ln = __fadd_rn(__fmul_rn((float)e, 0.693147180559945f), __fmul_rn(__fmul_rn(2.0f, s), pz));
  return __fadd_rn(__fmul_rn(1.02f, __fmul_rn(2.0f, ln)), 0.05f);
}

// Footprint record of a projected Gaussian: three float4 (48 bytes). The
// first holds Sigma' (a, b, c) and t; the other two hold the row spans,
// packed when the rectangle has at most kSpanRows rows and at most 255
// columns (fp_packed): row j's 16-bit field (word j / 2, bits 16 (j % 2)
// on) is its first tile column minus x0 in the low byte and its span length
// in the high byte; unpacked records leave these words zero and their spans
// are recomputed from the first float4.
constexpr int kFootVec = 3;     // float4 per record
constexpr int kSpanRows = 16;   // rows of packed spans

__host__ __device__ __forceinline__ bool fp_packed(int rows, int cols) {
  return rows <= kSpanRows && cols <= 255;
}

// Per-Gaussian constants of the row spans: the ellipse's half-height
// hy = sqrt(t c), the slope k = b / c of its centre line, mm = a - b k, its
// half-width hx = sqrt(t a) and the height yr = b sqrt(t / a) of its
// rightmost point.
struct FootRows {
  float hy, k, mm, hx, yr;
};

__device__ __forceinline__ FootRows fp_rows(float a, float b, float c, float t) {
  FootRows f;
  f.hy = __fsqrt_rn(__fmul_rn(t, c));
  f.k = __fdiv_rn(b, c);
  f.mm = fmaxf(__fsub_rn(a, __fmul_rn(b, f.k)), 0.0f);
  f.hx = __fsqrt_rn(__fmul_rn(t, a));
  f.yr = __fmul_rn(b, __fsqrt_rn(__fdiv_rn(t, a)));
  return f;
}

// Tile columns [tx0, tx1) of tile row ty, within [cx0, cx1), whose pixel
// centres (16 tx + 0.5 ... 16 tx + 15.5) meet the ellipse
// {(u, v) + d : d^T Sigma'^-1 d <= t}, Sigma' = [[a, b], [b, c]] (f from
// fp_rows). Cut to the row's pixel-centre strip, the ellipse spans x in
// [u + xmin, u + xmax]: its boundary at height dy is
// x = (b / c) dy +- sqrt((a - b^2 / c)(t - dy^2 / c)) and its extremes
// +-sqrt(t a) lie at dy = +-b sqrt(t / a). t = +inf: the whole row of the
// rectangle; t < 0: nothing.
__device__ __forceinline__ void fp_row_span(const FootRows& f, float u, float v, float c, float t, int ty,
                                            int cx0, int cx1, int& tx0, int& tx1) {
  tx0 = tx1 = cx0;
  if (!(t >= 0.0f)) return;
  if (isinf(t)) {
    tx1 = cx1;
    return;
  }
  const float tw = (float)kTile;
  const float Y0 = __fadd_rn((float)(ty * kTile), 0.5f);
  const float Y1 = __fadd_rn(Y0, __fsub_rn(tw, 1.0f));
  const float dy0 = __fsub_rn(Y0, v), dy1 = __fsub_rn(Y1, v);
  const float ya = fmaxf(dy0, -f.hy), yb = fminf(dy1, f.hy);
  if (!(ya <= yb)) return;
  const float wa = __fsqrt_rn(fmaxf(__fmul_rn(f.mm, __fsub_rn(t, __fdiv_rn(__fmul_rn(ya, ya), c))), 0.0f));
  const float wb = __fsqrt_rn(fmaxf(__fmul_rn(f.mm, __fsub_rn(t, __fdiv_rn(__fmul_rn(yb, yb), c))), 0.0f));
  const float kya = __fmul_rn(f.k, ya), kyb = __fmul_rn(f.k, yb);
  const float xmax = (f.yr >= ya && f.yr <= yb) ? f.hx : fmaxf(__fadd_rn(kya, wa), __fadd_rn(kyb, wb));
  const float xmin = (-f.yr >= ya && -f.yr <= yb) ? -f.hx : fminf(__fsub_rn(kya, wa), __fsub_rn(kyb, wb));
  // x / tw for the power-of-two tile width: the product by 1 / tw rounds the
  // same real number, so it equals the quotient bit for bit
  const float itw = 1.0f / (float)kTile;
  static_assert((kTile & (kTile - 1)) == 0, "tile width must be a power of two");
  float f0 = ceilf(__fmul_rn(__fsub_rn(__fadd_rn(u, xmin), __fsub_rn(tw, 0.5f)), itw));
  float f1 = __fadd_rn(floorf(__fmul_rn(__fsub_rn(__fadd_rn(u, xmax), 0.5f), itw)), 1.0f);
  f0 = fminf(fmaxf(f0, (float)cx0), (float)cx1);
  f1 = fminf(fmaxf(f1, (float)cx0), (float)cx1);
  if (f1 > f0) {
    tx0 = (int)f0;
    tx1 = (int)f1;
  }
}

}  // namespace hyrf
