// beta_internal.cuh -- device-side definitions shared by the CUDA translation
// units of the Beta rasterizer (sm_103a).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "beta_splat.h"

namespace beta {

constexpr int kThreads = 256;     // raster CTA: one 16x16 tile, one pixel per thread
constexpr int kGrad2d = 10;       // 2D gradient sums per record (see beta_raster.cu)
constexpr int kGrad2dStride = 12; // floats per record slot: 48 bytes, 16-byte aligned for vector atomics
constexpr int kRecordF4 = 3;      // raster record: 3 x float4 = 48 bytes

// Raster record of one (view, primitive), 48 bytes:
//   f4[0] = (mx_int, my_int, off_x, off_y)  centre mu' = mx_int + 0.5 - off_x
//   f4[1] = (p, q1, q2, beta)               whitening: u = p dx, v = q2 dx + q1 dy, r^2 = u^2 + v^2
//   f4[2] = (log2 o, c_r, c_g, c_b)
// Pixel (x, y) has dx = (x - mx_int) + off_x, which is exact up to one rounding.
// The support r^2 < 1 spans |dx| <= 1/p and |dy| <= sqrt(p^2 + q2^2) / (p q1).

struct ViewDev {
  float R[9];
  float t[3];
  float fx, fy, cx, cy, near_plane;
  float campos[3];
  float bg[3];
  int32_t width, height, ntx, nty;
  int32_t tile_off;
  int32_t pad0;
  int64_t pix_off;
};

struct ViewTable {
  int32_t n_views;
  int32_t total_tiles;
  int64_t total_pixels;
  ViewDev v[BETA_MAX_VIEWS];
};

struct RenderOpts {
  float t_eps, alpha_max, blur_eps, b_lo, b_hi;
  int32_t color_mode;
  int32_t tile_w, tile_h, batch_s;
};

// status helpers -------------------------------------------------------------
__device__ __forceinline__ void set_status(int32_t* st, int32_t code) {
  if (st) atomicCAS(st, 0, code);
}

// view lookup for a global tile id (binary search over the view table)
__device__ __forceinline__ int view_of_tile(const ViewTable& vt, int g) {
  int lo = 0, hi = vt.n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (vt.v[mid].tile_off <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Rule B1 (tile rectangle) and rule D (depth key): fixed fp32 operation
// sequences, every operation rounded to nearest, no contraction.  The same
// written rule is implemented independently by the CPU oracle; tile
// assignment and key order must agree bit for bit.
// ---------------------------------------------------------------------------

// exp in fp32 by Cody-Waite reduction and a degree-7 Taylor polynomial
// (Horner with fused multiply-adds): x in [-80, 80].  ln 2 is split into a
// high part with trailing zero bits (n * LN2_HI is exact for |n| < 2^12) and
// the remainder; the two fp32 values are the single-precision split that
// fdlibm's public expf uses.  The polynomial coefficients are 1/k!.
__device__ __forceinline__ float rule_exp(float x) {
  const float LOG2E = 1.44269504f;
  const float LN2_HI = 0.693145751953125f;
  const float LN2_LO = 1.42860677e-06f;
  float tt = __fmul_rn(x, LOG2E);
  float n = rintf(tt);
  float nh = __fmul_rn(n, LN2_HI);
  float nl = __fmul_rn(n, LN2_LO);
  float r = __fsub_rn(x, nh);
  r = __fsub_rn(r, nl);
  float p = 1.98412698e-04f;
  p = __fmaf_rn(p, r, 1.38888889e-03f);
  p = __fmaf_rn(p, r, 8.33333333e-03f);
  p = __fmaf_rn(p, r, 4.16666667e-02f);
  p = __fmaf_rn(p, r, 1.66666667e-01f);
  p = __fmaf_rn(p, r, 0.5f);
  p = __fmaf_rn(p, r, 1.0f);
  p = __fmaf_rn(p, r, 1.0f);
  int e = (int)n + 127;
  float scale = __int_as_float(e << 23);
  return __fmul_rn(p, scale);
}

// dot of three products, summed left to right, each step rounded
__device__ __forceinline__ float rn_dot3(float a0, float b0, float a1, float b1, float a2, float b2) {
  float s = __fadd_rn(__fmul_rn(a0, b0), __fmul_rn(a1, b1));
  return __fadd_rn(s, __fmul_rn(a2, b2));
}

// View-independent part of the rule chain: scales, normalised quaternion and
// its rotation matrix.
struct PrimGeo {
  float mu[3], s[3], q[4];   // q normalised
  float Rq[9];               // rotation of q
  float qn;                  // |q|
};

// Per-view part of the rule chain.
struct ViewGeo {
  float A[9];                // W Rq
  float tc[3];               // camera-space centre (rule D)
  float iz, j00, j11, j02, j12;
  float M0[3], M1[3];        // M = J W Rq S (2 x 3)
  float sxx, syy;            // diagonal of Sigma' (blur included)
  float pxc, pyc;            // projected centre (rule B1's fp32 value)
};

// Rule chain, view-independent part.  Returns false if the primitive is
// culled in every view (log-scale out of [-80, 80] or a zero quaternion).
__device__ __forceinline__ bool rule_prim(const float* p, PrimGeo& g) {
  g.mu[0] = p[0]; g.mu[1] = p[1]; g.mu[2] = p[2];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    float l = p[3 + k];
    if (!(l >= -80.0f && l <= 80.0f)) return false;
    g.s[k] = rule_exp(l);
  }
  float qw = p[6], qx = p[7], qy = p[8], qz = p[9];
  float qq = __fmul_rn(qw, qw);
  qq = __fadd_rn(qq, __fmul_rn(qx, qx));
  qq = __fadd_rn(qq, __fmul_rn(qy, qy));
  qq = __fadd_rn(qq, __fmul_rn(qz, qz));
  if (!(qq > 0.0f)) return false;
  float sq = __fsqrt_rn(qq);
  g.qn = sq;
  float rn = __fdiv_rn(1.0f, sq);
  float w = __fmul_rn(qw, rn), x = __fmul_rn(qx, rn), y = __fmul_rn(qy, rn), z = __fmul_rn(qz, rn);
  g.q[0] = w; g.q[1] = x; g.q[2] = y; g.q[3] = z;
  float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
  float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
  float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
  g.Rq[0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
  g.Rq[1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
  g.Rq[2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
  g.Rq[3] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
  g.Rq[4] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
  g.Rq[5] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
  g.Rq[6] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
  g.Rq[7] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
  g.Rq[8] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));
  return true;
}

// Camera-space centre and depth key (rule D).  Returns false at or behind
// the near plane.
__device__ __forceinline__ bool rule_depth(const PrimGeo& pg, const ViewDev& V, ViewGeo& g,
                                           uint32_t& key) {
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float s = __fadd_rn(__fmul_rn(V.R[r * 3 + 0], pg.mu[0]), __fmul_rn(V.R[r * 3 + 1], pg.mu[1]));
    s = __fadd_rn(s, __fmul_rn(V.R[r * 3 + 2], pg.mu[2]));
    g.tc[r] = __fadd_rn(s, V.t[r]);
  }
  key = __float_as_uint(g.tc[2]);
  return g.tc[2] > V.near_plane;
}

// Rule chain, per-view part after rule_depth: J, M, diagonal of Sigma' and
// the tile rectangle.  Returns false if the rectangle is empty.
__device__ __forceinline__ bool rule_view(const PrimGeo& pg, const ViewDev& V, float blur,
                                          int tile_shift_w, int tile_shift_h, ViewGeo& g,
                                          int rect[4]) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      g.A[r * 3 + c] = rn_dot3(V.R[r * 3 + 0], pg.Rq[0 * 3 + c], V.R[r * 3 + 1], pg.Rq[1 * 3 + c],
                               V.R[r * 3 + 2], pg.Rq[2 * 3 + c]);
  g.iz = __fdiv_rn(1.0f, g.tc[2]);
  g.j00 = __fmul_rn(V.fx, g.iz);
  g.j11 = __fmul_rn(V.fy, g.iz);
  g.j02 = -__fmul_rn(__fmul_rn(g.j00, g.tc[0]), g.iz);
  g.j12 = -__fmul_rn(__fmul_rn(g.j11, g.tc[1]), g.iz);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g.M0[c] = __fmul_rn(__fadd_rn(__fmul_rn(g.j00, g.A[0 * 3 + c]), __fmul_rn(g.j02, g.A[2 * 3 + c])), pg.s[c]);
    g.M1[c] = __fmul_rn(__fadd_rn(__fmul_rn(g.j11, g.A[1 * 3 + c]), __fmul_rn(g.j12, g.A[2 * 3 + c])), pg.s[c]);
  }
  float sxx = __fmul_rn(g.M0[0], g.M0[0]);
  sxx = __fadd_rn(sxx, __fmul_rn(g.M0[1], g.M0[1]));
  sxx = __fadd_rn(sxx, __fmul_rn(g.M0[2], g.M0[2]));
  sxx = __fadd_rn(sxx, blur);
  float syy = __fmul_rn(g.M1[0], g.M1[0]);
  syy = __fadd_rn(syy, __fmul_rn(g.M1[1], g.M1[1]));
  syy = __fadd_rn(syy, __fmul_rn(g.M1[2], g.M1[2]));
  syy = __fadd_rn(syy, blur);
  g.sxx = sxx;
  g.syy = syy;
  const float INFL = 1.000244140625f;  // 1 + 2^-12
  const float PAD = 0.015625f;         // 2^-6 pixel
  float ex = __fadd_rn(__fmul_rn(__fsqrt_rn(sxx), INFL), PAD);
  float ey = __fadd_rn(__fmul_rn(__fsqrt_rn(syy), INFL), PAD);
  float pxc = __fadd_rn(__fmul_rn(g.j00, g.tc[0]), V.cx);
  float pyc = __fadd_rn(__fmul_rn(g.j11, g.tc[1]), V.cy);
  g.pxc = pxc;
  g.pyc = pyc;
  float lox = __fsub_rn(__fsub_rn(pxc, ex), 0.5f), hix = __fsub_rn(__fadd_rn(pxc, ex), 0.5f);
  float loy = __fsub_rn(__fsub_rn(pyc, ey), 0.5f), hiy = __fsub_rn(__fadd_rn(pyc, ey), 0.5f);
  if (!(isfinite(lox) && isfinite(hix) && isfinite(loy) && isfinite(hiy))) return false;
  float i0 = __fadd_rn(floorf(lox), 1.0f), i1 = __fsub_rn(ceilf(hix), 1.0f);
  float j0 = __fadd_rn(floorf(loy), 1.0f), j1 = __fsub_rn(ceilf(hiy), 1.0f);
  if (i0 < 0.0f) i0 = 0.0f;
  if (j0 < 0.0f) j0 = 0.0f;
  float wm1 = (float)(V.width - 1), hm1 = (float)(V.height - 1);
  if (i1 > wm1) i1 = wm1;
  if (j1 > hm1) j1 = hm1;
  if (i0 > i1 || j0 > j1) return false;
  // pixel index / tile size for power-of-two tiles (indices are >= 0 here)
  rect[0] = (int)i0 >> tile_shift_w;
  rect[1] = (int)i1 >> tile_shift_w;
  rect[2] = (int)j0 >> tile_shift_h;
  rect[3] = (int)j1 >> tile_shift_h;
  return true;
}

// a*b - c*d with Kahan's fused multiply-add algorithm (one rounding error)
__device__ __forceinline__ float rule_dop(float a, float b, float c, float d) {
  const float w = __fmul_rn(c, d);
  const float e = __fmaf_rn(-c, d, w);
  const float f = __fmaf_rn(a, b, -w);
  return __fadd_rn(f, e);
}

// Rule B2: the tiles of the rule B1 rectangle that the support ellipse
// reaches (Sec. 3.1, Eq. 2: the Beta kernel is exactly zero outside r^2 < 1).
// For every tile row, the band of its pixel-centre rows (widened by PAD) is
// cut with the ellipse of Sigma' inflated by INFL: its x-range over the band
// is the whole half-width when the ellipse's rightmost (leftmost) point lies
// in the band, else the boundary at the band end nearest that point,
//   x = (b / c) y +- sqrt(K2 (det / c) max(0, 1 - y^2 (1 / (K2 c)))),  K2 = INFL^2,
// with a = sxx, c = syy (blur included), b = M0 . M1 and
// det = |M0 x M1|^2 + blur (a + c - blur) (minors by Kahan's algorithm).  The
// columns whose centres lie in that range widened by PAD give the row's
// tiles.  fp32, every operation rounded to nearest, in the order written (the
// oracle implements the same written rule).  The rule applies to rectangles
// of at least 2 x 2 and at most 32 tiles (one tile wide or high, a rectangle
// loses a tile only where an image edge cuts the ellipse); the others, and
// degenerate ellipses, keep every tile.  Returns the kept tiles as bit
// r w + q for tile (tx0 + q, ty0 + r) of a w x h rectangle (w h <= 32),
// 0xFFFFFFFF for larger rectangles.
__device__ __forceinline__ uint32_t rule_all_tiles(const int rect[4]) {
  const int wh = (rect[1] - rect[0] + 1) * (rect[3] - rect[2] + 1);
  return wh >= 32 ? 0xFFFFFFFFu : (1u << wh) - 1u;
}
// Does rule B2 apply to the rectangle (at least 2 x 2 and at most 32 tiles)?
__device__ __forceinline__ bool rule_tiles_apply(const int rect[4]) {
  const int w = rect[1] - rect[0] + 1, h = rect[3] - rect[2] + 1;
  return w >= 2 && h >= 2 && w * h <= 32;
}
__device__ __forceinline__ uint32_t rule_tiles(const ViewGeo& g, const ViewDev& V, float blur, int tile_shift_w,
                                               int tile_h, const int rect[4]) {
  const int w = rect[1] - rect[0] + 1, h = rect[3] - rect[2] + 1;
  if (w * h > 32) return 0xFFFFFFFFu;
  const uint32_t all = rule_all_tiles(rect);
  if (w < 2 || h < 2) return all;
  if (!(g.sxx > 0.0f && g.syy > 0.0f)) return all;
  const float INFL = 1.000244140625f;  // 1 + 2^-12
  const float PAD = 0.015625f;         // 2^-6 pixel
  const float b = rn_dot3(g.M0[0], g.M1[0], g.M0[1], g.M1[1], g.M0[2], g.M1[2]);
  const float m01 = rule_dop(g.M0[0], g.M1[1], g.M0[1], g.M1[0]);
  const float m02 = rule_dop(g.M0[0], g.M1[2], g.M0[2], g.M1[0]);
  const float m12 = rule_dop(g.M0[1], g.M1[2], g.M0[2], g.M1[1]);
  float det = __fmul_rn(m01, m01);
  det = __fadd_rn(det, __fmul_rn(m02, m02));
  det = __fadd_rn(det, __fmul_rn(m12, m12));
  det = __fadd_rn(det, __fmul_rn(blur, __fsub_rn(__fadd_rn(g.sxx, g.syy), blur)));
  const float sa = __fsqrt_rn(g.sxx), sc = __fsqrt_rn(g.syy);
  const float xfull = __fmul_rn(sa, INFL);
  const float ytop = __fmul_rn(sc, INFL);
  const float ystar = __fdiv_rn(__fmul_rn(b, INFL), sa);
  const float slope = __fdiv_rn(b, g.syy);
  const float K2 = __fmul_rn(INFL, INFL);
  const float hh = __fmul_rn(__fdiv_rn(det, g.syy), K2);
  const float cc = __fmul_rn(g.syy, K2);
  const float icc = __fdiv_rn(1.0f, cc);
  if (!(isfinite(ystar) && isfinite(slope) && isfinite(hh) && isfinite(icc) && cc > 0.0f)) return all;
  uint32_t mask = 0u;
  for (int r = 0; r < h; ++r) {
    const int y0 = (rect[2] + r) * tile_h;
    const int y1 = min(y0 + tile_h - 1, V.height - 1);
    float ya = __fsub_rn(__fsub_rn(__fadd_rn((float)y0, 0.5f), PAD), g.pyc);
    float yb = __fsub_rn(__fadd_rn(__fadd_rn((float)y1, 0.5f), PAD), g.pyc);
    if (ya < -ytop) ya = -ytop;
    if (yb > ytop) yb = ytop;
    if (!(ya <= yb)) continue;
    const bool in_r = (ya <= ystar) && (ystar <= yb);
    const bool in_l = (ya <= -ystar) && (-ystar <= yb);
    const float yr = ystar < ya ? ya : yb;     // band end nearest the rightmost point
    const float yl = -ystar < ya ? ya : yb;    // band end nearest the leftmost point
    float xmax, xmin;
    if (in_r) {
      xmax = xfull;
    } else {
      float t = __fsub_rn(1.0f, __fmul_rn(__fmul_rn(yr, yr), icc));
      if (t < 0.0f) t = 0.0f;
      xmax = __fadd_rn(__fmul_rn(slope, yr), __fsqrt_rn(__fmul_rn(hh, t)));
    }
    if (in_l) {
      xmin = -xfull;
    } else {
      float t = __fsub_rn(1.0f, __fmul_rn(__fmul_rn(yl, yl), icc));
      if (t < 0.0f) t = 0.0f;
      xmin = __fsub_rn(__fmul_rn(slope, yl), __fsqrt_rn(__fmul_rn(hh, t)));
    }
    const float lo = __fsub_rn(__fsub_rn(__fadd_rn(g.pxc, xmin), PAD), 0.5f);
    const float hi = __fsub_rn(__fadd_rn(__fadd_rn(g.pxc, xmax), PAD), 0.5f);
    uint32_t rowbits;
    if (!(isfinite(lo) && isfinite(hi))) {
      rowbits = w == 32 ? 0xFFFFFFFFu : ((1u << w) - 1u);
    } else {
      float i0 = __fadd_rn(floorf(lo), 1.0f), i1 = __fsub_rn(ceilf(hi), 1.0f);
      if (i0 < 0.0f) i0 = 0.0f;
      const float wm1 = (float)(V.width - 1);
      if (i1 > wm1) i1 = wm1;
      if (i0 > i1) continue;
      int q0 = (int)i0 >> tile_shift_w, q1 = (int)i1 >> tile_shift_w;
      q0 = max(q0, rect[0]);
      q1 = min(q1, rect[1]);
      if (q0 > q1) continue;
      q0 -= rect[0];
      q1 -= rect[0];
      rowbits = ((2u << q1) - 1u) & ~((1u << q0) - 1u);
    }
    mask |= rowbits << (r * w);
  }
  return mask;
}

// ---------------------------------------------------------------------------
// double-float helpers (error-free transformations) for the projected centre
// ---------------------------------------------------------------------------
struct dd { float hi, lo; };

__device__ __forceinline__ dd two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dd fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ dd two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  return {p, e};
}
__device__ __forceinline__ dd dd_add_f(dd a, float b) {
  dd s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, e);
}
// a / b in double-float
__device__ __forceinline__ dd dd_div(dd a, dd b) {
  float q = __fdiv_rn(a.hi, b.hi);
  dd pq = two_prod(q, b.hi);
  float r = __fsub_rn(__fsub_rn(a.hi, pq.hi), pq.lo);
  r = __fadd_rn(r, a.lo);
  r = __fsub_rn(r, __fmul_rn(q, b.lo));
  float q2 = __fdiv_rn(r, b.hi);
  return fast_two_sum(q, q2);
}
// a * b in double-float
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
  dd p = two_prod(a.hi, b.hi);
  return fast_two_sum(p.hi, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)));
}
__device__ __forceinline__ dd dd_mul_f(dd a, float b) {
  dd p = two_prod(a.hi, b);
  return fast_two_sum(p.hi, __fmaf_rn(a.lo, b, p.lo));
}

// camera-space coordinate r of the centre as a double-float (exact products)
__device__ __forceinline__ dd cam_coord_dd(const ViewDev& V, int r, const float mu[3]) {
  dd acc = two_prod(V.R[r * 3 + 0], mu[0]);
  acc = dd_add(acc, two_prod(V.R[r * 3 + 1], mu[1]));
  acc = dd_add(acc, two_prod(V.R[r * 3 + 2], mu[2]));
  return dd_add_f(acc, V.t[r]);
}

// a*b - c*d with one rounding error (Kahan's algorithm)
__device__ __forceinline__ float diff_of_products(float a, float b, float c, float d) {
  float w = c * d;
  float e = __fmaf_rn(-c, d, w);
  float f = __fmaf_rn(a, b, -w);
  return f + e;
}

__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// lobe count -> template instantiation (M = 0..8)
#define BETA_DISPATCH_M(M_, CALL) \
  switch (M_) {                   \
    case 0: return CALL(0);       \
    case 1: return CALL(1);       \
    case 2: return CALL(2);       \
    case 3: return CALL(3);       \
    case 4: return CALL(4);       \
    case 5: return CALL(5);       \
    case 6: return CALL(6);       \
    case 7: return CALL(7);       \
    case 8: return CALL(8);       \
    default: return cudaErrorInvalidValue; \
  }

// Optimiser-step constants (beta_optim.cu).
struct AdamDev {
  float lr[9];                 // mean, log-scale, quaternion, opacity, b, c0, lobe dir, lobe b, lobe colour
  float beta1, beta2, eps;
  float inv_c1, inv_c2;        // 1 / (1 - beta^t)
  float lambda_o, lambda_sigma;
  float noise_scale;           // lambda_eps * lr_mu
  float noise_pow;             // 4 e^b'
};

// ---------------------------------------------------------------------------
// host-side helpers and launchers (launchers are defined in the .cu files)
// ---------------------------------------------------------------------------

// Streaming multiprocessors of the current device, looked up once per device.
inline int device_sm_count() {
  constexpr int kDevices = 64;
  static std::atomic<int> cache[kDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return 1;
  if (dev >= kDevices) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }
  int n = cache[dev].load(std::memory_order_relaxed);
  if (n == 0) {
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cache[dev].store(n, std::memory_order_relaxed);
  }
  return n;
}
struct ProjBuffers {
  float4* rec;       // [V * pitch * 4]
  uint2* rect;       // [V * pitch]  (tx0 | tx1 << 16, ty0 | ty1 << 16), tx0 > tx1 if empty
  uint32_t* key;     // [V * pitch]  depth key, 0xFFFFFFFF if not binned
  uint32_t* tiles;   // [V * pitch]  rule B2 tiles of the rectangle (bit r w + q; all ones: every tile)
  uint32_t* work;    // records rule B2 applies to (k_tiles' worklist): projection block b owns
                     // entries [b kProjRegion V, (b + 1) kProjRegion V), in arbitrary order
  uint32_t* n_work;  // [projection blocks] entries of each block's region
};

constexpr int kProjRegion = 256;   // primitives per projection block (its worklist region)
inline int64_t proj_blocks(int32_t pitch) { return (pitch + kProjRegion - 1) / kProjRegion; }
size_t proj_bytes(int32_t pitch, int32_t n_views);
ProjBuffers proj_layout(void* proj, int32_t pitch, int32_t n_views);

cudaError_t launch_project(const float* planes, int n, int pitch, int n_lobes, const ViewTable& vt,
                           const RenderOpts& ro, ProjBuffers pb, cudaStream_t s);
cudaError_t launch_project_bwd(const float* planes, int n, int pitch, int n_lobes,
                               const ViewTable& vt, const RenderOpts& ro, float* grad2d,
                               float* grad_planes, const int32_t* status, cudaStream_t s);

struct SortWs;  // defined in beta_sort.cu
// fault-injection test hook of the scan's look-back (0 on success)
int set_scan_faults(int spin_limit, int64_t withhold_block);
size_t binsort_ws_bytes(int64_t n_items, int64_t cap, int total_tiles);
cudaError_t launch_bin_sort(const ViewTable& vt, int pitch, ProjBuffers pb, uint32_t* pair_vals,
                            int64_t cap, uint32_t* ranges, int64_t* d_count, int32_t* d_status,
                            void* ws, cudaStream_t s);

cudaError_t launch_adam(int n_lobes, float* planes, const float* grad, float* m, float* v,
                        const float* eta, int n, int pitch, const AdamDev& a, double* reg,
                        cudaStream_t s);
size_t ssim_ws_bytes(const ViewTable& vt);
cudaError_t launch_ssim_loss(const ViewTable& vt, const float* color, const float* target, float lambda,
                             float* loss, float* dL_dcolor, void* ws, cudaStream_t s);
size_t reloc_ws_bytes(int n);
cudaError_t launch_relocate(int n, int pitch, int n_planes, float* planes, float* m, float* v,
                            const uint32_t* rnd, float min_opacity, void* ws, int32_t* src_out,
                            int32_t* d_count, cudaStream_t s);
// optional hit-mask buffer shared by the raster forward and backward
struct HitMasks {
  uint32_t* words;   // nullptr: none (the backward recomputes its cover pass)
  size_t n_words;
};
size_t hit_mask_bytes(const ViewTable& vt, const RenderOpts& ro, int64_t cap);
cudaError_t launch_raster_fwd(const ViewTable& vt, const RenderOpts& ro, const float4* rec,
                              const uint32_t* vals, const uint32_t* ranges, float* color,
                              float* T_final, uint32_t* n_contrib, const int32_t* status,
                              uint32_t* sched, HitMasks hm, cudaStream_t s);
cudaError_t launch_raster_bwd(const ViewTable& vt, const RenderOpts& ro, const float4* rec,
                              const uint32_t* vals, const uint32_t* ranges, const float* T_final,
                              const uint32_t* n_contrib, const float* dL_dcolor, float* grad2d,
                              const int32_t* status, uint32_t* sched, HitMasks hm, cudaStream_t s);
size_t schedule_bytes(int total_tiles);
cudaError_t launch_schedule(const ViewTable& vt, const uint32_t* ranges, uint32_t* sched,
                            const int32_t* status, cudaStream_t s);
size_t fwd_l1_ws_bytes(const ViewTable& vt);
cudaError_t launch_raster_fwd_l1(const ViewTable& vt, const RenderOpts& ro, const float4* rec,
                                 const uint32_t* vals, const uint32_t* ranges, float* color,
                                 float* T_final, uint32_t* n_contrib, const int32_t* status,
                                 uint32_t* sched, const float* target, float* loss, float* dL_dcolor,
                                 float* ws, HitMasks hm, cudaStream_t s);
// forward + L1 + backward in one launch (tile shapes with pixel pairs)
bool raster_step_supported(const RenderOpts& ro);
cudaError_t launch_raster_step_l1(const ViewTable& vt, const RenderOpts& ro, const float4* rec,
                                  const uint32_t* vals, const uint32_t* ranges, float* color, float* T_final,
                                  uint32_t* n_contrib, const int32_t* status, uint32_t* sched, const float* target,
                                  float* loss, float* dL_dcolor, float* ws, float* grad2d, cudaStream_t s);
size_t l1_ws_bytes(const ViewTable& vt);
cudaError_t launch_l1(const ViewTable& vt, const float* color, const float* target, float* loss,
                      float* dL_dcolor, float* ws, cudaStream_t s);

}  // namespace beta
