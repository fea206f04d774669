// beta_project.cu -- per-(view, primitive) projection (forward) and the chain
// rule from 2D gradients back to the raw parameters (backward).
//
// Forward (Sec. 3.2 / Sec. 3.3 of arXiv 2501.18630), for primitive i, view v:
//   s = exp(log-scale), q_hat = q/|q|, R = R(q_hat), t = W mu + t_w,
//   J = d(pinhole)/dt, M = J W R S (2x3), Sigma' = M M^T + blur I,
//   mu' = (fx tx/tz + cx, fy ty/tz + cy), o = sigmoid(logit), beta = 4 e^b,
//   c = c0 + sum_m max(R_m . V, 0)^(4 e^{b_m}) c_m,  V = normalize(mu - campos).
// One thread per primitive loops over the views, so the parameters are read
// from HBM once per batch.
//
// Numerics: the tile rectangle and depth key follow the fixed fp32 rule in
// beta_internal.cuh.  The projected centre is computed in double-float so
// that the pixel offset x - mu' is exact to fp32 rounding; Sigma' is never
// inverted directly: its Cholesky factor gives the whitening (p, q1, q2)
// with r^2 = (p dx)^2 + (q2 dx + q1 dy)^2, and det Sigma' is the sum of the
// squared 2x2 minors of M (Cauchy-Binet), each minor by Kahan's
// difference-of-products.
#include <cuda_runtime.h>
#include <stdint.h>

#include "beta_internal.cuh"

namespace beta {

// Layout of the projection buffer: records, rectangles, keys and tile masks
// per (view, primitive), then the rule-B2 worklist (kProjRegion x V entries
// per projection block) and one entry count per block.
ProjBuffers proj_layout(void* proj, int32_t pitch, int32_t n_views) {
  ProjBuffers b;
  char* p = (char*)proj;
  const size_t nrec = (size_t)pitch * n_views;
  const size_t nwork = (size_t)proj_blocks(pitch) * kProjRegion * n_views;
  b.rec = (float4*)p;
  b.rect = (uint2*)(p + nrec * 16 * kRecordF4);
  b.key = (uint32_t*)(p + nrec * (16 * kRecordF4 + 8));
  b.tiles = (uint32_t*)(p + nrec * (16 * kRecordF4 + 12));
  b.work = (uint32_t*)(p + nrec * (16 * kRecordF4 + 16));
  b.n_work = (uint32_t*)(p + nrec * (16 * kRecordF4 + 16) + nwork * 4);
  return b;
}

size_t proj_bytes(int32_t pitch, int32_t n_views) {
  const size_t nrec = (size_t)pitch * n_views;
  const size_t nwork = (size_t)proj_blocks(pitch) * kProjRegion * n_views;
  return nrec * (16 * kRecordF4 + 16) + nwork * 4 + ((size_t)proj_blocks(pitch) * 4 + 15) / 16 * 16;
}

namespace {

constexpr float kLog2e = 1.4426950408889634f;

// Asynchronous 16-byte global -> shared copies (LDGSTS): the backward loads
// the 2D gradients of the views ahead without holding registers for them.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const size_t ga = __cvta_generic_to_global(gmem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(ga) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
constexpr float kLn2 = 0.6931471805599453f;

__device__ __forceinline__ float sigmoidf(float x) { return 1.0f / (1.0f + expf(-x)); }

// log2(sigmoid(x)) without cancellation
__device__ __forceinline__ float log2_sigmoid(float x) {
  return x >= 0.0f ? -log1pf(expf(-x)) * kLog2e : x * kLog2e - log1pf(expf(x)) * kLog2e;
}

template <int M>
__device__ __forceinline__ void load_params(const float* __restrict__ planes, int pitch, int i,
                                            float* p, bool& ok) {
  ok = true;
#pragma unroll
  for (int k = 0; k < 15 + 6 * M; ++k) {
    p[k] = planes[(size_t)k * pitch + i];
    ok = ok && isfinite(p[k]);
  }
}

// View-independent per-primitive quantities of the forward.
template <int M>
struct PrimAttr {
  float o, log2o, beta;
  float c0[3];
  float lobe_dir[M > 0 ? M : 1][3];
  float lobe_beta[M > 0 ? M : 1];
};

template <int M>
__device__ __forceinline__ void prim_attr(const float* p, int mode, PrimAttr<M>& a) {
  a.o = sigmoidf(p[10]);
  a.log2o = log2_sigmoid(p[10]);
  a.beta = 4.0f * expf(p[11]);
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) a.c0[ch] = (mode != 2) ? p[12 + ch] : 0.0f;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const float* L = p + 15 + 6 * m;
    float st, ct, sp, cp;
    sincosf(L[0], &st, &ct);
    sincosf(L[1], &sp, &cp);
    a.lobe_dir[m][0] = st * cp;
    a.lobe_dir[m][1] = st * sp;
    a.lobe_dir[m][2] = ct;
    a.lobe_beta[m] = 4.0f * expf(L[2]);
  }
}

// spherical-Beta colour for view direction V = normalize(mu - campos)
template <int M>
__device__ __forceinline__ void sb_colour(const float* p, const PrimAttr<M>& a, const ViewDev& V,
                                          int mode, float c[3]) {
  c[0] = a.c0[0];
  c[1] = a.c0[1];
  c[2] = a.c0[2];
  if (M > 0 && mode != 1) {
    float vx = p[0] - V.campos[0], vy = p[1] - V.campos[1], vz = p[2] - V.campos[2];
    float inv = rsqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz)));
    vx *= inv;
    vy *= inv;
    vz *= inv;
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const float* L = p + 15 + 6 * m;
      float dot = a.lobe_dir[m][0] * vx + a.lobe_dir[m][1] * vy + a.lobe_dir[m][2] * vz;
      if (dot > 0.0f) {
        // MUFU log2/exp2 (relative error ~1e-6 in w, far below the image tolerance)
        float w = ex2_approx(a.lobe_beta[m] * lg2_approx(dot));
        c[0] = fmaf(w, L[3], c[0]);
        c[1] = fmaf(w, L[4], c[1]);
        c[2] = fmaf(w, L[5], c[2]);
      }
    }
  }
}

constexpr int kFwdThreads = 256, kFwdBlocksPerSM = 1;

template <int M>
__global__ void __launch_bounds__(kFwdThreads, kFwdBlocksPerSM) k_project(const float* __restrict__ planes, int n, int pitch,
                                                 ViewTable vt, RenderOpts ro,
                                                 float4* __restrict__ rec, uint2* __restrict__ rect,
                                                 uint32_t* __restrict__ key, uint32_t* __restrict__ tiles,
                                                 uint32_t* __restrict__ work, uint32_t* __restrict__ n_work) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = i < pitch;   // threads past the pitch write nothing but join the warp's append
  float p[15 + 6 * M];
  bool ok = false;
  if (i < n) load_params<M>(planes, pitch, i, p, ok);
  if (ok) ok = (p[11] >= ro.b_lo) && (p[11] < ro.b_hi);
  PrimGeo pg;
  if (ok) ok = rule_prim(p, pg);
  PrimAttr<M> at;
  if (ok) prim_attr<M>(p, ro.color_mode, at);
  uint64_t need = 0;   // views whose record rule B2 applies to
  for (int v = 0; v < vt.n_views; ++v) {
    const ViewDev& V = vt.v[v];
    const size_t r = (size_t)v * pitch + i;
    ViewGeo g;
    int rc[4];
    uint32_t kk = 0xffffffffu;
    bool bin = ok && rule_depth(pg, V, g, kk) &&
               rule_view(pg, V, ro.blur_eps, __ffs(ro.tile_w) - 1, __ffs(ro.tile_h) - 1, g, rc);
    float4 o0, o1, o2;
    if (bin) {
      // projected centre in double-float
      dd tx = cam_coord_dd(V, 0, pg.mu), ty = cam_coord_dd(V, 1, pg.mu), tz = cam_coord_dd(V, 2, pg.mu);
      const dd rz = dd_div(dd{1.0f, 0.0f}, tz);   // one double-float division for both axes
      dd mx = dd_add_f(dd_mul_f(dd_mul(tx, rz), V.fx), V.cx);
      dd my = dd_add_f(dd_mul_f(dd_mul(ty, rz), V.fy), V.cy);
      float ix = floorf(mx.hi), iy = floorf(my.hi);
      float fx = (mx.hi - ix) + mx.lo, fy = (my.hi - iy) + my.lo;
      if (fx < 0.0f) { ix -= 1.0f; fx += 1.0f; }
      if (fx >= 1.0f) { ix += 1.0f; fx -= 1.0f; }
      if (fy < 0.0f) { iy -= 1.0f; fy += 1.0f; }
      if (fy >= 1.0f) { iy += 1.0f; fy -= 1.0f; }
      // Sigma' = M M^T + blur I, det by Cauchy-Binet
      float a0 = fmaf(g.M0[0], g.M0[0], fmaf(g.M0[1], g.M0[1], g.M0[2] * g.M0[2]));
      float c0 = fmaf(g.M1[0], g.M1[0], fmaf(g.M1[1], g.M1[1], g.M1[2] * g.M1[2]));
      float b = fmaf(g.M0[0], g.M1[0], fmaf(g.M0[1], g.M1[1], g.M0[2] * g.M1[2]));
      float m01 = diff_of_products(g.M0[0], g.M1[1], g.M0[1], g.M1[0]);
      float m02 = diff_of_products(g.M0[0], g.M1[2], g.M0[2], g.M1[0]);
      float m12 = diff_of_products(g.M0[1], g.M1[2], g.M0[2], g.M1[1]);
      float det = fmaf(m01, m01, fmaf(m02, m02, m12 * m12));
      float a = a0 + ro.blur_eps;
      if (ro.blur_eps != 0.0f) det = fmaf(ro.blur_eps, a0 + c0 + ro.blur_eps, det);
      bin = (det > 0.0f) && (a > 0.0f) && isfinite(det);
      if (bin) {
        const float pp = rsqrtf(a), isd = rsqrtf(det);
        const float q1 = (a * pp) * isd;
        const float q2 = -(b * pp) * isd;
        float col[3];
        sb_colour<M>(p, at, V, ro.color_mode, col);
        o0 = make_float4(ix, iy, 0.5f - fx, 0.5f - fy);
        o1 = make_float4(pp, q1, q2, at.beta);
        o2 = make_float4(at.log2o, col[0], col[1], col[2]);
      }
    }
    if (bin) {
      rec[r * kRecordF4 + 0] = o0;
      rec[r * kRecordF4 + 1] = o1;
      rec[r * kRecordF4 + 2] = o2;
      rect[r] = make_uint2((uint32_t)rc[0] | ((uint32_t)rc[1] << 16), (uint32_t)rc[2] | ((uint32_t)rc[3] << 16));
      key[r] = kk;
      tiles[r] = rule_all_tiles(rc);   // k_tiles narrows it where rule B2 applies
    } else if (live) {
      rect[r] = make_uint2(1u, 1u);
      key[r] = 0xffffffffu;
      tiles[r] = 0u;
    }
    if (bin && rule_tiles_apply(rc)) need |= 1ull << v;
  }
  // the records rule B2 applies to go on k_tiles' worklist, in this block's
  // region: one atomic per warp, after the view loop (every thread of the
  // warp gets here: none returned early)
  const int lane = threadIdx.x & 31;
  const int cnt = __popcll(need);
  int incl = cnt;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  const int total = __shfl_sync(0xffffffffu, incl, 31);
  if (total == 0) return;
  uint32_t base = 0;
  if (lane == 31) base = atomicAdd(&n_work[blockIdx.x], (uint32_t)total);
  base = __shfl_sync(0xffffffffu, base, 31) + (uint32_t)(incl - cnt);
  uint32_t* region = work + (size_t)blockIdx.x * kProjRegion * vt.n_views;
  for (uint64_t m = need; m; m &= m - 1ull) region[base++] = (uint32_t)(__ffsll((long long)m) - 1) * (uint32_t)pitch + (uint32_t)i;
}

__global__ void k_proj_prep(uint32_t* n_work, int nb) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += gridDim.x * blockDim.x) n_work[b] = 0u;
}

// Rule B2 for the records on the worklist: the rule chain recomputed (the
// same fp32 operations as k_project, so the same rectangle) and the tiles of
// the rectangle the support reaches.  The worklist packs the records that
// need it into full warps; CTA b takes projection block b's region.
__global__ void __launch_bounds__(256) k_tiles(const float* __restrict__ planes, int pitch, ViewTable vt,
                                               RenderOpts ro, const uint32_t* __restrict__ work,
                                               const uint32_t* __restrict__ n_work, uint32_t* __restrict__ tiles) {
  const uint32_t nw = n_work[blockIdx.x];
  const uint32_t* region = work + (size_t)blockIdx.x * kProjRegion * vt.n_views;
  const int sw = __ffs(ro.tile_w) - 1, sh = __ffs(ro.tile_h) - 1;
  for (uint32_t k = threadIdx.x; k < nw; k += blockDim.x) {
    const uint32_t r = region[k];
    const int v = (int)(r / (uint32_t)pitch), i = (int)(r - (uint32_t)v * (uint32_t)pitch);
    float p[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) p[q] = planes[(size_t)q * pitch + i];
    PrimGeo pg;
    ViewGeo g;
    uint32_t kk;
    int rc[4];
    const ViewDev& V = vt.v[v];
    if (rule_prim(p, pg) && rule_depth(pg, V, g, kk) && rule_view(pg, V, ro.blur_eps, sw, sh, g, rc))
      tiles[r] = rule_tiles(g, V, ro.blur_eps, sw, ro.tile_h, rc);
  }
}

// Per-view geometry for the backward: the same quantities as the rule chain
// (A = W Rq, J, M = J A S), at ordinary fp32 speed -- no tile rectangle: a
// record only holds 2D gradients if it was binned, so its rectangle was
// non-empty.
__device__ __forceinline__ void view_geo_bwd(const PrimGeo& pg, const ViewDev& V, ViewGeo& g) {
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int c = 0; c < 3; ++c)
      g.A[r * 3 + c] = fmaf(V.R[r * 3 + 0], pg.Rq[0 * 3 + c],
                            fmaf(V.R[r * 3 + 1], pg.Rq[1 * 3 + c], V.R[r * 3 + 2] * pg.Rq[2 * 3 + c]));
  g.iz = __frcp_rn(g.tc[2]);
  g.j00 = V.fx * g.iz;
  g.j11 = V.fy * g.iz;
  g.j02 = -(g.j00 * g.tc[0]) * g.iz;
  g.j12 = -(g.j11 * g.tc[1]) * g.iz;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    g.M0[c] = fmaf(g.j00, g.A[0 * 3 + c], g.j02 * g.A[2 * 3 + c]) * pg.s[c];
    g.M1[c] = fmaf(g.j11, g.A[1 * 3 + c], g.j12 * g.A[2 * 3 + c]) * pg.s[c];
  }
}

// ---------------------------------------------------------------------------
// backward: 2D gradients (d mu', d Sigma' (a, b, c), d o, d beta, d colour)
// of every view -> gradients of the raw parameters.  Gradients w.r.t. the
// rotation matrix, the scales and the lobe directions are summed over views
// first and taken through the view-independent maps once.
// ---------------------------------------------------------------------------
constexpr int kBwdThreads = 128, kBwdBlocksPerSM = 3;   // up to 170 registers a thread

template <int M>
__global__ void __launch_bounds__(kBwdThreads, kBwdBlocksPerSM) k_project_bwd(const float* __restrict__ planes, int n,
                                                     int pitch, ViewTable vt, RenderOpts ro,
                                                     float* __restrict__ grad2d,
                                                     float* __restrict__ gout,
                                                     const int32_t* __restrict__ status) {
  // 2D gradients of view v+1 in flight while view v is processed (one view
  // ahead measured faster than two or three):
  // [buffer][float4][thread], each thread reads only its own slots
  constexpr int kAhead = 1;
  __shared__ __align__(16) float4 s_g[kAhead + 1][3][kBwdThreads];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  constexpr int NP = 15 + 6 * M;
  constexpr int MM = M > 0 ? M : 1;
  float gp[NP];
#pragma unroll
  for (int k = 0; k < NP; ++k) gp[k] = 0.0f;
  float p[NP];
  bool ok = false;
  load_params<M>(planes, pitch, i, p, ok);
  if (ok) ok = (p[11] >= ro.b_lo) && (p[11] < ro.b_hi);
  if (*status != 0) ok = false;
  PrimGeo pg;
  if (ok) ok = rule_prim(p, pg);
  if (ok) {
    PrimAttr<M> at;
    prim_attr<M>(p, ro.color_mode, at);
    float dR[9], ds[3], dRm[MM][3];
#pragma unroll
    for (int k = 0; k < 9; ++k) dR[k] = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) ds[k] = 0.0f;
#pragma unroll
    for (int m = 0; m < MM; ++m) dRm[m][0] = dRm[m][1] = dRm[m][2] = 0.0f;
    float go = 0.0f, gbeta = 0.0f;
    const int tid = threadIdx.x;
    auto fetch = [&](int v) {
      if (v < vt.n_views) {
        const float4* src = reinterpret_cast<const float4*>(grad2d + ((size_t)v * pitch + i) * kGrad2dStride);
#pragma unroll
        for (int q = 0; q < 3; ++q) cp_async16(&s_g[v % (kAhead + 1)][q][tid], src + q);
      }
      cp_async_commit();   // one group per view, empty past the last
    };
#pragma unroll
    for (int a = 0; a < kAhead; ++a) fetch(a);
    for (int v = 0; v < vt.n_views; ++v) {
      const ViewDev& V = vt.v[v];
      float4* g2 = reinterpret_cast<float4*>(grad2d + ((size_t)v * pitch + i) * kGrad2dStride);
      cp_async_wait<kAhead - 1>();   // view v's group has landed
      const int sb = v % (kAhead + 1);
      const float4 ga4 = s_g[sb][0][tid], gb4 = s_g[sb][1][tid], gc4 = s_g[sb][2][tid];
      fetch(v + kAhead);
      const float G[kGrad2d] = {ga4.x, ga4.y, ga4.z, ga4.w, gb4.x, gb4.y, gb4.z, gb4.w, gc4.x, gc4.y};
      bool any = false;
#pragma unroll
      for (int k = 0; k < kGrad2d; ++k) any = any || (G[k] != 0.0f);
      if (!any) continue;
      // leave the accumulator zeroed for the next backward
      const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      g2[0] = z4;
      g2[1] = z4;
      g2[2] = z4;
      ViewGeo g;
      uint32_t kk;
      if (!rule_depth(pg, V, g, kk)) continue;
      view_geo_bwd(pg, V, g);
      // whitening of Sigma' (the forward's formulas) turns the whitened sums
      // into d mu' and d Sigma' = [[ga, gb/2], [gb/2, gc]] (gb: off-diagonal scalar)
      float gmx, gmy, ga, gb, gc;
      {
        const float a0 = fmaf(g.M0[0], g.M0[0], fmaf(g.M0[1], g.M0[1], g.M0[2] * g.M0[2]));
        const float c0 = fmaf(g.M1[0], g.M1[0], fmaf(g.M1[1], g.M1[1], g.M1[2] * g.M1[2]));
        const float bb = fmaf(g.M0[0], g.M1[0], fmaf(g.M0[1], g.M1[1], g.M0[2] * g.M1[2]));
        const float m01 = diff_of_products(g.M0[0], g.M1[1], g.M0[1], g.M1[0]);
        const float m02 = diff_of_products(g.M0[0], g.M1[2], g.M0[2], g.M1[0]);
        const float m12 = diff_of_products(g.M0[1], g.M1[2], g.M0[2], g.M1[1]);
        float det = fmaf(m01, m01, fmaf(m02, m02, m12 * m12));
        const float aa = a0 + ro.blur_eps;
        if (ro.blur_eps != 0.0f) det = fmaf(ro.blur_eps, a0 + c0 + ro.blur_eps, det);
        const float p = rsqrtf(aa), isd = rsqrtf(det);
        const float q1 = (aa * p) * isd, q2 = -(bb * p) * isd;
        const float b2 = 2.0f * at.beta;
        gmx = b2 * fmaf(p, G[0], q2 * G[1]);
        gmy = b2 * q1 * G[1];
        ga = at.beta * fmaf(p * p, G[2], fmaf(2.0f * p * q2, G[3], q2 * q2 * G[4]));
        gb = b2 * q1 * fmaf(p, G[3], q2 * G[4]);
        gc = at.beta * q1 * q1 * G[4];
      }
      // Sigma' = M M^T: dM0 = 2 ga M0 + gb M1, dM1 = gb M0 + 2 gc M1
      float dM0[3], dM1[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        dM0[k] = 2.0f * ga * g.M0[k] + gb * g.M1[k];
        dM1[k] = gb * g.M0[k] + 2.0f * gc * g.M1[k];
      }
      // M0k = (j00 A0k + j02 A2k) s_k ; M1k = (j11 A1k + j12 A2k) s_k
      float dA[9];
      float dj00 = 0.f, dj02 = 0.f, dj11 = 0.f, dj12 = 0.f;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        float u0 = g.j00 * g.A[0 * 3 + k] + g.j02 * g.A[2 * 3 + k];
        float u1 = g.j11 * g.A[1 * 3 + k] + g.j12 * g.A[2 * 3 + k];
        ds[k] += dM0[k] * u0 + dM1[k] * u1;
        dA[0 * 3 + k] = dM0[k] * g.j00 * pg.s[k];
        dA[1 * 3 + k] = dM1[k] * g.j11 * pg.s[k];
        dA[2 * 3 + k] = (dM0[k] * g.j02 + dM1[k] * g.j12) * pg.s[k];
        dj00 += dM0[k] * g.A[0 * 3 + k] * pg.s[k];
        dj02 += dM0[k] * g.A[2 * 3 + k] * pg.s[k];
        dj11 += dM1[k] * g.A[1 * 3 + k] * pg.s[k];
        dj12 += dM1[k] * g.A[2 * 3 + k] * pg.s[k];
      }
      // A = W Rq  ->  dRq += W^T dA
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int c = 0; c < 3; ++c)
          dR[a * 3 + c] += V.R[0 * 3 + a] * dA[0 * 3 + c] + V.R[1 * 3 + a] * dA[1 * 3 + c] +
                           V.R[2 * 3 + a] * dA[2 * 3 + c];
      // J(t) and mu'(t)
      const float tx = g.tc[0], ty = g.tc[1], iz = g.iz, iz2 = iz * iz, iz3 = iz2 * iz;
      float dtx = dj02 * (-V.fx * iz2) + gmx * V.fx * iz;
      float dty = dj12 * (-V.fy * iz2) + gmy * V.fy * iz;
      float dtz = dj00 * (-V.fx * iz2) + dj11 * (-V.fy * iz2) + dj02 * (2.f * V.fx * tx * iz3) +
                  dj12 * (2.f * V.fy * ty * iz3) - gmx * V.fx * tx * iz2 - gmy * V.fy * ty * iz2;
      // t = W mu + t_w
      gp[0] += V.R[0] * dtx + V.R[3] * dty + V.R[6] * dtz;
      gp[1] += V.R[1] * dtx + V.R[4] * dty + V.R[7] * dtz;
      gp[2] += V.R[2] * dtx + V.R[5] * dty + V.R[8] * dtz;
      go += G[5];                               // times 1/o below
      gbeta += G[6];                            // times ln 2 below
      // colour
      const float gr = G[7], gg = G[8], gbl = G[9];
      if (ro.color_mode != 2) {
        gp[12] += gr;
        gp[13] += gg;
        gp[14] += gbl;
      }
      if (M > 0 && ro.color_mode != 1) {
        float vx = p[0] - V.campos[0], vy = p[1] - V.campos[1], vz = p[2] - V.campos[2];
        float il = rsqrtf(fmaf(vx, vx, fmaf(vy, vy, vz * vz)));
        vx *= il;
        vy *= il;
        vz *= il;
        float dvx = 0.f, dvy = 0.f, dvz = 0.f;
#pragma unroll
        for (int m = 0; m < M; ++m) {
          const float* L = p + 15 + 6 * m;
          float* dL = gp + 15 + 6 * m;
          const float rx = at.lobe_dir[m][0], ry = at.lobe_dir[m][1], rz = at.lobe_dir[m][2];
          float dot = rx * vx + ry * vy + rz * vz;
          if (dot > 0.0f) {
            // w = dot^bm and d w / d dot = bm w / dot, with the MUFU log2/exp2
            // (relative error ~1e-6, far inside the gradient tolerance)
            float bm = at.lobe_beta[m];
            float lw = lg2_approx(dot);
            float wgt = ex2_approx(bm * lw);
            dL[3] += wgt * gr;
            dL[4] += wgt * gg;
            dL[5] += wgt * gbl;
            float gw = gr * L[3] + gg * L[4] + gbl * L[5];
            dL[2] += gw * wgt * (lw * kLn2) * bm;
            float ddot = gw * bm * wgt * __frcp_rn(dot);
            dRm[m][0] += ddot * vx;
            dRm[m][1] += ddot * vy;
            dRm[m][2] += ddot * vz;
            dvx += ddot * rx;
            dvy += ddot * ry;
            dvz += ddot * rz;
          }
        }
        float vd = vx * dvx + vy * dvy + vz * dvz;
        gp[0] += (dvx - vx * vd) * il;
        gp[1] += (dvy - vy * vd) * il;
        gp[2] += (dvz - vz * vd) * il;
      }
    }
    // scales: s = exp(log-scale)
#pragma unroll
    for (int k = 0; k < 3; ++k) gp[3 + k] = ds[k] * pg.s[k];
    // Rq(q_hat) -> d q_hat -> d q
    const float w = pg.q[0], x = pg.q[1], y = pg.q[2], z = pg.q[3];
    float dw = 2.f * (-z * dR[1] + y * dR[2] + z * dR[3] - x * dR[5] - y * dR[6] + x * dR[7]);
    float dx = 2.f * (y * dR[1] + z * dR[2] + y * dR[3] - 2.f * x * dR[4] - w * dR[5] + z * dR[6] +
                      w * dR[7] - 2.f * x * dR[8]);
    float dy = 2.f * (-2.f * y * dR[0] + x * dR[1] + w * dR[2] + x * dR[3] + z * dR[5] - w * dR[6] +
                      z * dR[7] - 2.f * y * dR[8]);
    float dz = 2.f * (-2.f * z * dR[0] - w * dR[1] + x * dR[2] + w * dR[3] - 2.f * z * dR[4] +
                      y * dR[5] + x * dR[6] + y * dR[7]);
    float qd = w * dw + x * dx + y * dy + z * dz;
    float iq = 1.0f / pg.qn;
    gp[6] = (dw - w * qd) * iq;
    gp[7] = (dx - x * qd) * iq;
    gp[8] = (dy - y * qd) * iq;
    gp[9] = (dz - z * qd) * iq;
    // opacity logit and shape
    // dL/do = (1/o) sum (dL/dalpha) alpha; sigmoid' = o (1 - o)
    gp[10] = go * (1.0f - at.o);
    // dL/dbeta = ln 2 sum (dL/dalpha) alpha log2(1 - r^2); dbeta/db = beta
    gp[11] = gbeta * kLn2 * at.beta;
    // lobe directions R = (sin t cos p, sin t sin p, cos t)
#pragma unroll
    for (int m = 0; m < M; ++m) {
      const float* L = p + 15 + 6 * m;
      float st, ct, sp, cp;
      sincosf(L[0], &st, &ct);
      sincosf(L[1], &sp, &cp);
      gp[15 + 6 * m + 0] = dRm[m][0] * ct * cp + dRm[m][1] * ct * sp - dRm[m][2] * st;
      gp[15 + 6 * m + 1] = -dRm[m][0] * st * sp + dRm[m][1] * st * cp;
    }
  }
#pragma unroll
  for (int k = 0; k < NP; ++k) gout[(size_t)k * pitch + i] = gp[k];
}

}  // namespace

template <int M>
static cudaError_t launch_project_m(const float* planes, int n, int pitch, const ViewTable& vt,
                                    const RenderOpts& ro, ProjBuffers pb, cudaStream_t s) {
  int grid = (pitch + kFwdThreads - 1) / kFwdThreads;
  if (grid < 1) return cudaSuccess;
  static_assert(kFwdThreads == kProjRegion, "a projection block owns one worklist region");
  k_proj_prep<<<(grid + 255) / 256, 256, 0, s>>>(pb.n_work, grid);
  k_project<M><<<grid, kFwdThreads, 0, s>>>(planes, n, pitch, vt, ro, pb.rec, pb.rect, pb.key, pb.tiles,
                                            pb.work, pb.n_work);
  k_tiles<<<grid, 256, 0, s>>>(planes, pitch, vt, ro, pb.work, pb.n_work, pb.tiles);
  return cudaGetLastError();
}

template <int M>
static cudaError_t launch_project_bwd_m(const float* planes, int n, int pitch, const ViewTable& vt,
                                        const RenderOpts& ro, float* grad2d, float* gout,
                                        const int32_t* status, cudaStream_t s) {
  int grid = (n + kBwdThreads - 1) / kBwdThreads;
  if (grid < 1) return cudaSuccess;
  k_project_bwd<M><<<grid, kBwdThreads, 0, s>>>(planes, n, pitch, vt, ro, grad2d, gout, status);
  return cudaGetLastError();
}

cudaError_t launch_project(const float* planes, int n, int pitch, int n_lobes, const ViewTable& vt,
                           const RenderOpts& ro, ProjBuffers pb, cudaStream_t s) {
#define CALL_P(m) launch_project_m<m>(planes, n, pitch, vt, ro, pb, s)
  BETA_DISPATCH_M(n_lobes, CALL_P)
#undef CALL_P
}

cudaError_t launch_project_bwd(const float* planes, int n, int pitch, int n_lobes,
                               const ViewTable& vt, const RenderOpts& ro, float* grad2d,
                               float* grad_planes, const int32_t* status, cudaStream_t s) {
#define CALL_B(m) launch_project_bwd_m<m>(planes, n, pitch, vt, ro, grad2d, grad_planes, status, s)
  BETA_DISPATCH_M(n_lobes, CALL_B)
#undef CALL_B
}

}  // namespace beta
