// beta_raster.cu -- tile compositing (forward), its reverse-order backward,
// the per-pixel L1 loss, and the longest-first tile schedule.
//
// Forward (Eq. C of arXiv 2501.18630): for every pixel of a tile, walk the
// tile's depth-sorted list, r^2 = (p dx)^2 + (q2 dx + q1 dy)^2, and for
// r^2 < 1 (the Beta kernel's bounded support, Eq. 2) composite
//   alpha = min(alpha_max, o (1 - r^2)^beta),  C += T alpha c,  T *= 1 - alpha,
// stopping before a primitive once T < t_eps.
//
// Layout: one CTA per TW x TH tile.  In 8 x 4 tiles (k_raster_fwd /
// k_raster_bwd) every thread owns one pixel and warp w an 8 x 4 block; in the
// others (k_raster_fwd2 / k_raster_bwd2, below) every thread owns two
// horizontally adjacent pixels and the warp a 16 x 4 or 8 x 8 block, "pixel"
// reading "pixel pair" in what follows.  Records of the tile's list are
// staged S at a time in shared memory (double-buffered cp.async, one batch
// ahead).  Each warp walks the staged records 32 at a time in two passes.
// First, lane k works out which
// of the block's 32 pixel centres record k may cover (per pixel row the
// support is an interval in x, solved in closed form and widened slightly),
// and a 32 x 32 bit transpose across the warp turns these into, per lane, the
// set of records that may cover its own pixel.  Then every lane composites (or
// differentiates) only its own records, in list order, after the exact r^2
// test: the warp iterates as often as its busiest lane rather than once per
// record touching the block (small Betas cover ~7 of a block's 32 pixels).
// Transmittance early exit is decided per warp (__all_sync) and per CTA
// (__syncthreads_or).
//
// Backward: the same tiling walks each tile list from the largest
// last-contributor position down, recovering T_k = T_{k+1} / (1 - alpha_k)
// and the suffix colour S (as g . S), and produces per-record 2D gradients
// (d mu', d Sigma', d o, d beta, d colour): every lane adds its ten values
// with three 16-byte vector atomics, except for records covering more than
// 12 of the block's lanes, which the warp processes together and sums with a
// 12-shuffle reduce-scatter, one atomic per value.
//
// Scheduling: with a schedule buffer (beta_schedule) the raster kernels are
// persistent -- a grid sized to the SMs takes tiles from a global counter in
// longest-list-first order (tiles bucketed by floor(log2 count)); the last
// CTA to leave resets the counter.  Without one, CTA b renders tile b.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <climits>

#include "beta_internal.cuh"

namespace beta {

namespace {

// 16-byte vector atomic add (sm_90+), into a 16-byte aligned slot
__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
               "f"(d)
               : "memory");
}

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// floor / ceil of x in [-1, 8] by one add rounded toward -inf / +inf: the
// floats near 1.5 * 2^23 are spaced by 1, so the rounded sum is that constant
// plus floor(x) / ceil(x) exactly (an FMA-pipe add instead of a round and a
// conversion on the narrow multi-function pipe).
constexpr float kRoundMagic = 12582912.0f;   // 1.5 * 2^23, bits 0x4B400000
__device__ __forceinline__ int floor_small(float x) { return __float_as_int(__fadd_rd(x, kRoundMagic)) - 0x4B400000; }
__device__ __forceinline__ int ceil_small(float x) { return __float_as_int(__fadd_ru(x, kRoundMagic)) - 0x4B400000; }

// Pixels of the 8x4 block with first pixel (bxf, byf) whose centre the
// record's support r^2 < 1 may cover: bit 8 r + j for row r, column j.  On a
// row, r^2 = (p dx)^2 + (q2 dx + q1 dy)^2 is a convex quadratic in dx, so its
// support is the interval dx in [xc - w, xc + w] with A = p^2 + q2^2,
// xc = -q1 q2 dy / A and w = sqrt(A - (p q1 dy)^2) / A (empty when the root
// is imaginary).  It is solved for r^2 < 1 + 1e-5 and widened by 1e-3 pixel
// plus 1e-5 of its extent, so every pixel the exact fp32 test of rec_r2
// accepts is covered (the compositing repeats that test); dy is formed as
// rec_r2 forms it.
__device__ __forceinline__ uint32_t block_cover(float4 f0, float4 f1, float bxf, float byf) {
  const float p = f1.x, q1 = f1.y, q2 = f1.z;
  const float X0 = (bxf - f0.x) + f0.z;              // dx of the block's first column
  const float A = fmaf(p, p, q2 * q2);
  const float iA = rcp_approx(A);
  const float A1 = A * 1.00001f;
  const float sxc = q1 * q2 * iA;
  const float pq = p * q1;
  uint32_t m = 0u;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const float dy = ((byf + (float)r) - f0.y) + f0.w;
    const float t = pq * dy;
    const float disc = fmaf(-t, t, A1);
    const float w = sqrt_approx(fmaxf(disc, 0.0f)) * iA;
    const float xc = fmaf(-sxc, dy, -X0);              // interval centre, in columns of the block
    const float e = fmaf(1e-5f, fabsf(xc) + w, 1e-3f);
    const int ilo = ceil_small(fminf(fmaxf(xc - w - e, 0.0f), 8.0f));     // in [0, 8]
    const int ihi = floor_small(fmaxf(fminf(xc + w + e, 7.0f), -1.0f));   // in [-1, 7]
    const uint32_t row = (0xFFu >> (7 - ihi)) & (0xFFu << ilo);   // columns ilo .. ihi
    m |= (disc > 0.0f ? row : 0u) << (8 * r);
  }
  return m;
}

// 32 x 32 bit-matrix transpose across the warp: on entry lane L holds row L,
// on return lane j holds column j (bit L of lane j's word = bit j of lane L's).
// Five exchange stages; at stage s lanes L and L ^ s swap the off-diagonal
// s x s blocks of their 2s x 2s block.
__device__ __forceinline__ uint32_t transpose32(uint32_t w, int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const uint32_t m = s == 16 ? 0x0000FFFFu : s == 8 ? 0x00FF00FFu : s == 4 ? 0x0F0F0F0Fu
                     : s == 2 ? 0x33333333u : 0x55555555u;
    const bool up = (lane & s) != 0;
    const uint32_t send = up ? (w & m) << s : (w & ~m) >> s;
    const uint32_t got = __shfl_xor_sync(0xffffffffu, send, s);
    w = (w & (up ? ~m : m)) | got;
  }
  return w;
}

// r^2 of a staged record at the pixel centre (xf, yf), with the whitened
// coordinates u, v.  One expression for every caller, so that the support
// test of the first pass and the compositing of the second see the same value.
__device__ __forceinline__ float rec_r2(float4 f0, float4 f1, float xf, float yf, float& u, float& vv) {
  const float dx = (xf - f0.x) + f0.z;
  const float dy = (yf - f0.y) + f0.w;
  u = f1.x * dx;
  vv = fmaf(f1.z, dx, f1.y * dy);
  return fmaf(u, u, vv * vv);
}

// Asynchronous 16-byte global -> shared copies (LDGSTS), so record staging
// for the next batch overlaps compositing of the current one.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const size_t ga = __cvta_generic_to_global(gmem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(ga) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
  const size_t ga = __cvta_generic_to_global(gmem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(ga) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Stage record r (48 bytes) into a shared slot.
__device__ __forceinline__ void stage_record(float4* dst, const float4* __restrict__ rec, uint32_t r) {
  const float4* src = rec + (size_t)r * kRecordF4;
#pragma unroll
  for (int q = 0; q < kRecordF4; ++q) cp_async16(dst + q, src + q);
}

// Records covering more than this many pixels of a warp's block are reduced
// across the warp before their atomics in the backward; for the others every
// lane adds its own terms.
constexpr int kLaneAtomics = 12;

// Hit masks (optional, written by the forward, read by the backward): per
// tile g, per chunk j of 32 list positions, NT words (word t: the records of
// the chunk that may cover pixel t of the tile, bit k = position 32 j + k,
// from block_cover and the transpose) and NW words (word w: the chunk's
// records covering more than kLaneAtomics pixels of warp w's block).  Chunk j
// of tile g is slot (ranges[g] >> 5) + g + j, so the slots of the tiles never
// overlap and (pairs >> 5) + tiles + 1 slots hold every list.  A tile whose
// slots do not all fit in the buffer uses none (the backward recomputes its
// cover pass); returns the tile's first slot, or nullptr.
template <int NT>
__device__ __forceinline__ uint32_t* hit_tile(uint32_t* hm, size_t hm_words, uint32_t range0, uint32_t range1,
                                              int g) {
  constexpr int NW = NT / 32;
  if (!hm) return nullptr;
  const size_t w0 = ((size_t)(range0 >> 5) + (size_t)g) * (size_t)(NT + NW);
  const size_t n = (size_t)((range1 - range0 + 31u) >> 5) * (size_t)(NT + NW);
  return w0 + n <= hm_words ? hm + w0 : nullptr;
}

// Resident CTAs per SM asked of the register allocator for `threads` threads
// per CTA and `per_sm` threads per SM, at most the 32 CTAs an SM holds.
constexpr int min_blocks(int threads, int per_sm) {
  return per_sm / threads < 32 ? per_sm / threads : 32;
}

// Tile assignment: CTA b renders tile b, or (persistent) tiles are taken from
// the schedule's counter in its longest-first order.  Returns -1 when done.
template <bool PERSIST>
__device__ __forceinline__ int next_tile(int iter, int total_tiles, uint32_t* ctr,
                                         const uint32_t* order, int* s_item) {
  if (!PERSIST) return iter == 0 ? (int)blockIdx.x : -1;
  if (threadIdx.x == 0) *s_item = (int)atomicAdd(ctr, 1u);
  __syncthreads();
  const int item = *s_item;
  __syncthreads();
  return item < total_tiles ? (int)order[item] : -1;
}

// The last CTA of a persistent grid to run out of work resets the counter.
template <bool PERSIST>
__device__ __forceinline__ void leave(uint32_t* ctr) {
  if (PERSIST && threadIdx.x == 0) {
    const uint32_t done = atomicAdd(ctr + 1, 1u);
    if (done == gridDim.x - 1) {
      ctr[0] = 0u;
      ctr[1] = 0u;
    }
  }
}

template <int TW, int TH, int S, bool PERSIST>
__global__ void __launch_bounds__(TW * TH, min_blocks(TW * TH, 1536)) k_raster_fwd(ViewTable vt, RenderOpts ro,
                                                       const float4* __restrict__ rec,
                                                       const uint32_t* __restrict__ vals,
                                                       const uint32_t* __restrict__ ranges,
                                                       float* __restrict__ color,
                                                       float* __restrict__ Tout,
                                                       uint32_t* __restrict__ ncontrib,
                                                       const int32_t* __restrict__ status,
                                                       uint32_t* ctr, const uint32_t* __restrict__ order,
                                                       const float* __restrict__ target,
                                                       float* __restrict__ dLdC,
                                                       float* __restrict__ l1_partial,
                                                       uint32_t* __restrict__ hm, size_t hm_words) {
  constexpr int NT = TW * TH, BXW = TW / 8, RPT = (S + NT - 1) / NT;
  __shared__ __align__(16) float4 s_rec[2][S][kRecordF4];
  __shared__ float s_l1[NT / 32];
  __shared__ float s_tgt[3][NT];   // the pixel's target, copied in while the tile composites
  __shared__ int s_item;
  if (*status != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float t_eps = ro.t_eps, amax = ro.alpha_max;
  for (int iter = 0;; ++iter) {
    const int g = next_tile<PERSIST>(iter, vt.total_tiles, ctr, order, &s_item);
    if (g < 0) break;
    const int v = view_of_tile(vt, g);
    const int W = vt.v[v].width, H = vt.v[v].height, ntx = vt.v[v].ntx;
    const int lt = g - vt.v[v].tile_off;
    const int ty = lt / ntx, tx = lt - ty * ntx;
    const int bx = tx * TW + (warp % BXW) * 8, by = ty * TH + (warp / BXW) * 4;
    const int x = bx + (lane & 7), y = by + (lane >> 3);
    const bool inside = x < W && y < H;
    const float xf = (float)x, yf = (float)y, bxf = (float)bx, byf = (float)by;
    const uint32_t start = ranges[g], end = ranges[g + 1];
    uint32_t* const hslot = hit_tile<NT>(hm, hm_words, start, end, g);
    if (target && inside) {
      const int64_t HW = (int64_t)W * H;
      const int64_t o = 3 * vt.v[v].pix_off + (int64_t)y * W + x;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) cp_async4(&s_tgt[ch][tid], target + o + ch * HW);
    }

    // batch 0 goes to buffer 0 now; the list entries of batch 1 are loaded
    // ahead so that its copies can be issued without waiting on them
    uint32_t rn[RPT];
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int jj = tid + q * NT;
      if (jj < S && start + jj < end) stage_record(s_rec[0][jj], rec, vals[start + jj]);
      const uint32_t j1 = start + S + jj;
      rn[q] = (jj < S && j1 < end) ? vals[j1] : 0u;
    }
    cp_async_commit();

    float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f;
    uint32_t last = 0;
    bool done = !inside;
    bool warp_done = __all_sync(0xffffffffu, done);

    int buf = 0;
    for (uint32_t base = start; base < end; base += S) {
      cp_async_wait_all();
      if (!__syncthreads_or(!done)) break;
      // copies of the next batch into the other buffer (free: every warp has
      // passed the barrier after compositing from it), entries of the one after
      const uint32_t nb = base + S;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int jj = tid + q * NT;
        if (jj < S && nb + jj < end) stage_record(s_rec[buf ^ 1][jj], rec, rn[q]);
        const uint32_t j2 = nb + S + jj;
        rn[q] = (jj < S && j2 < end) ? vals[j2] : 0u;
      }
      cp_async_commit();
      const int cnt = (int)min((uint32_t)S, end - base);
      for (int c = 0; c < cnt && !warp_done; c += 32) {
        // pass 1: lane k finds the pixels of this warp's block that record
        // c + k may cover; the transpose gives every lane the records that
        // may cover its own pixel
        const int idx = c + lane;
        const uint32_t cov = idx < cnt ? block_cover(s_rec[buf][idx][0], s_rec[buf][idx][1], bxf, byf) : 0u;
        uint32_t mine = transpose32(cov, lane);
        if (hslot) {
          // kept for the backward, which would otherwise redo this pass
          uint32_t* slot = hslot + (size_t)((base - start + c) >> 5) * (NT + NT / 32);
          const uint32_t wide = __ballot_sync(0xffffffffu, __popc(cov) > kLaneAtomics);
          slot[tid] = mine;
          if (lane == 0) slot[NT + warp] = wide;
        }
        if (done) mine = 0u;   // off-image lanes start done and stay done
        // pass 2: every lane composites its own hits in list order, so the
        // warp iterates as often as its busiest lane, not once per record
        // that touches the block
        while (mine) {
          const int k = __ffs(mine) - 1;
          mine &= mine - 1;
          const int s = c + k;
          const float4 f0 = s_rec[buf][s][0];
          const float4 f1 = s_rec[buf][s][1];
          float u, vv;
          const float r2 = rec_r2(f0, f1, xf, yf, u, vv);
          if (!(r2 < 1.0f)) continue;                  // outside the support (the cover is conservative)
          const float4 f2 = s_rec[buf][s][2];
          const float lb = lg2_approx(1.0f - r2);
          const float a = fminf(ex2_approx(fmaf(f1.w, lb, f2.x)), amax);
          const float w = a * T;
          C0 = fmaf(w, f2.y, C0);
          C1 = fmaf(w, f2.z, C1);
          C2 = fmaf(w, f2.w, C2);
          T = T * (1.0f - a);
          last = base - start + (uint32_t)s + 1u;
          if (T < t_eps) {
            done = true;
            mine = 0u;
          }
        }
        warp_done = __all_sync(0xffffffffu, done);
      }
      buf ^= 1;
    }
    cp_async_wait_all();   // no copy may still land in a buffer the next tile fills
    float l1 = 0.0f;
    if (inside) {
      const int64_t HW = (int64_t)W * H;
      const int64_t pix = vt.v[v].pix_off + (int64_t)y * W + x;
      const int64_t o = 3 * vt.v[v].pix_off + (int64_t)y * W + x;
      const float c[3] = {C0 + T * vt.v[v].bg[0], C1 + T * vt.v[v].bg[1], C2 + T * vt.v[v].bg[2]};
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) color[o + ch * HW] = c[ch];
      Tout[pix] = T;
      ncontrib[pix] = last;
      if (target) {
        // the per-pixel L1 term and its gradient, as beta_l1_loss computes them
        const float scale = 1.0f / (3.0f * (float)HW);
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
          const float d = c[ch] - s_tgt[ch][tid];   // landed: the copies were waited for above
          l1 += fabsf(d);
          dLdC[o + ch * HW] = d > 0.0f ? scale : (d < 0.0f ? -scale : 0.0f);
        }
      }
    }
    if (target) {
      // tile partial sum of |C - target|, reduced in a fixed order
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, off);
      if (lane == 0) s_l1[warp] = l1;
      __syncthreads();
      if (tid == 0) {
        float t = 0.0f;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) t += s_l1[w];
        l1_partial[g] = t;
      }
      __syncthreads();
    }
  }
  leave<PERSIST>(ctr);
}

// Sum of ten per-lane values over the warp, scattered: on return lane L holds
// the warp total of field warp_sum10_field(L) (lanes with bit 0 set, and for
// fields 2..4 / 7..9 also lanes with bit 1 set, hold duplicates).  12 shuffles.
__device__ __forceinline__ float warp_sum10(const float v[10], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  float a[5];
#pragma unroll
  for (int j = 0; j < 5; ++j) {
    const float send = b4 ? v[j] : v[j + 5];
    const float keep = b4 ? v[j + 5] : v[j];
    a[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float b[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float hi = j < 2 ? a[j + 3] : 0.0f;
    const float send = b3 ? a[j] : hi;
    const float keep = b3 ? hi : a[j];
    b[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  const float send0 = b3 ? (b2 ? b[0] : b[1]) : (b2 ? b[0] : b[2]);
  const float keep0 = b3 ? (b2 ? b[1] : b[0]) : (b2 ? b[2] : b[0]);
  const float c0 = keep0 + __shfl_xor_sync(0xffffffffu, send0, 4);
  const float send1 = (!b3 && b2) ? b[1] : 0.0f;
  const float keep1 = (!b3 && !b2) ? b[1] : 0.0f;
  const float c1 = keep1 + __shfl_xor_sync(0xffffffffu, send1, 4);
  const bool two = !b3 && !b2;
  const float sendd = two ? (b1 ? c0 : c1) : c0;
  const float keepd = two ? (b1 ? c1 : c0) : c0;
  float d = keepd + __shfl_xor_sync(0xffffffffu, sendd, 2);
  d += __shfl_xor_sync(0xffffffffu, d, 1);
  return d;
}

// field held by `lane` after warp_sum10, or -1 for a duplicate holder
__device__ __forceinline__ int warp_sum10_field(int lane) {
  if (lane & 1) return -1;
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4, b1 = lane & 2;
  int sub;
  if (!b3 && !b2) sub = b1 ? 1 : 0;
  else {
    if (b1) return -1;
    sub = b3 ? (b2 ? 4 : 3) : 2;
  }
  return (b4 ? 5 : 0) + sub;
}

// Per-lane terms of a record's 2D gradients at this lane's pixel, in whitened
// coordinates (u, v) = L^-1 (x - mu'); beta, 1/o, ln 2 and the whitening
// matrix are per-record constants applied by the projection backward:
//   G0..G4 = k (u, v, u^2, u v, v^2),  k = (dL/dalpha) alpha / (1 - r^2)
//   G5 = (dL/dalpha) alpha,  G6 = G5 log2(1 - r^2),  G7..9 = alpha T dL/dC.
// The forward's alpha is recomputed; T_k = T_{k+1} / (1 - alpha_k) and the
// suffix colour GS (as g . S) are updated only where `act` holds and the
// pixel lies inside the support (r^2 < 1); returns that condition.  ZERO:
// every term is exactly zero where the condition fails (t and the colour
// weight are zeroed, 1 - r^2 is clamped so that no term is 0 * inf), for a
// caller that sums the terms over the warp without selecting them.
template <bool ZERO>
__device__ __forceinline__ bool bwd_terms(float4 f0, float4 f1, float4 f2, float xf, float yf, float amax,
                                          bool act, float gx, float gy, float gz, float& T, float& GS,
                                          float G[kGrad2d]) {
  float u, vv;
  const float r2 = rec_r2(f0, f1, xf, yf, u, vv);
  act = act && r2 < 1.0f;
  const float beta = f1.w;
  // ZERO: 1 - r^2 >= 2^-24 wherever r^2 < 1, so the clamp changes nothing
  // there and keeps every term finite elsewhere
  const float base = ZERO ? fmaxf(1.0f - r2, 5.9604645e-8f) : 1.0f - r2;
  const float lb = lg2_approx(base);
  const float a0 = ex2_approx(fmaf(beta, lb, f2.x));   // the forward's alpha
  const float a = fminf(a0, amax);
  const float inv = rcp_approx(1.0f - a);
  const float Tk = T * inv;
  const float gc = fmaf(gx, f2.y, fmaf(gy, f2.z, gz * f2.w));
  const float dLa = fmaf(Tk, gc, -GS * inv);
  const float wgt = (!ZERO || act) ? a * Tk : 0.0f;
  G[7] = wgt * gx;
  G[8] = wgt * gy;
  G[9] = wgt * gz;
  const float t = (a0 < amax && (!ZERO || act)) ? dLa * a0 : 0.0f;   // clamped alpha: no o/beta/r^2 gradient
  const float kk = t * rcp_approx(base);
  G[0] = kk * u;
  G[1] = kk * vv;
  G[2] = G[0] * u;
  G[3] = G[0] * vv;
  G[4] = G[1] * vv;
  G[5] = t;
  G[6] = t * lb;
  GS = act ? fmaf(wgt, gc, GS) : GS;
  T = act ? Tk : T;
  return act;
}

template <int TW, int TH, int S, bool PERSIST>
__global__ void __launch_bounds__(TW * TH, min_blocks(TW * TH, 1280)) k_raster_bwd(ViewTable vt, RenderOpts ro,
                                                       const float4* __restrict__ rec,
                                                       const uint32_t* __restrict__ vals,
                                                       const uint32_t* __restrict__ ranges,
                                                       const float* __restrict__ Tfin,
                                                       const uint32_t* __restrict__ ncontrib,
                                                       const float* __restrict__ dLdC,
                                                       float* __restrict__ grad2d,
                                                       const int32_t* __restrict__ status,
                                                       uint32_t* ctr, const uint32_t* __restrict__ order,
                                                       const uint32_t* __restrict__ hm, size_t hm_words) {
  constexpr int NT = TW * TH, NW = NT / 32, BXW = TW / 8, RPT = (S + NT - 1) / NT;
  __shared__ __align__(16) float4 s_rec[2][S][kRecordF4];
  __shared__ uint32_t s_ridx[2][S];
  __shared__ uint32_t s_wmax[NW];
  __shared__ int s_item;
  if (*status != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float amax = ro.alpha_max;
  const int my_field = warp_sum10_field(lane);
  for (int iter = 0;; ++iter) {
    const int g = next_tile<PERSIST>(iter, vt.total_tiles, ctr, order, &s_item);
    if (g < 0) break;
    const int v = view_of_tile(vt, g);
    const int W = vt.v[v].width, H = vt.v[v].height, ntx = vt.v[v].ntx;
    const int lt = g - vt.v[v].tile_off;
    const int ty = lt / ntx, tx = lt - ty * ntx;
    const int bx = tx * TW + (warp % BXW) * 8, by = ty * TH + (warp / BXW) * 4;
    const int x = bx + (lane & 7), y = by + (lane >> 3);
    const bool inside = x < W && y < H;
    const float xf = (float)x, yf = (float)y, bxf = (float)bx, byf = (float)by;
    const uint32_t range0 = ranges[g];
    const uint32_t* lst = vals + range0;
    const uint32_t* const hslot = hit_tile<NT>(const_cast<uint32_t*>(hm), hm_words, range0, ranges[g + 1], g);

    float T = 1.0f, gx = 0.0f, gy = 0.0f, gz = 0.0f, GS = 0.0f;
    uint32_t nl = 0;
    if (inside) {
      const int64_t HW = (int64_t)W * H;
      const int64_t pix = vt.v[v].pix_off + (int64_t)y * W + x;
      const float* gb = dLdC + 3 * vt.v[v].pix_off + (int64_t)y * W + x;
      gx = gb[0];
      gy = gb[HW];
      gz = gb[2 * HW];
      T = Tfin[pix];
      nl = ncontrib[pix];
      GS = T * (gx * vt.v[v].bg[0] + gy * vt.v[v].bg[1] + gz * vt.v[v].bg[2]);
    }
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, nl);
    if (lane == 0) s_wmax[warp] = wmax;
    __syncthreads();
    int bmax = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) bmax = max(bmax, (int)s_wmax[w]);

    // Batch b covers list positions [b S, min(b S + S, bmax)), b = nb - 1 .. 0
    // (the forward's batches, so chunks start at multiples of 32).  The last
    // goes to buffer 0 now; the list entries of the one before it are loaded
    // ahead so that its copies issue without waiting.
    const int nb = (bmax + S - 1) / S;
    uint32_t rn[RPT];
    {
      const int lo0 = (nb - 1) * S, lo1 = lo0 - S;
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int jj = tid + q * NT;
        if (nb > 0 && jj < bmax - lo0) {
          const uint32_t r = lst[lo0 + jj];
          s_ridx[0][jj] = r;
          stage_record(s_rec[0][jj], rec, r);
        }
        rn[q] = (lo1 >= 0 && jj < S) ? lst[lo1 + jj] : 0u;
      }
      cp_async_commit();
    }

    // hit masks of the next chunk (chunks are walked from the last down),
    // loaded one chunk ahead so that their DRAM latency overlaps a chunk
    uint32_t pf_mine = 0u, pf_wide = 0u;
    int pf_chunk = -1;
    int buf = 0;
    for (int b = nb - 1; b >= 0; --b) {
      const int lo = b * S;
      const int cnt = min(S, bmax - lo);
      cp_async_wait_all();
      __syncthreads();
      {
        // copies of batch b - 1 (full) into the other buffer, entries of b - 2
#pragma unroll
        for (int q = 0; q < RPT; ++q) {
          const int jj = tid + q * NT;
          if (b >= 1 && jj < S) {
            s_ridx[buf ^ 1][jj] = rn[q];
            stage_record(s_rec[buf ^ 1][jj], rec, rn[q]);
          }
          rn[q] = (b >= 2 && jj < S) ? lst[(b - 2) * S + jj] : 0u;
        }
        cp_async_commit();
      }
      for (int c = ((cnt - 1) >> 5) << 5; c >= 0; c -= 32) {
        if ((uint32_t)(lo + c) >= wmax) continue;
        // pass 1: lane k finds the pixels of this warp's block that record
        // c + k may cover (records at or past the warp's last contributor
        // are skipped); records covering more than kLaneAtomics pixels are
        // marked `wide`; the transpose gives every lane its own records
        uint32_t wide, mine;
        if (hslot) {
          const int j = (lo + c) >> 5;
          if (pf_chunk == j) {                           // the forward's pass 1
            mine = pf_mine;
            wide = pf_wide;
          } else {
            const uint32_t* slot = hslot + (size_t)j * (NT + NW);
            mine = slot[tid];
            wide = slot[NT + warp];
          }
          if (j >= 1) {
            const uint32_t* nslot = hslot + (size_t)(j - 1) * (NT + NW);
            pf_mine = nslot[tid];
            pf_wide = nslot[NT + warp];
            pf_chunk = j - 1;
          }
          const int limw = (int)wmax - (lo + c);         // no lane of the warp reaches past wmax
          wide &= limw >= 32 ? 0xffffffffu : (1u << limw) - 1u;
        } else {
          const int idx = c + lane;
          const uint32_t cov = (idx < cnt && (uint32_t)(lo + idx) < wmax)
                                   ? block_cover(s_rec[buf][idx][0], s_rec[buf][idx][1], bxf, byf) : 0u;
          wide = __ballot_sync(0xffffffffu, __popc(cov) > kLaneAtomics);
          mine = transpose32(cov, lane);
        }
        const int lim = (int)nl - (lo + c);            // only positions before this pixel's last contributor
        mine &= lim >= 32 ? 0xffffffffu : (lim <= 0 ? 0u : (1u << lim) - 1u);
        // pass 2, in reverse list order: between wide records every lane walks
        // its own hits and adds its terms with three vector atomics; a wide
        // record is done by the whole warp together (reduce-scatter, one
        // atomic per value)
        for (;;) {
          const int kb = wide ? 31 - __clz(wide) : -1;                 // warp-uniform
          const uint32_t above = kb >= 0 ? ~((2u << kb) - 1u) : 0xffffffffu;
          uint32_t seg = mine & above;
          mine &= ~above;
          while (seg) {
            const int k = 31 - __clz(seg);
            seg &= ~(1u << k);
            const int s = c + k;
            float G[kGrad2d];
            if (!bwd_terms<false>(s_rec[buf][s][0], s_rec[buf][s][1], s_rec[buf][s][2], xf, yf, amax, true, gx, gy, gz,
                           T, GS, G))
              continue;                                // outside the support (the cover is conservative)
            float* gdst = grad2d + (size_t)s_ridx[buf][s] * kGrad2dStride;
            red_add_v4(gdst + 0, G[0], G[1], G[2], G[3]);
            red_add_v4(gdst + 4, G[4], G[5], G[6], G[7]);
            red_add_v4(gdst + 8, G[8], G[9], 0.0f, 0.0f);
          }
          if (kb < 0) break;
          wide &= ~(1u << kb);
          const bool mine_kb = (mine >> kb) & 1u;
          mine &= ~(1u << kb);
          const int s = c + kb;
          float G[kGrad2d];
          bwd_terms<true>(s_rec[buf][s][0], s_rec[buf][s][1], s_rec[buf][s][2], xf, yf, amax, mine_kb, gx, gy, gz, T,
                          GS, G);                    // zero terms where this pixel is not covered
          const float tot = warp_sum10(G, lane);
          float* gdst = grad2d + (size_t)s_ridx[buf][s] * kGrad2dStride;
          if (my_field >= 0 && tot != 0.0f) atomicAdd(gdst + my_field, tot);
        }
      }
      buf ^= 1;
    }
    cp_async_wait_all();   // no copy may still land in a buffer the next tile fills
    __syncthreads();
  }
  leave<PERSIST>(ctr);
}

// ---------------------------------------------------------------------------
// Pixel-pair raster kernels: every lane owns two horizontally adjacent pixels.
// Warp w of a tile owns a BW x BH block (16 x 4 in tiles at least 16 wide,
// else 8 x 8); lane L owns pixels (2 pc, r) and (2 pc + 1, r) of it, with
// pc = L mod PC, r = L / PC, PC = BW / 2 pair columns.  A record's cover mask
// has one bit per pair (bit L: the record may cover either pixel of lane L),
// and the lanes walk the union of their two pixels' records: one set of
// shared-memory record loads and, in the backward, one set of gradient
// atomics serve both pixels (neighbouring pixels share most records), and the
// warp-wide reductions of records covering many lanes serve 64 pixels.
// ---------------------------------------------------------------------------

// Threads per SM asked of the register allocator for the pixel-pair kernels:
// 1280 (48 registers) where the record buffers of 64-record batches leave
// room for that many CTAs, 1024 (64 registers) for larger batches, whose
// shared memory holds fewer CTAs anyway.
constexpr int pair_threads_per_sm(int S) { return S <= 64 ? 1280 : 1024; }

// Do TW x TH tiles hold whole pixel-pair blocks (16 x 4 in tiles at least
// 16 wide, 8 x 8 in 8-wide ones)?  Those use the pixel-pair kernels, the
// others (8 x 4) the one-pixel-per-lane ones; the hit-mask layout follows.
constexpr bool pair_tiles(int tw, int th) { return th % (tw % 16 == 0 ? 4 : 8) == 0; }

template <int TW>
struct PairBlock {
  static constexpr int BW = TW % 16 == 0 ? 16 : 8;   // block width in pixels
  static constexpr int BH = 64 / BW;                 // block height
  static constexpr int PC = BW / 2;                  // pair columns
  static constexpr int WX = TW / BW;                 // blocks per tile row
};

// Pairs of the BW x BH block with first pixel (bxf, byf) whose two pixel
// centres the record's support r^2 < 1 may reach: bit PC r + pc for row r,
// pair column pc.  Per row the support is the interval of block_cover (same
// closed form, margins and dy); the pairs are those holding a column of it.
template <int BW>
__device__ __forceinline__ uint32_t pair_cover(float4 f0, float4 f1, float bxf, float byf) {
  constexpr int BH = 64 / BW, PC = BW / 2;
  constexpr uint32_t kPcMask = (1u << PC) - 1u;
  const float p = f1.x, q1 = f1.y, q2 = f1.z;
  const float X0 = (bxf - f0.x) + f0.z;              // dx of the block's first column
  const float A = fmaf(p, p, q2 * q2);
  const float iA = rcp_approx(A);
  const float A1 = A * 1.00001f;
  const float sxc = q1 * q2 * iA;
  const float pq = p * q1;
  uint32_t m = 0u;
#pragma unroll
  for (int r = 0; r < BH; ++r) {
    const float dy = ((byf + (float)r) - f0.y) + f0.w;
    const float t = pq * dy;
    const float disc = fmaf(-t, t, A1);
    const float w = sqrt_approx(fmaxf(disc, 0.0f)) * iA;
    const float xc = fmaf(-sxc, dy, -X0);              // interval centre, in columns of the block
    const float e = fmaf(1e-5f, fabsf(xc) + w, 1e-3f);
    const int ilo = ceil_small(fminf(fmaxf(xc - w - e, 0.0f), (float)BW));         // in [0, BW]
    const int ihi = floor_small(fmaxf(fminf(xc + w + e, (float)(BW - 1)), -1.0f));  // in [-1, BW - 1]
    const int plo = ilo >> 1, phi = ihi >> 1;                                        // phi = -1 for ihi = -1
    const uint32_t row = (kPcMask >> (PC - 1 - phi)) & (kPcMask << plo);            // pairs plo .. phi
    m |= (disc > 0.0f && ilo <= ihi ? row : 0u) << (PC * r);
  }
  return m;
}

// r^2 of a staged record at the lane's two pixel centres (xf, yf) and
// (xf + 1, yf), with their whitened coordinates: each pixel's the values
// rec_r2 gives it (the row term q1 dy is shared), so that every pixel
// composites the same way whatever the tiling, and the forward and the
// backward see the same values.
__device__ __forceinline__ void rec_r2_pair(float4 f0, float4 f1, float xf, float yf, float& u0, float& v0,
                                            float& u1, float& v1, float& r2a, float& r2b) {
  const float dx0 = (xf - f0.x) + f0.z;
  const float dx1 = ((xf + 1.0f) - f0.x) + f0.z;
  const float dy = (yf - f0.y) + f0.w;
  const float qy = f1.y * dy;
  u0 = f1.x * dx0;
  v0 = fmaf(f1.z, dx0, qy);
  u1 = f1.x * dx1;
  v1 = fmaf(f1.z, dx1, qy);
  r2a = fmaf(u0, u0, v0 * v0);
  r2b = fmaf(u1, u1, v1 * v1);
}

// Per-lane state of the pixel-pair forward after a tile's walk: transmittance,
// accumulated colour and last contributor (1-based list position, 0 for none)
// of the lane's two pixels.
struct PairFwdState {
  float T0, T1, C00, C01, C02, C10, C11, C12;
  uint32_t last0, last1;
  int walked_batch, walked_buf;   // the last batch the walk composited and its s_rec buffer (-1: none)
};

// Forward walk of one tile's list [start, end) at the lane's pixel pair (xf,
// yf), (xf + 1, yf) of the warp block whose first pixel is (bxf, byf): records
// staged S per batch (double-buffered cp.async, the list entries of the next
// batch loaded one batch ahead); per 32-record chunk the warp's cover pass and
// bit transpose, then every lane composites its records in list order at both
// pixels (Eq. C), until T < t_eps at every pixel of the CTA.  With hslot the
// cover masks of the list's first hm_chunks chunks are stored for the
// backward; with ridx (a [2][S] array) the staged records' indices as well,
// so that a backward can start from the last batch still in s_rec.  Returns
// with every copy landed; the caller synchronises the CTA before s_rec is
// staged again.
template <int TW, int TH, int S>
__device__ __forceinline__ void pair_fwd_walk(float4 (&s_rec)[2][S][kRecordF4], uint32_t* ridx,
                                              const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
                                              uint32_t start, uint32_t end, uint32_t* hslot, int hm_chunks,
                                              float xf, float yf, float bxf, float byf, bool in0, bool in1,
                                              float t_eps, float amax, PairFwdState& st) {
  using PB = PairBlock<TW>;
  constexpr int NT = TW * TH / 2, NW = NT / 32, RPT = (S + NT - 1) / NT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  // batch 0 goes to buffer 0 now; the list entries of batch 1 are loaded
  // ahead so that its copies can be issued without waiting on them
  uint32_t rn[RPT];
#pragma unroll
  for (int q = 0; q < RPT; ++q) {
    const int jj = tid + q * NT;
    if (jj < S && start + jj < end) {
      const uint32_t r = vals[start + jj];
      if (ridx) ridx[jj] = r;
      stage_record(s_rec[0][jj], rec, r);
    }
    const uint32_t j1 = start + S + jj;
    rn[q] = (jj < S && j1 < end) ? vals[j1] : 0u;
  }
  cp_async_commit();

  float T0 = 1.0f, T1 = 1.0f, C00 = 0.0f, C01 = 0.0f, C02 = 0.0f, C10 = 0.0f, C11 = 0.0f, C12 = 0.0f;
  uint32_t last0 = 0, last1 = 0;
  bool done0 = !in0, done1 = !in1;
  bool warp_done = __all_sync(0xffffffffu, done0 && done1);

  int buf = 0, batch = 0, walked_batch = -1, walked_buf = -1;
  for (uint32_t base = start; base < end; base += S, ++batch) {
    cp_async_wait_all();
    if (!__syncthreads_or(!(done0 && done1))) break;
    const uint32_t nb = base + S;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int jj = tid + q * NT;
      if (jj < S && nb + jj < end) {
        if (ridx) ridx[(buf ^ 1) * S + jj] = rn[q];
        stage_record(s_rec[buf ^ 1][jj], rec, rn[q]);
      }
      const uint32_t j2 = nb + S + jj;
      rn[q] = (jj < S && j2 < end) ? vals[j2] : 0u;
    }
    cp_async_commit();
    walked_batch = batch;
    walked_buf = buf;
    const int cnt = (int)min((uint32_t)S, end - base);
    for (int c = 0; c < cnt && !warp_done; c += 32) {
      // pass 1: lane k finds the pairs of this warp's block that record
      // c + k may cover; the transpose gives every lane its records
      const int idx = c + lane;
      const uint32_t cov =
          idx < cnt ? pair_cover<PB::BW>(s_rec[buf][idx][0], s_rec[buf][idx][1], bxf, byf) : 0u;
      uint32_t mine = transpose32(cov, lane);
      const int jc = (int)((base - start + c) >> 5);
      if (hslot && jc < hm_chunks) {
        uint32_t* slot = hslot + (size_t)jc * (NT + NW);
        const uint32_t wide = __ballot_sync(0xffffffffu, __popc(cov) > kLaneAtomics);
        slot[tid] = mine;
        if (lane == 0) slot[NT + warp] = wide;
      }
      if (done0 && done1) mine = 0u;
      // pass 2: every lane composites its records in list order at both
      // of its pixels
      while (mine) {
        const int k = __ffs(mine) - 1;
        mine &= mine - 1;
        const int s = c + k;
        const float4 f0 = s_rec[buf][s][0];
        const float4 f1 = s_rec[buf][s][1];
        float u0, v0, u1, v1, r2a, r2b;
        rec_r2_pair(f0, f1, xf, yf, u0, v0, u1, v1, r2a, r2b);
        const bool h0 = !done0 && r2a < 1.0f, h1 = !done1 && r2b < 1.0f;
        if (!(h0 || h1)) continue;                    // outside the support (the cover is conservative)
        const float4 f2 = s_rec[buf][s][2];
        const uint32_t pos = base - start + (uint32_t)s + 1u;
        if (h0) {
          const float a = fminf(ex2_approx(fmaf(f1.w, lg2_approx(1.0f - r2a), f2.x)), amax);
          const float w = a * T0;
          C00 = fmaf(w, f2.y, C00);
          C01 = fmaf(w, f2.z, C01);
          C02 = fmaf(w, f2.w, C02);
          T0 = T0 * (1.0f - a);
          last0 = pos;
          done0 = T0 < t_eps;
        }
        if (h1) {
          const float a = fminf(ex2_approx(fmaf(f1.w, lg2_approx(1.0f - r2b), f2.x)), amax);
          const float w = a * T1;
          C10 = fmaf(w, f2.y, C10);
          C11 = fmaf(w, f2.z, C11);
          C12 = fmaf(w, f2.w, C12);
          T1 = T1 * (1.0f - a);
          last1 = pos;
          done1 = T1 < t_eps;
        }
        if (done0 && done1) mine = 0u;
      }
      warp_done = __all_sync(0xffffffffu, done0 && done1);
    }
    buf ^= 1;
  }
  cp_async_wait_all();   // no copy may still land in a buffer the next tile fills
  st.T0 = T0;
  st.T1 = T1;
  st.C00 = C00;
  st.C01 = C01;
  st.C02 = C02;
  st.C10 = C10;
  st.C11 = C11;
  st.C12 = C12;
  st.last0 = last0;
  st.last1 = last1;
  st.walked_batch = walked_batch;
  st.walked_buf = walked_buf;
}

// Epilogue of the pixel-pair forward at pixels (x, y), (x + 1, y) of view v:
// the colour C + T bg to color; T and the last contributor to Tout / ncontrib
// when those are given; with a target (tgt[ch][2 tid + i]: pixel i, channel
// ch, landed in shared memory) the L1 term, whose gradient
// sign(C - target) / (3 H W) goes to dLdC when given and to gv (pixel i,
// channel ch at gv[3 i + ch]; zero off the image or without a target).
// Returns the lane's sum of |C - target|.
template <int NT>
__device__ __forceinline__ float pair_fwd_out(const PairFwdState& st, const ViewTable& vt, int v, int x, int y,
                                              bool in0, bool in1, bool with_target, const float (&tgt)[3][2 * NT],
                                              float* __restrict__ color, float* __restrict__ Tout,
                                              uint32_t* __restrict__ ncontrib, float* __restrict__ dLdC,
                                              float (&gv)[6]) {
  const int tid = threadIdx.x;
  const int W = vt.v[v].width, H = vt.v[v].height;
  const int64_t HW = (int64_t)W * H;
  const int64_t pix = vt.v[v].pix_off + (int64_t)y * W + x;
  const int64_t o = 3 * vt.v[v].pix_off + (int64_t)y * W + x;
  const float scale = 1.0f / (3.0f * (float)HW);
  float l1 = 0.0f;
#pragma unroll
  for (int i = 0; i < 2; ++i) {
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) gv[3 * i + ch] = 0.0f;
    if (!(i == 0 ? in0 : in1)) continue;
    const float T = i == 0 ? st.T0 : st.T1;
    const float c[3] = {(i == 0 ? st.C00 : st.C10) + T * vt.v[v].bg[0], (i == 0 ? st.C01 : st.C11) + T * vt.v[v].bg[1],
                        (i == 0 ? st.C02 : st.C12) + T * vt.v[v].bg[2]};
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) color[o + i + ch * HW] = c[ch];
    if (Tout) Tout[pix + i] = T;
    if (ncontrib) ncontrib[pix + i] = i == 0 ? st.last0 : st.last1;
    if (with_target) {
      // the per-pixel L1 term and its gradient, as beta_l1_loss computes them
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        const float d = c[ch] - tgt[ch][2 * tid + i];
        l1 += fabsf(d);
        const float gd = d > 0.0f ? scale : (d < 0.0f ? -scale : 0.0f);
        gv[3 * i + ch] = gd;
        if (dLdC) dLdC[o + i + ch * HW] = gd;
      }
    }
  }
  return l1;
}

// The CTA's sum of the lanes' l1 in a fixed order (warp shuffles, then the
// warps in index order), stored to *out.  Synchronises the CTA on entry and
// exit.
template <int NW>
__device__ __forceinline__ void tile_l1_partial(float l1, float (&s_l1)[NW], float* out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) l1 += __shfl_xor_sync(0xffffffffu, l1, off);
  if (lane == 0) s_l1[warp] = l1;
  __syncthreads();
  if (tid == 0) {
    float t = 0.0f;
#pragma unroll
    for (int w = 0; w < NW; ++w) t += s_l1[w];
    *out = t;
  }
  __syncthreads();
}

template <int TW, int TH, int S, bool PERSIST>
__global__ void __launch_bounds__(TW * TH / 2, min_blocks(TW * TH / 2, pair_threads_per_sm(S))) k_raster_fwd2(
    ViewTable vt, RenderOpts ro, const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ ranges, float* __restrict__ color, float* __restrict__ Tout,
    uint32_t* __restrict__ ncontrib, const int32_t* __restrict__ status, uint32_t* ctr,
    const uint32_t* __restrict__ order, const float* __restrict__ target, float* __restrict__ dLdC,
    float* __restrict__ l1_partial, uint32_t* __restrict__ hm, size_t hm_words) {
  using PB = PairBlock<TW>;
  constexpr int NT = TW * TH / 2, NW = NT / 32;
  static_assert(pair_tiles(TW, TH) && TH % PB::BH == 0 && NT % 32 == 0, "tile must hold whole pair blocks");
  __shared__ __align__(16) float4 s_rec[2][S][kRecordF4];
  __shared__ float s_l1[NW];
  __shared__ float s_tgt[3][2 * NT];   // the pixels' targets, copied in while the tile composites
  __shared__ int s_item;
  if (*status != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float t_eps = ro.t_eps, amax = ro.alpha_max;
  for (int iter = 0;; ++iter) {
    const int g = next_tile<PERSIST>(iter, vt.total_tiles, ctr, order, &s_item);
    if (g < 0) break;
    const int v = view_of_tile(vt, g);
    const int W = vt.v[v].width, H = vt.v[v].height, ntx = vt.v[v].ntx;
    const int lt = g - vt.v[v].tile_off;
    const int ty = lt / ntx, tx = lt - ty * ntx;
    const int bx = tx * TW + (warp % PB::WX) * PB::BW, by = ty * TH + (warp / PB::WX) * PB::BH;
    const int x = bx + 2 * (lane % PB::PC), y = by + lane / PB::PC;   // pixels (x, y), (x + 1, y)
    const bool in0 = x < W && y < H, in1 = x + 1 < W && y < H;
    const uint32_t start = ranges[g], end = ranges[g + 1];
    uint32_t* const hslot = hit_tile<NT>(hm, hm_words, start, end, g);
    if (target) {
      const int64_t HW = (int64_t)W * H;
      const int64_t o = 3 * vt.v[v].pix_off + (int64_t)y * W + x;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        if (in0) cp_async4(&s_tgt[ch][2 * tid], target + o + ch * HW);
        if (in1) cp_async4(&s_tgt[ch][2 * tid + 1], target + o + 1 + ch * HW);
      }
    }
    PairFwdState fs;
    pair_fwd_walk<TW, TH, S>(s_rec, nullptr, rec, vals, start, end, hslot, INT_MAX, (float)x, (float)y, (float)bx,
                             (float)by, in0, in1, t_eps, amax, fs);
    float gv[6];
    const float l1 = pair_fwd_out<NT>(fs, vt, v, x, y, in0, in1, target != nullptr, s_tgt, color, Tout, ncontrib,
                                      dLdC, gv);
    // tile partial sum of |C - target|, reduced in a fixed order
    if (target) tile_l1_partial<NW>(l1, s_l1, l1_partial + g);
  }
  leave<PERSIST>(ctr);
}

// One pixel's terms (bwd_terms with ZERO) from its whitened coordinates,
// added to G when ADD.
template <bool ADD>
__device__ __forceinline__ bool pix_terms(float u, float vv, float r2, float4 f1, float4 f2, float amax, bool act,
                                          float gx, float gy, float gz, float& T, float& GS, float G[kGrad2d]) {
  act = act && r2 < 1.0f;
  const float beta = f1.w;
  const float base = fmaxf(1.0f - r2, 5.9604645e-8f);   // 1 - r^2 >= 2^-24 wherever r^2 < 1
  const float lb = lg2_approx(base);
  const float a0 = ex2_approx(fmaf(beta, lb, f2.x));   // the forward's alpha
  const float a = fminf(a0, amax);
  const float inv = rcp_approx(1.0f - a);
  const float Tk = T * inv;
  const float gc = fmaf(gx, f2.y, fmaf(gy, f2.z, gz * f2.w));
  const float dLa = fmaf(Tk, gc, -GS * inv);
  const float wgt = act ? a * Tk : 0.0f;
  const float t = (a0 < amax && act) ? dLa * a0 : 0.0f;   // clamped alpha: no o/beta/r^2 gradient
  const float kk = t * rcp_approx(base);
  const float g0 = kk * u, g1 = kk * vv;
  const float H[kGrad2d] = {g0, g1, g0 * u, g0 * vv, g1 * vv, t, t * lb, wgt * gx, wgt * gy, wgt * gz};
#pragma unroll
  for (int q = 0; q < kGrad2d; ++q) G[q] = ADD ? G[q] + H[q] : H[q];
  GS = act ? fmaf(wgt, gc, GS) : GS;
  T = act ? Tk : T;
  return act;
}

// Per-lane state the pixel-pair backward starts from: final transmittance,
// the suffix colour term g . S (the background's, T bg . g), dL/dC and the
// last-contributor position of the lane's two pixels (zeros off the image).
struct PairBwdState {
  float T0, T1, GS0, GS1, g0x, g0y, g0z, g1x, g1y, g1z;
  uint32_t nl0, nl1;
};

// Reverse walk of one tile's list lst at the lane's pixel pair, from the CTA's
// largest last-contributor position down: batches of S records staged as the
// forward staged them (so chunks start at multiples of 32), the list entries
// of the next batch down loaded one batch ahead; per chunk the cover masks
// (the forward's from hslot for the list's first hm_chunks chunks, else the
// cover pass again), then every lane's
// walk of its records in reverse list order at both pixels with three vector
// atomics per record, and records covering more than kLaneAtomics of the
// warp's pairs by the whole warp (reduce-scatter, one atomic per value).
// When the first batch it needs is reuse_batch, which a forward walk left
// complete in s_rec[reuse_buf] with its indices in s_ridx[reuse_buf], it
// starts from there instead of staging it again (reuse_batch = -1: never).
// Returns with every copy landed and the CTA synchronised.
template <int TW, int TH, int S>
__device__ __forceinline__ void pair_bwd_walk(float4 (&s_rec)[2][S][kRecordF4], uint32_t (&s_ridx)[2][S],
                                              uint32_t (&s_wmax)[TW * TH / 64], const float4* __restrict__ rec,
                                              const uint32_t* __restrict__ lst, const uint32_t* hslot,
                                              int hm_chunks, float* __restrict__ grad2d, float xf, float yf,
                                              float bxf, float byf, float amax, int my_field,
                                              const PairBwdState& st, int reuse_batch, int reuse_buf) {
  using PB = PairBlock<TW>;
  constexpr int NT = TW * TH / 2, NW = NT / 32, RPT = (S + NT - 1) / NT;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float T0 = st.T0, T1 = st.T1, GS0 = st.GS0, GS1 = st.GS1;
  const float g0x = st.g0x, g0y = st.g0y, g0z = st.g0z, g1x = st.g1x, g1y = st.g1y, g1z = st.g1z;
  const uint32_t nl0 = st.nl0, nl1 = st.nl1;
  const uint32_t nlm = max(nl0, nl1);
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, nlm);
  if (lane == 0) s_wmax[warp] = wmax;
  __syncthreads();
  int bmax = 0;
#pragma unroll
  for (int w = 0; w < NW; ++w) bmax = max(bmax, (int)s_wmax[w]);

  // Batch b covers list positions [b S, min(b S + S, bmax)), b = nb - 1 .. 0
  // (the forward's batches, so chunks start at multiples of 32).  The last
  // goes to buffer 0 now (or is already in reuse_buf); the list entries of
  // the one before it are loaded ahead so that its copies issue without
  // waiting.
  const int nb = (bmax + S - 1) / S;
  const bool reuse = nb > 0 && reuse_batch == nb - 1;   // CTA-uniform
  int buf = reuse ? reuse_buf : 0;
  uint32_t rn[RPT];
  {
    const int lo0 = (nb - 1) * S, lo1 = lo0 - S;
#pragma unroll
    for (int q = 0; q < RPT; ++q) {
      const int jj = tid + q * NT;
      if (!reuse && nb > 0 && jj < bmax - lo0) {
        const uint32_t r = lst[lo0 + jj];
        s_ridx[0][jj] = r;
        stage_record(s_rec[0][jj], rec, r);
      }
      rn[q] = (lo1 >= 0 && jj < S) ? lst[lo1 + jj] : 0u;
    }
    cp_async_commit();
  }

  // hit masks of the next chunk (chunks are walked from the last down),
  // loaded one chunk ahead so that their DRAM latency overlaps a chunk
  uint32_t pf_mine = 0u, pf_wide = 0u;
  int pf_chunk = -1;
  for (int b = nb - 1; b >= 0; --b) {
    const int lo = b * S;
    const int cnt = min(S, bmax - lo);
    cp_async_wait_all();
    __syncthreads();
    {
      // copies of batch b - 1 (full) into the other buffer, entries of b - 2
#pragma unroll
      for (int q = 0; q < RPT; ++q) {
        const int jj = tid + q * NT;
        if (b >= 1 && jj < S) {
          s_ridx[buf ^ 1][jj] = rn[q];
          stage_record(s_rec[buf ^ 1][jj], rec, rn[q]);
        }
        rn[q] = (b >= 2 && jj < S) ? lst[(b - 2) * S + jj] : 0u;
      }
      cp_async_commit();
    }
    for (int c = ((cnt - 1) >> 5) << 5; c >= 0; c -= 32) {
      if ((uint32_t)(lo + c) >= wmax) continue;
      uint32_t wide, mine;
      const int j = (lo + c) >> 5;
      if (hslot && j < hm_chunks) {
        if (pf_chunk == j) {                           // the forward's pass 1
          mine = pf_mine;
          wide = pf_wide;
        } else {
          const uint32_t* slot = hslot + (size_t)j * (NT + NW);
          mine = slot[tid];
          wide = slot[NT + warp];
        }
        const int limw = (int)wmax - (lo + c);         // no lane of the warp reaches past wmax
        wide &= limw >= 32 ? 0xffffffffu : (1u << limw) - 1u;
      } else {
        const int idx = c + lane;
        const uint32_t cov = (idx < cnt && (uint32_t)(lo + idx) < wmax)
                                 ? pair_cover<PB::BW>(s_rec[buf][idx][0], s_rec[buf][idx][1], bxf, byf) : 0u;
        wide = __ballot_sync(0xffffffffu, __popc(cov) > kLaneAtomics);
        mine = transpose32(cov, lane);
      }
      if (hslot && j >= 1 && j - 1 < hm_chunks) {     // the next chunk's stored masks, one chunk ahead
        const uint32_t* nslot = hslot + (size_t)(j - 1) * (NT + NW);
        pf_mine = nslot[tid];
        pf_wide = nslot[NT + warp];
        pf_chunk = j - 1;
      }
      const int lim = (int)nlm - (lo + c);           // only positions before a pixel's last contributor
      mine &= lim >= 32 ? 0xffffffffu : (lim <= 0 ? 0u : (1u << lim) - 1u);
      // pass 2, in reverse list order: between wide records every lane walks
      // its own records at both of its pixels and adds their summed terms
      // with three vector atomics; a wide record is done by the whole warp
      // together (reduce-scatter, one atomic per value)
      for (;;) {
        const int kb = wide ? 31 - __clz(wide) : -1;                 // warp-uniform
        const uint32_t above = kb >= 0 ? ~((2u << kb) - 1u) : 0xffffffffu;
        uint32_t seg = mine & above;
        mine &= ~above;
        while (seg) {
          const int k = 31 - __clz(seg);
          seg &= ~(1u << k);
          const int s = c + k;
          const uint32_t pos = (uint32_t)(lo + s);
          const float4 f0 = s_rec[buf][s][0], f1 = s_rec[buf][s][1], f2 = s_rec[buf][s][2];
          float u0, v0, u1, v1, r2a, r2b;
          rec_r2_pair(f0, f1, xf, yf, u0, v0, u1, v1, r2a, r2b);
          float G[kGrad2d];
          const bool a0 = pix_terms<false>(u0, v0, r2a, f1, f2, amax, pos < nl0, g0x, g0y, g0z, T0, GS0, G);
          const bool a1 = pix_terms<true>(u1, v1, r2b, f1, f2, amax, pos < nl1, g1x, g1y, g1z, T1, GS1, G);
          if (!(a0 || a1)) continue;                  // outside the support (the cover is conservative)
          float* gdst = grad2d + (size_t)s_ridx[buf][s] * kGrad2dStride;
          red_add_v4(gdst + 0, G[0], G[1], G[2], G[3]);
          red_add_v4(gdst + 4, G[4], G[5], G[6], G[7]);
          red_add_v4(gdst + 8, G[8], G[9], 0.0f, 0.0f);
        }
        if (kb < 0) break;
        wide &= ~(1u << kb);
        const bool mine_kb = (mine >> kb) & 1u;
        mine &= ~(1u << kb);
        const int s = c + kb;
        const uint32_t pos = (uint32_t)(lo + s);
        const float4 f0 = s_rec[buf][s][0], f1 = s_rec[buf][s][1], f2 = s_rec[buf][s][2];
        float u0, v0, u1, v1, r2a, r2b;
        rec_r2_pair(f0, f1, xf, yf, u0, v0, u1, v1, r2a, r2b);
        float G[kGrad2d];                              // zero where a pixel is not covered
        pix_terms<false>(u0, v0, r2a, f1, f2, amax, mine_kb && pos < nl0, g0x, g0y, g0z, T0, GS0, G);
        pix_terms<true>(u1, v1, r2b, f1, f2, amax, mine_kb && pos < nl1, g1x, g1y, g1z, T1, GS1, G);
        const float tot = warp_sum10(G, lane);
        float* gdst = grad2d + (size_t)s_ridx[buf][s] * kGrad2dStride;
        if (my_field >= 0 && tot != 0.0f) atomicAdd(gdst + my_field, tot);
      }
    }
    buf ^= 1;
  }
  cp_async_wait_all();   // no copy may still land in a buffer the next tile fills
  __syncthreads();
}

template <int TW, int TH, int S, bool PERSIST>
__global__ void __launch_bounds__(TW * TH / 2, min_blocks(TW * TH / 2, pair_threads_per_sm(S))) k_raster_bwd2(
    ViewTable vt, RenderOpts ro, const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ ranges, const float* __restrict__ Tfin, const uint32_t* __restrict__ ncontrib,
    const float* __restrict__ dLdC, float* __restrict__ grad2d, const int32_t* __restrict__ status, uint32_t* ctr,
    const uint32_t* __restrict__ order, const uint32_t* __restrict__ hm, size_t hm_words) {
  using PB = PairBlock<TW>;
  constexpr int NT = TW * TH / 2, NW = NT / 32;
  static_assert(pair_tiles(TW, TH) && TH % PB::BH == 0 && NT % 32 == 0, "tile must hold whole pair blocks");
  __shared__ __align__(16) float4 s_rec[2][S][kRecordF4];
  __shared__ uint32_t s_ridx[2][S];
  __shared__ uint32_t s_wmax[NW];
  __shared__ int s_item;
  if (*status != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float amax = ro.alpha_max;
  const int my_field = warp_sum10_field(lane);
  for (int iter = 0;; ++iter) {
    const int g = next_tile<PERSIST>(iter, vt.total_tiles, ctr, order, &s_item);
    if (g < 0) break;
    const int v = view_of_tile(vt, g);
    const int W = vt.v[v].width, H = vt.v[v].height, ntx = vt.v[v].ntx;
    const int lt = g - vt.v[v].tile_off;
    const int ty = lt / ntx, tx = lt - ty * ntx;
    const int bx = tx * TW + (warp % PB::WX) * PB::BW, by = ty * TH + (warp / PB::WX) * PB::BH;
    const int x = bx + 2 * (lane % PB::PC), y = by + lane / PB::PC;   // pixels (x, y), (x + 1, y)
    const bool in0 = x < W && y < H, in1 = x + 1 < W && y < H;
    const uint32_t range0 = ranges[g];
    const uint32_t* const hslot = hit_tile<NT>(const_cast<uint32_t*>(hm), hm_words, range0, ranges[g + 1], g);

    PairBwdState bs{1.0f, 1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0u, 0u};
    {
      const int64_t HW = (int64_t)W * H;
      const int64_t pix = vt.v[v].pix_off + (int64_t)y * W + x;
      const float* gb = dLdC + 3 * vt.v[v].pix_off + (int64_t)y * W + x;
      const float* bg = vt.v[v].bg;
      if (in0) {
        bs.g0x = gb[0];
        bs.g0y = gb[HW];
        bs.g0z = gb[2 * HW];
        bs.T0 = Tfin[pix];
        bs.nl0 = ncontrib[pix];
        bs.GS0 = bs.T0 * (bs.g0x * bg[0] + bs.g0y * bg[1] + bs.g0z * bg[2]);
      }
      if (in1) {
        bs.g1x = gb[1];
        bs.g1y = gb[HW + 1];
        bs.g1z = gb[2 * HW + 1];
        bs.T1 = Tfin[pix + 1];
        bs.nl1 = ncontrib[pix + 1];
        bs.GS1 = bs.T1 * (bs.g1x * bg[0] + bs.g1y * bg[1] + bs.g1z * bg[2]);
      }
    }
    pair_bwd_walk<TW, TH, S>(s_rec, s_ridx, s_wmax, rec, vals + range0, hslot, INT_MAX, grad2d, (float)x, (float)y,
                             (float)bx, (float)by, amax, my_field, bs, -1, 0);
  }
  leave<PERSIST>(ctr);
}

// Forward, L1 loss and backward of each tile in one CTA (the pixel-pair
// tilings): the forward walk and epilogue of k_raster_fwd2 with the L1 target,
// then the reverse walk of k_raster_bwd2 started from the lanes' registers
// (final T, last contributors, dL/dC), so that no per-pixel state goes through
// memory between the two and the backward's record gathers find the records
// the forward just staged in L2.  T, the last contributors and dL/dC are
// stored only when their buffers are given.  The forward's cover masks of
// each list's first kStepMaskChunks(NT) chunks of 32 records (192 records at
// 64 threads, 1.5 KB) are kept in shared memory; the backward repeats the
// cover passes of later chunks.  Colour, L1 partials, T, last contributors and dL/dC
// equal k_raster_fwd2's bit for bit, and every per-record term the backward
// adds equals k_raster_bwd2's (the sums differ only by the order of the
// floating-point atomics).
constexpr int kStepMaskChunks(int nt) { return nt >= 384 ? 1 : 384 / nt; }

template <int TW, int TH, int S, bool PERSIST>
__global__ void __launch_bounds__(TW * TH / 2, min_blocks(TW * TH / 2, pair_threads_per_sm(S))) k_raster_step2(
    ViewTable vt, RenderOpts ro, const float4* __restrict__ rec, const uint32_t* __restrict__ vals,
    const uint32_t* __restrict__ ranges, float* __restrict__ color, float* __restrict__ Tout,
    uint32_t* __restrict__ ncontrib, const int32_t* __restrict__ status, uint32_t* ctr,
    const uint32_t* __restrict__ order, const float* __restrict__ target, float* __restrict__ dLdC,
    float* __restrict__ l1_partial, float* __restrict__ grad2d) {
  using PB = PairBlock<TW>;
  constexpr int NT = TW * TH / 2, NW = NT / 32;
  static_assert(pair_tiles(TW, TH) && TH % PB::BH == 0 && NT % 32 == 0, "tile must hold whole pair blocks");
  __shared__ __align__(16) float4 s_rec[2][S][kRecordF4];
  __shared__ uint32_t s_ridx[2][S];
  __shared__ float s_l1[NW];
  __shared__ float s_tgt[3][2 * NT];   // the pixels' targets, copied in while the tile composites
  __shared__ uint32_t s_wmax[NW];
  __shared__ uint32_t s_hm[kStepMaskChunks(NT) * (NT + NW)];   // cover masks, hit-mask slot layout
  __shared__ int s_item;
  if (*status != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const float t_eps = ro.t_eps, amax = ro.alpha_max;
  const int my_field = warp_sum10_field(lane);
  for (int iter = 0;; ++iter) {
    const int g = next_tile<PERSIST>(iter, vt.total_tiles, ctr, order, &s_item);
    if (g < 0) break;
    const int v = view_of_tile(vt, g);
    const int W = vt.v[v].width, H = vt.v[v].height, ntx = vt.v[v].ntx;
    const int lt = g - vt.v[v].tile_off;
    const int ty = lt / ntx, tx = lt - ty * ntx;
    const int bx = tx * TW + (warp % PB::WX) * PB::BW, by = ty * TH + (warp / PB::WX) * PB::BH;
    const int x = bx + 2 * (lane % PB::PC), y = by + lane / PB::PC;   // pixels (x, y), (x + 1, y)
    const bool in0 = x < W && y < H, in1 = x + 1 < W && y < H;
    const float xf = (float)x, yf = (float)y, bxf = (float)bx, byf = (float)by;
    const uint32_t start = ranges[g], end = ranges[g + 1];
    {
      const int64_t HW = (int64_t)W * H;
      const int64_t o = 3 * vt.v[v].pix_off + (int64_t)y * W + x;
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        if (in0) cp_async4(&s_tgt[ch][2 * tid], target + o + ch * HW);
        if (in1) cp_async4(&s_tgt[ch][2 * tid + 1], target + o + 1 + ch * HW);
      }
    }
    PairFwdState fs;
    pair_fwd_walk<TW, TH, S>(s_rec, &s_ridx[0][0], rec, vals, start, end, s_hm, kStepMaskChunks(NT), xf, yf, bxf,
                             byf, in0, in1, t_eps, amax, fs);
    float gv[6];
    const float l1 = pair_fwd_out<NT>(fs, vt, v, x, y, in0, in1, true, s_tgt, color, Tout, ncontrib, dLdC, gv);
    // also the barrier after which no warp still reads the forward's s_rec
    // and every cover mask in s_hm is visible to the whole CTA
    tile_l1_partial<NW>(l1, s_l1, l1_partial + g);

    const float* bg = vt.v[v].bg;
    PairBwdState bs;
    bs.T0 = fs.T0;
    bs.T1 = fs.T1;
    bs.g0x = gv[0];
    bs.g0y = gv[1];
    bs.g0z = gv[2];
    bs.g1x = gv[3];
    bs.g1y = gv[4];
    bs.g1z = gv[5];
    bs.nl0 = fs.last0;
    bs.nl1 = fs.last1;
    bs.GS0 = in0 ? bs.T0 * (bs.g0x * bg[0] + bs.g0y * bg[1] + bs.g0z * bg[2]) : 0.0f;
    bs.GS1 = in1 ? bs.T1 * (bs.g1x * bg[0] + bs.g1y * bg[1] + bs.g1z * bg[2]) : 0.0f;
    pair_bwd_walk<TW, TH, S>(s_rec, s_ridx, s_wmax, rec, vals + start, s_hm, kStepMaskChunks(NT), grad2d, xf, yf,
                             bxf, byf, amax, my_field, bs, fs.walked_batch, fs.walked_buf);
  }
  leave<PERSIST>(ctr);
}

// ---------------------------------------------------------------------------
// longest-first schedule: bucket b = bit length of the tile's pair count,
// buckets emitted from the longest down (order inside a bucket is arbitrary:
// the result of a tile does not depend on when it runs).
// layout (u32): [0..1] forward counter, [2..3] backward counter, [16..79]
// bucket counts, [80..143] bucket cursors, [144..] order.
// ---------------------------------------------------------------------------
constexpr int kSchedHist = 16, kSchedCursor = 80, kSchedOrder = 144, kBuckets = 33;

__device__ __forceinline__ int tile_bucket(uint32_t count) {
  return count == 0u ? 0 : 32 - __clz(count);
}

__global__ void k_sched_prep(uint32_t* sched) {
  for (int i = threadIdx.x; i < kSchedOrder; i += blockDim.x) sched[i] = 0u;
}

__global__ void k_sched_hist(const uint32_t* __restrict__ ranges, int total_tiles, uint32_t* sched,
                             const int32_t* __restrict__ status) {
  __shared__ uint32_t h[kBuckets];
  if (*status != 0) return;
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total_tiles; g += gridDim.x * blockDim.x)
    atomicAdd(&h[tile_bucket(ranges[g + 1] - ranges[g])], 1u);
  __syncthreads();
  for (int i = threadIdx.x; i < kBuckets; i += blockDim.x)
    if (h[i]) atomicAdd(&sched[kSchedHist + i], h[i]);
}

__global__ void k_sched_scatter(const uint32_t* __restrict__ ranges, int total_tiles,
                                uint32_t* sched, const int32_t* __restrict__ status) {
  __shared__ uint32_t base[kBuckets];
  if (*status != 0) return;
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int b = kBuckets - 1; b >= 0; --b) {
      base[b] = run;
      run += sched[kSchedHist + b];
    }
  }
  __syncthreads();
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < total_tiles; g += gridDim.x * blockDim.x) {
    const int b = tile_bucket(ranges[g + 1] - ranges[g]);
    const uint32_t pos = base[b] + atomicAdd(&sched[kSchedCursor + b], 1u);
    sched[kSchedOrder + pos] = (uint32_t)g;
  }
}

// L1 loss: one thread per pixel; block partial sums then a deterministic
// per-view reduction.
__global__ void __launch_bounds__(256) k_l1(ViewTable vt, const float* __restrict__ color,
                                            const float* __restrict__ target, float* __restrict__ dLdC,
                                            float* __restrict__ partial) {
  __shared__ float s_w[8];
  const int b = blockIdx.x;
  int lo = 0, hi = vt.n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (vt.v[mid].pad0 <= b) lo = mid; else hi = mid - 1;
  }
  const int v = lo;
  const int64_t HW = (int64_t)vt.v[v].width * vt.v[v].height;
  const int64_t p = (int64_t)(b - vt.v[v].pad0) * 256 + threadIdx.x;
  float acc = 0.0f;
  if (p < HW) {
    const float scale = 1.0f / (3.0f * (float)HW);
    const int64_t o = 3 * vt.v[v].pix_off + p;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      float d = color[o + ch * HW] - target[o + ch * HW];
      acc += fabsf(d);
      dLdC[o + ch * HW] = d > 0.0f ? scale : (d < 0.0f ? -scale : 0.0f);
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < 8; ++w) t += s_w[w];
    partial[b] = t;
  }
}

__global__ void k_l1_reduce(ViewTable vt, const float* __restrict__ partial, int total_blocks,
                            float* __restrict__ loss) {
  __shared__ double s_w[32];
  const int v = blockIdx.x;
  const int b0 = vt.v[v].pad0;
  const int b1 = (v + 1 < vt.n_views) ? vt.v[v + 1].pad0 : total_blocks;
  double acc = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) acc += (double)partial[b];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
    const double HW = (double)vt.v[v].width * vt.v[v].height;
    loss[v] = (float)(t / (3.0 * HW));
  }
}

}  // namespace

size_t schedule_bytes(int total_tiles) { return (size_t)(kSchedOrder + total_tiles) * 4; }

cudaError_t launch_schedule(const ViewTable& vt, const uint32_t* ranges, uint32_t* sched,
                            const int32_t* status, cudaStream_t s) {
  const int T = vt.total_tiles;
  const int grid = std::max(1, std::min((T + 255) / 256, device_sm_count() * 4));
  k_sched_prep<<<1, 160, 0, s>>>(sched);
  k_sched_hist<<<grid, 256, 0, s>>>(ranges, T, sched, status);
  k_sched_scatter<<<grid, 256, 0, s>>>(ranges, T, sched, status);
  return cudaGetLastError();
}

namespace {

template <int TW, int TH>
constexpr bool kPairs = pair_tiles(TW, TH);
static_assert(pair_tiles(16, 8) && pair_tiles(8, 8) && !pair_tiles(8, 4), "pixel-pair tile rule");

template <typename K>
int persistent_grid(K kernel, int threads, int total_tiles) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return std::max(1, std::min(total_tiles, per_sm * device_sm_count()));
}

template <int TW, int TH, int S>
cudaError_t fwd_shape(const ViewTable& vt, const RenderOpts& ro, const float4* rec,
                      const uint32_t* vals, const uint32_t* ranges, float* color, float* T_final,
                      uint32_t* n_contrib, const int32_t* status, uint32_t* sched, const float* target,
                      float* dL_dcolor, float* l1_partial, HitMasks hm, cudaStream_t s) {
  if constexpr (kPairs<TW, TH>) {
    constexpr int NT = TW * TH / 2;
    if (sched) {
      auto k = k_raster_fwd2<TW, TH, S, true>;
      k<<<persistent_grid(k, NT, vt.total_tiles), NT, 0, s>>>(
          vt, ro, rec, vals, ranges, color, T_final, n_contrib, status, sched + 0, sched + kSchedOrder,
          target, dL_dcolor, l1_partial, hm.words, hm.n_words);
    } else {
      k_raster_fwd2<TW, TH, S, false><<<vt.total_tiles, NT, 0, s>>>(
          vt, ro, rec, vals, ranges, color, T_final, n_contrib, status, nullptr, nullptr, target, dL_dcolor,
          l1_partial, hm.words, hm.n_words);
    }
  } else {
    if (sched) {
      auto k = k_raster_fwd<TW, TH, S, true>;
      k<<<persistent_grid(k, TW * TH, vt.total_tiles), TW * TH, 0, s>>>(
          vt, ro, rec, vals, ranges, color, T_final, n_contrib, status, sched + 0, sched + kSchedOrder,
          target, dL_dcolor, l1_partial, hm.words, hm.n_words);
    } else {
      k_raster_fwd<TW, TH, S, false><<<vt.total_tiles, TW * TH, 0, s>>>(
          vt, ro, rec, vals, ranges, color, T_final, n_contrib, status, nullptr, nullptr, target, dL_dcolor,
          l1_partial, hm.words, hm.n_words);
    }
  }
  return cudaGetLastError();
}

template <int TW, int TH, int S>
cudaError_t bwd_shape(const ViewTable& vt, const RenderOpts& ro, const float4* rec,
                      const uint32_t* vals, const uint32_t* ranges, const float* T_final,
                      const uint32_t* n_contrib, const float* dL_dcolor, float* grad2d,
                      const int32_t* status, uint32_t* sched, HitMasks hm, cudaStream_t s) {
  if constexpr (kPairs<TW, TH>) {
    constexpr int NT = TW * TH / 2;
    if (sched) {
      auto k = k_raster_bwd2<TW, TH, S, true>;
      k<<<persistent_grid(k, NT, vt.total_tiles), NT, 0, s>>>(
          vt, ro, rec, vals, ranges, T_final, n_contrib, dL_dcolor, grad2d, status, sched + 2,
          sched + kSchedOrder, hm.words, hm.n_words);
    } else {
      k_raster_bwd2<TW, TH, S, false><<<vt.total_tiles, NT, 0, s>>>(
          vt, ro, rec, vals, ranges, T_final, n_contrib, dL_dcolor, grad2d, status, nullptr, nullptr,
          hm.words, hm.n_words);
    }
  } else {
    if (sched) {
      auto k = k_raster_bwd<TW, TH, S, true>;
      k<<<persistent_grid(k, TW * TH, vt.total_tiles), TW * TH, 0, s>>>(
          vt, ro, rec, vals, ranges, T_final, n_contrib, dL_dcolor, grad2d, status, sched + 2,
          sched + kSchedOrder, hm.words, hm.n_words);
    } else {
      k_raster_bwd<TW, TH, S, false><<<vt.total_tiles, TW * TH, 0, s>>>(
          vt, ro, rec, vals, ranges, T_final, n_contrib, dL_dcolor, grad2d, status, nullptr, nullptr,
          hm.words, hm.n_words);
    }
  }
  return cudaGetLastError();
}

// Forward + L1 + backward in one launch (pixel-pair tilings only).
template <int TW, int TH, int S>
cudaError_t step_shape(const ViewTable& vt, const RenderOpts& ro, const float4* rec, const uint32_t* vals,
                       const uint32_t* ranges, float* color, float* T_final, uint32_t* n_contrib,
                       const int32_t* status, uint32_t* sched, const float* target, float* dL_dcolor,
                       float* l1_partial, float* grad2d, cudaStream_t s) {
  if constexpr (kPairs<TW, TH>) {
    constexpr int NT = TW * TH / 2;
    if (sched) {
      auto k = k_raster_step2<TW, TH, S, true>;
      k<<<persistent_grid(k, NT, vt.total_tiles), NT, 0, s>>>(
          vt, ro, rec, vals, ranges, color, T_final, n_contrib, status, sched + 0, sched + kSchedOrder, target,
          dL_dcolor, l1_partial, grad2d);
    } else {
      k_raster_step2<TW, TH, S, false><<<vt.total_tiles, NT, 0, s>>>(
          vt, ro, rec, vals, ranges, color, T_final, n_contrib, status, nullptr, nullptr, target, dL_dcolor,
          l1_partial, grad2d);
    }
    return cudaGetLastError();
  } else {
    return cudaErrorInvalidValue;   // 8 x 4 tiles have no pixel-pair kernels
  }
}

// (tile shape, batch) -> instantiation.  Supported: 8x4 (one warp), 8x8,
// 16x8, 16x16, 32x16 tiles; batches of 64, 128 or 256 records (at most 8
// records per thread).
#define BETA_TILE_DISPATCH(FN, ...)                                                 \
  switch (ro.tile_w * 1000 + ro.tile_h) {                                           \
    case 8004:                                                                      \
      if (ro.batch_s == 64) return FN<8, 4, 64>(__VA_ARGS__);                       \
      if (ro.batch_s == 128) return FN<8, 4, 128>(__VA_ARGS__);                     \
      return FN<8, 4, 256>(__VA_ARGS__);                                            \
    case 8008:                                                                      \
      if (ro.batch_s == 64) return FN<8, 8, 64>(__VA_ARGS__);                       \
      if (ro.batch_s == 128) return FN<8, 8, 128>(__VA_ARGS__);                     \
      return FN<8, 8, 256>(__VA_ARGS__);                                            \
    case 16008:                                                                     \
      if (ro.batch_s == 64) return FN<16, 8, 64>(__VA_ARGS__);                      \
      if (ro.batch_s == 128) return FN<16, 8, 128>(__VA_ARGS__);                    \
      return FN<16, 8, 256>(__VA_ARGS__);                                           \
    case 16016:                                                                     \
      if (ro.batch_s == 64) return FN<16, 16, 64>(__VA_ARGS__);                     \
      if (ro.batch_s == 128) return FN<16, 16, 128>(__VA_ARGS__);                   \
      return FN<16, 16, 256>(__VA_ARGS__);                                          \
    case 32016:                                                                     \
      if (ro.batch_s == 64) return FN<32, 16, 64>(__VA_ARGS__);                     \
      if (ro.batch_s == 128) return FN<32, 16, 128>(__VA_ARGS__);                   \
      return FN<32, 16, 256>(__VA_ARGS__);                                          \
    default:                                                                        \
      return cudaErrorInvalidValue;                                                 \
  }

}  // namespace

cudaError_t launch_raster_fwd(const ViewTable& vt, const RenderOpts& ro, const float4* rec,
                              const uint32_t* vals, const uint32_t* ranges, float* color,
                              float* T_final, uint32_t* n_contrib, const int32_t* status,
                              uint32_t* sched, HitMasks hm, cudaStream_t s) {
  if (vt.total_tiles <= 0) return cudaSuccess;
  BETA_TILE_DISPATCH(fwd_shape, vt, ro, rec, vals, ranges, color, T_final, n_contrib, status, sched,
                     nullptr, nullptr, nullptr, hm, s)
}

size_t hit_mask_bytes(const ViewTable& vt, const RenderOpts& ro, int64_t cap) {
  // one word per lane (per pixel pair in the pixel-pair kernels) and one per warp
  const bool pairs = pair_tiles(ro.tile_w, ro.tile_h);
  const int64_t nt = (int64_t)ro.tile_w * ro.tile_h / (pairs ? 2 : 1);
  const int64_t slots = (std::max<int64_t>(cap, 0) >> 5) + vt.total_tiles + 1;
  return (size_t)slots * (size_t)(nt + nt / 32) * sizeof(uint32_t);
}

size_t fwd_l1_ws_bytes(const ViewTable& vt) { return (size_t)std::max(vt.total_tiles, 1) * sizeof(float); }

// Forward with the L1 loss in its epilogue: the kernel writes dL/dC and one
// partial sum per tile; k_l1_reduce then sums each view's tiles in order.
cudaError_t launch_raster_fwd_l1(const ViewTable& vt_in, const RenderOpts& ro, const float4* rec,
                                 const uint32_t* vals, const uint32_t* ranges, float* color,
                                 float* T_final, uint32_t* n_contrib, const int32_t* status,
                                 uint32_t* sched, const float* target, float* loss, float* dL_dcolor,
                                 float* ws, HitMasks hm, cudaStream_t s) {
  if (vt_in.total_tiles <= 0) return cudaSuccess;
  cudaError_t e = [&]() -> cudaError_t {
    const ViewTable& vt = vt_in;
    BETA_TILE_DISPATCH(fwd_shape, vt, ro, rec, vals, ranges, color, T_final, n_contrib, status, sched,
                       target, dL_dcolor, ws, hm, s)
  }();
  if (e != cudaSuccess) return e;
  ViewTable vt = vt_in;   // the reduce finds view v's partials from tile_off[v]
  for (int v = 0; v < vt.n_views; ++v) vt.v[v].pad0 = vt.v[v].tile_off;
  k_l1_reduce<<<vt.n_views, 256, 0, s>>>(vt, ws, vt.total_tiles, loss);
  return cudaGetLastError();
}

bool raster_step_supported(const RenderOpts& ro) { return pair_tiles(ro.tile_w, ro.tile_h); }

// Forward, L1 loss and backward in one launch; k_l1_reduce then sums each
// view's tile partials in order, as launch_raster_fwd_l1 does.
cudaError_t launch_raster_step_l1(const ViewTable& vt_in, const RenderOpts& ro, const float4* rec,
                                  const uint32_t* vals, const uint32_t* ranges, float* color, float* T_final,
                                  uint32_t* n_contrib, const int32_t* status, uint32_t* sched, const float* target,
                                  float* loss, float* dL_dcolor, float* ws, float* grad2d, cudaStream_t s) {
  if (vt_in.total_tiles <= 0) return cudaSuccess;
  if (!raster_step_supported(ro)) return cudaErrorInvalidValue;
  cudaError_t e = [&]() -> cudaError_t {
    const ViewTable& vt = vt_in;
    BETA_TILE_DISPATCH(step_shape, vt, ro, rec, vals, ranges, color, T_final, n_contrib, status, sched, target,
                       dL_dcolor, ws, grad2d, s)
  }();
  if (e != cudaSuccess) return e;
  ViewTable vt = vt_in;   // the reduce finds view v's partials from tile_off[v]
  for (int v = 0; v < vt.n_views; ++v) vt.v[v].pad0 = vt.v[v].tile_off;
  k_l1_reduce<<<vt.n_views, 256, 0, s>>>(vt, ws, vt.total_tiles, loss);
  return cudaGetLastError();
}

cudaError_t launch_raster_bwd(const ViewTable& vt, const RenderOpts& ro, const float4* rec,
                              const uint32_t* vals, const uint32_t* ranges, const float* T_final,
                              const uint32_t* n_contrib, const float* dL_dcolor, float* grad2d,
                              const int32_t* status, uint32_t* sched, HitMasks hm, cudaStream_t s) {
  if (vt.total_tiles <= 0) return cudaSuccess;
  BETA_TILE_DISPATCH(bwd_shape, vt, ro, rec, vals, ranges, T_final, n_contrib, dL_dcolor, grad2d,
                     status, sched, hm, s)
}

// the L1 block offsets of each view ride in ViewDev::pad0
static int l1_blocks(ViewTable& vt) {
  int b = 0;
  for (int v = 0; v < vt.n_views; ++v) {
    vt.v[v].pad0 = b;
    int64_t HW = (int64_t)vt.v[v].width * vt.v[v].height;
    b += (int)((HW + 255) / 256);
  }
  return b;
}

size_t l1_ws_bytes(const ViewTable& vt) {
  ViewTable t = vt;
  return (size_t)l1_blocks(t) * sizeof(float);
}

cudaError_t launch_l1(const ViewTable& vt_in, const float* color, const float* target, float* loss,
                      float* dL_dcolor, float* ws, cudaStream_t s) {
  ViewTable vt = vt_in;
  int nb = l1_blocks(vt);
  if (nb <= 0) return cudaSuccess;
  k_l1<<<nb, 256, 0, s>>>(vt, color, target, dL_dcolor, ws);
  k_l1_reduce<<<vt.n_views, 256, 0, s>>>(vt, ws, nb, loss);
  return cudaGetLastError();
}

}  // namespace beta
