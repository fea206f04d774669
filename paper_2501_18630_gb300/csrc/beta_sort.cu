// beta_sort.cu -- binning and depth ordering of (tile, record) pairs.
//
// Sec. 3.2 of arXiv 2501.18630 composites "after sorting overlapping
// primitives by depth relative to the camera".  Here every record (view,
// primitive) is first ordered by its depth key with a stable LSD radix sort;
// the pairs (global tile, record) are then emitted in that order and sorted
// stably by tile alone.  The result equals a sort of the pairs by
// (tile, depth key, primitive index) while moving only 32-bit keys.
//
// Both radix sorts are onesweep sorts (one digit histogram pass for all
// digits, then one scatter kernel per 8-bit digit whose CTAs chain their
// digit offsets by decoupled look-back).  Every look-back wait is bounded:
// after kSpinLimit polls the CTA records BETA_ERR_TIMEOUT and proceeds.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "beta_internal.cuh"

namespace beta {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;                            // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;     // 4096 keys per CTA tile
constexpr int kScanItems = 8;
constexpr int kScanTile = kSortThreads * kScanItems;     // 2048 records per scan block
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagInc = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr int kSpinLimit = 1 << 20;
constexpr int kLookWin = 8;   // look-back predecessors loaded per round
constexpr int kMaxPasses = 4;
constexpr int kOnesweepSmem = 2 * kSortTile * 4;  // staged keys + values (32 KB)

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Workspace carve-up (offsets are 256-byte aligned).
struct SortWs {
  uint32_t* dkey_a;
  uint32_t* dkey_b;
  uint32_t* dval_a;
  uint32_t* dval_b;
  unsigned long long* look_e;   // [nb_scan] emit look-back (flag | inclusive or aggregate count)
  uint32_t* pkey_a;
  uint32_t* pkey_b;
  uint32_t* pval_ws;
  uint32_t* ghist;      // [2][kMaxPasses][512]: depth sort, tile sort
  uint32_t* counters;   // [2][kMaxPasses] look-back tile counters, then the emit ticket
  uint32_t* look_d;     // [4][nblk_d][256]
  uint32_t* look_t;     // [npass_t][nblk_t][radix_t]
  size_t bytes;
};

// Digit plan of the tile-id sort: 8-bit passes, except that 17- or 18-bit
// tile ids take two 9-bit passes instead of three 8-bit ones.
struct TilePlan {
  int passes, bits;
};
static TilePlan tile_plan(int total_tiles) {
  int b = 0;
  while ((1ll << b) < (int64_t)total_tiles) ++b;
  if (b == 17 || b == 18) return {2, 9};
  return {(b + 7) / 8, 8};
}

static SortWs carve(void* base, int64_t n_items, int64_t cap, int total_tiles) {
  SortWs w{};
  char* p = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += align256(bytes);
    return q;
  };
  int64_t nblk_d = cdiv(n_items, kSortTile);
  int64_t nblk_t = cdiv(cap > 0 ? cap : 1, kSortTile);
  int64_t nb_scan = cdiv(n_items, kScanTile);
  const TilePlan tp = tile_plan(total_tiles);
  w.dkey_a = (uint32_t*)take(n_items * 4);
  w.dkey_b = (uint32_t*)take(n_items * 4);
  w.dval_a = (uint32_t*)take(n_items * 4);
  w.dval_b = (uint32_t*)take(n_items * 4);
  w.look_e = (unsigned long long*)take(nb_scan * 8);
  w.pkey_a = (uint32_t*)take(cap * 4);
  w.pkey_b = (uint32_t*)take(cap * 4);
  w.pval_ws = (uint32_t*)take(cap * 4);
  w.ghist = (uint32_t*)take(2 * kMaxPasses * 512 * 4);
  w.counters = (uint32_t*)take((2 * kMaxPasses + 1) * 4);
  w.look_d = (uint32_t*)take((size_t)4 * nblk_d * 256 * 4);
  w.look_t = (uint32_t*)take((size_t)(tp.passes > 0 ? tp.passes : 1) * nblk_t * (1 << tp.bits) * 4);
  w.bytes = off;
  return w;
}

size_t binsort_ws_bytes(int64_t n_items, int64_t cap, int total_tiles) {
  return carve(nullptr, n_items, cap, total_tiles).bytes;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

__global__ void k_sort_prep(uint32_t* ghist, uint32_t* counters, unsigned long long* look_e,
                            int64_t nb_scan, int64_t* d_count, int32_t* status) {
  int t = threadIdx.x;
  for (int i = t; i < 2 * kMaxPasses * 512; i += blockDim.x) ghist[i] = 0;
  for (int64_t i = t; i < nb_scan; i += blockDim.x) look_e[i] = 0ull;
  if (t < 2 * kMaxPasses + 1) counters[t] = 0;
  if (t == 0) {
    *d_count = 0;
    *status = 0;
  }
}

// Adds one key per lane to the per-pass digit histograms (BITS-bit digits).
// Per pass, the leader's digit and its peers cost one shared-memory atomic,
// the other lanes add themselves (a second leader round measured slower:
// spread digits rarely share).  Warp-uniform call.
template <int BITS>
__device__ __forceinline__ void hist_add(uint32_t k, bool valid, int npass, uint32_t (*h)[1 << BITS],
                                         int lane) {
  constexpr uint32_t kMask = (1u << BITS) - 1u;
  const uint32_t vmask = __ballot_sync(0xffffffffu, valid);
  if (vmask == 0u) return;
  for (int p = 0; p < npass; ++p) {
    const uint32_t d = (k >> (BITS * p)) & kMask;
    // the leader's digit and its peers: one atomic (a digit most of the warp
    // shares, as in the depth keys' top bytes); the rest add themselves
    const int leader = __ffs(vmask) - 1;
    const uint32_t dl = __shfl_sync(0xffffffffu, d, leader);
    const uint32_t peers = __ballot_sync(0xffffffffu, valid && d == dl);
    if (lane == leader) atomicAdd(&h[p][dl], (uint32_t)__popc(peers));
    if (valid && d != dl) atomicAdd(&h[p][d], 1u);
  }
}

// Digit histograms of every pass at once (at most NPMAX passes of BITS
// bits); also clears the look-back table of the sort (only the tiles that
// `count` needs).  Keys are read as 16-byte vectors, kHistVec of them per
// thread in flight; each warp counts into its own shared-memory histograms
// (no contention between warps), which are summed at the end.
constexpr int kHistVec = 4;

template <int BITS, int NPMAX>
__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const uint32_t* __restrict__ keys,
                                                             int64_t count_host,
                                                             const int64_t* __restrict__ d_count,
                                                             int64_t cap, int npass,
                                                             uint32_t* __restrict__ ghist,
                                                             uint32_t* __restrict__ look,
                                                             int64_t look_stride_tiles) {
  constexpr int R = 1 << BITS;
  __shared__ uint32_t h[kSortThreads / 32][NPMAX][R];
  const int64_t count = d_count ? min(*d_count, cap) : count_host;
  for (int i = threadIdx.x; i < (kSortThreads / 32) * NPMAX * R; i += blockDim.x) (&h[0][0][0])[i] = 0;
  // clear the look-back entries of the tiles this sort will use (per pass)
  const int64_t nblk = (count + kSortTile - 1) / kSortTile;
  const int64_t used = nblk * R;
  const int64_t gstride = (int64_t)gridDim.x * blockDim.x;
  for (int p = 0; p < npass; ++p) {
    uint32_t* lp = look + (int64_t)p * look_stride_tiles * R;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < used; i += gstride) lp[i] = 0;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t (*hw)[R] = h[warp];
  const int64_t nvec = count >> 2;
  const uint4* kv = reinterpret_cast<const uint4*>(keys);
  constexpr int64_t kRound = (int64_t)kSortThreads * kHistVec;
  for (int64_t g0 = (int64_t)blockIdx.x * kRound; g0 < nvec; g0 += (int64_t)gridDim.x * kRound) {
    uint4 q[kHistVec];
#pragma unroll
    for (int i = 0; i < kHistVec; ++i) {
      const int64_t idx = g0 + i * kSortThreads + threadIdx.x;
      q[i] = idx < nvec ? kv[idx] : make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int i = 0; i < kHistVec; ++i) {
      const bool ok = g0 + i * kSortThreads + threadIdx.x < nvec;
      hist_add<BITS>(q[i].x, ok, npass, hw, lane);
      hist_add<BITS>(q[i].y, ok, npass, hw, lane);
      hist_add<BITS>(q[i].z, ok, npass, hw, lane);
      hist_add<BITS>(q[i].w, ok, npass, hw, lane);
    }
  }
  // the last count mod 4 keys
  if (blockIdx.x == 0 && threadIdx.x < (int)(count & 3)) {
    const uint32_t k = keys[(nvec << 2) + threadIdx.x];
    for (int p = 0; p < npass; ++p) atomicAdd(&hw[p][(k >> (BITS * p)) & (uint32_t)(R - 1)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < npass * R; i += blockDim.x) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) c += (&h[w][0][0])[i];
    if (c) atomicAdd(&ghist[i], c);
  }
}

// Block-wide exclusive scan of DPT consecutive values per thread (thread t
// holds entries t*DPT .. t*DPT+DPT-1); returns the total.
template <int DPT>
__device__ __forceinline__ uint32_t block_scan_digits(const uint32_t (&c)[DPT], uint32_t (&excl)[DPT],
                                                      uint32_t* s_wsum) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t local = 0;
#pragma unroll
  for (int q = 0; q < DPT; ++q) local += c[q];
  uint32_t x = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s_wsum[warp] = x;
  __syncthreads();
  uint32_t wpre = 0, tot = 0;
  for (int w = 0; w < kSortThreads / 32; ++w) {
    if (w < warp) wpre += s_wsum[w];
    tot += s_wsum[w];
  }
  uint32_t run = wpre + x - local;
#pragma unroll
  for (int q = 0; q < DPT; ++q) {
    excl[q] = run;
    run += c[q];
  }
  __syncthreads();
  return tot;
}

// One onesweep scatter pass over the BITS-bit digit at `shift`.  Each CTA
// tile of 4096 keys is ranked per warp (each lane ORs its bit into its
// digit's peer mask in shared memory), its digit counts are chained to the
// preceding tiles by decoupled look-back, keys and then values are reordered
// by digit in shared memory, and both are written out so that consecutive
// threads write consecutive addresses of each digit's run.  Values are
// loaded only after the keys have been placed, so that keys and values are
// never live in registers together.  Thread t owns digits t*DPT .. +DPT-1 in
// the per-digit steps (scans, look-back).
template <int BITS>
__global__ void __launch_bounds__(kSortThreads, BITS == 8 ? 4 : 3) k_onesweep(
    const uint32_t* __restrict__ keys_in, const uint32_t* __restrict__ vals_in,
    uint32_t* __restrict__ keys_out, uint32_t* __restrict__ vals_out, int write_keys,
    const uint32_t* __restrict__ ghist, uint32_t* look, uint32_t* tile_counter, int64_t count_host,
    const int64_t* __restrict__ d_count, int64_t cap, int shift, int32_t* status) {
  constexpr int R = 1 << BITS, DPT = R / kSortThreads;
  constexpr uint32_t kMask = (uint32_t)R - 1u;
  extern __shared__ uint32_t s_dyn[];
  uint32_t* s_key = s_dyn;                    // [kSortTile] keys in block-sorted order
  uint32_t* s_val = s_dyn + kSortTile;        // [kSortTile]
  __shared__ uint32_t s_peer[kSortThreads / 32][R];
  __shared__ uint32_t s_whist[kSortThreads / 32][R];
  __shared__ uint32_t s_gbase[R];             // global start of each digit's run for this tile
  __shared__ uint32_t s_bexcl[R];             // start of each digit inside the tile
  __shared__ uint32_t s_gexcl[R];
  __shared__ uint32_t s_wsum[kSortThreads / 32];
  __shared__ uint32_t s_tile;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // counts fit in 31 bits (the pair capacity is checked on the host)
  const uint32_t count = (uint32_t)(d_count ? min(*d_count, cap) : count_host);
  const uint32_t nblk = (count + kSortTile - 1) / kSortTile;

  // exclusive scan of the global digit histogram (once per CTA)
  {
    uint32_t c[DPT], e[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) c[q] = ghist[tid * DPT + q];
    block_scan_digits<DPT>(c, e, s_wsum);
#pragma unroll
    for (int q = 0; q < DPT; ++q) s_gexcl[tid * DPT + q] = e[q];
  }

  for (int i = tid; i < (kSortThreads / 32) * R; i += kSortThreads) (&s_peer[0][0])[i] = 0u;
  for (;;) {
    if (tid == 0) s_tile = atomicAdd(tile_counter, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= nblk) break;
    for (int i = tid; i < (kSortThreads / 32) * R; i += kSortThreads) (&s_whist[0][0])[i] = 0u;
    __syncthreads();

    const uint32_t seg = tile * kSortTile + (uint32_t)warp * (32 * kSortItems) + lane;
    uint32_t key[kSortItems], loc[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const uint32_t idx = seg + it * 32;
      key[it] = idx < count ? keys_in[idx] : 0xffffffffu;
    }
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const bool valid = seg + it * 32 < count;
      const uint32_t d = (key[it] >> shift) & kMask;
      // peers with the same digit: each lane sets its bit in the digit's mask
      if (valid) atomicOr(&s_peer[warp][d], 1u << lane);
      __syncwarp();
      const uint32_t peers = valid ? s_peer[warp][d] : 0u;
      const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
      const int leader = __ffs(peers) - 1;
      const uint32_t base = valid ? s_whist[warp][d] : 0u;
      __syncwarp();
      if (valid && lane == leader) {
        s_whist[warp][d] = base + (uint32_t)__popc(peers);
        s_peer[warp][d] = 0u;
      }
      __syncwarp();
      loc[it] = base + rank;
    }
    __syncthreads();
    // per digit: exclusive prefix over warps and the tile total
    uint32_t total[DPT], bex[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = tid * DPT + q;
      uint32_t t = 0;
#pragma unroll
      for (int w = 0; w < kSortThreads / 32; ++w) {
        const uint32_t c = s_whist[w][d];
        s_whist[w][d] = t;
        t += c;
      }
      total[q] = t;
    }
    // start of each digit inside the tile: exclusive scan of the totals
    block_scan_digits<DPT>(total, bex, s_wsum);
    // post this tile's count of each of the thread's digits: the inclusive
    // prefix for tile 0, the tile's own aggregate otherwise
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = tid * DPT + q;
      s_bexcl[d] = bex[q];
      atomicExch(look + (size_t)tile * R + d, (tile == 0 ? kFlagInc : kFlagAgg) | total[q]);
    }
    // decoupled look-back, kLookWin predecessors per round: the loads of a
    // round are independent, so a chain of aggregates (the first wave of
    // tiles all post theirs at once) costs one latency per kLookWin tiles
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
      const int d = tid * DPT + q;
      uint32_t excl = 0;
      if (tile > 0) {
        for (int64_t j = (int64_t)tile - 1;; j -= kLookWin) {
          uint32_t v[kLookWin];
#pragma unroll
          for (int i = 0; i < kLookWin; ++i)
            v[i] = j - i >= 0 ? *(volatile const uint32_t*)(look + (j - i) * R + d) : kFlagInc;
          bool stop = false;
#pragma unroll
          for (int i = 0; i < kLookWin; ++i) {
            if (stop) break;
            int spins = 0;
            while ((v[i] & ~kCountMask) == 0u) {   // not posted yet
              if (++spins > kSpinLimit) {
                set_status(status, BETA_ERR_TIMEOUT);
                v[i] = kFlagInc;
                break;
              }
              __nanosleep(64);
              v[i] = *(volatile const uint32_t*)(look + (j - i) * R + d);
            }
            excl += v[i] & kCountMask;
            stop = (v[i] & ~kCountMask) != kFlagAgg;   // an inclusive prefix ends the walk
          }
          if (stop) break;
        }
        atomicExch(look + (size_t)tile * R + d, kFlagInc | (excl + total[q]));
      }
      s_gbase[d] = s_gexcl[d] + excl;
    }
    __syncthreads();
    // keys to their place inside the tile; loc becomes the tile position
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      if (seg + it * 32 < count) {
        const uint32_t d = (key[it] >> shift) & kMask;
        loc[it] += s_bexcl[d] + s_whist[warp][d];
        s_key[loc[it]] = key[it];
      }
    }
    // values follow the keys
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
      const uint32_t idx = seg + it * 32;
      if (idx < count) s_val[loc[it]] = vals_in ? vals_in[idx] : idx;
    }
    __syncthreads();
    // coalesced write-out: element i of the tile goes to its digit's run
    const int n_here = (int)min((uint32_t)kSortTile, count - tile * kSortTile);
#pragma unroll 4
    for (int i = tid; i < n_here; i += kSortThreads) {
      const uint32_t k = s_key[i];
      const uint32_t d = (k >> shift) & kMask;
      const uint32_t gpos = s_gbase[d] + ((uint32_t)i - s_bexcl[d]);
      if (write_keys) keys_out[gpos] = k;
      vals_out[gpos] = s_val[i];
    }
    __syncthreads();
  }
}

__device__ __forceinline__ uint32_t rect_count(uint2 r) {
  int tx0 = (int)(r.x & 0xffffu), tx1 = (int)(r.x >> 16);
  int ty0 = (int)(r.y & 0xffffu), ty1 = (int)(r.y >> 16);
  if (tx0 > tx1 || ty0 > ty1) return 0u;
  return (uint32_t)(tx1 - tx0 + 1) * (uint32_t)(ty1 - ty0 + 1);
}

// block-wide exclusive scan of 64-bit values (256 threads)
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long x,
                                                              unsigned long long* s_w,
                                                              unsigned long long& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned long long inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  unsigned long long pre = 0, tot = 0;
  for (int w = 0; w < kSortThreads / 32; ++w) {
    if (w < warp) pre += s_w[w];
    tot += s_w[w];
  }
  total = tot;
  __syncthreads();
  return pre + inc - x;
}

constexpr int kEmitStage = 4096;   // pairs staged in shared memory per emit block (32 KB)
constexpr unsigned long long kEAgg = 1ull << 62, kEInc = 2ull << 62, kECount = (1ull << 62) - 1;

// Pair counts of the records in depth order, their exclusive scan and the
// emission of (global tile, record) pairs, in one pass: each CTA takes the
// next block of kScanTile records from a ticket, reduces its counts, chains
// its offset to the preceding blocks by decoupled look-back (warp 0 inspects
// 32 predecessors at a time; bounded waits) and writes its pairs.  The last
// block publishes the pair count K and flags a capacity overflow.
__global__ void __launch_bounds__(kSortThreads) k_emit(const uint32_t* __restrict__ order,
                                                       const uint2* __restrict__ rects,
                                                       int64_t n_items, int pitch, ViewTable vt,
                                                       unsigned long long* look, uint32_t* ticket,
                                                       uint32_t* __restrict__ pkey,
                                                       uint32_t* __restrict__ pval, int64_t cap,
                                                       int64_t* d_count, int32_t* status) {
  __shared__ unsigned long long s_w[kSortThreads / 32];
  __shared__ unsigned long long s_base;
  __shared__ uint32_t s_blk;
  __shared__ uint32_t s_pk[kEmitStage], s_pv[kEmitStage];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_blk = atomicAdd(ticket, 1u);
  __syncthreads();
  const int64_t blk = s_blk;
  const int64_t nb = (n_items + kScanTile - 1) / kScanTile;
  if (blk >= nb) return;
  const int64_t base = blk * kScanTile + threadIdx.x * kScanItems;
  uint32_t rec[kScanItems];
  uint2 rc[kScanItems];
  unsigned long long cnt = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t j = base + k;
    rec[k] = j < n_items ? order[j] : 0u;
    rc[k] = j < n_items ? rects[rec[k]] : make_uint2(1u, 1u);
    cnt += rect_count(rc[k]);
  }
  unsigned long long total;
  const unsigned long long excl = block_excl_scan(cnt, s_w, total);
  if (warp == 0) {
    unsigned long long prefix = 0;
    if (blk == 0) {
      if (lane == 0) atomicExch(&look[0], kEInc | total);
    } else {
      if (lane == 0) atomicExch(&look[blk], kEAgg | total);
      for (int64_t j0 = blk - 1;; j0 -= 32) {
        const int64_t j = j0 - lane;            // lane 0: the nearest predecessor
        unsigned long long v = kEInc;           // before block 0: an inclusive zero
        if (j >= 0) {
          volatile unsigned long long* pj = look + j;
          v = *pj;
          int spins = 0;
          while ((v & ~kECount) == 0ull) {
            if (++spins > kSpinLimit) {
              set_status(status, BETA_ERR_TIMEOUT);
              v = kEInc;
              break;
            }
            __nanosleep(64);
            v = *pj;
          }
        }
        const uint32_t inc = __ballot_sync(0xffffffffu, (v & ~kECount) == kEInc);
        const int first = inc ? __ffs(inc) - 1 : 31;   // sum up to the nearest inclusive entry
        unsigned long long mine = lane <= first ? (v & kECount) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        prefix += mine;
        if (inc) break;
      }
      if (lane == 0) atomicExch(&look[blk], kEInc | (prefix + total));
    }
    if (lane == 0) {
      s_base = prefix;
      if (blk == nb - 1) {
        *d_count = (int64_t)(prefix + total);
        if ((int64_t)(prefix + total) > cap) set_status(status, BETA_ERR_CAPACITY);
      }
    }
  }
  __syncthreads();
  // pairs land in shared memory first (the block's first kEmitStage pairs),
  // then leave with coalesced stores; pairs past the stage (blocks of very
  // large primitives) are written directly
  const unsigned long long bbase = s_base;
  unsigned long long off = excl;   // relative to the block's first pair
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const uint32_t c = rect_count(rc[k]);
    if (c == 0) continue;
    const int v = (int)(rec[k] / (uint32_t)pitch);
    const int ntx = vt.v[v].ntx, toff = vt.v[v].tile_off;
    const int tx0 = (int)(rc[k].x & 0xffffu), tx1 = (int)(rc[k].x >> 16);
    const int ty0 = (int)(rc[k].y & 0xffffu), ty1 = (int)(rc[k].y >> 16);
    for (int ty = ty0; ty <= ty1; ++ty)
      for (int tx = tx0; tx <= tx1; ++tx) {
        const uint32_t key = (uint32_t)(toff + ty * ntx + tx);
        if (off < (unsigned long long)kEmitStage) {
          s_pk[off] = key;
          s_pv[off] = rec[k];
        } else if ((int64_t)(bbase + off) < cap) {
          pkey[bbase + off] = key;
          pval[bbase + off] = rec[k];
        }
        ++off;
      }
  }
  __syncthreads();
  const int n_stage = (int)min(total, (unsigned long long)kEmitStage);
  for (int i = threadIdx.x; i < n_stage; i += kSortThreads) {
    if ((int64_t)(bbase + i) < cap) {
      pkey[bbase + i] = s_pk[i];
      pval[bbase + i] = s_pv[i];
    }
  }
}

__global__ void k_tile_ranges(const uint32_t* __restrict__ keys, const int64_t* __restrict__ d_count,
                              int64_t cap, int total_tiles, uint32_t* __restrict__ ranges) {
  const int64_t K = min(*d_count, cap);
  if (K == 0) {
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g <= total_tiles;
         g += (int64_t)gridDim.x * blockDim.x)
      ranges[g] = 0u;
    return;
  }
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < K;
       k += (int64_t)gridDim.x * blockDim.x) {
    int64_t t = keys[k];
    int64_t prev = k > 0 ? (int64_t)keys[k - 1] : -1;
    for (int64_t g = prev + 1; g <= t; ++g) ranges[g] = (uint32_t)k;
    if (k == K - 1)
      for (int64_t g = t + 1; g <= total_tiles; ++g) ranges[g] = (uint32_t)K;
  }
}

// ---------------------------------------------------------------------------
// host launcher
// ---------------------------------------------------------------------------

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

cudaError_t launch_bin_sort(const ViewTable& vt, int pitch, ProjBuffers pb, uint32_t* pair_vals,
                            int64_t cap, uint32_t* ranges, int64_t* d_count, int32_t* d_status,
                            void* ws, cudaStream_t s) {
  const int64_t n_items = (int64_t)vt.n_views * pitch;
  const int total_tiles = vt.total_tiles;
  SortWs w = carve(ws, n_items, cap, total_tiles);
  const int64_t nblk_d = cdiv(n_items, kSortTile);
  const int64_t nblk_t = cdiv(cap > 0 ? cap : 1, kSortTile);
  const TilePlan tp = tile_plan(total_tiles);
  const int np_t = tp.passes, rt = 1 << tp.bits;
  const int persist = sm_count() * 4;
  uint32_t* gh_d = w.ghist;
  uint32_t* gh_t = w.ghist + kMaxPasses * 512;

  // 32 KB dynamic + 20 / 38 KB static shared memory per CTA (8 / 9-bit digits)
  static bool smem_set = false;
  if (!smem_set) {
    if (cudaFuncSetAttribute(k_onesweep<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOnesweepSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_onesweep<8>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess ||
        cudaFuncSetAttribute(k_onesweep<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, kOnesweepSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_onesweep<9>, cudaFuncAttributePreferredSharedMemoryCarveout, 100) != cudaSuccess)
      return cudaGetLastError();
    smem_set = true;
  }
  k_sort_prep<<<1, 256, 0, s>>>(w.ghist, w.counters, w.look_e, cdiv(n_items, kScanTile), d_count, d_status);

  // 1. stable sort of all records by depth key (4 passes of 8 bits)
  int grid_h = (int)std::min<int64_t>(cdiv(n_items, 4 * kSortThreads * kHistVec), (int64_t)persist * 2);
  if (grid_h < 1) grid_h = 1;
  k_digit_hist<8, kMaxPasses><<<grid_h, kSortThreads, 0, s>>>(pb.key, n_items, nullptr, n_items, 4, gh_d,
                                                               w.look_d, nblk_d);
  const uint32_t* kin = pb.key;
  const uint32_t* vin = nullptr;
  uint32_t* kbuf[2] = {w.dkey_a, w.dkey_b};
  uint32_t* vbuf[2] = {w.dval_a, w.dval_b};
  int grid_d = (int)std::min<int64_t>(nblk_d, persist);
  if (grid_d < 1) grid_d = 1;
  for (int p = 0; p < 4; ++p) {
    k_onesweep<8><<<grid_d, kSortThreads, kOnesweepSmem, s>>>(kin, vin, kbuf[p & 1], vbuf[p & 1], p < 3 ? 1 : 0,
                                               gh_d + p * 256, w.look_d + (size_t)p * nblk_d * 256,
                                               w.counters + p, n_items, nullptr, n_items, 8 * p,
                                               d_status);
    kin = kbuf[p & 1];
    vin = vbuf[p & 1];
  }
  const uint32_t* order = vbuf[1];

  // 2. pair counts in depth order -> offsets -> emit (tile, record) pairs
  const int64_t nb_scan = cdiv(n_items, kScanTile);
  // final tile-sorted values must land in pair_vals: choose the emit buffer by pass parity
  uint32_t* pval_emit = (np_t % 2 == 0) ? pair_vals : w.pval_ws;
  uint32_t* pval_other = (np_t % 2 == 0) ? w.pval_ws : pair_vals;
  if (nb_scan > 0)
    k_emit<<<(unsigned)nb_scan, kSortThreads, 0, s>>>(order, pb.rect, n_items, pitch, vt, w.look_e,
                                                       w.counters + 2 * kMaxPasses, w.pkey_a, pval_emit,
                                                       cap, d_count, d_status);

  // 3. stable sort of the pairs by global tile id
  const uint32_t* final_keys = w.pkey_a;
  if (np_t > 0) {
    int grid_th = (int)std::min<int64_t>(cdiv(cap, 4 * kSortThreads * kHistVec), (int64_t)persist * 2);
    if (grid_th < 1) grid_th = 1;
    if (tp.bits == 9)
      k_digit_hist<9, 2><<<grid_th, kSortThreads, 0, s>>>(w.pkey_a, 0, d_count, cap, np_t, gh_t, w.look_t,
                                                          nblk_t);
    else
      k_digit_hist<8, kMaxPasses><<<grid_th, kSortThreads, 0, s>>>(w.pkey_a, 0, d_count, cap, np_t, gh_t,
                                                                   w.look_t, nblk_t);
    int grid_t = (int)std::min<int64_t>(nblk_t, persist);
    if (grid_t < 1) grid_t = 1;
    uint32_t* pk[2] = {w.pkey_b, w.pkey_a};
    uint32_t* pv[2] = {pval_other, pval_emit};
    const uint32_t* ki = w.pkey_a;
    const uint32_t* vi = pval_emit;
    for (int p = 0; p < np_t; ++p) {
      auto k = tp.bits == 9 ? k_onesweep<9> : k_onesweep<8>;
      k<<<grid_t, kSortThreads, kOnesweepSmem, s>>>(ki, vi, pk[p & 1], pv[p & 1], 1, gh_t + p * rt,
                                                     w.look_t + (size_t)p * nblk_t * rt,
                                                     w.counters + kMaxPasses + p, 0, d_count, cap,
                                                     tp.bits * p, d_status);
      ki = pk[p & 1];
      vi = pv[p & 1];
    }
    final_keys = ki;
  }
  int grid_r = (int)std::min<int64_t>(cdiv(std::max<int64_t>(cap, total_tiles + 1), 256), (int64_t)persist * 2);
  if (grid_r < 1) grid_r = 1;
  k_tile_ranges<<<grid_r, 256, 0, s>>>(final_keys, d_count, cap, total_tiles, ranges);
  return cudaGetLastError();
}

}  // namespace beta
