// beta_sort.cu -- binning and depth ordering of (tile, record) pairs.
//
// Sec. 3.2 of arXiv 2501.18630 composites the primitives that overlap a
// pixel in order of their camera depth.  The pairs (global tile, record) are
// built as per-tile lists and each list is sorted on its own:
//   1. k_tile_count:   every record adds one to a counter of each tile of its
//                      rectangle that its support reaches (the rule B2 mask
//                      of the projection; kSub counters per tile, chosen by
//                      the record index, so that the atomics on a busy tile
//                      spread over several addresses);
//   2. k_tile_scan:    exclusive scan of the counters = the tile ranges (list
//                      g is pairs [ranges[g], ranges[g+1])), the pair count K
//                      and the capacity check; lists longer than a warp sorts
//                      are put on a separate work list;
//   3. k_tile_scatter: every record appends the 64-bit item
//                      (depth key << 32 | record) to each of its tiles' lists,
//                      slots taken with atomics (arbitrary order inside a list);
//   4. k_tile_sort:    each list is sorted by its items (a register sorting
//                      network per thread, then a shuffle bitonic network
//                      across the warp, or merge-path merges in shared memory
//                      for 16 items a lane and for CTA sorts), one warp per
//                      list up to kWarpMax items, one CTA per longer list, and
//                      the record ids are written out.
// The items of a list are distinct (the record index is part of them), so the
// sorted list does not depend on the order the atomics gave: it is the order
// (tile, depth key, record index), a stable sort of the pairs by depth in
// record order.  Every wait (the scan's look-back) is bounded: after
// kSpinLimit polls (or the test hook's smaller limit) the CTA records
// BETA_ERR_TIMEOUT and proceeds.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <atomic>

#include "beta_internal.cuh"

namespace beta {

namespace {

typedef unsigned long long u64;

constexpr int kSortThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kSortThreads * kScanItems;   // tiles per scan block
static_assert(kScanItems == 8, "the scan moves a thread's tiles as two 16-byte vectors");
constexpr int kWarpMax = 512;                      // longest list one warp sorts (16 items a lane)
constexpr int kCtaItems = 16;
constexpr int kCtaMax = kSortThreads * kCtaItems;      // longest list sorted in one shared-memory pass
constexpr int kTicketLists = 4;                    // short lists per warp ticket
constexpr int kSub = 16;                           // counters per tile (record index mod kSub): spreads
                                                   // the atomics on a busy tile over kSub addresses
constexpr int kSpinLimit = 1 << 20;
constexpr u64 kAgg = 1ull << 62, kInc = 2ull << 62, kCountMask = (1ull << 62) - 1;
constexpr u64 kPad = ~0ull;                        // above every item (depth keys are < 2^31)

// counters: [0] scan ticket, [1] long-list ticket, [2] short-list ticket,
// [3] number of long lists
constexpr int kCounters = 4;

__host__ __device__ inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }
// counter row length: a multiple of kScanItems, so the scan moves 16-byte vectors
__host__ __device__ inline int64_t crow(int total_tiles) { return cdiv(total_tiles, kScanItems) * kScanItems; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Workspace carve-up (offsets are 256-byte aligned).
struct SortWs {
  uint32_t* cnt;       // [kSub][row] pairs per tile and record class (row = tiles rounded up to 8)
  uint32_t* cursor;    // [kSub][row] next free slot of each class's part of a list
  uint32_t* longl;     // [total_tiles] tiles whose list is longer than kWarpMax
  u64* look;           // [nb_scan] scan look-back (flag | aggregate or inclusive sum)
  uint32_t* counters;  // [kCounters]
  u64* items;          // [cap] list items, then merge buffer of the longest lists
  u64* tmp;            // [cap] merge buffer of lists longer than kCtaMax
  size_t bytes;
};

static SortWs carve(void* base, int64_t cap, int total_tiles) {
  SortWs w{};
  char* p = (char*)base;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* q = p ? p + off : nullptr;
    off += align256(bytes);
    return q;
  };
  const int64_t nb_scan = cdiv(total_tiles, kScanTile);
  const int64_t c = cap > 0 ? cap : 1;
  w.cnt = (uint32_t*)take((size_t)kSub * crow(total_tiles) * 4);
  w.cursor = (uint32_t*)take((size_t)kSub * crow(total_tiles) * 4);
  w.longl = (uint32_t*)take((size_t)total_tiles * 4);
  w.look = (u64*)take((size_t)nb_scan * 8);
  w.counters = (uint32_t*)take(kCounters * 4);
  w.items = (u64*)take((size_t)c * 8);
  w.tmp = (u64*)take((size_t)c * 8);
  w.bytes = off;
  return w;
}

size_t binsort_ws_bytes(int64_t n_items, int64_t cap, int total_tiles) {
  (void)n_items;
  return carve(nullptr, cap, total_tiles).bytes;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------

__global__ void k_sort_prep(uint32_t* cnt, int total_tiles, u64* look, int64_t nb_scan,
                            uint32_t* counters, int64_t* d_count, int32_t* status) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t i = t; i < (int64_t)kSub * crow(total_tiles); i += stride) cnt[i] = 0u;
  for (int64_t i = t; i < nb_scan; i += stride) look[i] = 0ull;
  if (t < kCounters) counters[t] = 0u;
  if (t == 0) {
    *d_count = 0;
    *status = 0;
  }
}

// Tiles of a record: its rectangle (tx0 | tx1 << 16, ty0 | ty1 << 16),
// inclusive, empty (tx0 > tx1) for records that are not binned, and the mask
// of the rectangle's tiles that its support reaches (rule B2: bit dy w + dx;
// rectangles of more than 32 tiles keep every tile).
struct Rect {
  int tx0, ty0, w, h, n;
  bool full;
  uint32_t mask;
};
__device__ __forceinline__ Rect rect_of(uint2 r, uint32_t mask) {
  Rect q;
  q.tx0 = (int)(r.x & 0xffffu);
  q.ty0 = (int)(r.y & 0xffffu);
  const int tx1 = (int)(r.x >> 16), ty1 = (int)(r.y >> 16);
  q.w = tx1 - q.tx0 + 1;
  q.h = ty1 - q.ty0 + 1;
  const bool empty = tx1 < q.tx0 || ty1 < q.ty0;
  q.full = !empty && q.w * q.h > 32;
  q.mask = mask;
  q.n = empty ? 0 : (q.full ? q.w * q.h : __popc(mask));
  return q;
}

// Walks the kept tiles of a masked rectangle (not `full`) row by row, without
// divisions: next() gives the offset dy * ntx + dx of the next tile.
struct TileWalk {
  uint32_t mask, rowmask, rm;
  int w, h, dy, ntx;
  __device__ __forceinline__ TileWalk(const Rect& q, int ntx_) : mask(q.mask), w(q.w), h(q.h), dy(0), ntx(ntx_) {
    rowmask = w >= 32 ? 0xffffffffu : (1u << w) - 1u;
    rm = mask & rowmask;
  }
  __device__ __forceinline__ bool next(int& off) {
    while (rm == 0u) {
      if (++dy >= h) return false;
      rm = (mask >> (dy * w)) & rowmask;
    }
    const int dx = __ffs(rm) - 1;
    rm &= rm - 1u;
    off = dy * ntx + dx;
    return true;
  }
};

// 1. pairs per tile
__global__ void __launch_bounds__(kSortThreads) k_tile_count(const uint2* __restrict__ rects,
                                                         const uint32_t* __restrict__ tiles, int64_t n_items,
                                                         int pitch, ViewTable vt, int total_tiles,
                                                         uint32_t* cnt) {
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_items;
       r += (int64_t)gridDim.x * blockDim.x) {
    const Rect q = rect_of(rects[r], tiles[r]);
    if (q.n == 0) continue;
    const int v = (int)((uint32_t)r / (uint32_t)pitch);
    const int ntx = vt.v[v].ntx;
    uint32_t* c = cnt + (size_t)(r & (kSub - 1)) * crow(total_tiles) + vt.v[v].tile_off + q.ty0 * ntx + q.tx0;
    if (q.full) {
      for (int dy = 0; dy < q.h; ++dy, c += ntx)
        for (int dx = 0; dx < q.w; ++dx) atomicAdd(&c[dx], 1u);
    } else {
      TileWalk it(q, ntx);
      int off;
      while (it.next(off)) atomicAdd(&c[off], 1u);
    }
  }
}

// block-wide exclusive scan of 64-bit values (kSortThreads threads)
__device__ __forceinline__ u64 block_excl_scan(u64 x, u64* s_w, u64& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  u64 inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const u64 y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  u64 pre = 0, tot = 0;
  for (int w = 0; w < kSortThreads / 32; ++w) {
    if (w < warp) pre += s_w[w];
    tot += s_w[w];
  }
  total = tot;
  __syncthreads();
  return pre + inc - x;
}

// 2. exclusive scan of the tile counters: each CTA takes the next block of
// kScanTile tiles from a ticket, reduces it, chains its offset to the
// preceding blocks by decoupled look-back (warp 0 inspects 32 predecessors
// at a time; bounded waits) and writes ranges and cursors.  The last block
// writes ranges[total_tiles] and the pair count and flags a capacity overflow.
__global__ void __launch_bounds__(kSortThreads) k_tile_scan(const uint32_t* __restrict__ cnt, int total_tiles,
                                                        u64* look, uint32_t* counters,
                                                        uint32_t* __restrict__ ranges,
                                                        uint32_t* __restrict__ cursor,
                                                        uint32_t* __restrict__ longl, int64_t cap,
                                                        int64_t* d_count, int32_t* status,
                                                        int spin_limit, int64_t withhold) {
  __shared__ u64 s_w[kSortThreads / 32];
  __shared__ u64 s_base;
  __shared__ uint32_t s_blk;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_blk = atomicAdd(&counters[0], 1u);
  __syncthreads();
  const int64_t blk = s_blk;
  const int64_t nb = cdiv(total_tiles, kScanTile);
  if (blk >= nb) return;
  const int64_t base = blk * kScanTile + threadIdx.x * kScanItems;
  // the thread's kScanItems tiles: per class two 16-byte loads (rows are
  // padded to a multiple of kScanItems and zeroed, so no tail guard)
  const int64_t row = crow(total_tiles);
  const bool mine = base < total_tiles;
  uint32_t c[kScanItems];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) c[k] = 0u;
  if (mine)
#pragma unroll 4
    for (int q = 0; q < kSub; ++q) {
      const uint4* src = reinterpret_cast<const uint4*>(cnt + q * row + base);
      const uint4 a = src[0], b = src[1];
      c[0] += a.x; c[1] += a.y; c[2] += a.z; c[3] += a.w;
      c[4] += b.x; c[5] += b.y; c[6] += b.z; c[7] += b.w;
    }
  u64 sum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) sum += c[k];
  u64 total;
  const u64 excl = block_excl_scan(sum, s_w, total);
  if (warp == 0) {
    u64 prefix = 0;
    // `withhold` (a test hook, -1 normally) names a block that never posts
    // its look-back entry, so that its successors' bounded waits run out
    const bool post = blk != withhold;
    if (blk == 0) {
      if (lane == 0 && post) atomicExch(&look[0], kInc | total);
    } else {
      if (lane == 0 && post) atomicExch(&look[blk], kAgg | total);
      for (int64_t j0 = blk - 1;; j0 -= 32) {
        const int64_t j = j0 - lane;   // lane 0: the nearest predecessor
        u64 v = kInc;                  // before block 0: an inclusive zero
        if (j >= 0) {
          volatile u64* pj = look + j;
          v = *pj;
          int spins = 0;
          while ((v & ~kCountMask) == 0ull) {
            if (++spins > spin_limit) {
              set_status(status, BETA_ERR_TIMEOUT);
              v = kInc;
              break;
            }
            __nanosleep(64);
            v = *pj;
          }
        }
        const uint32_t inc = __ballot_sync(0xffffffffu, (v & ~kCountMask) == kInc);
        const int first = inc ? __ffs(inc) - 1 : 31;   // sum up to the nearest inclusive entry
        u64 mine = lane <= first ? (v & kCountMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
        prefix += mine;
        if (inc) break;
      }
      if (lane == 0 && post) atomicExch(&look[blk], kInc | (prefix + total));
    }
    if (lane == 0) {
      s_base = prefix;
      if (blk == nb - 1) {
        const u64 K = prefix + total;
        ranges[total_tiles] = (uint32_t)K;
        *d_count = (int64_t)K;
        if ((int64_t)K > cap) set_status(status, BETA_ERR_CAPACITY);
      }
    }
  }
  __syncthreads();
  u64 run = s_base + excl;
  if (!mine) return;
  uint32_t start[kScanItems];
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    const int64_t g = base + k;
    start[k] = (uint32_t)run;
    if (g < total_tiles) {
      ranges[g] = (uint32_t)run;
      if (c[k] > (uint32_t)kWarpMax) longl[atomicAdd(&counters[3], 1u)] = (uint32_t)g;
    }
    run += c[k];
  }
  // class q's part of a list starts after classes 0 .. q-1
#pragma unroll 4
  for (int q = 0; q < kSub; ++q) {
    const uint4* src = reinterpret_cast<const uint4*>(cnt + q * row + base);
    uint4* dst = reinterpret_cast<uint4*>(cursor + q * row + base);
    const uint4 a = src[0], b = src[1];
    dst[0] = make_uint4(start[0], start[1], start[2], start[3]);
    dst[1] = make_uint4(start[4], start[5], start[6], start[7]);
    start[0] += a.x; start[1] += a.y; start[2] += a.z; start[3] += a.w;
    start[4] += b.x; start[5] += b.y; start[6] += b.z; start[7] += b.w;
  }
}

// 3. every record appends its item to the lists of its tiles; up to four
// slots are claimed before the first store so that the atomics overlap.
__global__ void __launch_bounds__(kSortThreads) k_tile_scatter(const uint2* __restrict__ rects,
                                                           const uint32_t* __restrict__ tiles,
                                                           const uint32_t* __restrict__ keys,
                                                           int64_t n_items, int pitch, ViewTable vt,
                                                           int total_tiles, uint32_t* cursor,
                                                           u64* __restrict__ items,
                                                           int64_t cap, const int32_t* __restrict__ status) {
  if (*status != 0) return;   // capacity overflow (or a failed scan): no list is written
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n_items;
       r += (int64_t)gridDim.x * blockDim.x) {
    const Rect q = rect_of(rects[r], tiles[r]);
    if (q.n == 0) continue;
    const int v = (int)((uint32_t)r / (uint32_t)pitch);
    const int ntx = vt.v[v].ntx;
    uint32_t* cur = cursor + (size_t)(r & (kSub - 1)) * crow(total_tiles) + vt.v[v].tile_off + q.ty0 * ntx + q.tx0;
    const u64 item = ((u64)keys[r] << 32) | (u64)(uint32_t)r;
    if (q.full) {
      int dx = 0, row = 0;   // tile j of the rectangle, row-major, walked incrementally
      for (int j0 = 0; j0 < q.n; j0 += 4) {
        uint32_t slot[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          slot[u] = 0xffffffffu;
          if (j0 + u < q.n) {
            slot[u] = atomicAdd(&cur[row + dx], 1u);
            if (++dx == q.w) {
              dx = 0;
              row += ntx;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j0 + u < q.n && (int64_t)slot[u] < cap) items[slot[u]] = item;
      }
    } else {
      TileWalk it(q, ntx);
      for (int j0 = 0; j0 < q.n; j0 += 4) {
        uint32_t slot[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          int off;
          slot[u] = (j0 + u < q.n && it.next(off)) ? atomicAdd(&cur[off], 1u) : 0xffffffffu;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (j0 + u < q.n && (int64_t)slot[u] < cap) items[slot[u]] = item;
      }
    }
  }
}

// Shared-memory index of item i of a sorted run: one pad word per 16 items
// makes the blocked stores (thread t writes items t*E .. t*E+E-1, E = 1..16)
// free of bank conflicts.
__device__ __forceinline__ int sidx(int i) { return i + (i >> 4); }

template <int G>
__device__ __forceinline__ void group_sync() {
  if (G == 32) __syncwarp();
  else __syncthreads();
}

// Ascending bitonic sorting network over a thread's E registers.
template <int E>
__device__ __forceinline__ void sort_regs(u64 (&k)[E]) {
#pragma unroll
  for (int size = 2; size <= E; size <<= 1)
#pragma unroll
    for (int stride = size >> 1; stride > 0; stride >>= 1)
#pragma unroll
      for (int i = 0; i < E; ++i) {
        const int j = i ^ stride;
        if (j > i) {
          const bool up = (i & size) == 0;
          const u64 a = k[i], b = k[j];
          const bool sw = up ? (a > b) : (a < b);
          k[i] = sw ? b : a;
          k[j] = sw ? a : b;
        }
      }
}

// Merge sort across a group of G threads, each holding a sorted run of E
// items: at every level thread t produces outputs t*E .. t*E+E-1 of the
// merge of two neighbouring runs, starting where the merge path crosses its
// first output (binary search), ties to the left run.  `sm` holds G*E items
// (padded by sidx).
template <int G, int E>
__device__ __forceinline__ void group_merge(u64 (&k)[E], u64* sm, int t) {
#pragma unroll 1
  for (int run = E; run < G * E; run <<= 1) {
#pragma unroll
    for (int j = 0; j < E; ++j) sm[sidx(t * E + j)] = k[j];
    group_sync<G>();
    const int d = t * E;
    const int a0 = d & ~(2 * run - 1), b0 = a0 + run;
    const int diag = d - a0;
    int lo = max(0, diag - run), hi = min(diag, run);
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sm[sidx(a0 + mid)] <= sm[sidx(b0 + diag - 1 - mid)]) lo = mid + 1;
      else hi = mid;
    }
    int ia = lo, ib = diag - lo;
    u64 a = ia < run ? sm[sidx(a0 + ia)] : kPad;
    u64 b = ib < run ? sm[sidx(b0 + ib)] : kPad;
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const bool ta = a <= b;
      k[j] = ta ? a : b;
      ia += ta ? 1 : 0;
      ib += ta ? 0 : 1;
      const bool more = ta ? ia < run : ib < run;
      const u64 nx = more ? sm[sidx(ta ? a0 + ia : b0 + ib)] : kPad;
      a = ta ? nx : a;
      b = ta ? b : nx;
    }
    group_sync<G>();
  }
}

// Bitonic network across the warp for lane-sorted runs (E registers a lane,
// item i = lane * E + j): from run size 2E up to 32E, strides >= E exchange
// with lane ^ (stride / E) through shuffles and strides < E are
// compare-exchanges inside the lane; a run's direction is bit log2(size) of
// its first item.  No shared memory and no dependent loads.
template <int E>
__device__ __forceinline__ void warp_bitonic(u64 (&k)[E], int lane) {
  // lane runs must alternate ascending / descending for the first merge
  if (lane & 1) {
#pragma unroll
    for (int j = 0; j < E / 2; ++j) {
      const u64 t = k[j];
      k[j] = k[E - 1 - j];
      k[E - 1 - j] = t;
    }
  }
#pragma unroll 1
  for (int size = 2 * E; size <= 32 * E; size <<= 1) {
    const bool up = ((lane * E) & size) == 0;
#pragma unroll 1
    for (int stride = size >> 1; stride >= E; stride >>= 1) {
      const int lm = stride / E;
      const bool take_min = ((lane & lm) == 0) == up;
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const u64 o = __shfl_xor_sync(0xffffffffu, k[j], lm);
        k[j] = (take_min == (o < k[j])) ? o : k[j];
      }
    }
#pragma unroll
    for (int stride = E / 2; stride > 0; stride >>= 1)
#pragma unroll
      for (int j = 0; j < E; ++j) {
        const int jj = j ^ stride;
        if (jj > j) {
          const u64 a = k[j], b = k[jj];
          const bool sw = up ? (a > b) : (a < b);
          k[j] = sw ? b : a;
          k[jj] = sw ? a : b;
        }
      }
  }
}

// Sorts list items[0, n) (n <= 32 E) with one warp and writes the record ids:
// E <= 8 by the shuffle network, E = 16 by merge-path merges in shared memory.
template <int E>
__device__ __forceinline__ void warp_list_sort(const u64* items, int n, uint32_t* __restrict__ out,
                                               u64* sm, int lane) {
  u64 k[E];
  if (E <= 8) {
#pragma unroll
    for (int j = 0; j < E; ++j) {
      const int p = lane * E + j;
      k[j] = p < n ? items[p] : kPad;
    }
    sort_regs<E>(k);
    warp_bitonic<E>(k, lane);
  } else {
    for (int p = lane; p < 32 * E; p += 32) sm[sidx(p)] = p < n ? items[p] : kPad;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < E; ++j) k[j] = sm[sidx(lane * E + j)];
    __syncwarp();
    sort_regs<E>(k);
    group_merge<32, E>(k, sm, lane);
  }
#pragma unroll
  for (int j = 0; j < E; ++j) sm[sidx(lane * E + j)] = k[j];
  __syncwarp();
  for (int p = lane; p < n; p += 32) out[p] = (uint32_t)sm[sidx(p)];
  __syncwarp();
}

// Sorts up to kSortThreads * E items of `src` (m of them) with the whole
// CTA; the sorted items are left in sm[sidx(0 .. m-1)].
template <int E>
__device__ __forceinline__ void cta_chunk_sort(const u64* src, int m, u64* sm, int tid) {
  for (int p = tid; p < kSortThreads * E; p += kSortThreads) sm[sidx(p)] = p < m ? src[p] : kPad;
  __syncthreads();
  u64 k[E];
#pragma unroll
  for (int j = 0; j < E; ++j) k[j] = sm[sidx(tid * E + j)];
  __syncthreads();
  sort_regs<E>(k);
  group_merge<kSortThreads, E>(k, sm, tid);
#pragma unroll
  for (int j = 0; j < E; ++j) sm[sidx(tid * E + j)] = k[j];
  __syncthreads();
}

// Sorts a list longer than kWarpMax with the whole CTA.  Lists of up to
// kCtaMax items are sorted in shared memory (4, 8 or 16 items a thread, the
// fewest that hold the list); longer ones are sorted in chunks of kCtaMax
// into `tmp`, then merged pairwise through global memory (merge path per 16
// outputs, buffers alternating between tmp and items) until one run is left.
// items/tmp are read after this CTA wrote them, so they are plain (coherent)
// loads.
__device__ void cta_list_sort(u64* items, u64* tmp, uint32_t n, uint32_t* __restrict__ out, u64* sm,
                              int tid) {
  if (n <= (uint32_t)kCtaMax) {
    if (n <= 4u * kSortThreads) cta_chunk_sort<4>(items, (int)n, sm, tid);
    else if (n <= 8u * kSortThreads) cta_chunk_sort<8>(items, (int)n, sm, tid);
    else cta_chunk_sort<kCtaItems>(items, (int)n, sm, tid);
    for (int p = tid; p < (int)n; p += kSortThreads) out[p] = (uint32_t)sm[sidx(p)];
    __syncthreads();
    return;
  }
  for (uint32_t c0 = 0; c0 < n; c0 += kCtaMax) {
    const int m = (int)min((uint32_t)kCtaMax, n - c0);
    cta_chunk_sort<kCtaItems>(items + c0, m, sm, tid);
    for (int p = tid; p < m; p += kSortThreads) tmp[c0 + p] = sm[sidx(p)];
    __syncthreads();
  }
  u64* src = tmp;
  u64* dst = items;
  for (uint32_t run = kCtaMax; run < n; run <<= 1) {
    for (uint32_t o0 = 0; o0 < n; o0 += kCtaMax) {
      const uint32_t d = o0 + (uint32_t)tid * kCtaItems;
      if (d < n) {
        const uint32_t a0 = d - d % (2 * run);
        const uint32_t la = min(run, n - a0);
        const uint32_t lb = min(run, n - a0 - la);
        const u64* A = src + a0;
        const u64* B = A + la;
        const uint32_t diag = d - a0;
        uint32_t lo = diag > lb ? diag - lb : 0u, hi = min(diag, la);
        while (lo < hi) {
          const uint32_t mid = (lo + hi) >> 1;
          if (A[mid] <= B[diag - 1 - mid]) lo = mid + 1;
          else hi = mid;
        }
        uint32_t ia = lo, ib = diag - lo;
        for (int j = 0; j < kCtaItems && d + j < n; ++j) {
          const u64 a = ia < la ? A[ia] : kPad;
          const u64 b = ib < lb ? B[ib] : kPad;
          const bool ta = a <= b;
          dst[d + j] = ta ? a : b;
          ia += ta ? 1u : 0u;
          ib += ta ? 0u : 1u;
        }
      }
    }
    __syncthreads();
    u64* t = src;
    src = dst;
    dst = t;
  }
  for (uint32_t p = tid; p < n; p += kSortThreads) out[p] = (uint32_t)src[p];
  __syncthreads();
}

// 4. per-list sort.  Long lists first (one CTA each, from a ticket), then
// short lists (one warp each, kTicketLists tiles per ticket).
__global__ void __launch_bounds__(kSortThreads, 3) k_tile_sort(const uint32_t* __restrict__ ranges,
                                                           int total_tiles,
                                                           const uint32_t* __restrict__ longl,
                                                           uint32_t* counters, u64* items, u64* tmp,
                                                           uint32_t* __restrict__ vals,
                                                           const int32_t* __restrict__ status) {
  constexpr int kWarpSm = kWarpMax + kWarpMax / 16;
  __shared__ u64 sm[kCtaMax + kCtaMax / 16];
  __shared__ uint32_t s_t;
  static_assert((kSortThreads / 32) * kWarpSm <= kCtaMax + kCtaMax / 16, "warp regions exceed the CTA's");
  if (*status != 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t n_long = counters[3];
  for (;;) {
    if (tid == 0) s_t = atomicAdd(&counters[1], 1u);
    __syncthreads();
    const uint32_t i = s_t;
    __syncthreads();
    if (i >= n_long) break;
    const uint32_t g = longl[i];
    const uint32_t s = ranges[g];
    cta_list_sort(items + s, tmp + s, ranges[g + 1] - s, vals + s, sm, tid);
  }
  u64* wsm = sm + warp * kWarpSm;
  for (;;) {
    uint32_t t0 = 0;
    if (lane == 0) t0 = atomicAdd(&counters[2], (uint32_t)kTicketLists);
    t0 = __shfl_sync(0xffffffffu, t0, 0);
    if (t0 >= (uint32_t)total_tiles) break;
    for (int q = 0; q < kTicketLists; ++q) {
      const int g = (int)t0 + q;
      if (g >= total_tiles) break;
      const uint32_t s = ranges[g];
      const int n = (int)(ranges[g + 1] - s);
      if (n <= 1) {
        if (n == 1 && lane == 0) vals[s] = (uint32_t)items[s];
        continue;
      }
      if (n > kWarpMax) continue;
      if (n <= 32) warp_list_sort<1>(items + s, n, vals + s, wsm, lane);
      else if (n <= 64) warp_list_sort<2>(items + s, n, vals + s, wsm, lane);
      else if (n <= 128) warp_list_sort<4>(items + s, n, vals + s, wsm, lane);
      else if (n <= 256) warp_list_sort<8>(items + s, n, vals + s, wsm, lane);
      else warp_list_sort<16>(items + s, n, vals + s, wsm, lane);
    }
  }
}

// ---------------------------------------------------------------------------
// host launcher
// ---------------------------------------------------------------------------

// Scan look-back settings: the poll limit, and the scan block that withholds
// its look-back entry (-1: none).  Changed only by the fault-injection test
// hook beta_debug_scan_faults.
static std::atomic<int> g_spin_limit{kSpinLimit};
static std::atomic<int64_t> g_withhold{-1};

int set_scan_faults(int spin_limit, int64_t withhold_block) {
  if (spin_limit == 0) spin_limit = kSpinLimit;
  if (spin_limit < 1 || spin_limit > kSpinLimit || withhold_block < -1) return -1;
  g_spin_limit.store(spin_limit);
  g_withhold.store(withhold_block);
  return 0;
}

cudaError_t launch_bin_sort(const ViewTable& vt, int pitch, ProjBuffers pb, uint32_t* pair_vals,
                            int64_t cap, uint32_t* ranges, int64_t* d_count, int32_t* d_status,
                            void* ws, cudaStream_t s) {
  const int64_t n_items = (int64_t)vt.n_views * pitch;
  const int total_tiles = vt.total_tiles;
  SortWs w = carve(ws, cap, total_tiles);
  const int64_t nb_scan = cdiv(total_tiles, kScanTile);
  const int64_t grid_p = std::min<int64_t>(cdiv(std::max<int64_t>((int64_t)kSub * crow(total_tiles), nb_scan), kSortThreads), 1024);
  const int64_t grid_r = std::max<int64_t>(1, std::min<int64_t>(cdiv(n_items, kSortThreads), 1 << 20));

  k_sort_prep<<<(unsigned)std::max<int64_t>(grid_p, 1), kSortThreads, 0, s>>>(w.cnt, total_tiles, w.look, nb_scan,
                                                                          w.counters, d_count, d_status);
  k_tile_count<<<(unsigned)grid_r, kSortThreads, 0, s>>>(pb.rect, pb.tiles, n_items, pitch, vt, total_tiles, w.cnt);
  k_tile_scan<<<(unsigned)nb_scan, kSortThreads, 0, s>>>(w.cnt, total_tiles, w.look, w.counters, ranges, w.cursor,
                                                     w.longl, cap, d_count, d_status, g_spin_limit.load(),
                                                     g_withhold.load());
  k_tile_scatter<<<(unsigned)grid_r, kSortThreads, 0, s>>>(pb.rect, pb.tiles, pb.key, n_items, pitch, vt, total_tiles,
                                                       w.cursor, w.items, cap, d_status);
  k_tile_sort<<<(unsigned)(device_sm_count() * 3), kSortThreads, 0, s>>>(ranges, total_tiles, w.longl, w.counters, w.items,
                                                              w.tmp, pair_vals, d_status);
  return cudaGetLastError();
}

}  // namespace beta
