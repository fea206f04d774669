/*
 * beta_splat.h -- C ABI of the GB300 (sm_103a) Beta-splatting rasterizer.
 *
 * Deformable Beta Splatting (arXiv 2501.18630): 3D ellipsoidal Beta
 * primitives {mu, o, q, s, b, f} (Sec. 3.2) are projected with EWA
 * (Sigma' = J W Sigma W^T J^T), binned into pixel tiles (16x16 by default), depth-sorted,
 * and composited front to back with the Beta kernel
 *     alpha = min(alpha_max, o (1 - r^2)^beta),  beta = 4 e^b    (Eq. 2, Eq. eq:beta)
 *     C(x) = sum_i c_i alpha_i prod_{j<i} (1 - alpha_j)              (Eq. C)
 * with view-dependent spherical-Beta colour                          (Sec. 3.3)
 *     c(V) = c0 + sum_m max(R_m . V, 0)^(4 e^{b_m}) c_m.
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 *  - Memory: the caller owns every buffer.  The library never allocates or
 *    frees device memory; sizes come from the *_bytes() queries.  Pointers
 *    are DEVICE pointers unless the argument is documented as host.
 *  - Streams: every compute call is asynchronous on `stream` (a
 *    cudaStream_t; NULL means the legacy default stream), never
 *    synchronises, and issues only kernel launches.
 *  - Errors: host-detectable argument errors (null pointers, bad sizes,
 *    unsupported options, too small workspace) are returned immediately as
 *    a negative beta_status and nothing is launched.  A failed launch
 *    returns BETA_ERR_CUDA.  Data-dependent errors (pair capacity overflow,
 *    a bounded spin-wait that ran out) are written to the device status word
 *    `d_status` (int32), which the caller reads after synchronising; every
 *    kernel downstream of a non-zero status skips its work.
 *  - Culling: non-finite primitives, centres with camera depth <= near and
 *    primitives whose support misses the image touch no tile.  They are not
 *    errors.
 *
 * Primitive parameters: one float32 plane per scalar, planes of `pitch`
 * floats (pitch >= n, multiple of 4), plane index
 *     0-2 mean xyz | 3-5 log-scale | 6-9 quaternion wxyz (unnormalised) |
 *     10 opacity logit | 11 shape b | 12-14 base colour c0 |
 *     15+6m+{0..5}: lobe m theta, phi, b_m, c_m rgb          (3+6M features)
 * i.e. 15 + 6M planes.  s = exp(log-scale), o = sigmoid(logit),
 * R_m = (sin theta cos phi, sin theta sin phi, cos theta).
 *
 * Batches of views: V <= BETA_MAX_VIEWS cameras.  View v has
 * ntx_v x nty_v tiles, ntx_v = ceil(W_v / tile_w); global tile ids run view
 * by view (row-major inside a view).  Pixel outputs of view v start at
 * pixel offset P_v = sum_{u<v} W_u H_u: colour is planar per view,
 * color[3 P_v + ch W_v H_v + y W_v + x]; T_final and n_contrib are
 * [P_v + y W_v + x].  A record is (view, primitive) = v * pitch + i.
 */
#ifndef BETA_SPLAT_H
#define BETA_SPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* beta_stream_t; /* == cudaStream_t */

typedef enum {
  BETA_OK = 0,
  BETA_ERR_ARG = -1,         /* invalid argument (host-detected)                  */
  BETA_ERR_CAPACITY = -2,    /* more (tile, primitive) pairs than pair_capacity   */
  BETA_ERR_CUDA = -3,        /* a kernel launch failed                            */
  BETA_ERR_TIMEOUT = -4,     /* a bounded device spin-wait gave up                */
  BETA_ERR_UNSUPPORTED = -5, /* option outside the supported set                  */
  BETA_ERR_WORKSPACE = -6    /* workspace smaller than the *_bytes() query        */
} beta_status;

#define BETA_MAX_LOBES 8
#define BETA_MAX_VIEWS 64

/* Primitive parameters (host struct; `planes` is a device pointer). */
typedef struct {
  int32_t n;          /* number of primitives, >= 0                           */
  int32_t pitch;      /* floats per plane, >= n, multiple of 4                */
  int32_t n_lobes;    /* spherical-Beta lobes M, 0..BETA_MAX_LOBES            */
  int32_t reserved;   /* must be 0                                            */
  const float* planes;/* device, (15 + 6M) x pitch float32, layout above     */
} beta_params;

/* Pinhole camera (host struct).  World point X maps to camera space as
 * R X + t (OpenCV axes: x right, y down, z forward); pixel (i, j) is
 * sampled at its centre (i + 1/2, j + 1/2). */
typedef struct {
  float R[9];          /* row-major world->camera rotation                    */
  float t[3];
  float fx, fy, cx, cy;
  float near_plane;    /* centres with camera z <= near_plane are culled      */
  int32_t width, height;
  float bg[3];         /* background, weighted by the final transmittance     */
} beta_camera;

/* Render options (host struct).  beta_default_opts() fills the defaults. */
typedef struct {
  int32_t tile_w, tile_h; /* pixel tile: 8x4, 8x8, 16x8, 16x16 (default) or 32x16 */
  int32_t batch_s;        /* records staged per raster batch: 64, 128 or 256 */
  int32_t color_mode;     /* 0: c0 + lobes, 1: c0 only (diffuse), 2: lobes only (specular) */
  float t_eps;            /* stop before a primitive once T < t_eps (2^-19)   */
  float alpha_max;        /* alpha = min(alpha_max, o B)   (0.99)             */
  float blur_eps;         /* added to the diagonal of Sigma' (0)              */
  float b_lo, b_hi;       /* render only primitives with b_lo <= b < b_hi (geometry
                             decomposition, Sec. 4.3); -inf / +inf by default */
} beta_opts;

void beta_default_opts(beta_opts* opt /* host */);
const char* beta_status_string(int code);
int32_t beta_version(void);

/* Fault-injection hook for tests of the bounded waits (host-only, no device
 * work; the paper has no counterpart).  The tile scan of beta_bin_sort chains
 * its blocks by a decoupled look-back in which each block polls its
 * predecessors' entries; every poll loop gives up after `spin_limit` polls
 * and writes BETA_ERR_TIMEOUT to d_status, and the kernels after it then
 * skip their work.  This call sets the poll limit of later launches
 * (1 .. 2^20; 0 restores the default 2^20) and names one scan block
 * (`withhold_block`, in units of 2048 tiles; -1 for none, the default) that
 * never posts its entry, so that its successors' waits run out.  Process-wide
 * and not thread-safe: for tests only.  Returns BETA_ERR_ARG outside those
 * ranges. */
int beta_debug_scan_faults(int32_t spin_limit, int64_t withhold_block);

/* ---- sizes (host-only queries, no device work) ------------------------ */

/* Bytes of the projection buffer `proj` for V views: 64 bytes per record
 * (48-byte raster record, 8-byte tile rectangle, 4-byte depth key, 4-byte
 * mask of the rectangle's tiles the support reaches), then a worklist of
 * 4 x V bytes per primitive (pitch rounded up to a multiple of 256) and one
 * 4-byte count per 256 primitives, rounded up to 16 bytes. */
size_t beta_proj_bytes(int32_t pitch, int32_t n_views);
/* Total tiles of a batch of views (the length of tile_ranges is this + 1). */
int64_t beta_total_tiles(const beta_camera* cams /* host */, int32_t n_views, const beta_opts* opt);
/* Total pixels of a batch of views. */
int64_t beta_total_pixels(const beta_camera* cams /* host */, int32_t n_views);
/* Workspace of beta_bin_sort for a pair capacity (tile counters and list
 * cursors, the scan's look-back flags, 16 bytes of list items and merge
 * buffer per pair). */
size_t beta_binsort_workspace_bytes(int32_t pitch, int32_t n_views, int64_t pair_capacity,
                                    const beta_camera* cams /* host */, const beta_opts* opt);
/* Workspace of beta_raster_bwd: per-record 2D gradient sums, a 48-byte slot
 * (10 floats used) per record. */
size_t beta_grad2d_bytes(int32_t pitch, int32_t n_views);
/* Workspace of beta_l1_loss (per-block partial sums). */
size_t beta_l1_workspace_bytes(const beta_camera* cams /* host */, int32_t n_views);

/* ---- the hot path ----------------------------------------------------- */

/* Step 1 (Sec. 3.2, Sec. 3.3): per (view, primitive) activations, EWA
 * projection Sigma' = J W R S S^T R^T W^T J^T, projected centre, Beta shape
 * beta = 4 e^b, spherical-Beta colour, tile rectangle, the tiles of the
 * rectangle that the support ellipse reaches (Sec. 3.1, Eq. 2) and depth key.
 * Writes `proj` (beta_proj_bytes(pitch, n_views) bytes, 16-byte aligned). */
int beta_project(const beta_params* prm /* host */, const beta_camera* cams /* host [n_views] */,
                 int32_t n_views, const beta_opts* opt /* host */, void* proj,
                 beta_stream_t stream);

/* Step 2 (Sec. 3.2: overlapping primitives are composited in depth order): forms one
 * (tile, record) pair per tile of each record's rectangle that its support
 * ellipse reaches (the tile mask beta_project wrote), as per-tile
 * lists (atomic counts, their scan, atomic slots), sorts every list by its
 * unique (depth key, record index) items, and writes the per-tile ranges:
 * the pairs end up sorted by (global tile, depth key, primitive index).
 *   pair_vals   [pair_capacity] out: record of every sorted pair
 *   tile_ranges [total_tiles + 1] out: pairs of tile g are
 *               pair_vals[tile_ranges[g] .. tile_ranges[g + 1])
 *   d_pair_count (int64) out: number of pairs K (also when K > capacity)
 *   d_status    out: reset to BETA_OK, then BETA_ERR_CAPACITY if
 *               K > pair_capacity or BETA_ERR_TIMEOUT if a spin gave up.
 *   ws, ws_bytes: workspace of beta_binsort_workspace_bytes(). */
int beta_bin_sort(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                  const beta_opts* opt, const void* proj, uint32_t* pair_vals,
                  int64_t pair_capacity, uint32_t* tile_ranges, int64_t* d_pair_count,
                  int32_t* d_status, void* ws, size_t ws_bytes, beta_stream_t stream);

/* Size of the library's own device scratch array used by
 * beta_bin_sort_static (32 MiB). */
#define BETA_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* beta_bin_sort without a caller workspace.  The paper has no counterpart:
 * this is a deployment convenience.  Some callers cannot allocate device
 * memory at all -- a plugin whose host application owns every device
 * allocation, a real-time loop where cudaMalloc's implicit device
 * synchronisation is not allowed, or a deployment that must reserve all
 * memory when the library is loaded.  They call this variant instead: it is
 * beta_bin_sort with its workspace taken from a file-scope __device__ array
 * of BETA_STATIC_SCRATCH_BYTES inside the library (every GPU that loads the
 * library holds that array until the process exits).  The caller still
 * passes the inputs and outputs, and the call allocates nothing.
 *   - Problems whose workspace (beta_binsort_workspace_bytes) exceeds
 *     BETA_STATIC_SCRATCH_BYTES are rejected with BETA_ERR_WORKSPACE before
 *     anything is launched.
 *   - Each call made outside stream capture looks up the array's device
 *     address (cudaGetSymbolAddress) with the calling device current, so the
 *     first call on a device does the set-up; a call on a capturing stream
 *     reuses the address of an earlier uncaptured call on that device and
 *     returns BETA_ERR_CUDA if there was none.  Make the first call on each
 *     device before any stream capture.
 *   - All calls on a device share the one array, and it keeps what the last
 *     call left in it (the call clears every part that must start at zero).
 *     Calls whose kernels overlap on the GPU (different streams, or
 *     different host threads without ordering) race on the array: order them
 *     on one stream.
 * Arguments, outputs and status codes are those of beta_bin_sort. */
int beta_bin_sort_static(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                         const beta_opts* opt, const void* proj, uint32_t* pair_vals,
                         int64_t pair_capacity, uint32_t* tile_ranges, int64_t* d_pair_count,
                         int32_t* d_status, beta_stream_t stream);

/* Longest-first tile schedule for the persistent raster kernels.  Reads the
 * tile ranges written by beta_bin_sort and writes into `sched`
 * (beta_schedule_bytes() bytes, 4-byte aligned): the tiles ordered by
 * decreasing pair count (bucketed by bit length) and two work counters that
 * the raster kernels consume and reset.  Without a schedule (sched = NULL in
 * the raster calls) CTA b renders tile b. */
size_t beta_schedule_bytes(const beta_camera* cams /* host */, int32_t n_views, const beta_opts* opt);
int beta_schedule(const beta_camera* cams, int32_t n_views, const beta_opts* opt,
                  const uint32_t* tile_ranges, void* sched, const int32_t* d_status,
                  beta_stream_t stream);

/* Bytes of the optional hit-mask buffer of beta_raster_fwd(_l1) and
 * beta_raster_bwd for a pair capacity: per tile and per 32 list positions,
 * one 32-bit word per thread of the tile's raster CTA (which of the 32
 * primitives may cover its pixels: a pair of horizontally adjacent pixels,
 * or one pixel in 8x4 tiles) and one per warp (which cover more than 12 of
 * its threads' pixels): ((pair_capacity >> 5) + total_tiles + 1) x
 * (L x 33/32) x 4 bytes, L = tile pixels / 2 (tile pixels for 8x4 tiles).
 * 0 for invalid arguments. */
size_t beta_hit_mask_bytes(const beta_camera* cams /* host */, int32_t n_views, const beta_opts* opt,
                           int64_t pair_capacity);

/* Step 3 (Eq. C): front-to-back compositing of every tile's sorted list.
 *   color     [3 x total_pixels] out: C + T_final * bg (planar per view)
 *   T_final   [total_pixels] out: final transmittance
 *   n_contrib [total_pixels] out: 1 + position (inside the tile's list) of
 *             the last primitive that contributed, 0 if none.
 *   sched     beta_schedule() output for a persistent launch, or NULL
 *   hit_masks, hit_mask_bytes: NULL / 0, or a 4-byte aligned buffer of
 *             beta_hit_mask_bytes() for the pair capacity of the binning;
 *             the forward writes which primitives may cover each pixel, and
 *             a beta_raster_bwd given the same buffer reads them instead of
 *             working them out again (the results are the same either way;
 *             parts of the lists beyond a shorter buffer are recomputed).
 *   d_status  in: if non-zero the kernel writes nothing. */
int beta_raster_fwd(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                    const beta_opts* opt, const void* proj, const uint32_t* pair_vals,
                    const uint32_t* tile_ranges, void* sched, void* hit_masks, size_t hit_mask_bytes,
                    float* color, float* T_final, uint32_t* n_contrib, const int32_t* d_status,
                    beta_stream_t stream);

/* beta_raster_fwd followed by beta_l1_loss in one pass: the forward kernel
 * computes the L1 term and dL_dcolor of each pixel it writes, and one partial
 * sum per tile, which a second kernel adds per view in tile order.  Outputs
 * color, T_final, n_contrib as beta_raster_fwd, and loss, dL_dcolor as
 * beta_l1_loss (dL_dcolor bit for bit; loss to fp32 summation order).
 *   target   [3 x total_pixels] in (layout of color)
 *   loss     device float[n_views] out;  dL_dcolor: layout of color, out
 *   ws       beta_raster_fwd_l1_workspace_bytes() bytes (one float per tile),
 *            4-byte aligned
 * Returns BETA_ERR_ARG for null pointers, BETA_ERR_WORKSPACE for a short or
 * misaligned ws. */
size_t beta_raster_fwd_l1_workspace_bytes(const beta_camera* cams /* host */, int32_t n_views,
                                          const beta_opts* opt);
int beta_raster_fwd_l1(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                       const beta_opts* opt, const void* proj, const uint32_t* pair_vals,
                       const uint32_t* tile_ranges, void* sched, void* hit_masks, size_t hit_mask_bytes,
                       float* color, float* T_final, uint32_t* n_contrib, const float* target, float* loss,
                       float* dL_dcolor, void* ws, size_t ws_bytes, const int32_t* d_status,
                       beta_stream_t stream);

/* Per-pixel L1 loss of a batch of views (Sec. 3.4, the L1 term):
 *   loss[v] = mean over 3 W_v H_v of |color - target|   (device float[n_views], out)
 *   dL_dcolor = sign(color - target) / (3 W_v H_v)       (same layout as color, out)
 * so the gradient is that of sum_v loss[v].  ws: beta_l1_workspace_bytes(). */
int beta_l1_loss(const beta_camera* cams, int32_t n_views, const float* color,
                 const float* target, float* loss, float* dL_dcolor, void* ws, size_t ws_bytes,
                 beta_stream_t stream);

/* Step 4a (backward of Eq. C): walks each pixel's list from its last
 * contributor down, recovering T by division, and accumulates ten per-record
 * sums with vector or warp-reduced atomics into grad2d: in whitened coordinates
 * (u, v) = L^-1 (x - mu') (Sigma' = L L^T) and with k = (dL/dalpha) alpha /
 * (1 - r^2) -- sum k (u, v, u^2, u v, v^2), sum (dL/dalpha) alpha, the same
 * times log2(1 - r^2), and sum alpha T dL/dC (3).  beta_project_bwd turns
 * them into d mu', d Sigma', d o, d beta and d colour.
 *   sched     beta_schedule() output (persistent launch) or NULL
 *   hit_masks, hit_mask_bytes: the buffer the forward of these lists wrote
 *             (beta_raster_fwd), or NULL / 0
 *   dL_dcolor [3 x total_pixels] in (layout of color)
 *   grad2d    [beta_grad2d_bytes()] in/out: one 48-byte slot per record (16-byte
 *             aligned buffer), ACCUMULATED.
 *             It must hold zeros on entry: zero it once after allocation;
 *             beta_project_bwd clears every slot it consumes. */
int beta_raster_bwd(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                    const beta_opts* opt, const void* proj, const uint32_t* pair_vals,
                    const uint32_t* tile_ranges, void* sched, const void* hit_masks, size_t hit_mask_bytes,
                    const float* T_final, const uint32_t* n_contrib, const float* dL_dcolor, float* grad2d,
                    const int32_t* d_status, beta_stream_t stream);

/* Steps 3 and 4a with the L1 loss between them, in one launch (Eq. C, the
 * L1 term of Sec. 3.4 and the reverse-mode derivative of Eq. C): for every
 * tile, one CTA composites the tile's pixels, forms their L1 term and
 * dL/dC = sign(C - target) / (3 W_v H_v) in registers, and then walks the
 * tile's list in reverse from those registers, adding the ten per-record sums
 * of beta_raster_bwd into grad2d.  No per-pixel state passes through memory
 * between the forward and the backward, and the backward finds the records
 * the forward of the same tile just read in L2.
 * The results are those of beta_raster_fwd_l1 followed by beta_raster_bwd on
 * the same lists: color, T_final, n_contrib, dL_dcolor bit for bit, loss to
 * the same fp32 summation order, and every term added to grad2d the same,
 * with the sums differing only in the order of the floating-point atomic
 * additions.
 *   T_final, n_contrib, dL_dcolor  optional outputs (NULL: not written)
 *   target, loss, ws, ws_bytes     as beta_raster_fwd_l1
 *   grad2d    as beta_raster_bwd (zeros on entry, accumulated)
 *   sched     beta_schedule() output for a persistent launch, or NULL
 * Only tile shapes whose raster kernels give each thread a pair of pixels
 * (every supported shape but 8 x 4) have this kernel: BETA_ERR_ARG for 8 x 4
 * tiles (run beta_raster_fwd_l1 and beta_raster_bwd there), for null
 * required pointers and a grad2d that is not 16-byte aligned;
 * BETA_ERR_WORKSPACE for a short or misaligned ws. */
/* 1 if beta_raster_fwd_bwd_l1 serves these options (valid options whose tile
 * shape has pixel-pair raster kernels: every supported shape but 8 x 4), else
 * 0.  Host-only; needs no GPU. */
int beta_raster_fwd_bwd_l1_supported(const beta_opts* opt /* host */);
int beta_raster_fwd_bwd_l1(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                           const beta_opts* opt, const void* proj, const uint32_t* pair_vals,
                           const uint32_t* tile_ranges, void* sched, float* color, float* T_final,
                           uint32_t* n_contrib, const float* target, float* loss, float* dL_dcolor,
                           float* grad2d, void* ws, size_t ws_bytes, const int32_t* d_status,
                           beta_stream_t stream);

/* Step 4b (backward of Sec. 3.2 / Sec. 3.3): chains the 2D gradients of every
 * view through Sigma' = M M^T, M = J W R(q) S, mu'(t), t = W mu + t_w, the
 * sigmoid, beta = 4 e^b and the spherical-Beta colour to the raw parameters,
 * summing over views, then writes zeros back into grad2d.
 *   grad_planes out: (15 + 6M) x pitch float32, same layout as the params,
 *             overwritten for i < n (padding lanes are left untouched).
 *   d_status  in: if non-zero, the gradients are written as zeros. */
int beta_project_bwd(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                     const beta_opts* opt, float* grad2d, float* grad_planes,
                     const int32_t* d_status, beta_stream_t stream);

/* ---- the optimiser step after the backward (Sec. 3.4) ----------------- */

/* Options of beta_adam_step (host struct).  beta_adam_default_opts() fills the
 * appendix "Hyperparameters" values: lr = {1.6e-4 (mean, the initial
 * lambda_lr; the caller applies its decay), 5e-3 (log-scale), 1e-3
 * (quaternion), 5e-2 (opacity logit), 1e-3 (b), 2.5e-3 (c0), 2.5e-3 (lobe
 * direction theta, phi), 2.5e-3 (lobe b_m), 2.5e-3 (lobe colour)},
 * lambda_o = lambda_Sigma = 0.01, lambda_eps = 5e4, b' = ln 25; Adam
 * beta1 0.9, beta2 0.999, eps 1e-15 (the paper does not state them). */
typedef struct {
  float lr[9];
  float beta1, beta2, eps;
  float lambda_o, lambda_sigma; /* regulariser weights of the composite loss          */
  float lambda_eps, noise_b;    /* position-noise weight and the Beta kernel's b'     */
  int32_t step;                 /* Adam step t >= 1 (bias correction 1 - beta^t)     */
} beta_adam_opts;

void beta_adam_default_opts(beta_adam_opts* opt /* host */);

/* One optimiser step on the first n primitives (Sec. 3.4 "Optimization" and
 * the composite loss):
 *   g  = grad + lambda_o d(sum |o|) + lambda_Sigma d(sum_j sqrt(eig_j Sigma))
 *        (= lambda_o o (1 - o) on the opacity logit, lambda_Sigma s_j on log-scale j)
 *   Adam with one learning rate per parameter group (lr[] above),
 *   mu += lambda_eps lr[0] (1 - o)^(4 e^b') Sigma eta,  Sigma = R diag(s^2) R^T,
 * with o, s, R taken before the step.
 *   planes     [15 + 6M][pitch] in/out: raw parameters (beta_params layout)
 *   grad       [15 + 6M][pitch] in: dL/d(raw parameters) (beta_project_bwd's output)
 *   adam_m, adam_v [15 + 6M][pitch] in/out: moments (zero before the first step)
 *   eta        [3][pitch] in: standard normal samples, one triple per primitive
 *   reg_loss   device double[2] or NULL: lambda_o sum o and lambda_Sigma sum_j s_j
 *              are ADDED to it
 * All device pointers 16-byte aligned.  Returns BETA_ERR_ARG for null pointers,
 * n > pitch, pitch not a multiple of 4, n_lobes > 8, step < 1, or betas outside
 * [0, 1). */
int beta_adam_step(int32_t n, int32_t pitch, int32_t n_lobes, float* planes, const float* grad,
                   float* adam_m, float* adam_v, const float* eta, const beta_adam_opts* opt,
                   double* reg_loss, beta_stream_t stream);

/* Relocation of dead primitives (Sec. 3.4 "Densification", Eq. eq:densify),
 * run every few hundred steps.  Primitive i < n is dead when its opacity,
 * by the fixed fp32 rule o = 1 / (1 + e(-clamp(logit, -80, 80))) (e: the
 * Cody-Waite / degree-7 Taylor exp of the binning rule, every operation
 * rounded to nearest), is below min_opacity.  Each dead primitive draws a
 * live source with probability proportional to opacity: weights
 * floor(o 2^24), inclusive 64-bit prefix sums W, its random word r[i] picks
 * t = floor(r[i] W_total / 2^32) and the source is the first j with W_j > t.
 * Every parameter of the source is copied to it; a source with N copies in
 * all (itself included) gets o' = 1 - (1 - o)^(1/N) on each; the copies'
 * Adam moments are zeroed.  Nothing changes when no primitive is live.
 *   planes [15 + 6M][pitch] in/out; adam_m, adam_v same layout, in/out, or NULL
 *   rnd     [n] in: uniform 32-bit random words
 *   ws      beta_relocate_workspace_bytes(n) bytes, 256-byte aligned
 *   src_out [n] out or NULL: source index of each primitive, -1 if kept
 *   d_count device int32 out: number of relocated primitives */
size_t beta_relocate_workspace_bytes(int32_t n);
int beta_relocate(int32_t n, int32_t pitch, int32_t n_lobes, float* planes, float* adam_m,
                  float* adam_v, const uint32_t* rnd, float min_opacity, void* ws, size_t ws_bytes,
                  int32_t* src_out, int32_t* d_count, beta_stream_t stream);

/* ---- the composite loss with the DSSIM term (Sec. 3.4) -------------- */

/* Per view v, colour x and target y (layout of beta_raster_fwd's colour):
 *   loss[v] = (1 - lambda_ssim) mean|x - y| + lambda_ssim (1 - mean SSIM(x, y))
 * with SSIM from Gaussian-weighted local statistics (11 taps, sigma 1.5,
 * separable, zero outside the image, C1 = 0.01^2, C2 = 0.03^2, dynamic range
 * 1), means over the view's 3 W H values; dL_dcolor = d(sum_v loss[v])/dx
 * (sign(0) = 0 in the L1 part).  The appendix uses lambda_ssim = 0.2;
 * lambda_ssim = 0 is the plain L1 loss of beta_l1_loss.
 *   loss      device float[n_views] out;  dL_dcolor: layout of color, out
 *   ws        beta_dssim_workspace_bytes() bytes, 256-byte aligned
 * Returns BETA_ERR_ARG for null pointers or lambda_ssim outside [0, 1]. */
size_t beta_dssim_workspace_bytes(const beta_camera* cams /* host */, int32_t n_views);
int beta_l1_dssim_loss(const beta_camera* cams, int32_t n_views, const float* color,
                       const float* target, float lambda_ssim, float* loss, float* dL_dcolor,
                       void* ws, size_t ws_bytes, beta_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* BETA_SPLAT_H */
