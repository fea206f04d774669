// beta_api.cu -- the C ABI declared in include/beta_splat.h: argument
// validation, view tables, workspace carving and kernel launches.  Every
// entry point only enqueues kernels on the caller's stream.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "beta_internal.cuh"
#include "beta_splat.h"

using namespace beta;

namespace {

constexpr int32_t kVersion = 1;

bool valid_params(const beta_params* p) {
  if (!p) return false;
  if (p->n < 0 || p->pitch < p->n || p->pitch % 4 != 0 || p->pitch <= 0) return false;
  if (p->n_lobes < 0 || p->n_lobes > BETA_MAX_LOBES || p->reserved != 0) return false;
  if (p->n > 0 && !p->planes) return false;
  if (((uintptr_t)p->planes & 15u) != 0) return false;
  return true;
}

int check_opts(const beta_opts* o) {
  if (!o) return BETA_ERR_ARG;
  const int shape = o->tile_w * 1000 + o->tile_h;
  if (shape != 8004 && shape != 8008 && shape != 16008 && shape != 16016 && shape != 32016)
    return BETA_ERR_UNSUPPORTED;
  if (o->batch_s != 64 && o->batch_s != 128 && o->batch_s != 256) return BETA_ERR_UNSUPPORTED;
  if (o->color_mode < 0 || o->color_mode > 2) return BETA_ERR_ARG;
  if (!(o->t_eps >= 0.0f && o->t_eps < 1.0f)) return BETA_ERR_ARG;
  if (!(o->alpha_max > 0.0f && o->alpha_max < 1.0f)) return BETA_ERR_ARG;
  if (!(o->blur_eps >= 0.0f) || !isfinite(o->blur_eps)) return BETA_ERR_ARG;
  if (isnan(o->b_lo) || isnan(o->b_hi)) return BETA_ERR_ARG;
  return BETA_OK;
}

int build_views(const beta_camera* cams, int32_t n_views, const beta_opts* opt, ViewTable& vt) {
  if (!cams || n_views <= 0 || n_views > BETA_MAX_VIEWS) return BETA_ERR_ARG;
  memset(&vt, 0, sizeof(vt));
  vt.n_views = n_views;
  int64_t tiles = 0, pix = 0;
  for (int v = 0; v < n_views; ++v) {
    const beta_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || c.width > 65535 * 16 || c.height > 65535 * 16) return BETA_ERR_ARG;
    for (int k = 0; k < 9; ++k)
      if (!isfinite(c.R[k])) return BETA_ERR_ARG;
    for (int k = 0; k < 3; ++k)
      if (!isfinite(c.t[k]) || !isfinite(c.bg[k])) return BETA_ERR_ARG;
    if (!isfinite(c.fx) || !isfinite(c.fy) || !isfinite(c.cx) || !isfinite(c.cy) || !(c.near_plane > 0.0f))
      return BETA_ERR_ARG;
    ViewDev& d = vt.v[v];
    memcpy(d.R, c.R, sizeof(d.R));
    memcpy(d.t, c.t, sizeof(d.t));
    d.fx = c.fx;
    d.fy = c.fy;
    d.cx = c.cx;
    d.cy = c.cy;
    d.near_plane = c.near_plane;
    // camera position -R^T t (fp64, rounded once)
    for (int r = 0; r < 3; ++r)
      d.campos[r] = (float)-((double)c.R[0 * 3 + r] * c.t[0] + (double)c.R[1 * 3 + r] * c.t[1] +
                              (double)c.R[2 * 3 + r] * c.t[2]);
    memcpy(d.bg, c.bg, sizeof(d.bg));
    d.width = c.width;
    d.height = c.height;
    d.ntx = (c.width + opt->tile_w - 1) / opt->tile_w;
    d.nty = (c.height + opt->tile_h - 1) / opt->tile_h;
    d.tile_off = (int32_t)tiles;
    d.pix_off = pix;
    tiles += (int64_t)d.ntx * d.nty;
    pix += (int64_t)c.width * c.height;
  }
  if (tiles >= (1ll << 30)) return BETA_ERR_ARG;
  vt.total_tiles = (int32_t)tiles;
  vt.total_pixels = pix;
  return BETA_OK;
}

RenderOpts render_opts(const beta_opts* o) {
  RenderOpts r;
  r.t_eps = o->t_eps;
  r.alpha_max = o->alpha_max;
  r.blur_eps = o->blur_eps;
  r.b_lo = o->b_lo;
  r.b_hi = o->b_hi;
  r.color_mode = o->color_mode;
  r.tile_w = o->tile_w;
  r.tile_h = o->tile_h;
  r.batch_s = o->batch_s;
  return r;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

int cuda_status(cudaError_t e) { return e == cudaSuccess ? BETA_OK : BETA_ERR_CUDA; }

// Device scratch of beta_bin_sort_static: a fixed array inside the library,
// so callers that cannot allocate need not provide a workspace.
static __device__ __align__(256) unsigned char g_binsort_scratch[BETA_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_binsort_scratch on the current device (the host-side
// symbol itself is not a device address).  Looked up with the device current
// on every call made outside stream capture, so a device reset between calls
// is picked up; a call on a capturing stream takes the address an earlier
// uncaptured call on that device looked up, and fails without one.
int static_scratch(cudaStream_t stream, void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return BETA_ERR_CUDA;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  const cudaError_t q = cudaStreamIsCapturing(stream, &cap);
  if (q != cudaSuccess) cudaGetLastError();   // a refused query (legacy stream during a capture) is not kept
  const bool capturing = q != cudaSuccess || cap != cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!capturing) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_binsort_scratch) != cudaSuccess || !p) return BETA_ERR_CUDA;
    g_scratch_ptr[dev] = p;
  }
  if (!g_scratch_ptr[dev]) return BETA_ERR_CUDA;
  *out = g_scratch_ptr[dev];
  return BETA_OK;
}

}  // namespace

extern "C" {

void beta_default_opts(beta_opts* o) {
  if (!o) return;
  o->tile_w = 16;
  o->tile_h = 16;
  o->batch_s = 256;
  o->color_mode = 0;
  o->t_eps = 1.9073486328125e-06f;  // 2^-19
  o->alpha_max = 0.99f;
  o->blur_eps = 0.0f;
  o->b_lo = -INFINITY;
  o->b_hi = INFINITY;
}

const char* beta_status_string(int code) {
  switch (code) {
    case BETA_OK: return "ok";
    case BETA_ERR_ARG: return "invalid argument";
    case BETA_ERR_CAPACITY: return "pair capacity exceeded";
    case BETA_ERR_CUDA: return "CUDA launch failed";
    case BETA_ERR_TIMEOUT: return "device spin-wait timed out";
    case BETA_ERR_UNSUPPORTED: return "unsupported option";
    case BETA_ERR_WORKSPACE: return "workspace too small";
    default: return "unknown status";
  }
}

int32_t beta_version(void) { return kVersion; }

int beta_debug_scan_faults(int32_t spin_limit, int64_t withhold_block) {
  return set_scan_faults(spin_limit, withhold_block) == 0 ? BETA_OK : BETA_ERR_ARG;
}

size_t beta_proj_bytes(int32_t pitch, int32_t n_views) {
  if (pitch <= 0 || n_views <= 0) return 0;
  return proj_bytes(pitch, n_views);
}

int64_t beta_total_tiles(const beta_camera* cams, int32_t n_views, const beta_opts* opt) {
  ViewTable vt;
  if (check_opts(opt) != BETA_OK || build_views(cams, n_views, opt, vt) != BETA_OK) return -1;
  return vt.total_tiles;
}

int64_t beta_total_pixels(const beta_camera* cams, int32_t n_views) {
  beta_opts o;
  beta_default_opts(&o);
  ViewTable vt;
  if (build_views(cams, n_views, &o, vt) != BETA_OK) return -1;
  return vt.total_pixels;
}

size_t beta_binsort_workspace_bytes(int32_t pitch, int32_t n_views, int64_t cap,
                                    const beta_camera* cams, const beta_opts* opt) {
  ViewTable vt;
  if (pitch <= 0 || cap < 0 || check_opts(opt) != BETA_OK || build_views(cams, n_views, opt, vt) != BETA_OK)
    return 0;
  return binsort_ws_bytes((int64_t)pitch * n_views, cap, vt.total_tiles);
}

size_t beta_grad2d_bytes(int32_t pitch, int32_t n_views) {
  if (pitch <= 0 || n_views <= 0) return 0;
  return (size_t)pitch * n_views * kGrad2dStride * sizeof(float);
}

size_t beta_l1_workspace_bytes(const beta_camera* cams, int32_t n_views) {
  beta_opts o;
  beta_default_opts(&o);
  ViewTable vt;
  if (build_views(cams, n_views, &o, vt) != BETA_OK) return 0;
  return l1_ws_bytes(vt);
}

int beta_project(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                 const beta_opts* opt, void* proj, beta_stream_t stream) {
  if (!valid_params(prm) || !proj || !aligned16(proj)) return BETA_ERR_ARG;
  int e = check_opts(opt);
  if (e != BETA_OK) return e;
  ViewTable vt;
  if ((e = build_views(cams, n_views, opt, vt)) != BETA_OK) return e;
  if ((int64_t)prm->pitch * n_views >= (1ll << 32)) return BETA_ERR_ARG;
  ProjBuffers pb = proj_layout(proj, prm->pitch, n_views);
  return cuda_status(launch_project(prm->planes, prm->n, prm->pitch, prm->n_lobes, vt,
                                    render_opts(opt), pb, (cudaStream_t)stream));
}

int beta_bin_sort(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                  const beta_opts* opt, const void* proj, uint32_t* pair_vals,
                  int64_t pair_capacity, uint32_t* tile_ranges, int64_t* d_pair_count,
                  int32_t* d_status, void* ws, size_t ws_bytes, beta_stream_t stream) {
  if (!valid_params(prm) || !proj || !aligned16(proj) || !tile_ranges || !d_pair_count || !d_status)
    return BETA_ERR_ARG;
  if (pair_capacity < 0 || pair_capacity > 0x7fffffffll || (pair_capacity > 0 && !pair_vals))
    return BETA_ERR_ARG;
  int e = check_opts(opt);
  if (e != BETA_OK) return e;
  ViewTable vt;
  if ((e = build_views(cams, n_views, opt, vt)) != BETA_OK) return e;
  if ((int64_t)prm->pitch * n_views >= (1ll << 32)) return BETA_ERR_ARG;
  size_t need = binsort_ws_bytes((int64_t)prm->pitch * n_views, pair_capacity, vt.total_tiles);
  if (!ws || ws_bytes < need || ((uintptr_t)ws & 255u) != 0) return BETA_ERR_WORKSPACE;
  ProjBuffers pb = proj_layout((void*)proj, prm->pitch, n_views);
  return cuda_status(launch_bin_sort(vt, prm->pitch, pb, pair_vals, pair_capacity, tile_ranges,
                                     d_pair_count, d_status, ws, (cudaStream_t)stream));
}

int beta_bin_sort_static(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                         const beta_opts* opt, const void* proj, uint32_t* pair_vals,
                         int64_t pair_capacity, uint32_t* tile_ranges, int64_t* d_pair_count,
                         int32_t* d_status, beta_stream_t stream) {
  if (!valid_params(prm) || !proj || !aligned16(proj) || !tile_ranges || !d_pair_count || !d_status)
    return BETA_ERR_ARG;
  if (pair_capacity < 0 || pair_capacity > 0x7fffffffll || (pair_capacity > 0 && !pair_vals))
    return BETA_ERR_ARG;
  int e = check_opts(opt);
  if (e != BETA_OK) return e;
  ViewTable vt;
  if ((e = build_views(cams, n_views, opt, vt)) != BETA_OK) return e;
  if ((int64_t)prm->pitch * n_views >= (1ll << 32)) return BETA_ERR_ARG;
  size_t need = binsort_ws_bytes((int64_t)prm->pitch * n_views, pair_capacity, vt.total_tiles);
  if (need > (size_t)BETA_STATIC_SCRATCH_BYTES) return BETA_ERR_WORKSPACE;
  void* ws = nullptr;
  if ((e = static_scratch((cudaStream_t)stream, &ws)) != BETA_OK) return e;
  ProjBuffers pb = proj_layout((void*)proj, prm->pitch, n_views);
  return cuda_status(launch_bin_sort(vt, prm->pitch, pb, pair_vals, pair_capacity, tile_ranges,
                                     d_pair_count, d_status, ws, (cudaStream_t)stream));
}

size_t beta_hit_mask_bytes(const beta_camera* cams, int32_t n_views, const beta_opts* opt,
                           int64_t pair_capacity) {
  ViewTable vt;
  if (pair_capacity < 0 || check_opts(opt) != BETA_OK || build_views(cams, n_views, opt, vt) != BETA_OK) return 0;
  return hit_mask_bytes(vt, render_opts(opt), pair_capacity);
}

int beta_raster_fwd(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                    const beta_opts* opt, const void* proj, const uint32_t* pair_vals,
                    const uint32_t* tile_ranges, void* sched, void* hit_masks, size_t hit_mask_bytes,
                    float* color, float* T_final, uint32_t* n_contrib, const int32_t* d_status,
                    beta_stream_t stream) {
  if (!valid_params(prm) || !proj || !aligned16(proj) || !tile_ranges || !color || !T_final ||
      !n_contrib || !d_status)
    return BETA_ERR_ARG;
  int e = check_opts(opt);
  if (e != BETA_OK) return e;
  ViewTable vt;
  if ((e = build_views(cams, n_views, opt, vt)) != BETA_OK) return e;
  ProjBuffers pb = proj_layout((void*)proj, prm->pitch, n_views);
  if (sched && ((uintptr_t)sched & 3u)) return BETA_ERR_ARG;
  if (hit_masks && ((uintptr_t)hit_masks & 3u)) return BETA_ERR_ARG;
  const HitMasks hm{hit_masks ? (uint32_t*)hit_masks : nullptr, hit_masks ? hit_mask_bytes / 4 : 0};
  return cuda_status(launch_raster_fwd(vt, render_opts(opt), pb.rec, pair_vals, tile_ranges, color,
                                       T_final, n_contrib, d_status, (uint32_t*)sched, hm,
                                       (cudaStream_t)stream));
}

size_t beta_raster_fwd_l1_workspace_bytes(const beta_camera* cams, int32_t n_views, const beta_opts* opt) {
  ViewTable vt;
  if (check_opts(opt) != BETA_OK || build_views(cams, n_views, opt, vt) != BETA_OK) return 0;
  return fwd_l1_ws_bytes(vt);
}

int beta_raster_fwd_l1(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                       const beta_opts* opt, const void* proj, const uint32_t* pair_vals,
                       const uint32_t* tile_ranges, void* sched, void* hit_masks, size_t hit_mask_bytes,
                       float* color, float* T_final, uint32_t* n_contrib, const float* target, float* loss,
                       float* dL_dcolor, void* ws, size_t ws_bytes, const int32_t* d_status,
                       beta_stream_t stream) {
  if (!valid_params(prm) || !proj || !aligned16(proj) || !tile_ranges || !color || !T_final ||
      !n_contrib || !d_status || !target || !loss || !dL_dcolor)
    return BETA_ERR_ARG;
  int e = check_opts(opt);
  if (e != BETA_OK) return e;
  ViewTable vt;
  if ((e = build_views(cams, n_views, opt, vt)) != BETA_OK) return e;
  if (sched && ((uintptr_t)sched & 3u)) return BETA_ERR_ARG;
  if (!ws || ws_bytes < fwd_l1_ws_bytes(vt) || ((uintptr_t)ws & 3u)) return BETA_ERR_WORKSPACE;
  if (hit_masks && ((uintptr_t)hit_masks & 3u)) return BETA_ERR_ARG;
  ProjBuffers pb = proj_layout((void*)proj, prm->pitch, n_views);
  const HitMasks hm{hit_masks ? (uint32_t*)hit_masks : nullptr, hit_masks ? hit_mask_bytes / 4 : 0};
  return cuda_status(launch_raster_fwd_l1(vt, render_opts(opt), pb.rec, pair_vals, tile_ranges, color,
                                          T_final, n_contrib, d_status, (uint32_t*)sched, target, loss,
                                          dL_dcolor, (float*)ws, hm, (cudaStream_t)stream));
}

size_t beta_schedule_bytes(const beta_camera* cams, int32_t n_views, const beta_opts* opt) {
  ViewTable vt;
  if (check_opts(opt) != BETA_OK || build_views(cams, n_views, opt, vt) != BETA_OK) return 0;
  return schedule_bytes(vt.total_tiles);
}

int beta_schedule(const beta_camera* cams, int32_t n_views, const beta_opts* opt,
                  const uint32_t* tile_ranges, void* sched, const int32_t* d_status,
                  beta_stream_t stream) {
  if (!tile_ranges || !sched || !d_status || ((uintptr_t)sched & 3u)) return BETA_ERR_ARG;
  int e = check_opts(opt);
  if (e != BETA_OK) return e;
  ViewTable vt;
  if ((e = build_views(cams, n_views, opt, vt)) != BETA_OK) return e;
  return cuda_status(launch_schedule(vt, tile_ranges, (uint32_t*)sched, d_status, (cudaStream_t)stream));
}

int beta_l1_loss(const beta_camera* cams, int32_t n_views, const float* color, const float* target,
                 float* loss, float* dL_dcolor, void* ws, size_t ws_bytes, beta_stream_t stream) {
  if (!color || !target || !loss || !dL_dcolor) return BETA_ERR_ARG;
  beta_opts o;
  beta_default_opts(&o);
  ViewTable vt;
  int e = build_views(cams, n_views, &o, vt);
  if (e != BETA_OK) return e;
  if (!ws || ws_bytes < l1_ws_bytes(vt)) return BETA_ERR_WORKSPACE;
  return cuda_status(launch_l1(vt, color, target, loss, dL_dcolor, (float*)ws, (cudaStream_t)stream));
}

int beta_raster_bwd(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                    const beta_opts* opt, const void* proj, const uint32_t* pair_vals,
                    const uint32_t* tile_ranges, void* sched, const void* hit_masks, size_t hit_mask_bytes,
                    const float* T_final, const uint32_t* n_contrib, const float* dL_dcolor, float* grad2d,
                    const int32_t* d_status, beta_stream_t stream) {
  if (!valid_params(prm) || !proj || !aligned16(proj) || !tile_ranges || !T_final || !n_contrib ||
      !dL_dcolor || !grad2d || !d_status || !aligned16(grad2d))
    return BETA_ERR_ARG;
  int e = check_opts(opt);
  if (e != BETA_OK) return e;
  ViewTable vt;
  if ((e = build_views(cams, n_views, opt, vt)) != BETA_OK) return e;
  ProjBuffers pb = proj_layout((void*)proj, prm->pitch, n_views);
  if (sched && ((uintptr_t)sched & 3u)) return BETA_ERR_ARG;
  if (hit_masks && ((uintptr_t)hit_masks & 3u)) return BETA_ERR_ARG;
  const HitMasks hm{hit_masks ? (uint32_t*)hit_masks : nullptr, hit_masks ? hit_mask_bytes / 4 : 0};
  return cuda_status(launch_raster_bwd(vt, render_opts(opt), pb.rec, pair_vals, tile_ranges,
                                       T_final, n_contrib, dL_dcolor, grad2d, d_status,
                                       (uint32_t*)sched, hm, (cudaStream_t)stream));
}

int beta_raster_fwd_bwd_l1_supported(const beta_opts* opt) {
  return check_opts(opt) == BETA_OK && raster_step_supported(render_opts(opt)) ? 1 : 0;
}

int beta_raster_fwd_bwd_l1(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                           const beta_opts* opt, const void* proj, const uint32_t* pair_vals,
                           const uint32_t* tile_ranges, void* sched, float* color, float* T_final,
                           uint32_t* n_contrib, const float* target, float* loss, float* dL_dcolor,
                           float* grad2d, void* ws, size_t ws_bytes, const int32_t* d_status,
                           beta_stream_t stream) {
  if (!valid_params(prm) || !proj || !aligned16(proj) || !tile_ranges || !color || !target || !loss ||
      !grad2d || !aligned16(grad2d) || !d_status)
    return BETA_ERR_ARG;
  int e = check_opts(opt);
  if (e != BETA_OK) return e;
  if (!raster_step_supported(render_opts(opt))) return BETA_ERR_ARG;
  ViewTable vt;
  if ((e = build_views(cams, n_views, opt, vt)) != BETA_OK) return e;
  if (sched && ((uintptr_t)sched & 3u)) return BETA_ERR_ARG;
  if (!ws || ws_bytes < fwd_l1_ws_bytes(vt) || ((uintptr_t)ws & 3u)) return BETA_ERR_WORKSPACE;
  ProjBuffers pb = proj_layout((void*)proj, prm->pitch, n_views);
  return cuda_status(launch_raster_step_l1(vt, render_opts(opt), pb.rec, pair_vals, tile_ranges, color, T_final,
                                           n_contrib, d_status, (uint32_t*)sched, target, loss, dL_dcolor,
                                           (float*)ws, grad2d, (cudaStream_t)stream));
}

int beta_project_bwd(const beta_params* prm, const beta_camera* cams, int32_t n_views,
                     const beta_opts* opt, float* grad2d, float* grad_planes,
                     const int32_t* d_status, beta_stream_t stream) {
  if (!valid_params(prm) || !grad2d || !grad_planes || !d_status || !aligned16(grad2d))
    return BETA_ERR_ARG;
  int e = check_opts(opt);
  if (e != BETA_OK) return e;
  ViewTable vt;
  if ((e = build_views(cams, n_views, opt, vt)) != BETA_OK) return e;
  return cuda_status(launch_project_bwd(prm->planes, prm->n, prm->pitch, prm->n_lobes, vt,
                                        render_opts(opt), grad2d, grad_planes, d_status,
                                        (cudaStream_t)stream));
}

void beta_adam_default_opts(beta_adam_opts* o) {
  if (!o) return;
  const float lr[9] = {1.6e-4f, 5e-3f, 1e-3f, 5e-2f, 1e-3f, 2.5e-3f, 2.5e-3f, 2.5e-3f, 2.5e-3f};
  for (int k = 0; k < 9; ++k) o->lr[k] = lr[k];
  o->beta1 = 0.9f;
  o->beta2 = 0.999f;
  o->eps = 1e-15f;
  o->lambda_o = 0.01f;
  o->lambda_sigma = 0.01f;
  o->lambda_eps = 5e4f;
  o->noise_b = 3.2188758248682006f;   // ln 25
  o->step = 1;
}

int beta_adam_step(int32_t n, int32_t pitch, int32_t n_lobes, float* planes, const float* grad,
                   float* adam_m, float* adam_v, const float* eta, const beta_adam_opts* opt,
                   double* reg_loss, beta_stream_t stream) {
  if (!opt || n < 0 || pitch < n || pitch % 4 != 0 || n_lobes < 0 || n_lobes > BETA_MAX_LOBES)
    return BETA_ERR_ARG;
  if (!planes || !grad || !adam_m || !adam_v || !eta) return BETA_ERR_ARG;
  if (!aligned16(planes) || !aligned16(grad) || !aligned16(adam_m) || !aligned16(adam_v) || !aligned16(eta))
    return BETA_ERR_ARG;
  if (opt->step < 1 || !(opt->beta1 >= 0.0f && opt->beta1 < 1.0f) || !(opt->beta2 >= 0.0f && opt->beta2 < 1.0f) ||
      !(opt->eps > 0.0f) || !isfinite(opt->noise_b))
    return BETA_ERR_ARG;
  AdamDev a;
  for (int k = 0; k < 9; ++k) a.lr[k] = opt->lr[k];
  a.beta1 = opt->beta1;
  a.beta2 = opt->beta2;
  a.eps = opt->eps;
  a.inv_c1 = (float)(1.0 / (1.0 - pow((double)opt->beta1, (double)opt->step)));
  a.inv_c2 = (float)(1.0 / (1.0 - pow((double)opt->beta2, (double)opt->step)));
  a.lambda_o = opt->lambda_o;
  a.lambda_sigma = opt->lambda_sigma;
  a.noise_scale = opt->lambda_eps * opt->lr[0];
  a.noise_pow = (float)(4.0 * exp((double)opt->noise_b));
  return cuda_status(launch_adam(n_lobes, planes, grad, adam_m, adam_v, eta, n, pitch, a, reg_loss,
                                 (cudaStream_t)stream));
}

size_t beta_relocate_workspace_bytes(int32_t n) { return n > 0 ? reloc_ws_bytes(n) : 0; }

int beta_relocate(int32_t n, int32_t pitch, int32_t n_lobes, float* planes, float* adam_m,
                  float* adam_v, const uint32_t* rnd, float min_opacity, void* ws, size_t ws_bytes,
                  int32_t* src_out, int32_t* d_count, beta_stream_t stream) {
  if (n < 0 || pitch < n || pitch % 4 != 0 || n_lobes < 0 || n_lobes > BETA_MAX_LOBES) return BETA_ERR_ARG;
  if (!planes || !rnd || !d_count || !(min_opacity >= 0.0f && min_opacity <= 1.0f)) return BETA_ERR_ARG;
  if (n > 0 && (!ws || ws_bytes < reloc_ws_bytes(n) || ((uintptr_t)ws & 255u) != 0)) return BETA_ERR_WORKSPACE;
  return cuda_status(launch_relocate(n, pitch, 15 + 6 * n_lobes, planes, adam_m, adam_v, rnd, min_opacity,
                                     ws, src_out, d_count, (cudaStream_t)stream));
}

size_t beta_dssim_workspace_bytes(const beta_camera* cams, int32_t n_views) {
  beta_opts o;
  beta_default_opts(&o);
  ViewTable vt;
  if (build_views(cams, n_views, &o, vt) != BETA_OK) return 0;
  return ssim_ws_bytes(vt);
}

int beta_l1_dssim_loss(const beta_camera* cams, int32_t n_views, const float* color,
                       const float* target, float lambda_ssim, float* loss, float* dL_dcolor,
                       void* ws, size_t ws_bytes, beta_stream_t stream) {
  if (!color || !target || !loss || !dL_dcolor || !(lambda_ssim >= 0.0f && lambda_ssim <= 1.0f))
    return BETA_ERR_ARG;
  beta_opts o;
  beta_default_opts(&o);
  ViewTable vt;
  int e;
  if ((e = build_views(cams, n_views, &o, vt)) != BETA_OK) return e;
  if (!ws || ws_bytes < ssim_ws_bytes(vt) || ((uintptr_t)ws & 255u) != 0) return BETA_ERR_WORKSPACE;
  return cuda_status(launch_ssim_loss(vt, color, target, lambda_ssim, loss, dL_dcolor, ws,
                                      (cudaStream_t)stream));
}

}  // extern "C"
