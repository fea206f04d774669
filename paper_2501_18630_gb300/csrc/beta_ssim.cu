// beta_ssim.cu -- the image side of the composite loss with the DSSIM term
// (Sec. 3.4 of arXiv 2501.18630; lambda_SSIM = 0.2 in the appendix):
//
//   loss_v = (1 - lambda) mean|x - y| + lambda (1 - mean SSIM(x, y))
//
// per view v (colour x, target y, means over its 3 H W values), SSIM from
// Gaussian-weighted local statistics (11 taps, sigma 1.5, separable, zero
// outside the image; C1 = 0.01^2, C2 = 0.03^2):
//   mu = G * x,  sigma_x^2 = G * x^2 - mu_x^2,  sigma_xy = G * x y - mu_x mu_y,
//   S = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(sigma_x^2 + sigma_y^2 + C2)).
// Its gradient: with A1, A2, B1, B2 the four factors of S and d = 1/(B1 B2),
// S depends on x through (mu_x, G * x^2, G * x y):
//   a = dS/dmu_x = 2 mu_y A2 d - 2 mu_x S / B1 + 2 mu_x S / B2 - 2 mu_y A1 d
//   b = 2 dS/dG*x^2 = -2 S / B2,   c = dS/dG*xy = 2 A1 d
//   dL/dx = (1 - lambda) sign(x - y) / N - lambda / N (G*a + x G*b + y G*c).
//
// k_ssim_stats: one CTA per 32 x 32 pixel tile of one channel: x and y over
//   the tile and a 5-pixel halo in shared memory, the
//   horizontal and vertical 11-tap passes with each thread sliding a register
//   window over 4 outputs (one shared-memory load per input instead of one per
//   tap), then S, (a, b, c) to the workspace and the tile's sums of S and
//   |x - y| as per-block partials.
// k_ssim_grad:  the same tiling over (a, b, c): blur them and form dL/dx.
// k_ssim_loss:  per view, the sum of its blocks' partials (fixed order: the
//   loss is deterministic) and the loss.
// HBM traffic per channel-pixel: x, y read twice, (a, b, c) written and read
// once, dL/dx written: 44 bytes.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "beta_internal.cuh"

namespace beta {

namespace {

constexpr int kTX = 32, kTY = 32, kR = 5, kWin = 2 * kR + 1;
constexpr int kRun = 4;   // outputs per thread in each filter pass (sliding register window)
constexpr int kHX = kTX + 2 * kR, kHY = kTY + 2 * kR;
// row stride of the staged halo tiles: 45 = 1 (mod 4), so the four rows a
// warp reads in the horizontal pass (8 lanes each, 4 columns apart) fall in
// distinct banks
constexpr int kSX = 45;
// row stride of the horizontal-pass results: 33, so the same pass's stores
// (rows apart by one, 4 columns apart) fall in distinct banks
constexpr int kSH = kTX + 1;
constexpr float kC1 = 1e-4f, kC2 = 9e-4f;

// normalised Gaussian taps (sigma 1.5), computed by the host launcher and
// passed by value (kernel parameter space)
struct SsimWin {
  float g[kWin];
};

// view of an SSIM block (the per-view first block rides in ViewDev::pad0) and
// the channel and tile of the block inside the view
struct SsimBlock {
  int v, ch, x0, y0, W, H;
};

__device__ __forceinline__ SsimBlock ssim_block(const ViewTable& vt, int b) {
  int lo = 0, hi = vt.n_views - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (vt.v[mid].pad0 <= b) lo = mid; else hi = mid - 1;
  }
  SsimBlock r;
  r.v = lo;
  r.W = vt.v[lo].width;
  r.H = vt.v[lo].height;
  const int ntx = (r.W + kTX - 1) / kTX, nty = (r.H + kTY - 1) / kTY;
  int k = b - vt.v[lo].pad0;
  r.ch = k / (ntx * nty);
  k -= r.ch * ntx * nty;
  r.y0 = (k / ntx) * kTY;
  r.x0 = (k % ntx) * kTX;
  return r;
}

// Block sum (valid in thread 0): warp sums in fp32, the warps' sums in FP64
// (GB300's FP64 pipe is narrow: no per-thread FP64 arithmetic).
__device__ __forceinline__ double block_sum_d(float x, double* s_w) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = (double)x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
  return t;
}

// Horizontal pass over a staged (kHY x kHX) tile: row r, columns c0 .. c0 +
// kRun - 1 of the output, from a register window of kRun + 2 kR inputs.
// PRODUCTS: the sources are x and y, and the five filtered quantities are
// x, y, x^2, y^2, x y (formed in registers).
template <int Q, bool PRODUCTS>
__device__ __forceinline__ void hpass_run(const float (*src)[kHY][kSX], const SsimWin& win, int r, int c0,
                                          float (&out)[Q][kRun]) {
#pragma unroll
  for (int q = 0; q < Q; ++q)
#pragma unroll
    for (int j = 0; j < kRun; ++j) out[q][j] = 0.0f;
#pragma unroll
  for (int t = 0; t < kRun + 2 * kR; ++t) {
    float v[Q];
    if (PRODUCTS) {
      const float xv = src[0][r][c0 + t], yv = src[1][r][c0 + t];
      v[0] = xv;
      v[1] = yv;
      v[2] = xv * xv;
      v[3] = yv * yv;
      v[4] = xv * yv;
    } else {
#pragma unroll
      for (int q = 0; q < Q; ++q) v[q] = src[q][r][c0 + t];
    }
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
      const int k = t - j;                 // tap of input t for output j
      if (k >= 0 && k < kWin) {
#pragma unroll
        for (int q = 0; q < Q; ++q) out[q][j] = fmaf(win.g[k], v[q], out[q][j]);
      }
    }
  }
}

__global__ void __launch_bounds__(256) k_ssim_stats(ViewTable vt, SsimWin win, const float* __restrict__ color,
                                                    const float* __restrict__ target,
                                                    float* __restrict__ abc, int64_t plane,
                                                    double* __restrict__ acc) {
  __shared__ float s_in[2][kHY][kSX];     // x, y over the tile and its halo
  __shared__ float s_h[5][kHY][kSH];      // their horizontal pass
  __shared__ double s_w[8];
  const SsimBlock B = ssim_block(vt, blockIdx.x);
  const int64_t HW = (int64_t)B.W * B.H;
  const int64_t base = 3 * vt.v[B.v].pix_off + B.ch * HW;
  const float* xs = color + base;
  const float* ys = target + base;
  {
    constexpr int kLd = (kHY * kHX + 255) / 256;
    float lx[kLd], ly[kLd];
#pragma unroll
    for (int i = 0; i < kLd; ++i) {
      const int k = threadIdx.x + i * 256;
      const int r = k / kHX, c = k - r * kHX;
      const int gy = B.y0 - kR + r, gx = B.x0 - kR + c;
      const bool in = k < kHY * kHX && gx >= 0 && gx < B.W && gy >= 0 && gy < B.H;
      lx[i] = in ? xs[(int64_t)gy * B.W + gx] : 0.0f;
      ly[i] = in ? ys[(int64_t)gy * B.W + gx] : 0.0f;
    }
#pragma unroll
    for (int i = 0; i < kLd; ++i) {
      const int k = threadIdx.x + i * 256;
      if (k < kHY * kHX) {
        const int r = k / kHX, c = k - r * kHX;
        s_in[0][r][c] = lx[i];
        s_in[1][r][c] = ly[i];
      }
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kHY * (kTX / kRun); k += blockDim.x) {
    const int r = k / (kTX / kRun), c0 = (k - r * (kTX / kRun)) * kRun;
    float h[5][kRun];
    hpass_run<5, true>(s_in, win, r, c0, h);
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int j = 0; j < kRun; ++j) s_h[q][r][c0 + j] = h[q][j];
  }
  __syncthreads();
  // vertical pass: column c, rows r0 .. r0 + kRun - 1 from a register window
  // per-thread sums of 4 values in fp32 (GB300's FP64 rate is a small fraction
  // of FP32); the block and view sums are FP64
  float sum_s = 0.0f, sum_l1 = 0.0f;
  {
    const int c = threadIdx.x % kTX, r0 = (threadIdx.x / kTX) * kRun;
    float m[5][kRun];
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
      for (int j = 0; j < kRun; ++j) m[q][j] = 0.0f;
#pragma unroll
    for (int t = 0; t < kRun + 2 * kR; ++t) {
      float v[5];
#pragma unroll
      for (int q = 0; q < 5; ++q) v[q] = s_h[q][r0 + t][c];
#pragma unroll
      for (int j = 0; j < kRun; ++j) {
        const int k = t - j;
        if (k >= 0 && k < kWin) {
#pragma unroll
          for (int q = 0; q < 5; ++q) m[q][j] = fmaf(win.g[k], v[q], m[q][j]);
        }
      }
    }
    const int gx = B.x0 + c;
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
      const int gy = B.y0 + r0 + j;
      if (gx >= B.W || gy >= B.H) continue;
      const float mx = m[0][j], my = m[1][j];
      const float sxx = m[2][j] - mx * mx, syy = m[3][j] - my * my, sxy = m[4][j] - mx * my;
      const float A1 = 2.0f * mx * my + kC1, A2 = 2.0f * sxy + kC2;
      const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
      const float iB1 = __frcp_rn(B1), iB2 = __frcp_rn(B2);
      const float d = iB1 * iB2;
      const float S = A1 * A2 * d;
      const float a = 2.0f * my * A2 * d - 2.0f * mx * S * iB1 + 2.0f * mx * S * iB2 - 2.0f * my * A1 * d;
      const int64_t at = base + (int64_t)gy * B.W + gx;
      abc[at] = a;
      abc[plane + at] = -2.0f * S * iB2;
      abc[2 * plane + at] = 2.0f * A1 * d;
      sum_s += S;
      sum_l1 += fabsf(s_in[0][r0 + j + kR][c + kR] - s_in[1][r0 + j + kR][c + kR]);
    }
  }
  const double ts = block_sum_d(sum_s, s_w);
  __syncthreads();
  const double tl = block_sum_d(sum_l1, s_w);
  if (threadIdx.x == 0) {   // per-block partial sums, reduced per view by k_ssim_loss
    acc[2 * blockIdx.x] = ts;
    acc[2 * blockIdx.x + 1] = tl;
  }
}

__global__ void __launch_bounds__(256) k_ssim_grad(ViewTable vt, SsimWin win, const float* __restrict__ color,
                                                   const float* __restrict__ target,
                                                   const float* __restrict__ abc, int64_t plane, float lambda,
                                                   float* __restrict__ dLdC) {
  __shared__ float s_m[3][kHY][kSX];
  __shared__ float s_h[3][kHY][kSH];
  const SsimBlock B = ssim_block(vt, blockIdx.x);
  const int64_t HW = (int64_t)B.W * B.H;
  const int64_t base = 3 * vt.v[B.v].pix_off + B.ch * HW;
  // all of a thread's halo loads are issued before any store (memory-level
  // parallelism: the loads are the kernel's latency)
  constexpr int kLd = (kHY * kHX + 255) / 256;
  float ld[kLd][3];
#pragma unroll
  for (int i = 0; i < kLd; ++i) {
    const int k = threadIdx.x + i * 256;
    const int r = k / kHX, c = k - r * kHX;
    const int gy = B.y0 - kR + r, gx = B.x0 - kR + c;
    const bool in = k < kHY * kHX && gx >= 0 && gx < B.W && gy >= 0 && gy < B.H;
    const int64_t at = base + (int64_t)gy * B.W + gx;
#pragma unroll
    for (int q = 0; q < 3; ++q) ld[i][q] = in ? abc[q * plane + at] : 0.0f;
  }
#pragma unroll
  for (int i = 0; i < kLd; ++i) {
    const int k = threadIdx.x + i * 256;
    if (k < kHY * kHX) {
      const int r = k / kHX, c = k - r * kHX;
#pragma unroll
      for (int q = 0; q < 3; ++q) s_m[q][r][c] = ld[i][q];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kHY * (kTX / kRun); k += blockDim.x) {
    const int r = k / (kTX / kRun), c0 = (k - r * (kTX / kRun)) * kRun;
    float h[3][kRun];
    hpass_run<3, false>(s_m, win, r, c0, h);
#pragma unroll
    for (int q = 0; q < 3; ++q)
#pragma unroll
      for (int j = 0; j < kRun; ++j) s_h[q][r][c0 + j] = h[q][j];
  }
  __syncthreads();
  const float inv_n = 1.0f / (3.0f * (float)HW);
  const int c = threadIdx.x % kTX, r0 = (threadIdx.x / kTX) * kRun;
  float m[3][kRun];
#pragma unroll
  for (int q = 0; q < 3; ++q)
#pragma unroll
    for (int j = 0; j < kRun; ++j) m[q][j] = 0.0f;
#pragma unroll
  for (int t = 0; t < kRun + 2 * kR; ++t) {
    float v[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) v[q] = s_h[q][r0 + t][c];
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
      const int k = t - j;
      if (k >= 0 && k < kWin) {
#pragma unroll
        for (int q = 0; q < 3; ++q) m[q][j] = fmaf(win.g[k], v[q], m[q][j]);
      }
    }
  }
  const int gx = B.x0 + c;
#pragma unroll
  for (int j = 0; j < kRun; ++j) {
    const int gy = B.y0 + r0 + j;
    if (gx >= B.W || gy >= B.H) continue;
    const int64_t at = base + (int64_t)gy * B.W + gx;
    const float xv = color[at], yv = target[at];
    const float dif = xv - yv;
    const float sgn = dif > 0.0f ? 1.0f : (dif < 0.0f ? -1.0f : 0.0f);
    const float dS = m[0][j] + xv * m[1][j] + yv * m[2][j];
    dLdC[at] = inv_n * ((1.0f - lambda) * sgn - lambda * dS);
  }
}

// per view: the sums of its blocks' partials (fixed order), then the loss
__global__ void __launch_bounds__(256) k_ssim_loss(ViewTable vt, const double* __restrict__ acc, int nb,
                                                   float lambda, float* __restrict__ loss) {
  const int v = blockIdx.x;
  const int b0 = vt.v[v].pad0, b1 = v + 1 < vt.n_views ? vt.v[v + 1].pad0 : nb;
  double ss = 0.0, sl = 0.0;
  for (int b = b0 + threadIdx.x; b < b1; b += blockDim.x) {
    ss += acc[2 * b];
    sl += acc[2 * b + 1];
  }
  // one CTA per view: FP64 throughout (a few thousand values)
  __shared__ double s_a[256], s_b[256];
  s_a[threadIdx.x] = ss;
  s_b[threadIdx.x] = sl;
  __syncthreads();
  double ts = 0.0, tl = 0.0;
  if (threadIdx.x == 0)
    for (int t = 0; t < (int)blockDim.x; ++t) {
      ts += s_a[t];
      tl += s_b[t];
    }
  if (threadIdx.x == 0) {
    const double n = 3.0 * (double)vt.v[v].width * vt.v[v].height;
    loss[v] = (float)((1.0 - lambda) * tl / n + lambda * (1.0 - ts / n));
  }
}

int ssim_blocks(ViewTable& vt) {
  int b = 0;
  for (int v = 0; v < vt.n_views; ++v) {
    vt.v[v].pad0 = b;
    const int ntx = (vt.v[v].width + kTX - 1) / kTX, nty = (vt.v[v].height + kTY - 1) / kTY;
    b += 3 * ntx * nty;
  }
  return b;
}

}  // namespace

size_t ssim_ws_bytes(const ViewTable& vt) {
  // (a, b, c) planes over every view's pixels and channels, then two partial sums per block
  ViewTable t = vt;
  return ((size_t)9 * vt.total_pixels * sizeof(float) + 255) / 256 * 256 + (size_t)2 * ssim_blocks(t) * sizeof(double);
}

cudaError_t launch_ssim_loss(const ViewTable& vt_in, const float* color, const float* target, float lambda,
                             float* loss, float* dL_dcolor, void* ws, cudaStream_t s) {
  SsimWin win;
  {
    double sum = 0.0, gd[kWin];
    for (int t = 0; t < kWin; ++t) {
      const double k = t - kR;
      gd[t] = exp(-k * k / (2.0 * 1.5 * 1.5));
      sum += gd[t];
    }
    for (int t = 0; t < kWin; ++t) win.g[t] = (float)(gd[t] / sum);
  }
  ViewTable vt = vt_in;
  const int nb = ssim_blocks(vt);
  if (nb <= 0) return cudaSuccess;
  const int64_t plane = 3 * vt.total_pixels;
  float* abc = (float*)ws;
  double* acc = (double*)((char*)ws + ((size_t)9 * vt.total_pixels * sizeof(float) + 255) / 256 * 256);
  k_ssim_stats<<<nb, 256, 0, s>>>(vt, win, color, target, abc, plane, acc);
  k_ssim_grad<<<nb, 256, 0, s>>>(vt, win, color, target, abc, plane, lambda, dL_dcolor);
  k_ssim_loss<<<vt.n_views, 256, 0, s>>>(vt, acc, nb, lambda, loss);
  return cudaGetLastError();
}

}  // namespace beta
