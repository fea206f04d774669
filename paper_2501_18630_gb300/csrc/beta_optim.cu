// beta_optim.cu -- the optimiser step that follows the rasterizer's backward
// in the training loop (Sec. 3.4 of arXiv 2501.18630, "Optimization" and the
// composite loss; hyperparameters from the appendix):
//
//   g   = dL/dp + d/dp [lambda_o sum |o| + lambda_Sigma sum_j sqrt(eig_j Sigma)]
//         (o = sigmoid(logit): lambda_o o (1 - o);  sqrt(eig_j Sigma) = s_j =
//         exp(log-scale_j): lambda_Sigma s_j)
//   Adam: m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
//         p -= lr_group (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
//   mu  += lambda_eps lr_mu B(o; b') Sigma eta,  B(o; b') = (1 - o)^(4 e^b'),
//         Sigma = R diag(s^2) R^T, eta ~ N(0, I_3) given by the caller.
//
// One thread per four primitives walks their parameter planes with 16-byte
// accesses (SoA: coalesced); the opacity, scales and rotation the noise and
// the regularisers need are read once, before the update.  The
// kernel is HBM-bound: per primitive it reads parameters, gradients and both
// moments and writes parameters and moments, 7 x 4 (15 + 6M) bytes, plus
// 12 bytes of noise samples.
#include <cuda_runtime.h>
#include <stdint.h>

#include "beta_internal.cuh"

namespace beta {

namespace {

// Per-primitive part of the step: the noise vector and the regulariser
// gradients' inputs, from the parameters before the step.
struct PrimPre {
  float o, omo;        // opacity and 1 - opacity
  float s[3];          // scales
  float noise[3];      // lambda_eps lr_mu B(o; b') Sigma eta
};

__device__ __forceinline__ PrimPre prim_pre(const float* __restrict__ planes, const float* __restrict__ eta,
                                            int pitch, int i, const AdamDev& a) {
  PrimPre r;
  const float logit = planes[(size_t)10 * pitch + i];
  r.o = 1.0f / (1.0f + expf(-logit));
  r.omo = 1.0f / (1.0f + expf(logit));
#pragma unroll
  for (int j = 0; j < 3; ++j) r.s[j] = expf(planes[(size_t)(3 + j) * pitch + i]);
  // rotation of the normalised quaternion (w, x, y, z)
  float qw = planes[(size_t)6 * pitch + i], qx = planes[(size_t)7 * pitch + i];
  float qy = planes[(size_t)8 * pitch + i], qz = planes[(size_t)9 * pitch + i];
  const float qn = rsqrtf(fmaf(qw, qw, fmaf(qx, qx, fmaf(qy, qy, qz * qz))));
  qw *= qn; qx *= qn; qy *= qn; qz *= qn;
  const float R[9] = {1.0f - 2.0f * (qy * qy + qz * qz), 2.0f * (qx * qy - qw * qz), 2.0f * (qx * qz + qw * qy),
                      2.0f * (qx * qy + qw * qz), 1.0f - 2.0f * (qx * qx + qz * qz), 2.0f * (qy * qz - qw * qx),
                      2.0f * (qx * qz - qw * qy), 2.0f * (qy * qz + qw * qx), 1.0f - 2.0f * (qx * qx + qy * qy)};
  // Sigma eta = R diag(s^2) R^T eta
  const float e0 = eta[i], e1 = eta[(size_t)pitch + i], e2 = eta[(size_t)2 * pitch + i];
  float t[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) t[j] = (R[0 * 3 + j] * e0 + R[1 * 3 + j] * e1 + R[2 * 3 + j] * e2) * (r.s[j] * r.s[j]);
  // B(o; b') = (1 - o)^(4 e^b'); 0 for an opaque primitive
  const float bk = r.omo > 0.0f ? exp2f(a.noise_pow * log2f(r.omo)) : 0.0f;
  const float nscale = a.noise_scale * bk;
#pragma unroll
  for (int q = 0; q < 3; ++q) r.noise[q] = nscale * (R[q * 3 + 0] * t[0] + R[q * 3 + 1] * t[1] + R[q * 3 + 2] * t[2]);
  return r;
}

// learning-rate group of parameter plane k
__device__ __forceinline__ int plane_group(int k) {
  if (k < 3) return 0;
  if (k < 6) return 1;
  if (k < 10) return 2;
  if (k < 15) return k == 10 ? 3 : (k == 11 ? 4 : 5);
  const int l = (k - 15) % 6;
  return l < 2 ? 6 : (l == 2 ? 7 : 8);
}

// element j (runtime, 0..2) of a three-vector, by selects: registers only
__device__ __forceinline__ float pick3(const float (&x)[3], int j) {
  return j == 0 ? x[0] : (j == 1 ? x[1] : x[2]);
}

// learning rate of plane k (constant indices only, so the parameter block
// stays in the constant bank)
__device__ __forceinline__ float group_lr(const AdamDev& a, int k) {
  const int g = plane_group(k);
  float lr = a.lr[0];
#pragma unroll
  for (int j = 1; j < 9; ++j)
    if (g == j) lr = a.lr[j];
  return lr;
}

// Adam update of one value (the gradient already includes the regularisers)
__device__ __forceinline__ void adam1(float& p, float& m, float& v, float g, float lr, const AdamDev& a) {
  m = fmaf(a.beta1, m, (1.0f - a.beta1) * g);
  v = fmaf(a.beta2, v, (1.0f - a.beta2) * g * g);
  p -= lr * (m * a.inv_c1) / (sqrtf(v * a.inv_c2) + a.eps);
}

// Thread t updates primitives 4t .. 4t+3 with 16-byte loads and stores (the
// plane pitch is a multiple of 4), so each thread keeps four times the bytes
// in flight of a one-primitive thread; a group running past n takes the
// scalar path so that padding columns are never written.
template <int M>
__global__ void __launch_bounds__(256, 4) k_adam(float* __restrict__ planes, const float* __restrict__ grad,
                                              float* __restrict__ adam_m, float* __restrict__ adam_v,
                                              const float* __restrict__ eta, int n, int pitch, AdamDev a,
                                              double* __restrict__ reg) {
  constexpr int NP = 15 + 6 * M;
  __shared__ double s_red[2][8];
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  // regulariser sums in fp32 within a warp, FP64 across the warps
  float f_o = 0.0f, f_s = 0.0f;
  if (i0 < n) {
    const int cnt = min(4, n - i0);
    PrimPre pre[4];
#pragma unroll
    for (int l = 0; l < 4; ++l)
      if (l < cnt) {
        pre[l] = prim_pre(planes, eta, pitch, i0 + l, a);
        f_o += a.lambda_o * pre[l].o;
        f_s += a.lambda_sigma * (pre[l].s[0] + pre[l].s[1] + pre[l].s[2]);
      }
    if (cnt == 4) {
#pragma unroll 2
      for (int k = 0; k < NP; ++k) {
        const size_t at = (size_t)k * pitch + i0;
        float4 p4 = *reinterpret_cast<const float4*>(planes + at);
        const float4 g4 = *reinterpret_cast<const float4*>(grad + at);
        float4 m4 = *reinterpret_cast<const float4*>(adam_m + at);
        float4 v4 = *reinterpret_cast<const float4*>(adam_v + at);
        float* pp = &p4.x;
        float* mm = &m4.x;
        float* vv = &v4.x;
        const float* gg = &g4.x;
        const float lr = group_lr(a, k);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          float g = gg[l];
          if (k == 10) g += a.lambda_o * pre[l].o * pre[l].omo;
          if (k >= 3 && k < 6) g += a.lambda_sigma * pick3(pre[l].s, k - 3);
          adam1(pp[l], mm[l], vv[l], g, lr, a);
          if (k < 3) pp[l] += pick3(pre[l].noise, k);
        }
        *reinterpret_cast<float4*>(planes + at) = p4;
        *reinterpret_cast<float4*>(adam_m + at) = m4;
        *reinterpret_cast<float4*>(adam_v + at) = v4;
      }
    } else {
      for (int k = 0; k < NP; ++k) {
        const float lr = group_lr(a, k);
#pragma unroll
        for (int l = 0; l < 4; ++l) {
          if (l >= cnt) break;
          const size_t at = (size_t)k * pitch + i0 + l;
          float p = planes[at], m = adam_m[at], v = adam_v[at], g = grad[at];
          if (k == 10) g += a.lambda_o * pre[l].o * pre[l].omo;
          if (k >= 3 && k < 6) g += a.lambda_sigma * pick3(pre[l].s, k - 3);
          adam1(p, m, v, g, lr, a);
          if (k < 3) p += pick3(pre[l].noise, k);
          planes[at] = p;
          adam_m[at] = m;
          adam_v[at] = v;
        }
      }
    }
  }
  if (reg) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      f_o += __shfl_xor_sync(0xffffffffu, f_o, off);
      f_s += __shfl_xor_sync(0xffffffffu, f_s, off);
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
      s_red[0][warp] = f_o;
      s_red[1][warp] = f_s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double so = 0.0, ss = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        so += s_red[0][w];
        ss += s_red[1][w];
      }
      atomicAdd(&reg[0], so);
      atomicAdd(&reg[1], ss);
    }
  }
}

template <int M>
cudaError_t launch_m(float* planes, const float* grad, float* m, float* v, const float* eta, int n,
                     int pitch, const AdamDev& a, double* reg, cudaStream_t s) {
  const int grid = ((n + 3) / 4 + 255) / 256;
  if (grid < 1) return cudaSuccess;
  k_adam<M><<<grid, 256, 0, s>>>(planes, grad, m, v, eta, n, pitch, a, reg);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_adam(int n_lobes, float* planes, const float* grad, float* m, float* v,
                        const float* eta, int n, int pitch, const AdamDev& a, double* reg,
                        cudaStream_t s) {
#define BETA_ADAM_M(MM) launch_m<MM>(planes, grad, m, v, eta, n, pitch, a, reg, s)
  BETA_DISPATCH_M(n_lobes, BETA_ADAM_M)
#undef BETA_ADAM_M
}


// ---------------------------------------------------------------------------
// Relocation of dead primitives (Sec. 3.4 "Densification", Eq. eq:densify).
// A primitive whose opacity is below min_opacity is dead and is respawned as
// a copy of a live primitive drawn with probability proportional to opacity
// (one draw per dead primitive, with replacement); a source that ends with N
// copies in all gets o' = 1 - (1 - o)^(1/N) on every copy, its other
// parameters unchanged, and the copies' moments are reset.
//
// The decisions are integers computed from a fixed fp32 opacity rule
// (o = 1 / (1 + rule_exp(-clamp(logit, -80, 80))), every operation rounded
// to nearest): dead = o < min_opacity, weight = floor(o 2^24) for live
// primitives, W = inclusive 64-bit prefix sums, and the caller's 32-bit
// random word r of a dead primitive picks t = floor(r W_total / 2^32), the
// source being the first i with W_i > t.
//
//   k_reloc_weights  weights (bit 31: dead) and per-block sums
//   k_reloc_scan     exclusive scan of the block sums (one CTA)
//   k_reloc_cdf      per-primitive inclusive prefix W
//   k_reloc_sample   binary search per dead primitive, copy counts
//   k_reloc_opacity  new opacity logit of every source
//   k_reloc_copy     the copies (after the sources' new logits)
// ---------------------------------------------------------------------------
namespace {

constexpr uint32_t kDeadBit = 0x80000000u;

__device__ __forceinline__ float rule_opacity(float x) {
  if (!(x >= -80.0f)) x = -80.0f;
  if (x > 80.0f) x = 80.0f;
  const float e = rule_exp(-x);
  return __fdiv_rn(1.0f, __fadd_rn(1.0f, e));
}

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long x, unsigned long long* s_w) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (lane == 0) s_w[warp] = x;
  __syncthreads();
  unsigned long long t = 0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += s_w[w];
  __syncthreads();
  return t;
}

__global__ void __launch_bounds__(256) k_reloc_weights(const float* __restrict__ planes, int n, int pitch,
                                                       float min_opacity, uint32_t* __restrict__ w,
                                                       unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long s_w[8];
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t wi = 0;
  if (i < n) {
    const float o = rule_opacity(planes[(size_t)10 * pitch + i]);
    wi = o < min_opacity ? kDeadBit : (uint32_t)__fmul_rn(o, 16777216.0f);
    w[i] = wi;
  }
  const unsigned long long t = block_sum_u64(wi & ~kDeadBit, s_w);
  if (threadIdx.x == 0) bsum[blockIdx.x] = t;
}

__global__ void __launch_bounds__(1024) k_reloc_scan(unsigned long long* __restrict__ bsum, int nb,
                                                     unsigned long long* __restrict__ total) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < nb; c0 += 1024) {
    const int i = c0 + threadIdx.x;
    const unsigned long long x = i < nb ? bsum[i] : 0ull;
    unsigned long long inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += y;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    unsigned long long pre = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < warp) pre += s_w[w];
      tot += s_w[w];
    }
    const unsigned long long carry = s_carry;
    if (i < nb) bsum[i] = carry + pre + inc - x;   // exclusive block offsets, in place
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = s_carry;
}

__global__ void __launch_bounds__(256) k_reloc_cdf(const uint32_t* __restrict__ w, int n,
                                                   const unsigned long long* __restrict__ boff,
                                                   unsigned long long* __restrict__ cdf) {
  __shared__ unsigned long long s_w[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned long long x = i < n ? (unsigned long long)(w[i] & ~kDeadBit) : 0ull;
  unsigned long long inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) s_w[warp] = inc;
  __syncthreads();
  unsigned long long pre = 0;
  for (int ww = 0; ww < warp; ++ww) pre += s_w[ww];
  if (i < n) cdf[i] = boff[blockIdx.x] + pre + inc;
}

__global__ void __launch_bounds__(256) k_reloc_sample(const uint32_t* __restrict__ w, int n,
                                                      const unsigned long long* __restrict__ cdf,
                                                      const unsigned long long* __restrict__ total,
                                                      const uint32_t* __restrict__ rnd,
                                                      int32_t* __restrict__ src, uint32_t* __restrict__ copies,
                                                      int32_t* __restrict__ d_count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long T = *total;
  int32_t s = -1;
  if ((w[i] & kDeadBit) && T > 0) {
    // t = floor(r T / 2^32), exactly: T = hi 2^32 + lo
    const unsigned long long r = rnd[i];
    const unsigned long long t = r * (T >> 32) + ((r * (T & 0xffffffffull)) >> 32);
    int lo = 0, hi = n - 1;                      // first index with cdf > t
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cdf[mid] > t) hi = mid; else lo = mid + 1;
    }
    s = lo;
    atomicAdd(&copies[s], 1u);
    atomicAdd(d_count, 1);
  }
  src[i] = s;
}

__global__ void __launch_bounds__(256) k_reloc_opacity(float* __restrict__ planes, int n, int pitch,
                                                       const uint32_t* __restrict__ copies) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || copies[i] == 0u) return;
  const float inv_n = 1.0f / (float)(copies[i] + 1u);
  float* lp = planes + (size_t)10 * pitch + i;
  // -log(1 - o) = softplus(logit), from the logit (1 - o by subtraction loses
  // the digits of an opacity near 1); q = -log(1 - o') = softplus / N
  const float x = *lp;
  const float q = (x > 0.0f ? x + log1pf(expf(-x)) : log1pf(expf(x))) * inv_n;
  const float o_new = -expm1f(-q);                       // 1 - (1 - o)^(1/N)
  *lp = logf(o_new) + q;                                 // log o' - log(1 - o')
}

__global__ void __launch_bounds__(256) k_reloc_copy(float* __restrict__ planes, float* __restrict__ m,
                                                    float* __restrict__ v, int n, int pitch, int np,
                                                    const int32_t* __restrict__ src) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = src[i];
  if (s < 0) return;
  for (int k = 0; k < np; ++k) {
    const size_t at = (size_t)k * pitch;
    planes[at + i] = planes[at + s];
    if (m) m[at + i] = 0.0f;
    if (v) v[at + i] = 0.0f;
  }
}

}  // namespace

// workspace carve-up: weights u32[n], cdf u64[n], block sums u64[nb], total
// u64, copies u32[n], sources i32[n] (256-byte aligned pieces)
static size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

size_t reloc_ws_bytes(int n) {
  const size_t nb = (size_t)(n + 255) / 256;
  return al256((size_t)n * 4) + al256((size_t)n * 8) + al256(nb * 8) + al256(8) + al256((size_t)n * 4) +
         al256((size_t)n * 4);
}

cudaError_t launch_relocate(int n, int pitch, int n_planes, float* planes, float* m, float* v,
                            const uint32_t* rnd, float min_opacity, void* ws, int32_t* src_out,
                            int32_t* d_count, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int nb = (n + 255) / 256;
  char* p = (char*)ws;
  uint32_t* w = (uint32_t*)p;                   p += al256((size_t)n * 4);
  unsigned long long* cdf = (unsigned long long*)p; p += al256((size_t)n * 8);
  unsigned long long* bsum = (unsigned long long*)p; p += al256((size_t)nb * 8);
  unsigned long long* total = (unsigned long long*)p; p += al256(8);
  uint32_t* copies = (uint32_t*)p;              p += al256((size_t)n * 4);
  int32_t* src = src_out ? src_out : (int32_t*)p;
  cudaError_t e;
  if ((e = cudaMemsetAsync(copies, 0, (size_t)n * 4, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(d_count, 0, 4, s)) != cudaSuccess) return e;
  k_reloc_weights<<<nb, 256, 0, s>>>(planes, n, pitch, min_opacity, w, bsum);
  k_reloc_scan<<<1, 1024, 0, s>>>(bsum, nb, total);
  k_reloc_cdf<<<nb, 256, 0, s>>>(w, n, bsum, cdf);
  k_reloc_sample<<<nb, 256, 0, s>>>(w, n, cdf, total, rnd, src, copies, d_count);
  k_reloc_opacity<<<nb, 256, 0, s>>>(planes, n, pitch, copies);
  k_reloc_copy<<<nb, 256, 0, s>>>(planes, m, v, n, pitch, n_planes, src);
  return cudaGetLastError();
}

}  // namespace beta
