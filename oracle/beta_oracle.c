/*
 * beta_oracle.c -- plain FP64 CPU reference of the Beta-splatting rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header or constant with the CUDA path.
 *
 * What it computes (Deformable Beta Splatting, arXiv 2501.18630):
 *   - Beta kernel B(x; b) = (1 - x)^beta, beta = 4 e^b              (Eq. 2, Eq. eq:beta)
 *   - primitive {mu, o, q, s, b, f}                                 (Sec. 3.2)
 *   - Sigma = R S S^T R^T, Sigma' = J W Sigma W^T J^T, centre mu'     (Sec. 3.2)
 *   - r_i(x)^2 = (x - mu')^T Sigma'^-1 (x - mu')                     (Sec. 3.2, Eq. r)
 *   - depth-sorted front-to-back compositing
 *       C(x) = sum_i c_i o_i B(r_i^2; b_i) prod_{j<i} (1 - o_j B(r_j^2; b_j))  (Sec. 3.2, Eq. C)
 *   - spherical-Beta colour c(V) = c0 + sum_m B(1 - R_m . V; b_m) c_m (Sec. 3.3)
 *
 * Readings where the paper is silent:
 *   raw parameters are log-scale, opacity logit and an unnormalised
 *   quaternion (w,x,y,z); the lobe direction is (sin t cos p, sin t sin p,
 *   cos t); the lobe term is 0 when R_m . V <= 0; V = normalize(mu - campos);
 *   alpha = min(alpha_max, o B); compositing stops before primitive k when
 *   T < t_eps; pixel (i, j) is sampled at (i + 1/2, j + 1/2); the depth
 *   order is the camera-space z of the centre, rounded to fp32 by the rule
 *   below, ties broken by primitive index.
 *
 * Two pieces are not the paper's mathematics but fixed rules of this
 * implementation, and both sides implement them from the same written rule:
 *   (D) the depth key: float bits of tz computed in fp32 as
 *       ((R20*x + R21*y) + R22*z) + t2, every operation rounded;
 *   (B1) the tile rectangle of a primitive, a conservative bound of its
 *       support ellipse evaluated by a fixed fp32 operation sequence.
 * The per-pixel renderer below does not use B1 at all.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fPIC -shared (see build.py).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  double R[9];  /* world -> camera rotation, row-major */
  double t[3];
  double fx, fy, cx, cy, near_plane;
  int32_t width, height;
  double bg[3];
} ocam;

typedef struct {
  double t_eps;      /* stop before primitive k when T < t_eps            */
  double alpha_max;  /* alpha = min(alpha_max, o B)                       */
  double blur_eps;   /* added to the diagonal of Sigma'                   */
  int32_t color_mode;/* 0: c0 + lobes, 1: c0 only, 2: lobes only          */
  int32_t n_threads;
  double b_lo, b_hi; /* geometry decomposition (Sec. 4.3): keep b_lo <= b < b_hi */
} oopts;

typedef struct {
  int32_t valid;
  uint32_t key;      /* rule D depth key                                  */
  double depth;      /* camera-space z of the centre (fp64)               */
  double mu2[2];     /* projected centre, pixels                          */
  double cov[3];     /* Sigma' = [[a, b], [b, c]] -> (a, b, c)            */
  double conic[3];   /* Sigma'^-1 -> (A, B, C)                            */
  double o, beta;
  double color[3];
} oprim;

/* ------------------------------------------------------------------------ */
/* rule D: the fp32 depth key                                               */
/* ------------------------------------------------------------------------ */

static float rule_tz(const ocam* cam, float x, float y, float z) {
  float r6 = (float)cam->R[6], r7 = (float)cam->R[7], r8 = (float)cam->R[8];
  float t2 = (float)cam->t[2];
  float a = r6 * x;
  float b = r7 * y;
  float c = r8 * z;
  float s = a + b;
  s = s + c;
  s = s + t2;
  return s;
}

static uint32_t float_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  return u;
}

/* ------------------------------------------------------------------------ */
/* per-primitive quantities in FP64 (Sec. 3.2, Sec. 3.3)                    */
/* ------------------------------------------------------------------------ */

static void quat_to_rot(const double q[4], double R[9]) {
  /* unit quaternion (w, x, y, z) -> rotation matrix, row-major */
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1.0 - 2.0 * (y * y + z * z);
  R[1] = 2.0 * (x * y - w * z);
  R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);
  R[4] = 1.0 - 2.0 * (x * x + z * z);
  R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);
  R[7] = 2.0 * (y * z + w * x);
  R[8] = 1.0 - 2.0 * (x * x + y * y);
}

void oracle_project_one(const double* planes, int32_t pitch, int32_t n_lobes, int32_t i,
                        const ocam* cam, const oopts* op, oprim* out) {
  memset(out, 0, sizeof(*out));
  int np = 15 + 6 * n_lobes;
  double p[15 + 6 * 8];
  for (int k = 0; k < np; ++k) {
    p[k] = planes[(size_t)k * pitch + i];
    if (!isfinite(p[k])) return; /* non-finite primitive: culled */
  }
  const double* mu = p + 0;
  const double* ls = p + 3;
  const double* q = p + 6;
  /* geometry decomposition by the Beta shape parameter (Sec. 4.3) */
  if (!(p[11] >= op->b_lo && p[11] < op->b_hi)) return;

  /* rule D key and the near-plane cull (on the fp32 centre) */
  float tzf = rule_tz(cam, (float)mu[0], (float)mu[1], (float)mu[2]);
  out->key = float_bits(tzf);
  if (!(tzf > (float)cam->near_plane)) return;

  double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  if (!(qn > 0.0)) return;
  double qh[4] = {q[0] / qn, q[1] / qn, q[2] / qn, q[3] / qn};
  double Rq[9];
  quat_to_rot(qh, Rq);
  double s[3] = {exp(ls[0]), exp(ls[1]), exp(ls[2])};

  /* Sigma = R S S^T R^T */
  double Sig[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double acc = 0.0;
      for (int k = 0; k < 3; ++k) acc += Rq[r * 3 + k] * s[k] * s[k] * Rq[c * 3 + k];
      Sig[r * 3 + c] = acc;
    }

  /* t = W mu + t_w */
  const double* W = cam->R;
  double t[3];
  for (int r = 0; r < 3; ++r)
    t[r] = W[r * 3 + 0] * mu[0] + W[r * 3 + 1] * mu[1] + W[r * 3 + 2] * mu[2] + cam->t[r];
  out->depth = t[2];

  /* J: Jacobian of the pinhole projection at t */
  double J[6] = {cam->fx / t[2], 0.0, -cam->fx * t[0] / (t[2] * t[2]),
                 0.0, cam->fy / t[2], -cam->fy * t[1] / (t[2] * t[2])};
  /* T = J W (2x3); Sigma' = T Sigma T^T */
  double T[6];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c)
      T[r * 3 + c] = J[r * 3 + 0] * W[0 * 3 + c] + J[r * 3 + 1] * W[1 * 3 + c] + J[r * 3 + 2] * W[2 * 3 + c];
  double TS[6];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 3; ++c)
      TS[r * 3 + c] = T[r * 3 + 0] * Sig[0 * 3 + c] + T[r * 3 + 1] * Sig[1 * 3 + c] + T[r * 3 + 2] * Sig[2 * 3 + c];
  double cov[4];
  for (int r = 0; r < 2; ++r)
    for (int c = 0; c < 2; ++c)
      cov[r * 2 + c] = TS[r * 3 + 0] * T[c * 3 + 0] + TS[r * 3 + 1] * T[c * 3 + 1] + TS[r * 3 + 2] * T[c * 3 + 2];
  double a = cov[0] + op->blur_eps, b = 0.5 * (cov[1] + cov[2]), c = cov[3] + op->blur_eps;
  double det = a * c - b * b;
  if (!(det > 0.0)) return;
  out->cov[0] = a;
  out->cov[1] = b;
  out->cov[2] = c;
  out->conic[0] = c / det;
  out->conic[1] = -b / det;
  out->conic[2] = a / det;

  out->mu2[0] = cam->fx * t[0] / t[2] + cam->cx;
  out->mu2[1] = cam->fy * t[1] / t[2] + cam->cy;
  out->o = 1.0 / (1.0 + exp(-p[10]));
  out->beta = 4.0 * exp(p[11]);

  /* spherical Beta colour, V = normalize(mu - campos), campos = -W^T t_w */
  double cp[3];
  for (int r = 0; r < 3; ++r)
    cp[r] = -(W[0 * 3 + r] * cam->t[0] + W[1 * 3 + r] * cam->t[1] + W[2 * 3 + r] * cam->t[2]);
  double V[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
  double vn = sqrt(V[0] * V[0] + V[1] * V[1] + V[2] * V[2]);
  for (int r = 0; r < 3; ++r) V[r] /= vn;
  double col[3] = {0.0, 0.0, 0.0};
  if (op->color_mode != 2)
    for (int ch = 0; ch < 3; ++ch) col[ch] = p[12 + ch];
  if (op->color_mode != 1) {
    for (int m = 0; m < n_lobes; ++m) {
      const double* L = p + 15 + 6 * m;
      double Rm[3] = {sin(L[0]) * cos(L[1]), sin(L[0]) * sin(L[1]), cos(L[0])};
      double dot = Rm[0] * V[0] + Rm[1] * V[1] + Rm[2] * V[2];
      if (dot > 0.0) {
        /* B(1 - R.V; b_m) = (R.V)^(4 e^{b_m}) on the kernel's domain */
        double w = pow(dot, 4.0 * exp(L[2]));
        for (int ch = 0; ch < 3; ++ch) col[ch] += w * L[3 + ch];
      }
    }
  }
  for (int ch = 0; ch < 3; ++ch) out->color[ch] = col[ch];
  out->valid = 1;
}

void oracle_project(const double* planes, int32_t n, int32_t pitch, int32_t n_lobes,
                    const ocam* cam, const oopts* op, oprim* out) {
  for (int32_t i = 0; i < n; ++i) oracle_project_one(planes, pitch, n_lobes, i, cam, op, out + i);
}

/* ------------------------------------------------------------------------ */
/* rendering: per pixel, every primitive, depth order (Eq. C)               */
/* ------------------------------------------------------------------------ */

typedef struct {
  uint32_t key;
  int32_t idx;
} okey;

static int okey_cmp(const void* a, const void* b) {
  const okey* x = (const okey*)a;
  const okey* y = (const okey*)b;
  if (x->key != y->key) return x->key < y->key ? -1 : 1;
  return (x->idx > y->idx) - (x->idx < y->idx);
}

typedef struct {
  const oprim* prims;
  const int32_t* order;
  int32_t n_order;
  const ocam* cam;
  const oopts* op;
  const int32_t* px;
  const int32_t* py;
  int32_t p0, p1;
  double* out_C;
  double* out_T;
  int32_t* out_last;
  int32_t* out_count;
} ojob;

static void render_pixel(const ojob* jb, int32_t k) {
  double X = jb->px[k] + 0.5, Y = jb->py[k] + 0.5;
  double T = 1.0, C[3] = {0.0, 0.0, 0.0};
  int32_t last = -1, count = 0;
  for (int32_t j = 0; j < jb->n_order; ++j) {
    if (T < jb->op->t_eps) break;
    const oprim* P = jb->prims + jb->order[j];
    double dx = X - P->mu2[0], dy = Y - P->mu2[1];
    double r2 = P->conic[0] * dx * dx + 2.0 * P->conic[1] * dx * dy + P->conic[2] * dy * dy;
    if (!(r2 < 1.0)) continue; /* outside the bounded support */
    double alpha = P->o * pow(1.0 - r2, P->beta);
    if (alpha > jb->op->alpha_max) alpha = jb->op->alpha_max;
    for (int ch = 0; ch < 3; ++ch) C[ch] += T * alpha * P->color[ch];
    T *= (1.0 - alpha);
    last = jb->order[j];
    ++count;
  }
  for (int ch = 0; ch < 3; ++ch) jb->out_C[(size_t)k * 3 + ch] = C[ch] + T * jb->cam->bg[ch];
  jb->out_T[k] = T;
  jb->out_last[k] = last;
  jb->out_count[k] = count;
}

static void* render_worker(void* arg) {
  ojob* jb = (ojob*)arg;
  for (int32_t k = jb->p0; k < jb->p1; ++k) render_pixel(jb, k);
  return NULL;
}

/* Renders npix pixels (px[k], py[k]).  out_C: npix x 3 (RGB, background
 * included), out_T: final transmittance, out_last: id of the last primitive
 * that contributed (-1 if none), out_count: number of contributors.
 * Returns the number of valid (not culled) primitives. */
int32_t oracle_render(const double* planes, int32_t n, int32_t pitch, int32_t n_lobes,
                      const ocam* cam, const oopts* op, const int32_t* px, const int32_t* py,
                      int32_t npix, double* out_C, double* out_T, int32_t* out_last,
                      int32_t* out_count) {
  oprim* prims = (oprim*)malloc(sizeof(oprim) * (size_t)(n > 0 ? n : 1));
  okey* keys = (okey*)malloc(sizeof(okey) * (size_t)(n > 0 ? n : 1));
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  oracle_project(planes, n, pitch, n_lobes, cam, op, prims);
  int32_t nv = 0;
  for (int32_t i = 0; i < n; ++i)
    if (prims[i].valid) {
      keys[nv].key = prims[i].key;
      keys[nv].idx = i;
      ++nv;
    }
  qsort(keys, (size_t)nv, sizeof(okey), okey_cmp);
  for (int32_t j = 0; j < nv; ++j) order[j] = keys[j].idx;

  int nt = op->n_threads > 0 ? op->n_threads : 1;
  if (nt > 256) nt = 256;
  if (nt > npix) nt = npix > 0 ? npix : 1;
  pthread_t th[256];
  ojob jobs[256];
  for (int t = 0; t < nt; ++t) {
    jobs[t] = (ojob){prims, order, nv, cam, op, px, py,
                     (int32_t)((int64_t)npix * t / nt), (int32_t)((int64_t)npix * (t + 1) / nt),
                     out_C, out_T, out_last, out_count};
  }
  if (nt == 1) {
    render_worker(&jobs[0]);
  } else {
    for (int t = 0; t < nt; ++t) pthread_create(&th[t], NULL, render_worker, &jobs[t]);
    for (int t = 0; t < nt; ++t) pthread_join(th[t], NULL);
  }
  free(prims);
  free(keys);
  free(order);
  return nv;
}

/* Per-pixel r^2 of one primitive (diagnostics for the tests). */
double oracle_r2(const oprim* P, double X, double Y) {
  double dx = X - P->mu2[0], dy = Y - P->mu2[1];
  return P->conic[0] * dx * dx + 2.0 * P->conic[1] * dx * dy + P->conic[2] * dy * dy;
}

/* ------------------------------------------------------------------------ */
/* rule B1: the tile rectangle, fp32, fixed operation order                 */
/* ------------------------------------------------------------------------ */

/* exp in fp32: n = rint(x log2 e); r = (x - n ln2_hi) - n ln2_lo;
 * degree-7 Taylor polynomial of e^r by Horner with fused multiply-adds
 * (Cody-Waite reduction); result = p * 2^n.  Defined for x in [-80, 80].
 * ln2_hi carries trailing zero bits so that n * ln2_hi is exact; the hi/lo
 * pair is the single-precision split of fdlibm's public expf. */
float oracle_rule_exp(float x) {
  const float LOG2E = 1.44269504f;
  const float LN2_HI = 0.693145751953125f;
  const float LN2_LO = 1.42860677e-06f;
  float tt = x * LOG2E;
  float n = rintf(tt);
  float nh = n * LN2_HI;
  float nl = n * LN2_LO;
  float r = x - nh;
  r = r - nl;
  float p = 1.98412698e-04f;      /* 1/7! */
  p = fmaf(p, r, 1.38888889e-03f); /* 1/6! */
  p = fmaf(p, r, 8.33333333e-03f); /* 1/5! */
  p = fmaf(p, r, 4.16666667e-02f); /* 1/4! */
  p = fmaf(p, r, 1.66666667e-01f); /* 1/3! */
  p = fmaf(p, r, 0.5f);
  p = fmaf(p, r, 1.0f);
  p = fmaf(p, r, 1.0f);
  int32_t e = (int32_t)n + 127;
  uint32_t bits = (uint32_t)e << 23;
  float scale;
  memcpy(&scale, &bits, 4);
  return p * scale;
}

/* Opacity by a fixed fp32 rule, for the relocation step's decisions (Sec. 3.4
 * Densification: dead primitives and sampling weights):
 * o = 1 / (1 + rule_exp(-x)), x = the logit clamped to [-80, 80] (NaN -> -80),
 * every operation rounded to nearest in float. */
void oracle_rule_opacity(const float* logit, int32_t n, float* o) {
  for (int32_t i = 0; i < n; ++i) {
    float x = logit[i];
    if (!(x >= -80.0f)) x = -80.0f;
    if (x > 80.0f) x = 80.0f;
    float e = oracle_rule_exp(-x);
    float d = 1.0f + e;
    o[i] = 1.0f / d;
  }
}

/* a*b - c*d with Kahan's fused multiply-add algorithm (one rounding error) */
static float rule_dop(float a, float b, float c, float d) {
  float w = c * d;
  float e = fmaf(-c, d, w);
  float f = fmaf(a, b, -w);
  return f + e;
}

/* Rule B2: which tiles of the rule B1 rectangle the support ellipse reaches
 * (Sec. 3.1 / Eq. 2: the Beta kernel is exactly zero outside r^2 < 1, so a
 * tile no pixel centre of which lies inside the support gets no pair).
 * For every tile row, the band of its pixel-centre rows (widened by PAD) is
 * cut with the ellipse of Sigma' inflated by INFL; the ellipse's x-range over
 * the band is the whole half-width when its rightmost (leftmost) point lies in
 * the band, else the boundary at the band end nearest that point; the columns
 * whose centres lie within that range widened by PAD give the row's tiles.
 * Sigma' = [[a, b], [b, c]] with a = sxx, c = syy (blur included),
 * b = M0 . M1 and det = |M0 x M1|^2 + blur (a + c - blur), minors by Kahan's
 * algorithm; at height y (from the centre) the boundary is
 *   x = (b / c) y +- sqrt(K2 (det / c) max(0, 1 - y^2 (1 / (K2 c)))),  K2 = INFL^2.
 * Every operation is fp32, rounded to nearest, in the order written.  The
 * rule applies to rectangles of at least 2 x 2 and at most 32 tiles (a
 * rectangle one tile wide or high loses a tile only where an image edge cuts
 * the ellipse); the others, and degenerate ellipses, keep every tile.
 * Returns the tiles as bit r w + q for tile (tx0 + q, ty0 + r) of a w x h
 * rectangle (w h <= 32), 0xFFFFFFFF for larger rectangles. */
static uint32_t rule_tiles(const float M0[3], const float M1[3], float sxx, float syy, float blur,
                           float pxc, float pyc, const int32_t rect[4], int32_t width, int32_t height,
                           int32_t tile_w, int32_t tile_h) {
  const int32_t w = rect[1] - rect[0] + 1, h = rect[3] - rect[2] + 1;
  if (w * h > 32) return 0xFFFFFFFFu;
  const uint32_t all = w * h == 32 ? 0xFFFFFFFFu : ((1u << (w * h)) - 1u);
  if (w < 2 || h < 2) return all;
  if (!(sxx > 0.0f && syy > 0.0f)) return all;
  const float INFL = 1.000244140625f; /* 1 + 2^-12 */
  const float PAD = 0.015625f;        /* 2^-6 pixel */
  float b = M0[0] * M1[0];
  b = b + M0[1] * M1[1];
  b = b + M0[2] * M1[2];
  float m01 = rule_dop(M0[0], M1[1], M0[1], M1[0]);
  float m02 = rule_dop(M0[0], M1[2], M0[2], M1[0]);
  float m12 = rule_dop(M0[1], M1[2], M0[2], M1[1]);
  float det = m01 * m01;
  det = det + m02 * m02;
  det = det + m12 * m12;
  det = det + blur * ((sxx + syy) - blur);
  float sa = sqrtf(sxx), sc = sqrtf(syy);
  float xfull = sa * INFL;
  float ytop = sc * INFL;
  float ystar = (b * INFL) / sa;
  float slope = b / syy;
  float K2 = INFL * INFL;
  float hh = (det / syy) * K2;
  float cc = syy * K2;
  float icc = 1.0f / cc;
  if (!(isfinite(ystar) && isfinite(slope) && isfinite(hh) && isfinite(icc) && cc > 0.0f)) return all;
  uint32_t mask = 0u;
  for (int32_t r = 0; r < h; ++r) {
    int32_t y0 = (rect[2] + r) * tile_h;
    int32_t y1 = y0 + tile_h - 1;
    if (y1 > height - 1) y1 = height - 1;
    float ya = (((float)y0 + 0.5f) - PAD) - pyc;
    float yb = (((float)y1 + 0.5f) + PAD) - pyc;
    if (ya < -ytop) ya = -ytop;
    if (yb > ytop) yb = ytop;
    if (!(ya <= yb)) continue;
    int in_r = (ya <= ystar) && (ystar <= yb);
    int in_l = (ya <= -ystar) && (-ystar <= yb);
    float yr = ystar < ya ? ya : yb;     /* band end nearest the rightmost point */
    float yl = -ystar < ya ? ya : yb;    /* band end nearest the leftmost point  */
    float xmax, xmin;
    if (in_r) {
      xmax = xfull;
    } else {
      float t = 1.0f - (yr * yr) * icc;
      if (t < 0.0f) t = 0.0f;
      xmax = slope * yr + sqrtf(hh * t);
    }
    if (in_l) {
      xmin = -xfull;
    } else {
      float t = 1.0f - (yl * yl) * icc;
      if (t < 0.0f) t = 0.0f;
      xmin = slope * yl - sqrtf(hh * t);
    }
    float lo = ((pxc + xmin) - PAD) - 0.5f;
    float hi = ((pxc + xmax) + PAD) - 0.5f;
    uint32_t rowbits;
    if (!(isfinite(lo) && isfinite(hi))) {
      rowbits = w == 32 ? 0xFFFFFFFFu : ((1u << w) - 1u);
    } else {
      float i0 = floorf(lo) + 1.0f, i1 = ceilf(hi) - 1.0f;
      if (i0 < 0.0f) i0 = 0.0f;
      if (i1 > (float)(width - 1)) i1 = (float)(width - 1);
      if (i0 > i1) continue;
      int32_t q0 = (int32_t)i0 / tile_w, q1 = (int32_t)i1 / tile_w;
      if (q0 < rect[0]) q0 = rect[0];
      if (q1 > rect[1]) q1 = rect[1];
      if (q0 > q1) continue;
      q0 -= rect[0];
      q1 -= rect[0];
      rowbits = ((2u << q1) - 1u) & ~((1u << q0) - 1u);
    }
    mask |= rowbits << (r * w);
  }
  return mask;
}

/* Tile rectangle of primitive i under rule B1.  rect = (tx0, tx1, ty0, ty1),
 * inclusive tile indices, tx0 > tx1 when the primitive touches no tile.
 * Returns 1 if the primitive is binned, 0 otherwise.  key receives the
 * rule D depth key, tiles (if not NULL) the rule B2 tiles of the rectangle. */
int32_t oracle_rule_rect_one(const float* planes, int32_t pitch, int32_t n_lobes, int32_t i,
                             const ocam* cam, float blur, float b_lo, float b_hi, int32_t tile_w,
                             int32_t tile_h, int32_t rect[4], uint32_t* key, uint32_t* tiles) {
  if (tiles) *tiles = 0u;
  rect[0] = 0;
  rect[1] = -1;
  rect[2] = 0;
  rect[3] = -1;
  int np = 15 + 6 * n_lobes;
  for (int k = 0; k < np; ++k)
    if (!isfinite(planes[(size_t)k * pitch + i])) {
      *key = 0xFFFFFFFFu;
      return 0;
    }
  {
    float bb = planes[11 * (size_t)pitch + i];
    if (!(bb >= b_lo && bb < b_hi)) return 0;
  }
  float mx = planes[0 * (size_t)pitch + i], my = planes[1 * (size_t)pitch + i], mz = planes[2 * (size_t)pitch + i];
  float W[9], tw[3];
  for (int k = 0; k < 9; ++k) W[k] = (float)cam->R[k];
  for (int k = 0; k < 3; ++k) tw[k] = (float)cam->t[k];
  float fx = (float)cam->fx, fy = (float)cam->fy, cx = (float)cam->cx, cy = (float)cam->cy;

  float tc[3];
  for (int r = 0; r < 3; ++r) {
    float a = W[r * 3 + 0] * mx;
    float b = W[r * 3 + 1] * my;
    float c = W[r * 3 + 2] * mz;
    float s = a + b;
    s = s + c;
    tc[r] = s + tw[r];
  }
  *key = float_bits(tc[2]);
  if (!(tc[2] > (float)cam->near_plane)) return 0;

  float s3[3];
  for (int k = 0; k < 3; ++k) {
    float l = planes[(size_t)(3 + k) * pitch + i];
    if (!(l >= -80.0f && l <= 80.0f)) return 0;
    s3[k] = oracle_rule_exp(l);
  }
  float qw = planes[6 * (size_t)pitch + i], qx = planes[7 * (size_t)pitch + i];
  float qy = planes[8 * (size_t)pitch + i], qz = planes[9 * (size_t)pitch + i];
  float qq = qw * qw;
  qq = qq + qx * qx;
  qq = qq + qy * qy;
  qq = qq + qz * qz;
  if (!(qq > 0.0f)) return 0;
  float rn = 1.0f / sqrtf(qq);
  float w = qw * rn, x = qx * rn, y = qy * rn, z = qz * rn;
  float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  float Rq[9];
  Rq[0] = 1.0f - 2.0f * (yy + zz);
  Rq[1] = 2.0f * (xy - wz);
  Rq[2] = 2.0f * (xz + wy);
  Rq[3] = 2.0f * (xy + wz);
  Rq[4] = 1.0f - 2.0f * (xx + zz);
  Rq[5] = 2.0f * (yz - wx);
  Rq[6] = 2.0f * (xz - wy);
  Rq[7] = 2.0f * (yz + wx);
  Rq[8] = 1.0f - 2.0f * (xx + yy);
  /* A = W Rq */
  float A[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      float a = W[r * 3 + 0] * Rq[0 * 3 + c];
      float b = W[r * 3 + 1] * Rq[1 * 3 + c];
      float d = W[r * 3 + 2] * Rq[2 * 3 + c];
      float s = a + b;
      A[r * 3 + c] = s + d;
    }
  float iz = 1.0f / tc[2];
  float j00 = fx * iz;
  float j11 = fy * iz;
  float j02 = -((j00 * tc[0]) * iz);
  float j12 = -((j11 * tc[1]) * iz);
  float M0[3], M1[3];
  for (int c = 0; c < 3; ++c) {
    float a = j00 * A[0 * 3 + c];
    float b = j02 * A[2 * 3 + c];
    M0[c] = (a + b) * s3[c];
    float d = j11 * A[1 * 3 + c];
    float e = j12 * A[2 * 3 + c];
    M1[c] = (d + e) * s3[c];
  }
  float sxx = M0[0] * M0[0];
  sxx = sxx + M0[1] * M0[1];
  sxx = sxx + M0[2] * M0[2];
  sxx = sxx + blur;
  float syy = M1[0] * M1[0];
  syy = syy + M1[1] * M1[1];
  syy = syy + M1[2] * M1[2];
  syy = syy + blur;
  const float INFL = 1.000244140625f; /* 1 + 2^-12 */
  const float PAD = 0.015625f;        /* 2^-6 pixel */
  float ex = sqrtf(sxx) * INFL;
  ex = ex + PAD;
  float ey = sqrtf(syy) * INFL;
  ey = ey + PAD;
  float pxc = j00 * tc[0];
  pxc = pxc + cx;
  float pyc = j11 * tc[1];
  pyc = pyc + cy;
  float lox = (pxc - ex) - 0.5f, hix = (pxc + ex) - 0.5f;
  float loy = (pyc - ey) - 0.5f, hiy = (pyc + ey) - 0.5f;
  if (!(isfinite(lox) && isfinite(hix) && isfinite(loy) && isfinite(hiy))) return 0;
  float i0 = floorf(lox) + 1.0f, i1 = ceilf(hix) - 1.0f;
  float j0 = floorf(loy) + 1.0f, j1 = ceilf(hiy) - 1.0f;
  if (i0 < 0.0f) i0 = 0.0f;
  if (j0 < 0.0f) j0 = 0.0f;
  if (i1 > (float)(cam->width - 1)) i1 = (float)(cam->width - 1);
  if (j1 > (float)(cam->height - 1)) j1 = (float)(cam->height - 1);
  if (i0 > i1 || j0 > j1) return 0;
  rect[0] = (int32_t)i0 / tile_w;
  rect[1] = (int32_t)i1 / tile_w;
  rect[2] = (int32_t)j0 / tile_h;
  rect[3] = (int32_t)j1 / tile_h;
  if (tiles)
    *tiles = rule_tiles(M0, M1, sxx, syy, blur, pxc, pyc, rect, cam->width, cam->height, tile_w, tile_h);
  return 1;
}

void oracle_rule_rects(const float* planes, int32_t n, int32_t pitch, int32_t n_lobes,
                       const ocam* cam, float blur, float b_lo, float b_hi, int32_t tile_w,
                       int32_t tile_h, int32_t* rects, uint32_t* keys, int32_t* binned, uint32_t* tiles) {
  for (int32_t i = 0; i < n; ++i)
    binned[i] = oracle_rule_rect_one(planes, pitch, n_lobes, i, cam, blur, b_lo, b_hi, tile_w,
                                     tile_h, rects + 4 * (size_t)i, keys + i, tiles ? tiles + i : NULL);
}
