/*
 * sv_oracle.c -- plain FP64 CPU oracle of the StereoVAE hot path
 * (Chang et al., "StereoVAE: A lightweight stereo-matching system using
 * embedded GPUs", arXiv 2305.11566).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this code:
 * only the tests, the smoke check and the benchmark's CPU-baseline leg load it.
 * It shares no code, header, table or helper with the CUDA library.
 *
 * Every function is the plain definition of one step, written as direct loops
 * in double precision (integers where the step is integer).  OpenMP only
 * distributes independent output rows over threads; it never changes the
 * arithmetic of an output element.
 *
 * Steps and the passages they follow:
 *   orc_downsample4      quarter-size input of the coarse matcher (Sec. I, III-B1, IV-A):
 *                        4x4 box sums S (integer, no division: ZNCC is gain invariant)
 *   orc_zncc_at          ZNCC score of one (x, y, d) by Eq. 1-3 with window means
 *   orc_zncc_wta         winner-take-all of Eq. 6 (argmax of rho = argmin of 1 - rho),
 *                        decided by exact integer comparison
 *   orc_upsample4        "linear scaling" of the small map (Sec. IV-C), bilinear x4, values x4
 *   orc_conv2d           direct convolution (encoder, latent heads, decoder, final layer;
 *                        Sec. III-B, Table I), optional nearest x2 upsample + crop of its input
 *   orc_refine_forward   the refinement net and the residual onto the upsampled map
 *   orc_loss             smooth-L1 reconstruction + KL of the latent (Sec. III-B2, Eq. 9-11)
 *   orc_refine_backward  hand-derived gradient of orc_loss through the net (FP64)
 *   orc_sgm_path         semi-global aggregation along one direction (Sec. III-A, Eq. 4)
 *   orc_sgm              sum over directions (Eq. 5); orc_sgm_wta: Eq. 6 on the sum
 *   orc_smp, orc_median3 single-matching-phase occlusion check and median filter (Eq. 7
 *                        and the text after it)
 *   orc_census_volume    census matching cost (Sec. IV-C settings S1, S2)
 *   orc_dt_aggregate     domain-transform cost aggregation (Sec. IV-C settings S1, S3)
 *   orc_t1_*             the paper's Table I network (Sec. III-B1) and its loss (Eq. 8-11)
 *   orc_refine_forward_q the FP8 (E4M3) quantised refinement (Sec. V future work) and orc_e4m3
 *
 * Readings of the paper (where it is silent, garbled or inconsistent):
 *   - cost range: Eq. 1 gives 1 - rho, which lies in [0, 2], not [0, 1]; the
 *     oracle returns rho in [-1, 1] and WTA takes argmax rho (== argmin 1 - rho).
 *   - Eq. 1-3 reuse (x, y) as window index; the window is the k x k square of
 *     offsets (i, j) in [-r, r]^2 around each centre; each window has its own mean.
 *   - window pixels outside the image take the nearest edge pixel (clamp).
 *   - a candidate d is valid iff x - d >= 0; d = 0 is always valid.
 *   - a window with zero variance gives rho = 0 (exact integer test).
 *   - ties go to the lowest d.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* ------------------------------------------------------------------ a1
 * Quarter-size input (Sec. I; Sec. IV-A "initial quarter size"): S(x, y) is the
 * sum of the 4x4 block of full-resolution pixels (4x+i, 4y+j), i, j < 4.
 * w = W / 4, h = H / 4 (floor); trailing columns/rows are dropped. */
void orc_downsample4(const uint8_t* img, int W, int H, int pitch, int32_t* S) {
  int w = W / 4, h = H / 4;
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int32_t s = 0;
      for (int j = 0; j < 4; ++j)
        for (int i = 0; i < 4; ++i) s += img[(size_t)(4 * y + j) * pitch + 4 * x + i];
      S[(size_t)y * w + x] = s;
    }
}

/* ------------------------------------------------------------------ a2-a3
 * Eq. 1-3: rho = sum dL * dR / (sigma_L * sigma_R), dI = I - mean over the
 * window, sigma = sqrt(sum dI^2).  Left window centred at (x, y), right window
 * centred at (x - d, y).  Returns NAN when x - d < 0 (no candidate). */
double orc_zncc_at(const int32_t* SL, const int32_t* SR, int w, int h, int k, int x, int y, int d) {
  if (x - d < 0) return NAN;
  const int r = k / 2;
  const int N = k * k;
  double mL = 0.0, mR = 0.0;
  for (int j = -r; j <= r; ++j)
    for (int i = -r; i <= r; ++i) {
      int yy = clampi(y + j, 0, h - 1);
      mL += SL[(size_t)yy * w + clampi(x + i, 0, w - 1)];
      mR += SR[(size_t)yy * w + clampi(x - d + i, 0, w - 1)];
    }
  mL /= N;
  mR /= N;
  double num = 0.0, sLL = 0.0, sRR = 0.0;
  for (int j = -r; j <= r; ++j)
    for (int i = -r; i <= r; ++i) {
      int yy = clampi(y + j, 0, h - 1);
      double dl = SL[(size_t)yy * w + clampi(x + i, 0, w - 1)] - mL;
      double dr = SR[(size_t)yy * w + clampi(x - d + i, 0, w - 1)] - mR;
      num += dl * dr;
      sLL += dl * dl;
      sRR += dr * dr;
    }
  /* zero variance is decided exactly on the integer sums below */
  int64_t s1 = 0, s2 = 0, t1 = 0, t2 = 0;
  for (int j = -r; j <= r; ++j)
    for (int i = -r; i <= r; ++i) {
      int yy = clampi(y + j, 0, h - 1);
      int64_t a = SL[(size_t)yy * w + clampi(x + i, 0, w - 1)];
      int64_t b = SR[(size_t)yy * w + clampi(x - d + i, 0, w - 1)];
      s1 += a; s2 += a * a; t1 += b; t2 += b * b;
    }
  if ((int64_t)N * s2 - s1 * s1 == 0 || (int64_t)N * t2 - t1 * t1 == 0) return 0.0;
  return num / (sqrt(sLL) * sqrt(sRR));
}

/* Full cost volume rho[(y * w + x) * D + d] (NAN where x - d < 0). */
void orc_zncc_volume(const int32_t* SL, const int32_t* SR, int w, int h, int k, int D, double* rho) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x)
      for (int d = 0; d < D; ++d) rho[((size_t)y * w + x) * D + d] = orc_zncc_at(SL, SR, w, h, k, x, y, d);
}

/* Exact window sums for one candidate: n = N*sum(LR) - sum(L)*sum(R),
 * vL = N*sum(L^2) - sum(L)^2, vR = N*sum(R^2) - sum(R)^2 (all exact integers).
 * rho = n / sqrt(vL * vR) by Eq. 1-3 after multiplying through by N. */
static void exact_terms(const int32_t* SL, const int32_t* SR, int w, int h, int k, int x, int y, int d,
                        int64_t* n, int64_t* vL, int64_t* vR) {
  const int r = k / 2;
  const int64_t N = (int64_t)k * k;
  int64_t sl = 0, sr = 0, sll = 0, srr = 0, slr = 0;
  for (int j = -r; j <= r; ++j)
    for (int i = -r; i <= r; ++i) {
      int yy = clampi(y + j, 0, h - 1);
      int64_t a = SL[(size_t)yy * w + clampi(x + i, 0, w - 1)];
      int64_t b = SR[(size_t)yy * w + clampi(x - d + i, 0, w - 1)];
      sl += a; sr += b; sll += a * a; srr += b * b; slr += a * b;
    }
  *n = N * slr - sl * sr;
  *vL = N * sll - sl * sl;
  *vR = N * srr - sr * sr;
}

/* Exact comparison of two candidates at the same pixel (common vL > 0):
 * rho_1 > rho_2  <=>  n1 / sqrt(vR1) > n2 / sqrt(vR2).  A zero-variance right
 * window counts as n = 0.  Returns +1, 0, -1. */
static int cmp_exact(int64_t n1, int64_t v1, int64_t n2, int64_t v2) {
  if (v1 == 0) n1 = 0, v1 = 1;
  if (v2 == 0) n2 = 0, v2 = 1;
  int s1 = (n1 > 0) - (n1 < 0), s2 = (n2 > 0) - (n2 < 0);
  if (s1 != s2) return s1 > s2 ? 1 : -1;
  if (s1 == 0) return 0;
  __int128 a = (__int128)n1 * n1 * v2; /* |n| <= v_max ~ 2.7e10, so n^2 v < 2^127 */
  __int128 b = (__int128)n2 * n2 * v1;
  int c = (a > b) - (a < b);
  return s1 > 0 ? c : -c;
}

/* Eq. 6 winner-take-all over d in [0, D) restricted to x - d >= 0: disp = argmax rho
 * (lowest d on exact ties), decided exactly; best = rho(disp), second = largest rho over
 * the other valid candidates (-2 when there is none), both in FP64 from orc_zncc_at. */
void orc_zncc_wta(const int32_t* SL, const int32_t* SR, int w, int h, int k, int D,
                  int32_t* disp, double* best, double* second) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int64_t bn = 0, bvL = 0, bvR = 0;
      int bd = 0;
      exact_terms(SL, SR, w, h, k, x, y, 0, &bn, &bvL, &bvR);
      int dmax = D - 1 < x ? D - 1 : x;
      for (int d = 1; d <= dmax; ++d) {
        int64_t n, vL, vR;
        exact_terms(SL, SR, w, h, k, x, y, d, &n, &vL, &vR);
        if (vL == 0) continue; /* every rho is 0: keep d = 0 */
        if (cmp_exact(n, vR, bn, bvR) > 0) { bn = n; bvR = vR; bd = d; }
      }
      disp[(size_t)y * w + x] = bd;
      double b = orc_zncc_at(SL, SR, w, h, k, x, y, bd);
      double s = -2.0;
      for (int d = 0; d <= dmax; ++d) {
        if (d == bd) continue;
        double v = orc_zncc_at(SL, SR, w, h, k, x, y, d);
        if (v > s) s = v;
      }
      if (best) best[(size_t)y * w + x] = b;
      if (second) second[(size_t)y * w + x] = s;
    }
}

/* ------------------------------------------------------------------ a5
 * Linear scaling of the small map to full resolution (Sec. IV-C, "Mini+Linear";
 * Sec. III-B1: the net refines an upscaled coarse map).  Half-pixel centres:
 * source coordinate s = (X + 1/2) / 4 - 1/2, clamped to [0, w-1]; bilinear
 * weights; values multiplied by 4 (disparity in full-resolution pixels). */
void orc_upsample4(const double* disp, int w, int h, int W, int H, double* U) {
  for (int Y = 0; Y < H; ++Y) {
    double sy = (Y + 0.5) / 4.0 - 0.5;
    if (sy < 0) sy = 0;
    if (sy > h - 1) sy = h - 1;
    int y0 = (int)floor(sy);
    int y1 = y0 + 1 < h ? y0 + 1 : h - 1;
    double fy = sy - y0;
    for (int X = 0; X < W; ++X) {
      double sx = (X + 0.5) / 4.0 - 0.5;
      if (sx < 0) sx = 0;
      if (sx > w - 1) sx = w - 1;
      int x0 = (int)floor(sx);
      int x1 = x0 + 1 < w ? x0 + 1 : w - 1;
      double fx = sx - x0;
      double top = (1 - fx) * disp[(size_t)y0 * w + x0] + fx * disp[(size_t)y0 * w + x1];
      double bot = (1 - fx) * disp[(size_t)y1 * w + x0] + fx * disp[(size_t)y1 * w + x1];
      U[(size_t)Y * W + X] = 4.0 * ((1 - fy) * top + fy * bot);
    }
  }
}

/* Transpose of orc_upsample4 (gradient of sum(gU * U) w.r.t. disp). */
void orc_upsample4_backward(const double* gU, int w, int h, int W, int H, double* gdisp) {
  memset(gdisp, 0, sizeof(double) * (size_t)w * h);
  for (int Y = 0; Y < H; ++Y) {
    double sy = (Y + 0.5) / 4.0 - 0.5;
    if (sy < 0) sy = 0;
    if (sy > h - 1) sy = h - 1;
    int y0 = (int)floor(sy);
    int y1 = y0 + 1 < h ? y0 + 1 : h - 1;
    double fy = sy - y0;
    for (int X = 0; X < W; ++X) {
      double sx = (X + 0.5) / 4.0 - 0.5;
      if (sx < 0) sx = 0;
      if (sx > w - 1) sx = w - 1;
      int x0 = (int)floor(sx);
      int x1 = x0 + 1 < w ? x0 + 1 : w - 1;
      double fx = sx - x0;
      double g = 4.0 * gU[(size_t)Y * W + X];
      gdisp[(size_t)y0 * w + x0] += g * (1 - fy) * (1 - fx);
      gdisp[(size_t)y0 * w + x1] += g * (1 - fy) * fx;
      gdisp[(size_t)y1 * w + x0] += g * fy * (1 - fx);
      gdisp[(size_t)y1 * w + x1] += g * fy * fx;
    }
  }
}

/* ------------------------------------------------------------------ a7-a11
 * Direct 2-D convolution, NHWC activations, weights wt[co][ky][kx][ci], bias b[co].
 * out(y, x, co) = b[co] + sum_{ky, kx, ci} wt * V(y*stride + ky - pad, x*stride + kx - pad, ci)
 * where V is the input, zero outside [0, Hv) x [0, Wv).  With up2 = 1 the input is
 * first upsampled by nearest x2 and cropped to (Hv, Wv) = (Ho, Wo):
 * V(Y, X) = in(Y / 2, X / 2).  relu = 1 applies max(0, .) to the output. */
void orc_conv2d(const double* in, int Hi, int Wi, int Ci, const float* wt, const float* b, int Co, int ks,
                int stride, int pad, int up2, int Ho, int Wo, int relu, double* out) {
  const int Hv = up2 ? Ho : Hi, Wv = up2 ? Wo : Wi;
#pragma omp parallel for schedule(dynamic, 1)
  for (int y = 0; y < Ho; ++y)
    for (int x = 0; x < Wo; ++x)
      for (int co = 0; co < Co; ++co) {
        double acc = b ? (double)b[co] : 0.0;
        for (int ky = 0; ky < ks; ++ky) {
          int vy = y * stride + ky - pad;
          if (vy < 0 || vy >= Hv) continue;
          int iy = up2 ? vy / 2 : vy;
          for (int kx = 0; kx < ks; ++kx) {
            int vx = x * stride + kx - pad;
            if (vx < 0 || vx >= Wv) continue;
            int ix = up2 ? vx / 2 : vx;
            const double* ip = in + ((size_t)iy * Wi + ix) * Ci;
            const float* wp = wt + (((size_t)co * ks + ky) * ks + kx) * Ci;
            for (int ci = 0; ci < Ci; ++ci) acc += (double)wp[ci] * ip[ci];
          }
        }
        if (relu && acc < 0) acc = 0;
        out[((size_t)y * Wo + x) * Co + co] = acc;
      }
}

/* Gradient of orc_conv2d (without the ReLU, which the caller applies to gout):
 * gin += d/d in, gw += d/d wt, gb += d/d b.  Any of gin/gw/gb may be NULL. */
void orc_conv2d_backward(const double* in, int Hi, int Wi, int Ci, const float* wt, int Co, int ks, int stride,
                         int pad, int up2, int Ho, int Wo, const double* gout, double* gin, double* gw, double* gb) {
  const int Hv = up2 ? Ho : Hi, Wv = up2 ? Wo : Wi;
  if (gb)
    for (int co = 0; co < Co; ++co) {
      double s = 0;
      for (size_t p = 0; p < (size_t)Ho * Wo; ++p) s += gout[p * Co + co];
      gb[co] += s;
    }
  if (gw) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int co = 0; co < Co; ++co)
      for (int ky = 0; ky < ks; ++ky)
        for (int kx = 0; kx < ks; ++kx)
          for (int ci = 0; ci < Ci; ++ci) {
            double s = 0;
            for (int y = 0; y < Ho; ++y) {
              int vy = y * stride + ky - pad;
              if (vy < 0 || vy >= Hv) continue;
              int iy = up2 ? vy / 2 : vy;
              for (int x = 0; x < Wo; ++x) {
                int vx = x * stride + kx - pad;
                if (vx < 0 || vx >= Wv) continue;
                int ix = up2 ? vx / 2 : vx;
                s += gout[((size_t)y * Wo + x) * Co + co] * in[((size_t)iy * Wi + ix) * Ci + ci];
              }
            }
            gw[(((size_t)co * ks + ky) * ks + kx) * Ci + ci] += s;
          }
  }
  if (gin) {
    /* scatter form, serial: every (output, tap) adds wt * gout to the input it read */
    for (int y = 0; y < Ho; ++y)
      for (int x = 0; x < Wo; ++x)
        for (int ky = 0; ky < ks; ++ky) {
          int vy = y * stride + ky - pad;
          if (vy < 0 || vy >= Hv) continue;
          int iy = up2 ? vy / 2 : vy;
          for (int kx = 0; kx < ks; ++kx) {
            int vx = x * stride + kx - pad;
            if (vx < 0 || vx >= Wv) continue;
            int ix = up2 ? vx / 2 : vx;
            double* gp = gin + ((size_t)iy * Wi + ix) * Ci;
            for (int co = 0; co < Co; ++co) {
              double g = gout[((size_t)y * Wo + x) * Co + co];
              const float* wp = wt + (((size_t)co * ks + ky) * ks + kx) * Ci;
              for (int ci = 0; ci < Ci; ++ci) gp[ci] += g * wp[ci];
            }
          }
        }
  }
}

/* ------------------------------------------------------------------ the net
 * Refinement network of the build contract: input x0 = concat(L / 256, U / 256)
 * at full resolution (Sec. III-B2: inputs normalised, factor 256); encoder
 * 3 x [3x3 conv stride 2 pad 1, ReLU] with widths enc[0..2]; latent heads
 * mu, logvar = two 1x1 convs (Table I "mu & sigma", 1x1 kernels); z = mu at
 * inference, z = mu + eps * exp(logvar / 2) in training (reparameterisation, Eq. 8,
 * in its standard form); decoder 3 x [nearest x2 upsample cropped to the matching
 * encoder level, 3x3 conv pad 1, ReLU] with widths dec[0..2]; final 3x3 conv to
 * 1 channel, no activation, added to U (the residual onto the upsampled map).
 *
 * Weight vector: per layer in the order enc1, enc2, enc3, mu, logvar, dec1, dec2,
 * dec3, final: W[cout][kh][kw][cin] followed by b[cout], FP32. */
typedef struct {
  int enc[3];
  int lat;
  int dec[3];
} orc_net;

enum { L_ENC1, L_ENC2, L_ENC3, L_MU, L_LV, L_DEC1, L_DEC2, L_DEC3, L_FINAL, L_COUNT };

static void layer_dims(const orc_net* n, int l, int* co, int* ci, int* ks) {
  switch (l) {
    case L_ENC1: *co = n->enc[0]; *ci = 2; *ks = 3; break;
    case L_ENC2: *co = n->enc[1]; *ci = n->enc[0]; *ks = 3; break;
    case L_ENC3: *co = n->enc[2]; *ci = n->enc[1]; *ks = 3; break;
    case L_MU: *co = n->lat; *ci = n->enc[2]; *ks = 1; break;
    case L_LV: *co = n->lat; *ci = n->enc[2]; *ks = 1; break;
    case L_DEC1: *co = n->dec[0]; *ci = n->lat; *ks = 3; break;
    case L_DEC2: *co = n->dec[1]; *ci = n->dec[0]; *ks = 3; break;
    case L_DEC3: *co = n->dec[2]; *ci = n->dec[1]; *ks = 3; break;
    default: *co = 1; *ci = n->dec[2]; *ks = 3; break;
  }
}

/* offsets of W and b of layer l in the flat vector; returns total count when l == L_COUNT */
size_t orc_param_offset(const int* widths7, int l, int want_bias) {
  orc_net n = {{widths7[0], widths7[1], widths7[2]}, widths7[3], {widths7[4], widths7[5], widths7[6]}};
  size_t off = 0;
  for (int i = 0; i < L_COUNT; ++i) {
    int co, ci, ks;
    layer_dims(&n, i, &co, &ci, &ks);
    size_t nw = (size_t)co * ks * ks * ci;
    if (i == l) return want_bias ? off + nw : off;
    off += nw + co;
  }
  return off;
}

/* Activations of one forward pass (all FP64, NHWC). */
typedef struct {
  int H, W, H1, W1, H2, W2, H3, W3;
  double *U, *x0, *e1, *e2, *e3, *mu, *lv, *z, *d1, *d2, *d3, *Y;
} orc_acts;

static void level_sizes(int H, int W, orc_acts* a) {
  a->H = H; a->W = W;
  a->H1 = (H + 1) / 2; a->W1 = (W + 1) / 2;
  a->H2 = (a->H1 + 1) / 2; a->W2 = (a->W1 + 1) / 2;
  a->H3 = (a->H2 + 1) / 2; a->W3 = (a->W2 + 1) / 2;
}

static void acts_alloc(const orc_net* n, int H, int W, orc_acts* a) {
  level_sizes(H, W, a);
  size_t P0 = (size_t)H * W, P1 = (size_t)a->H1 * a->W1, P2 = (size_t)a->H2 * a->W2, P3 = (size_t)a->H3 * a->W3;
  a->U = calloc(P0, sizeof(double));
  a->x0 = calloc(P0 * 2, sizeof(double));
  a->e1 = calloc(P1 * n->enc[0], sizeof(double));
  a->e2 = calloc(P2 * n->enc[1], sizeof(double));
  a->e3 = calloc(P3 * n->enc[2], sizeof(double));
  a->mu = calloc(P3 * n->lat, sizeof(double));
  a->lv = calloc(P3 * n->lat, sizeof(double));
  a->z = calloc(P3 * n->lat, sizeof(double));
  a->d1 = calloc(P2 * n->dec[0], sizeof(double));
  a->d2 = calloc(P1 * n->dec[1], sizeof(double));
  a->d3 = calloc(P0 * n->dec[2], sizeof(double));
  a->Y = calloc(P0, sizeof(double));
}

static void acts_free(orc_acts* a) {
  free(a->U); free(a->x0); free(a->e1); free(a->e2); free(a->e3); free(a->mu); free(a->lv);
  free(a->z); free(a->d1); free(a->d2); free(a->d3); free(a->Y);
}

static const float* Wl(const float* p, const int* w7, int l) { return p + orc_param_offset(w7, l, 0); }
static const float* Bl(const float* p, const int* w7, int l) { return p + orc_param_offset(w7, l, 1); }

static void net_forward(const orc_net* n, const int* w7, const float* params, const uint8_t* left, int pitch,
                        const double* coarse, int w, int h, const float* eps, orc_acts* a) {
  const int H = a->H, W = a->W;
  int co, ci, ks;
  orc_upsample4(coarse, w, h, W, H, a->U);
  for (int Y = 0; Y < H; ++Y)
    for (int X = 0; X < W; ++X) {
      a->x0[((size_t)Y * W + X) * 2 + 0] = left[(size_t)Y * pitch + X] / 256.0;
      a->x0[((size_t)Y * W + X) * 2 + 1] = a->U[(size_t)Y * W + X] / 256.0;
    }
  layer_dims(n, L_ENC1, &co, &ci, &ks);
  orc_conv2d(a->x0, H, W, 2, Wl(params, w7, L_ENC1), Bl(params, w7, L_ENC1), co, 3, 2, 1, 0, a->H1, a->W1, 1, a->e1);
  layer_dims(n, L_ENC2, &co, &ci, &ks);
  orc_conv2d(a->e1, a->H1, a->W1, ci, Wl(params, w7, L_ENC2), Bl(params, w7, L_ENC2), co, 3, 2, 1, 0, a->H2, a->W2, 1, a->e2);
  layer_dims(n, L_ENC3, &co, &ci, &ks);
  orc_conv2d(a->e2, a->H2, a->W2, ci, Wl(params, w7, L_ENC3), Bl(params, w7, L_ENC3), co, 3, 2, 1, 0, a->H3, a->W3, 1, a->e3);
  orc_conv2d(a->e3, a->H3, a->W3, n->enc[2], Wl(params, w7, L_MU), Bl(params, w7, L_MU), n->lat, 1, 1, 0, 0, a->H3, a->W3, 0, a->mu);
  orc_conv2d(a->e3, a->H3, a->W3, n->enc[2], Wl(params, w7, L_LV), Bl(params, w7, L_LV), n->lat, 1, 1, 0, 0, a->H3, a->W3, 0, a->lv);
  size_t nl = (size_t)a->H3 * a->W3 * n->lat;
  for (size_t i = 0; i < nl; ++i) a->z[i] = eps ? a->mu[i] + (double)eps[i] * exp(0.5 * a->lv[i]) : a->mu[i];
  orc_conv2d(a->z, a->H3, a->W3, n->lat, Wl(params, w7, L_DEC1), Bl(params, w7, L_DEC1), n->dec[0], 3, 1, 1, 1, a->H2, a->W2, 1, a->d1);
  orc_conv2d(a->d1, a->H2, a->W2, n->dec[0], Wl(params, w7, L_DEC2), Bl(params, w7, L_DEC2), n->dec[1], 3, 1, 1, 1, a->H1, a->W1, 1, a->d2);
  orc_conv2d(a->d2, a->H1, a->W1, n->dec[1], Wl(params, w7, L_DEC3), Bl(params, w7, L_DEC3), n->dec[2], 3, 1, 1, 1, H, W, 1, a->d3);
  orc_conv2d(a->d3, H, W, n->dec[2], Wl(params, w7, L_FINAL), Bl(params, w7, L_FINAL), 1, 3, 1, 1, 0, H, W, 0, a->Y);
  for (size_t p = 0; p < (size_t)H * W; ++p) a->Y[p] += a->U[p];
}

/* Forward of one pair.  widths7 = {enc0, enc1, enc2, lat, dec0, dec1, dec2}.
 * coarse: h x w coarse disparities (coarse px, as doubles); eps: latent noise
 * (H3 * W3 * lat, NULL at inference).  Outputs (each nullable): Y [H*W] refined
 * disparity, U [H*W], mu and logvar [H3*W3*lat]. */
void orc_refine_forward(const int* widths7, const float* params, const uint8_t* left, int W, int H, int pitch,
                        const double* coarse, int w, int h, const float* eps, double* Y, double* U, double* mu,
                        double* logvar) {
  orc_net n = {{widths7[0], widths7[1], widths7[2]}, widths7[3], {widths7[4], widths7[5], widths7[6]}};
  orc_acts a;
  acts_alloc(&n, H, W, &a);
  net_forward(&n, widths7, params, left, pitch, coarse, w, h, eps, &a);
  size_t P0 = (size_t)H * W, nl = (size_t)a.H3 * a.W3 * n.lat;
  if (Y) memcpy(Y, a.Y, P0 * sizeof(double));
  if (U) memcpy(U, a.U, P0 * sizeof(double));
  if (mu) memcpy(mu, a.mu, nl * sizeof(double));
  if (logvar) memcpy(logvar, a.lv, nl * sizeof(double));
  acts_free(&a);
}

/* Intermediate activation of a forward pass, for layer-by-layer checks.
 * which: 0 U, 1 e1, 2 e2, 3 e3, 4 mu, 5 logvar, 6 z, 7 d1, 8 d2, 9 d3, 10 Y. */
void orc_refine_activation(const int* widths7, const float* params, const uint8_t* left, int W, int H, int pitch,
                           const double* coarse, int w, int h, const float* eps, int which, double* out) {
  orc_net n = {{widths7[0], widths7[1], widths7[2]}, widths7[3], {widths7[4], widths7[5], widths7[6]}};
  orc_acts a;
  acts_alloc(&n, H, W, &a);
  net_forward(&n, widths7, params, left, pitch, coarse, w, h, eps, &a);
  size_t P0 = (size_t)H * W, P1 = (size_t)a.H1 * a.W1, P2 = (size_t)a.H2 * a.W2, P3 = (size_t)a.H3 * a.W3;
  const double* src = a.Y;
  size_t cnt = P0;
  switch (which) {
    case 0: src = a.U; cnt = P0; break;
    case 1: src = a.e1; cnt = P1 * n.enc[0]; break;
    case 2: src = a.e2; cnt = P2 * n.enc[1]; break;
    case 3: src = a.e3; cnt = P3 * n.enc[2]; break;
    case 4: src = a.mu; cnt = P3 * n.lat; break;
    case 5: src = a.lv; cnt = P3 * n.lat; break;
    case 6: src = a.z; cnt = P3 * n.lat; break;
    case 7: src = a.d1; cnt = P2 * n.dec[0]; break;
    case 8: src = a.d2; cnt = P1 * n.dec[1]; break;
    case 9: src = a.d3; cnt = P0 * n.dec[2]; break;
    default: break;
  }
  memcpy(out, src, cnt * sizeof(double));
  acts_free(&a);
}

/* ------------------------------------------------------------------ a12 loss
 * Reconstruction term: smooth-L1 with beta = 1 px, summed over pixels and divided
 * by n_pix (the batch's pixel count); KL term of the latent against N(0, 1),
 * 0.5 * (mu^2 + exp(lv) - 1 - lv) summed and divided by n_lat, weighted by kl_w.
 * (Eq. 11 of the paper is garbled; this is its standard VAE form.)
 * Returns this pair's contribution: rec_sum / n_pix + kl_w * kl_sum / n_lat. */
double orc_loss(const double* Y, const float* gt, size_t P, const double* mu, const double* lv, size_t nl, double n_pix,
                double n_lat, double kl_w, double* rec_out, double* kl_out) {
  double rec = 0, kl = 0;
  for (size_t p = 0; p < P; ++p) {
    double e = Y[p] - (double)gt[p];
    double a = fabs(e);
    rec += a < 1.0 ? 0.5 * e * e : a - 0.5;
  }
  for (size_t i = 0; i < nl; ++i) kl += 0.5 * (mu[i] * mu[i] + exp(lv[i]) - 1.0 - lv[i]);
  if (rec_out) *rec_out = rec / n_pix;
  if (kl_out) *kl_out = kl / n_lat;
  return rec / n_pix + kl_w * kl / n_lat;
}

/* Loss of one pair by forward pass (training form: eps given). */
double orc_refine_loss(const int* widths7, const float* params, const uint8_t* left, int W, int H, int pitch,
                       const double* coarse, int w, int h, const float* eps, const float* gt, double n_pix,
                       double n_lat, double kl_w) {
  orc_net n = {{widths7[0], widths7[1], widths7[2]}, widths7[3], {widths7[4], widths7[5], widths7[6]}};
  orc_acts a;
  acts_alloc(&n, H, W, &a);
  net_forward(&n, widths7, params, left, pitch, coarse, w, h, eps, &a);
  double L = orc_loss(a.Y, gt, (size_t)H * W, a.mu, a.lv, (size_t)a.H3 * a.W3 * n.lat, n_pix, n_lat, kl_w, 0, 0);
  acts_free(&a);
  return L;
}

static void relu_mask(double* g, const double* act, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!(act[i] > 0)) g[i] = 0;
}

/* Gradient of orc_refine_loss w.r.t. the parameters (added into gparams, FP64,
 * same layout as params) and, if gcoarse != NULL, w.r.t. the coarse map (both
 * through the residual and through the network input channel U / 256).
 * Returns the loss. */
double orc_refine_backward(const int* widths7, const float* params, const uint8_t* left, int W, int H, int pitch,
                           const double* coarse, int w, int h, const float* eps, const float* gt, double n_pix,
                           double n_lat, double kl_w, double* gparams, double* gcoarse) {
  orc_net n = {{widths7[0], widths7[1], widths7[2]}, widths7[3], {widths7[4], widths7[5], widths7[6]}};
  orc_acts a;
  acts_alloc(&n, H, W, &a);
  net_forward(&n, widths7, params, left, pitch, coarse, w, h, eps, &a);
  const size_t P0 = (size_t)H * W, P1 = (size_t)a.H1 * a.W1, P2 = (size_t)a.H2 * a.W2, P3 = (size_t)a.H3 * a.W3;
  const size_t nl = P3 * n.lat;
  double L = orc_loss(a.Y, gt, P0, a.mu, a.lv, nl, n_pix, n_lat, kl_w, 0, 0);
#define GW(l) (gparams + orc_param_offset(widths7, l, 0))
#define GB(l) (gparams + orc_param_offset(widths7, l, 1))
  double* gY = calloc(P0, sizeof(double));
  for (size_t p = 0; p < P0; ++p) {
    double e = a.Y[p] - (double)gt[p];
    gY[p] = (fabs(e) < 1.0 ? e : (e > 0 ? 1.0 : -1.0)) / n_pix;
  }
  double* gU = calloc(P0, sizeof(double));
  for (size_t p = 0; p < P0; ++p) gU[p] = gY[p]; /* Y = U + r */
  double* gd3 = calloc(P0 * n.dec[2], sizeof(double));
  orc_conv2d_backward(a.d3, H, W, n.dec[2], Wl(params, widths7, L_FINAL), 1, 3, 1, 1, 0, H, W, gY, gd3, GW(L_FINAL), GB(L_FINAL));
  relu_mask(gd3, a.d3, P0 * n.dec[2]);
  double* gd2 = calloc(P1 * n.dec[1], sizeof(double));
  orc_conv2d_backward(a.d2, a.H1, a.W1, n.dec[1], Wl(params, widths7, L_DEC3), n.dec[2], 3, 1, 1, 1, H, W, gd3, gd2, GW(L_DEC3), GB(L_DEC3));
  relu_mask(gd2, a.d2, P1 * n.dec[1]);
  double* gd1 = calloc(P2 * n.dec[0], sizeof(double));
  orc_conv2d_backward(a.d1, a.H2, a.W2, n.dec[0], Wl(params, widths7, L_DEC2), n.dec[1], 3, 1, 1, 1, a.H1, a.W1, gd2, gd1, GW(L_DEC2), GB(L_DEC2));
  relu_mask(gd1, a.d1, P2 * n.dec[0]);
  double* gz = calloc(nl, sizeof(double));
  orc_conv2d_backward(a.z, a.H3, a.W3, n.lat, Wl(params, widths7, L_DEC1), n.dec[0], 3, 1, 1, 1, a.H2, a.W2, gd1, gz, GW(L_DEC1), GB(L_DEC1));
  double* gmu = calloc(nl, sizeof(double));
  double* glv = calloc(nl, sizeof(double));
  for (size_t i = 0; i < nl; ++i) {
    gmu[i] = gz[i] + kl_w * a.mu[i] / n_lat;
    glv[i] = kl_w * 0.5 * (exp(a.lv[i]) - 1.0) / n_lat;
    if (eps) glv[i] += gz[i] * (double)eps[i] * 0.5 * exp(0.5 * a.lv[i]);
  }
  double* ge3 = calloc(P3 * n.enc[2], sizeof(double));
  orc_conv2d_backward(a.e3, a.H3, a.W3, n.enc[2], Wl(params, widths7, L_MU), n.lat, 1, 1, 0, 0, a.H3, a.W3, gmu, ge3, GW(L_MU), GB(L_MU));
  orc_conv2d_backward(a.e3, a.H3, a.W3, n.enc[2], Wl(params, widths7, L_LV), n.lat, 1, 1, 0, 0, a.H3, a.W3, glv, ge3, GW(L_LV), GB(L_LV));
  relu_mask(ge3, a.e3, P3 * n.enc[2]);
  double* ge2 = calloc(P2 * n.enc[1], sizeof(double));
  orc_conv2d_backward(a.e2, a.H2, a.W2, n.enc[1], Wl(params, widths7, L_ENC3), n.enc[2], 3, 2, 1, 0, a.H3, a.W3, ge3, ge2, GW(L_ENC3), GB(L_ENC3));
  relu_mask(ge2, a.e2, P2 * n.enc[1]);
  double* ge1 = calloc(P1 * n.enc[0], sizeof(double));
  orc_conv2d_backward(a.e1, a.H1, a.W1, n.enc[0], Wl(params, widths7, L_ENC2), n.enc[1], 3, 2, 1, 0, a.H2, a.W2, ge2, ge1, GW(L_ENC2), GB(L_ENC2));
  relu_mask(ge1, a.e1, P1 * n.enc[0]);
  double* gx0 = calloc(P0 * 2, sizeof(double));
  orc_conv2d_backward(a.x0, H, W, 2, Wl(params, widths7, L_ENC1), n.enc[0], 3, 2, 1, 0, a.H1, a.W1, ge1, gx0, GW(L_ENC1), GB(L_ENC1));
  if (gcoarse) {
    for (size_t p = 0; p < P0; ++p) gU[p] += gx0[p * 2 + 1] / 256.0;
    orc_upsample4_backward(gU, w, h, W, H, gcoarse);
  }
#undef GW
#undef GB
  free(gY); free(gU); free(gd3); free(gd2); free(gd1); free(gz); free(gmu); free(glv);
  free(ge3); free(ge2); free(ge1); free(gx0);
  acts_free(&a);
  return L;
}

/* ------------------------------------------------------------------ Adam
 * One Adam step (Sec. IV-A: Adam, beta1 = 0.99, beta2 = 0.999, lr 5e-4) on FP64
 * state: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr * mhat / (sqrt(vhat) + eps)
 * with bias corrections mhat = m / (1 - b1^t), vhat = v / (1 - b2^t). */
void orc_adam(double* p, double* m, double* v, const double* g, size_t n, int t, double lr, double b1, double b2,
              double eps) {
  double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (size_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1 - b1) * g[i];
    v[i] = b2 * v[i] + (1 - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
  }
}

/* ------------------------------------------------------------------ semi-global matching
 * Sec. III-A (Eq. 4-6) on a coarse cost volume C [h][w][D], C = 1 - rho of Eq. 1.
 * Readings (the paper leaves them open): candidates with x - d < 0 carry the largest cost
 * of Eq. 1, 2; four path directions; P1, P2 are arguments.
 *
 * orc_sgm_path: the cost C_r aggregated along one direction r by Eq. 4.  dir 0: r = (1, 0),
 * paths run left to right along each row; 1: right to left; 2: top to bottom along each
 * column; 3: bottom to top.  The first pixel of a path keeps its own cost (no predecessor).
 * The terms with d - 1 < 0 or d + 1 >= D are absent.  Eq. 4's minimum over i excludes d and
 * d +- 1; taking it over all disparities gives the same value, since those three are
 * already in the minimum with smaller penalties. */
void orc_sgm_path(const double* C, int w, int h, int D, double P1, double P2, int dir, double* Cr) {
  const int dx = dir == 0 ? 1 : dir == 1 ? -1 : 0;
  const int dy = dir == 2 ? 1 : dir == 3 ? -1 : 0;
  const int nlines = dy == 0 ? h : w, len = dy == 0 ? w : h;
#pragma omp parallel for schedule(static)
  for (int line = 0; line < nlines; ++line) {
    for (int s = 0; s < len; ++s) {
      const int x = dx == 0 ? line : dx > 0 ? s : w - 1 - s;
      const int y = dy == 0 ? line : dy > 0 ? s : h - 1 - s;
      const double* c = C + ((size_t)y * w + x) * D;
      double* cur = Cr + ((size_t)y * w + x) * D;
      if (s == 0) {
        for (int d = 0; d < D; ++d) cur[d] = c[d];
        continue;
      }
      const double* prev = Cr + ((size_t)(y - dy) * w + (x - dx)) * D;
      double mprev = prev[0];
      for (int k = 1; k < D; ++k)
        if (prev[k] < mprev) mprev = prev[k];
      for (int d = 0; d < D; ++d) {
        double best = prev[d];
        if (d > 0 && prev[d - 1] + P1 < best) best = prev[d - 1] + P1;
        if (d + 1 < D && prev[d + 1] + P1 < best) best = prev[d + 1] + P1;
        if (mprev + P2 < best) best = mprev + P2;
        cur[d] = c[d] + best - mprev;
      }
    }
  }
}

/* C_SGM = sum over the first npaths directions of orc_sgm_path (Eq. 5), npaths in 1..4. */
void orc_sgm(const double* C, int w, int h, int D, double P1, double P2, int npaths, double* Csgm) {
  const size_t n = (size_t)w * h * D;
  double* Cr = malloc(n * sizeof(double));
  for (size_t i = 0; i < n; ++i) Csgm[i] = 0.0;
  for (int dir = 0; dir < npaths; ++dir) {
    orc_sgm_path(C, w, h, D, P1, P2, dir, Cr);
    for (size_t i = 0; i < n; ++i) Csgm[i] += Cr[i];
  }
  free(Cr);
}

/* Eq. 6 on an aggregated volume: the disparity of the smallest cost, lowest d on ties. */
void orc_sgm_wta(const double* Csgm, int w, int h, int D, int32_t* disp) {
  for (size_t p = 0; p < (size_t)w * h; ++p) {
    const double* c = Csgm + p * D;
    int best = 0;
    for (int d = 1; d < D; ++d)
      if (c[d] < c[best]) best = d;
    disp[p] = best;
  }
}

/* ------------------------------------------------------------------ post-processing
 * Sec. III-A (Eq. 7 and the text after it), on a coarse disparity map disp [h][w].
 * Readings: Eq. 7 as printed (|x - D(x) - (x - k - D(x - k))| <= 1 for every k in (0, D))
 * contradicts the uniqueness it states in words ("no pixel of the reference image is matched
 * by two or more pixels of the target image"); the oracle takes the words: pixel x is valid
 * iff no pixel x - k to its left, 0 < k < D, is matched to the same target column
 * (x - D(x) != x - k - D(x - k)), so of two pixels sharing a target the left one keeps it.
 * An invalid pixel takes the disparity of the nearest valid pixel of its row (the left one
 * at equal distance); a row without a valid pixel is left as it is. */
void orc_smp(const int32_t* disp, int w, int h, int D, int32_t* out) {
  unsigned char* valid = malloc((size_t)w);
  for (int y = 0; y < h; ++y) {
    const int32_t* row = disp + (size_t)y * w;
    int any = 0;
    for (int x = 0; x < w; ++x) {
      int ok = 1;
      for (int k = 1; k < D && x - k >= 0; ++k)
        if (x - row[x] == x - k - row[x - k]) ok = 0;
      valid[x] = (unsigned char)ok;
      any |= ok;
    }
    for (int x = 0; x < w; ++x) {
      int v = row[x];
      if (!valid[x] && any) {
        for (int dist = 1; dist < w; ++dist) {
          if (x - dist >= 0 && valid[x - dist]) { v = row[x - dist]; break; }
          if (x + dist < w && valid[x + dist]) { v = row[x + dist]; break; }
        }
      }
      out[(size_t)y * w + x] = v;
    }
  }
  free(valid);
}

/* The median filter of the same passage (size not given; reading: 3 x 3, window pixels
 * outside the map take the nearest edge pixel): the 5th smallest of the 9 values. */
void orc_median3(const int32_t* disp, int w, int h, int32_t* out) {
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      int32_t v[9];
      int n = 0;
      for (int j = -1; j <= 1; ++j)
        for (int i = -1; i <= 1; ++i) v[n++] = disp[(size_t)clampi(y + j, 0, h - 1) * w + clampi(x + i, 0, w - 1)];
      for (int a = 1; a < 9; ++a)  /* insertion sort */
        for (int b = a; b > 0 && v[b - 1] > v[b]; --b) {
          int32_t t = v[b];
          v[b] = v[b - 1];
          v[b - 1] = t;
        }
      out[(size_t)y * w + x] = v[4];
    }
}

/* ------------------------------------------------------------------ census cost
 * Sec. IV-C (settings S1 "Census+DT" and S2 "Census+SGM"): the census matching cost as an
 * alternative to ZNCC.  The paper names the method only; the reading taken here is the
 * textbook census transform on the quarter-size images (4 x 4 box sums S):
 *   census(x, y) = the bit string over the kc x kc window offsets (i, j) != (0, 0) (raster
 *                  order) with bit = 1 iff S(x + i, y + j) < S(x, y), window pixels clamped
 *                  to the image as for ZNCC;
 *   C(x, y, d)   = number of differing bits of census_L(x, y) and census_R(x - d, y), for
 *                  x - d >= 0; candidates with x - d < 0 take the largest cost, kc^2 - 1.
 * kc is odd, 3..7 (at most 48 bits).  The cost is an integer, stored as a double. */
static uint64_t census_code(const int32_t* S, int w, int h, int kc, int x, int y) {
  const int r = kc / 2;
  const int32_t c = S[(size_t)y * w + x];
  uint64_t code = 0;
  int bit = 0;
  for (int j = -r; j <= r; ++j)
    for (int i = -r; i <= r; ++i) {
      if (i == 0 && j == 0) continue;
      const int32_t v = S[(size_t)clampi(y + j, 0, h - 1) * w + clampi(x + i, 0, w - 1)];
      if (v < c) code |= (uint64_t)1 << bit;
      ++bit;
    }
  return code;
}

static int popcount64(uint64_t v) {
  int n = 0;
  for (; v; v &= v - 1) ++n;
  return n;
}

void orc_census_volume(const int32_t* SL, const int32_t* SR, int w, int h, int kc, int D, double* C) {
#pragma omp parallel for schedule(static)
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      const uint64_t cl = census_code(SL, w, h, kc, x, y);
      for (int d = 0; d < D; ++d) {
        double* out = C + ((size_t)y * w + x) * D + d;
        if (x - d < 0) {
          *out = (double)(kc * kc - 1);
          continue;
        }
        *out = (double)popcount64(cl ^ census_code(SR, w, h, kc, x - d, y));
      }
    }
}

/* ------------------------------------------------------------------ domain-transform aggregation
 * Sec. IV-C (settings S1 "Census+DT" and S3 "ZNCC+DT").  The paper does not define DT; the
 * reading taken here is cost aggregation by the domain transform, each disparity slice of the
 * cost volume smoothed by the recursive edge-aware filter of the domain transform, guided by
 * the left quarter-size image I = S_L / 16 (mean intensity of each 4 x 4 block, 0..255):
 *   between neighbours n - 1 and n of a row (or a column) the transformed distance is
 *   t(n) = 1 + (sigma_s / sigma_r) |I(n) - I(n - 1)|;
 *   iteration i = 1..N uses sigma_i = sigma_s sqrt(3) 2^(N - i) / sqrt(4^N - 1) and
 *   a_i = exp(-sqrt(2) / sigma_i); one iteration filters every row left to right,
 *   J(n) = J(n) + a_i^t(n) (J(n - 1) - J(n)), then right to left,
 *   J(n) = J(n) + a_i^t(n + 1) (J(n + 1) - J(n)), then every column the same way, top to
 *   bottom and bottom to top.
 * C, out: [h][w][D] (out may equal C).  guide: [h][w] box sums of the left image. */
void orc_dt_aggregate(const double* C, int w, int h, int D, const int32_t* guide, double sigma_s, double sigma_r,
                      int iters, double* out) {
  const size_t n = (size_t)w * h * D;
  if (out != C)
    for (size_t i = 0; i < n; ++i) out[i] = C[i];
  const double ratio = sigma_s / sigma_r;
  for (int it = 1; it <= iters; ++it) {
    const double sig = sigma_s * sqrt(3.0) * pow(2.0, iters - it) / sqrt(pow(4.0, iters) - 1.0);
    const double lna = -sqrt(2.0) / sig; /* log a_i */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < h; ++y)
      for (int d = 0; d < D; ++d) {
        for (int x = 1; x < w; ++x) {
          const double t = 1.0 + ratio * fabs(guide[(size_t)y * w + x] / 16.0 - guide[(size_t)y * w + x - 1] / 16.0);
          const double a = exp(lna * t);
          double* J = out + ((size_t)y * w + x) * D + d;
          *J += a * (*(J - D) - *J);
        }
        for (int x = w - 2; x >= 0; --x) {
          const double t = 1.0 + ratio * fabs(guide[(size_t)y * w + x + 1] / 16.0 - guide[(size_t)y * w + x] / 16.0);
          const double a = exp(lna * t);
          double* J = out + ((size_t)y * w + x) * D + d;
          *J += a * (*(J + D) - *J);
        }
      }
#pragma omp parallel for schedule(static)
    for (int x = 0; x < w; ++x)
      for (int d = 0; d < D; ++d) {
        const size_t row = (size_t)w * D;
        for (int y = 1; y < h; ++y) {
          const double t = 1.0 + ratio * fabs(guide[(size_t)y * w + x] / 16.0 - guide[(size_t)(y - 1) * w + x] / 16.0);
          const double a = exp(lna * t);
          double* J = out + ((size_t)y * w + x) * D + d;
          *J += a * (*(J - row) - *J);
        }
        for (int y = h - 2; y >= 0; --y) {
          const double t = 1.0 + ratio * fabs(guide[(size_t)(y + 1) * w + x] / 16.0 - guide[(size_t)y * w + x] / 16.0);
          const double a = exp(lna * t);
          double* J = out + ((size_t)y * w + x) * D + d;
          *J += a * (*(J + row) - *J);
        }
      }
  }
}

/* ------------------------------------------------------------------ the paper's Table I network
 * Sec. III-B1 (Table I) and Sec. III-B2 (Eq. 8-11).  Readings (the paper leaves them open):
 *  - inputs at half resolution Hh x Wh = ceil(H/2) x ceil(W/2) ("quarter size" = a quarter of
 *    the pixels, Table I "H/2 * W/2"): X_1 = the left image's 2 x 2 box mean / 256 (the last row
 *    / column of an odd size clamped), X_0 = the coarse disparity map (quarter-size matcher, in
 *    coarse pixels) upsampled bilinearly x2 with half-pixel centres and clamped sources, times 4
 *    (full-resolution pixels), / 256 (Sec. III-B2: data normalised, factor 256);
 *  - every conv and deconv has a bias and "same" zero padding (2 for 5 x 5); stride-2 convs give
 *    ceil(n / 2); the 5 x 5 stride-2 deconvolutions give 2 n, cropped to the size of the level
 *    they return to (H/4, H/2, H); a 1 x 1 deconvolution is a 1 x 1 conv;
 *  - leaky ReLU with slope 0.1 after every layer except the mu / sigma heads and the output;
 *  - "mu & sigma" is one 1 x 1 conv with two output channels (channel 0 mu, 1 sigma);
 *  - the inputs of a layer listed as "A & B & ..." are concatenated along channels in that
 *    order; the decoder's residual blocks D_1_R, D_2_R are single 5 x 5 stride-1 convs;
 *  - Eq. 8 as printed: gaussian = (mu - 1) + eps exp(sigma - 1), eps ~ N(0, 1) (inference:
 *    eps = 0); the network's output Y is the normalised disparity, 256 Y the disparity in
 *    full-resolution pixels (no residual onto the input map: Table I feeds X_0 to the last
 *    layer instead).
 * Layers (index: name, input -> output channels, kernel, kind):
 *   0 FE_1 1->32 5 conv   1 FE_2 1->32 5 conv   2 EN_1 64->16 5 conv s2  3 EN_1_R 16->8 5 conv
 *   4 EN_2 24->32 5 conv s2  5 EN_2_R 32->16 5 conv  6 heads 48->2 1 conv  7 D_1 1->32 1 deconv
 *   8 D_1_R 80->16 5 conv  9 D_2 96->16 5 deconv s2  10 D_2_R 40->8 5 conv  11 D 48->16 5 deconv s2
 *   12 Y 81->1 5 deconv s2.  Parameters: per layer W[co][ky][kx][ci] then b[co]. */
static const int T1_CO[13] = {32, 32, 16, 8, 32, 16, 2, 32, 16, 16, 8, 16, 1};
static const int T1_CI[13] = {1, 1, 64, 16, 24, 32, 48, 1, 80, 96, 40, 48, 81};
static const int T1_K[13] = {5, 5, 5, 5, 5, 5, 1, 1, 5, 5, 5, 5, 5};

size_t orc_t1_param_offset(int l, int want_bias) {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += (size_t)T1_CO[i] * T1_K[i] * T1_K[i] * T1_CI[i] + T1_CO[i];
  if (want_bias) o += (size_t)T1_CO[l] * T1_K[l] * T1_K[l] * T1_CI[l];
  return o;
}

size_t orc_t1_param_count(void) { return orc_t1_param_offset(13, 0); }

/* Generic layer of the Table I network.  mode 0: conv stride 1, 1: conv stride 2, 2: deconv
 * stride 2 (out(oy, ox) += in(iy, ix) w(ky, kx) for oy = 2 iy + ky - pad, ox = 2 ix + kx - pad,
 * outputs outside [0, Ho) x [0, Wo) dropped: the 2n output cropped).  pad = ks / 2.
 * act 1: leaky ReLU 0.1. */
void orc_t1_layer(const double* in, int Hi, int Wi, int Ci, const float* wt, const float* b, int Co, int ks, int mode,
                  int Ho, int Wo, int act, double* out) {
  const int pad = ks / 2;
  for (size_t i = 0; i < (size_t)Ho * Wo * Co; ++i) out[i] = b[i % Co];
  if (mode < 2) {
    const int s = mode == 1 ? 2 : 1;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ho; ++y)
      for (int x = 0; x < Wo; ++x)
        for (int co = 0; co < Co; ++co) {
          double acc = 0.0;
          for (int ky = 0; ky < ks; ++ky) {
            const int iy = y * s + ky - pad;
            if (iy < 0 || iy >= Hi) continue;
            for (int kx = 0; kx < ks; ++kx) {
              const int ix = x * s + kx - pad;
              if (ix < 0 || ix >= Wi) continue;
              const double* ip = in + ((size_t)iy * Wi + ix) * Ci;
              const float* wp = wt + (((size_t)co * ks + ky) * ks + kx) * Ci;
              for (int ci = 0; ci < Ci; ++ci) acc += (double)wp[ci] * ip[ci];
            }
          }
          out[((size_t)y * Wo + x) * Co + co] += acc;
        }
  } else {
    /* scatter form, written as a gather per output row so that rows are independent */
#pragma omp parallel for schedule(static)
    for (int oy = 0; oy < Ho; ++oy)
      for (int iy = 0; iy < Hi; ++iy) {
        const int ky = oy - 2 * iy + pad;
        if (ky < 0 || ky >= ks) continue;
        for (int ix = 0; ix < Wi; ++ix)
          for (int kx = 0; kx < ks; ++kx) {
            const int ox = 2 * ix + kx - pad;
            if (ox < 0 || ox >= Wo) continue;
            const double* ip = in + ((size_t)iy * Wi + ix) * Ci;
            double* op = out + ((size_t)oy * Wo + ox) * Co;
            for (int co = 0; co < Co; ++co) {
              const float* wp = wt + (((size_t)co * ks + ky) * ks + kx) * Ci;
              double acc = 0.0;
              for (int ci = 0; ci < Ci; ++ci) acc += (double)wp[ci] * ip[ci];
              op[co] += acc;
            }
          }
      }
  }
  if (act)
    for (size_t i = 0; i < (size_t)Ho * Wo * Co; ++i)
      if (out[i] < 0) out[i] *= 0.1;
}

/* Network inputs at half resolution: X_0 (disparity) and X_1 (left image), see above. */
void orc_t1_inputs(const uint8_t* left, int W, int H, int pitch, const double* coarse, int w, int h, double* X0,
                   double* X1) {
  const int Wh = (W + 1) / 2, Hh = (H + 1) / 2;
  for (int y = 0; y < Hh; ++y)
    for (int x = 0; x < Wh; ++x) {
      const int y1 = 2 * y + 1 < H ? 2 * y + 1 : H - 1, x1 = 2 * x + 1 < W ? 2 * x + 1 : W - 1;
      const double s = (double)left[(size_t)(2 * y) * pitch + 2 * x] + left[(size_t)(2 * y) * pitch + x1] +
                       left[(size_t)y1 * pitch + 2 * x] + left[(size_t)y1 * pitch + x1];
      X1[(size_t)y * Wh + x] = s / 4.0 / 256.0;
      double sx = (x + 0.5) / 2.0 - 0.5, sy = (y + 0.5) / 2.0 - 0.5;
      if (sx < 0) sx = 0;
      if (sx > w - 1) sx = w - 1;
      if (sy < 0) sy = 0;
      if (sy > h - 1) sy = h - 1;
      const int a = (int)floor(sx), c = (int)floor(sy);
      const int a1 = a + 1 < w ? a + 1 : w - 1, c1 = c + 1 < h ? c + 1 : h - 1;
      const double fx = sx - a, fy = sy - c;
      const double top = (1 - fx) * coarse[(size_t)c * w + a] + fx * coarse[(size_t)c * w + a1];
      const double bot = (1 - fx) * coarse[(size_t)c1 * w + a] + fx * coarse[(size_t)c1 * w + a1];
      X0[(size_t)y * Wh + x] = 4.0 * ((1 - fy) * top + fy * bot) / 256.0;
    }
}

/* channel concatenation of up to four NHWC tensors of the same spatial size */
static double* t1_cat(size_t P, const double* a, int ca, const double* b, int cb, const double* c, int cc,
                      const double* d, int cd) {
  const int C = ca + cb + cc + cd;
  double* o = malloc(P * C * sizeof(double));
  for (size_t p = 0; p < P; ++p) {
    double* q = o + p * C;
    for (int i = 0; i < ca; ++i) *q++ = a[p * ca + i];
    for (int i = 0; i < cb; ++i) *q++ = b[p * cb + i];
    for (int i = 0; i < cc; ++i) *q++ = c[p * cc + i];
    for (int i = 0; i < cd; ++i) *q++ = d[p * cd + i];
  }
  return o;
}

/* Forward pass of the Table I network.  coarse: h x w map in coarse pixels (real valued);
 * eps: H8 x W8 noise or NULL (inference, eps = 0).  Y: H x W normalised disparity (256 Y in
 * pixels); mu, sigma: H8 x W8 (nullable).  acts (nullable): receives a copy of activation
 * `which` (0 FE_1, 1 FE_2, 2 EN_1, 3 EN_1_R, 4 EN_2, 5 EN_2_R, 6 heads, 7 D_1, 8 D_1_R, 9 D_2,
 * 10 D_2_R, 11 D, 12 X_0, 13 X_1). */
void orc_t1_forward(const float* params, const uint8_t* left, int W, int H, int pitch, const double* coarse, int w,
                    int h, const double* eps, double* Y, double* mu, double* sigma, int which, double* acts) {
  const int H2 = (H + 1) / 2, W2 = (W + 1) / 2, H4 = (H2 + 1) / 2, W4 = (W2 + 1) / 2, H8 = (H4 + 1) / 2,
            W8 = (W4 + 1) / 2;
  const size_t P2 = (size_t)H2 * W2, P4 = (size_t)H4 * W4, P8 = (size_t)H8 * W8;
#define T1W(l) (params + orc_t1_param_offset(l, 0))
#define T1B(l) (params + orc_t1_param_offset(l, 1))
  double* X0 = malloc(P2 * sizeof(double));
  double* X1 = malloc(P2 * sizeof(double));
  orc_t1_inputs(left, W, H, pitch, coarse, w, h, X0, X1);
  double* fe1 = malloc(P2 * 32 * sizeof(double));
  double* fe2 = malloc(P2 * 32 * sizeof(double));
  orc_t1_layer(X0, H2, W2, 1, T1W(0), T1B(0), 32, 5, 0, H2, W2, 1, fe1);
  orc_t1_layer(X1, H2, W2, 1, T1W(1), T1B(1), 32, 5, 0, H2, W2, 1, fe2);
  double* in = t1_cat(P2, fe1, 32, fe2, 32, NULL, 0, NULL, 0);
  double* en1 = malloc(P4 * 16 * sizeof(double));
  orc_t1_layer(in, H2, W2, 64, T1W(2), T1B(2), 16, 5, 1, H4, W4, 1, en1);
  free(in);
  double* en1r = malloc(P4 * 8 * sizeof(double));
  orc_t1_layer(en1, H4, W4, 16, T1W(3), T1B(3), 8, 5, 0, H4, W4, 1, en1r);
  in = t1_cat(P4, en1, 16, en1r, 8, NULL, 0, NULL, 0);
  double* en2 = malloc(P8 * 32 * sizeof(double));
  orc_t1_layer(in, H4, W4, 24, T1W(4), T1B(4), 32, 5, 1, H8, W8, 1, en2);
  free(in);
  double* en2r = malloc(P8 * 16 * sizeof(double));
  orc_t1_layer(en2, H8, W8, 32, T1W(5), T1B(5), 16, 5, 0, H8, W8, 1, en2r);
  in = t1_cat(P8, en2, 32, en2r, 16, NULL, 0, NULL, 0);
  double* heads = malloc(P8 * 2 * sizeof(double));
  orc_t1_layer(in, H8, W8, 48, T1W(6), T1B(6), 2, 1, 0, H8, W8, 0, heads);
  free(in);
  double* g = malloc(P8 * sizeof(double));
  for (size_t p = 0; p < P8; ++p) {
    const double m = heads[2 * p], s = heads[2 * p + 1];
    g[p] = (m - 1.0) + (eps ? eps[p] * exp(s - 1.0) : 0.0);
    if (mu) mu[p] = m;
    if (sigma) sigma[p] = s;
  }
  double* d1 = malloc(P8 * 32 * sizeof(double));
  orc_t1_layer(g, H8, W8, 1, T1W(7), T1B(7), 32, 1, 0, H8, W8, 1, d1);
  in = t1_cat(P8, d1, 32, en2, 32, en2r, 16, NULL, 0);
  double* d1r = malloc(P8 * 16 * sizeof(double));
  orc_t1_layer(in, H8, W8, 80, T1W(8), T1B(8), 16, 5, 0, H8, W8, 1, d1r);
  free(in);
  in = t1_cat(P8, d1, 32, en2, 32, en2r, 16, d1r, 16);
  double* d2 = malloc(P4 * 16 * sizeof(double));
  orc_t1_layer(in, H8, W8, 96, T1W(9), T1B(9), 16, 5, 2, H4, W4, 1, d2);
  free(in);
  in = t1_cat(P4, d2, 16, en1, 16, en1r, 8, NULL, 0);
  double* d2r = malloc(P4 * 8 * sizeof(double));
  orc_t1_layer(in, H4, W4, 40, T1W(10), T1B(10), 8, 5, 0, H4, W4, 1, d2r);
  free(in);
  in = t1_cat(P4, d2, 16, en1, 16, en1r, 8, d2r, 8);
  double* dd = malloc(P2 * 16 * sizeof(double));
  orc_t1_layer(in, H4, W4, 48, T1W(11), T1B(11), 16, 5, 2, H2, W2, 1, dd);
  free(in);
  in = t1_cat(P2, dd, 16, X0, 1, fe1, 32, fe2, 32);
  orc_t1_layer(in, H2, W2, 81, T1W(12), T1B(12), 1, 5, 2, H, W, 0, Y);
  free(in);
  if (acts) {
    const double* src[14] = {fe1, fe2, en1, en1r, en2, en2r, heads, d1, d1r, d2, d2r, dd, X0, X1};
    const size_t n[14] = {P2 * 32, P2 * 32, P4 * 16, P4 * 8, P8 * 32, P8 * 16, P8 * 2, P8 * 32, P8 * 16, P4 * 16,
                          P4 * 8, P2 * 16, P2, P2};
    if (which >= 0 && which < 14) memcpy(acts, src[which], n[which] * sizeof(double));
  }
  free(X0); free(X1); free(fe1); free(fe2); free(en1); free(en1r); free(en2); free(en2r); free(heads); free(g);
  free(d1); free(d1r); free(d2); free(d2r); free(dd);
#undef T1W
#undef T1B
}

/* Loss of Sec. III-B2 for the Table I network (Eq. 9-11), readings:
 *   Loss_1 (Eq. 10): (sum over non-occluded pixels of |gt / 256 - Y| + sum over all pixels of
 *            |gt / 256 - Y|) / (number of pixels): non-occluded pixels weigh twice the
 *            occluded ones, as the text states (gt_noc: the ground truth where the pixel is
 *            visible in both views, gt_occ: everywhere);
 *   Loss_2 (Eq. 11, garbled): the KL divergence of N(mu - 1, exp(sigma - 1)^2) (the
 *            distribution Eq. 8 samples) from N(0, 1), 0.5 ((mu - 1)^2 + exp(2 (sigma - 1)) - 1
 *            - 2 (sigma - 1)), averaged over the latent elements (zero at mu = sigma = 1);
 *   Loss_total (Eq. 9) = 256 (Loss_1 + Loss_2).
 * noc[p] != 0 marks a non-occluded pixel.  parts (nullable): Loss_1, Loss_2. */
double orc_t1_loss(const double* Y, const float* gt, const uint8_t* noc, size_t P, const double* mu,
                   const double* sigma, size_t nl, double* parts) {
  double l1 = 0.0, l2 = 0.0;
  for (size_t p = 0; p < P; ++p) {
    const double e = fabs((double)gt[p] / 256.0 - Y[p]);
    l1 += noc[p] ? 2.0 * e : e;
  }
  l1 /= (double)P;
  for (size_t i = 0; i < nl; ++i) {
    const double m = mu[i] - 1.0, s = sigma[i] - 1.0;
    l2 += 0.5 * (m * m + exp(2.0 * s) - 1.0 - 2.0 * s);
  }
  l2 /= (double)nl;
  if (parts) {
    parts[0] = l1;
    parts[1] = l2;
  }
  return 256.0 * (l1 + l2);
}

/* ------------------------------------------------------------------ quantised refinement
 * Sec. V (future work: "compress the network through quantization").  The paper gives no
 * scheme; the one defined here is the FP8 form of this build, written out step by step:
 *   - number format E4M3 (1 sign, 4 exponent bits with bias 7, 3 mantissa bits, subnormals,
 *     largest finite 448, no infinity); rounding to nearest, ties to even, saturating at 448;
 *   - weights of a tensor-core layer quantised per output channel co: scale s[co] =
 *     max |v| / 448 over the values v the layer multiplies (FP32, 1 if all are zero), codes
 *     e4m3(v / s[co]) (the division in FP32);  for the nearest-x2 decoder layers the values
 *     are the phase-folded weights (the 3 x 3 kernel rows / columns {0} and {1, 2} for phase
 *     0, {0, 1} and {2} for phase 1, summed in FP32 in row-major tap order), for stride-2
 *     and 1 x 1 layers the weights themselves;
 *   - the quantised layers are enc2, enc3, the latent head, dec1 and dec2; their inputs (e1,
 *     e2, e3, z, d1) are rounded to E4M3 with scale 1, e1 first to BF16 (the first layer's
 *     output format);
 *   - the last decoder layer stays as in the BF16 form: d2 is rounded to BF16, dec3 uses the
 *     FP32 weights (phase-folded sums as above, unquantised) and d3 is rounded to BF16 (the
 *     final conv's input format);
 *   - a layer's output: relu(s[co] * sum(a_code * w_code) + b[co]) (no relu after the
 *     latent head); inference uses z = mu;
 *   - decoder border pixels left wrong by the phase folding (the last output row of an odd
 *     height, the last column of an odd width) use the 3 x 3 weights unfolded, quantised
 *     per output channel the same way, on the cropped up-sampled input;
 *   - the first layer (2 input channels) and the final conv keep FP32 weights (FP64 here),
 *     as in the BF16 form.
 * quant = 0 skips every rounding (codes = values, scales 1): the result must then equal
 * orc_refine_forward up to the order of the sums. */

/* E4M3 round to nearest even, saturating to +-448. */
double orc_e4m3(double x) {
  if (x != x) return x;
  const double a = fabs(x);
  if (a == 0.0) return x;
  if (a >= 448.0) return x < 0 ? -448.0 : 448.0;
  int e;
  frexp(a, &e);            /* a = f 2^e, f in [0.5, 1): the leading bit has weight 2^(e-1) */
  int q = e - 1 - 3;       /* quantum of a normal number: 3 mantissa bits below the leading one */
  if (q < -9) q = -9;      /* subnormal quantum 2^-9 (exponent field 0) */
  const double r = ldexp(nearbyint(ldexp(a, -q)), q);  /* default rounding mode: to nearest even */
  return x < 0 ? -(r > 448.0 ? 448.0 : r) : (r > 448.0 ? 448.0 : r);
}

/* BF16 round to nearest even of a double (through FP32, as the GPU stores FP32 results). */
static double orc_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return f;
  u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
  memcpy(&f, &u, 4);
  return f;
}

/* phase-folded weights of a nearest-x2 + 3 x 3 layer, FP32 sums in row-major tap order:
 * Wf[((ph * 4 + t) * co_n + co) * ci_n + ci], ph = 2 py + px, t = 2 a + b */
static void fold_weights(const float* Wt, int co_n, int ci_n, float* Wf) {
  for (int ph = 0; ph < 4; ++ph)
    for (int t = 0; t < 4; ++t)
      for (int co = 0; co < co_n; ++co)
        for (int ci = 0; ci < ci_n; ++ci) {
          const int py = ph >> 1, px = ph & 1, a = t >> 1, b = t & 1;
          const int ky0 = py == 0 ? (a == 0 ? 0 : 1) : (a == 0 ? 0 : 2);
          const int ky1 = py == 0 ? (a == 0 ? 0 : 2) : (a == 0 ? 1 : 2);
          const int kx0 = px == 0 ? (b == 0 ? 0 : 1) : (b == 0 ? 0 : 2);
          const int kx1 = px == 0 ? (b == 0 ? 0 : 2) : (b == 0 ? 1 : 2);
          float v = 0.f;
          for (int ky = ky0; ky <= ky1; ++ky)
            for (int kx = kx0; kx <= kx1; ++kx) v += Wt[((size_t)co * 9 + ky * 3 + kx) * ci_n + ci];
          Wf[((size_t)(ph * 4 + t) * co_n + co) * ci_n + ci] = v;
        }
}

/* per-output-channel scales and codes of n_per_co values per channel laid out
 * [group][co][...]: values v(co, j) at vals[(g * co_n + co) * per + j] for g < groups */
static void quantise_per_co(const float* vals, int groups, int co_n, int per, int quant, float* scale, double* codes) {
  for (int co = 0; co < co_n; ++co) {
    float m = 0.f;
    for (int g = 0; g < groups; ++g)
      for (int j = 0; j < per; ++j) {
        const float a = fabsf(vals[((size_t)g * co_n + co) * per + j]);
        if (a > m) m = a;
      }
    const float s = (quant && m > 0.f) ? m / 448.0f : 1.0f;
    scale[co] = s;
    for (int g = 0; g < groups; ++g)
      for (int j = 0; j < per; ++j) {
        const size_t i = ((size_t)g * co_n + co) * per + j;
        codes[i] = quant ? orc_e4m3((double)(vals[i] / s)) : (double)vals[i];
      }
  }
}

/* one quantised conv layer: mode 0 stride 2 (3 x 3, pad 1), 1 pointwise (1 x 1), 2 nearest x2
 * + crop + 3 x 3 (folded interior, unfolded border). in: [Hi][Wi][Ci] codes; out values. */
static void qconv(const double* in, int Hi, int Wi, int Ci, const float* Wt, const float* bias, int Co, int mode,
                  int Ho, int Wo, int relu, int quant, double* out) {
  if (mode != 2) {
    const int ks = mode == 0 ? 3 : 1, per = ks * ks * Ci;
    float* sc = malloc(sizeof(float) * Co);
    double* q = malloc(sizeof(double) * Co * per);
    quantise_per_co(Wt, 1, Co, per, quant, sc, q);
#pragma omp parallel for schedule(static)
    for (int y = 0; y < Ho; ++y)
      for (int x = 0; x < Wo; ++x)
        for (int co = 0; co < Co; ++co) {
          double acc = 0.0;
          for (int ky = 0; ky < ks; ++ky)
            for (int kx = 0; kx < ks; ++kx) {
              const int iy = mode == 0 ? 2 * y + ky - 1 : y, ix = mode == 0 ? 2 * x + kx - 1 : x;
              if (iy < 0 || ix < 0 || iy >= Hi || ix >= Wi) continue;
              const double* ip = in + ((size_t)iy * Wi + ix) * Ci;
              const double* wp = q + (size_t)co * per + (ky * ks + kx) * Ci;
              for (int ci = 0; ci < Ci; ++ci) acc += ip[ci] * wp[ci];
            }
          double v = (double)sc[co] * acc + (double)bias[co];
          if (relu && v < 0) v = 0;
          out[((size_t)y * Wo + x) * Co + co] = v;
        }
    free(sc);
    free(q);
    return;
  }
  float* Wf = malloc(sizeof(float) * 16 * Co * Ci);
  fold_weights(Wt, Co, Ci, Wf);
  float* scf = malloc(sizeof(float) * Co);
  float* scu = malloc(sizeof(float) * Co);
  double* qf = malloc(sizeof(double) * 16 * Co * Ci);
  double* qu = malloc(sizeof(double) * 9 * Co * Ci);
  /* folded values of one channel: 16 groups (phase, tap) of Ci each */
  quantise_per_co(Wf, 16, Co, Ci, quant, scf, qf);
  quantise_per_co(Wt, 1, Co, 9 * Ci, quant, scu, qu);
#pragma omp parallel for schedule(static)
  for (int oy = 0; oy < Ho; ++oy)
    for (int ox = 0; ox < Wo; ++ox) {
      const int border = ((Ho & 1) && oy == Ho - 1) || ((Wo & 1) && ox == Wo - 1);
      for (int co = 0; co < Co; ++co) {
        double acc = 0.0, s;
        if (border) {
          for (int ky = 0; ky < 3; ++ky)
            for (int kx = 0; kx < 3; ++kx) {
              const int vy = oy + ky - 1, vx = ox + kx - 1;
              if (vy < 0 || vx < 0 || vy >= Ho || vx >= Wo) continue;
              const double* ip = in + ((size_t)(vy / 2) * Wi + vx / 2) * Ci;
              const double* wp = qu + ((size_t)co * 9 + ky * 3 + kx) * Ci;
              for (int ci = 0; ci < Ci; ++ci) acc += ip[ci] * wp[ci];
            }
          s = scu[co];
        } else {
          const int py = oy & 1, px = ox & 1, i = oy >> 1, j = ox >> 1, ph = 2 * py + px;
          for (int t = 0; t < 4; ++t) {
            const int a = t >> 1, b = t & 1, iy = i + py + a - 1, ix = j + px + b - 1;
            if (iy < 0 || ix < 0 || iy >= Hi || ix >= Wi) continue;
            const double* ip = in + ((size_t)iy * Wi + ix) * Ci;
            const double* wp = qf + ((size_t)(ph * 4 + t) * Co + co) * Ci;
            for (int ci = 0; ci < Ci; ++ci) acc += ip[ci] * wp[ci];
          }
          s = scf[co];
        }
        double v = s * acc + (double)bias[co];
        if (relu && v < 0) v = 0;
        out[((size_t)oy * Wo + ox) * Co + co] = v;
      }
    }
  free(Wf); free(scf); free(scu); free(qf); free(qu);
}

static void round_act(double* a, size_t n, int quant, int bf16_first) {
  if (!quant) return;
  for (size_t i = 0; i < n; ++i) a[i] = orc_e4m3(bf16_first ? orc_bf16(a[i]) : a[i]);
}

/* One layer of the FP8 form on its own: in [Hi][Wi][Ci] (the values the previous layer passed
 * on), the layer's FP32 weights W[co][ky][kx][ci] and bias; mode 0 stride 2 (3 x 3, pad 1),
 * 1 pointwise, 2 nearest x2 + crop + 3 x 3; weights quantised per output channel as in
 * orc_refine_forward_q when quant_w (else the FP32 values, as the form's last decoder layer);
 * out_round 0 passes the values on, 1 rounds them to E4M3, 2 to BF16. */
void orc_qconv_layer(const double* in, int Hi, int Wi, int Ci, const float* Wt, const float* bias, int Co, int mode,
                     int Ho, int Wo, int relu, int quant_w, int out_round, double* out) {
  qconv(in, Hi, Wi, Ci, Wt, bias, Co, mode, Ho, Wo, relu, quant_w, out);
  const size_t n = (size_t)Ho * Wo * Co;
  if (out_round == 1) round_act(out, n, 1, 0);
  if (out_round == 2)
    for (size_t i = 0; i < n; ++i) out[i] = orc_bf16(out[i]);
}

/* The FP8 form's refinement (inference, z = mu); outputs as orc_refine_activation /
 * orc_refine_forward: Y [H*W]; act (nullable) receives activation `which` (0 e1 .. 6 d3, the
 * values each layer passes on: codes for e1-d1, BF16 values for d2 and d3). */
void orc_refine_forward_q(const int* widths7, const float* params, const uint8_t* left, int W, int H, int pitch,
                          const double* coarse, int w, int h, int quant, double* Y, int which, double* act) {
  orc_net n = {{widths7[0], widths7[1], widths7[2]}, widths7[3], {widths7[4], widths7[5], widths7[6]}};
  orc_acts a;
  acts_alloc(&n, H, W, &a);
  int co, ci, ks;
  orc_upsample4(coarse, w, h, W, H, a.U);
  for (int yy = 0; yy < H; ++yy)
    for (int xx = 0; xx < W; ++xx) {
      a.x0[((size_t)yy * W + xx) * 2 + 0] = left[(size_t)yy * pitch + xx] / 256.0;
      a.x0[((size_t)yy * W + xx) * 2 + 1] = a.U[(size_t)yy * W + xx] / 256.0;
    }
  const size_t P0 = (size_t)H * W, P1 = (size_t)a.H1 * a.W1, P2 = (size_t)a.H2 * a.W2, P3 = (size_t)a.H3 * a.W3;
  layer_dims(&n, L_ENC1, &co, &ci, &ks);
  orc_conv2d(a.x0, H, W, 2, Wl(params, widths7, L_ENC1), Bl(params, widths7, L_ENC1), co, 3, 2, 1, 0, a.H1, a.W1, 1,
             a.e1);
  round_act(a.e1, P1 * n.enc[0], quant, 1);
  qconv(a.e1, a.H1, a.W1, n.enc[0], Wl(params, widths7, L_ENC2), Bl(params, widths7, L_ENC2), n.enc[1], 0, a.H2, a.W2, 1,
        quant, a.e2);
  round_act(a.e2, P2 * n.enc[1], quant, 0);
  qconv(a.e2, a.H2, a.W2, n.enc[1], Wl(params, widths7, L_ENC3), Bl(params, widths7, L_ENC3), n.enc[2], 0, a.H3, a.W3, 1,
        quant, a.e3);
  round_act(a.e3, P3 * n.enc[2], quant, 0);
  qconv(a.e3, a.H3, a.W3, n.enc[2], Wl(params, widths7, L_MU), Bl(params, widths7, L_MU), n.lat, 1, a.H3, a.W3, 0, quant,
        a.z);
  round_act(a.z, P3 * n.lat, quant, 0);
  qconv(a.z, a.H3, a.W3, n.lat, Wl(params, widths7, L_DEC1), Bl(params, widths7, L_DEC1), n.dec[0], 2, a.H2, a.W2, 1,
        quant, a.d1);
  round_act(a.d1, P2 * n.dec[0], quant, 0);
  qconv(a.d1, a.H2, a.W2, n.dec[0], Wl(params, widths7, L_DEC2), Bl(params, widths7, L_DEC2), n.dec[1], 2, a.H1, a.W1, 1,
        quant, a.d2);
  if (quant)
    for (size_t i = 0; i < P1 * n.dec[1]; ++i) a.d2[i] = orc_bf16(a.d2[i]);
  qconv(a.d2, a.H1, a.W1, n.dec[1], Wl(params, widths7, L_DEC3), Bl(params, widths7, L_DEC3), n.dec[2], 2, H, W, 1, 0,
        a.d3);
  if (quant)
    for (size_t i = 0; i < P0 * n.dec[2]; ++i) a.d3[i] = orc_bf16(a.d3[i]);
  orc_conv2d(a.d3, H, W, n.dec[2], Wl(params, widths7, L_FINAL), Bl(params, widths7, L_FINAL), 1, 3, 1, 1, 0, H, W, 0,
             a.Y);
  for (size_t p = 0; p < P0; ++p) a.Y[p] += a.U[p];
  if (Y) memcpy(Y, a.Y, P0 * sizeof(double));
  if (act && which >= 0 && which <= 6) {
    const double* src[7] = {a.e1, a.e2, a.e3, a.z, a.d1, a.d2, a.d3};
    const size_t nn[7] = {P1 * n.enc[0], P2 * n.enc[1], P3 * n.enc[2], P3 * n.lat, P2 * n.dec[0], P1 * n.dec[1],
                          P0 * n.dec[2]};
    memcpy(act, src[which], nn[which] * sizeof(double));
  }
  acts_free(&a);
}
