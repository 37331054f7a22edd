// sv_internal.cuh -- internal declarations shared by the CUDA translation units of
// the StereoVAE library (context, device descriptors, kernel launchers).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <array>
#include <cstdint>
#include <cstring>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/stereovae.h"

namespace sv {

// ------------------------------------------------------------------ coarse stage
// Device descriptor of one pair for the coarse matcher.
struct ZPair {
  const uint8_t* L;
  const uint8_t* R;
  int W, H, pitch, D;
  int w, h;          // coarse size = (W / 4, H / 4)
  int16_t* disp;     // [h][w]
  float* best;       // [h][w] or nullptr
  float* second;     // [h][w] or nullptr
  float* cost;       // [h][w][D] cost volume 1 - rho (2 where x - d < 0), or nullptr
};

// One CTA job: rows [y0, y0 + kZnccTY) and columns [x0, x0 + group width) of a pair.
struct ZJob {
  int pair, y0, x0, pad;
};

constexpr int kZnccTY = 8;      // coarse rows per job
constexpr int kZnccWarps = 8;   // warps per CTA; each owns a column tile of TX(KD) columns

inline int zncc_kd(int D) { return (D + 31) / 32; }
inline int zncc_tx(int kd) { return kd == 1 ? 32 : kd == 2 ? 20 : kd == 3 ? 16 : 12; }

// Shared-memory layout of one ZNCC job (window radius r, disparity count D, tile TX).
struct ZLayout {
  int nlc, nrc, gx, nrs;  // staged left / right columns, job width, right-window columns
  size_t off_sl, off_sr, off_suml, off_invl, off_statr, off_cs, off_cs2, total;
};
__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }
__host__ __device__ inline ZLayout zlayout(int r, int D, int tx) {
  ZLayout z;
  const int TY = kZnccTY;
  z.gx = kZnccWarps * tx;
  z.nlc = z.gx + 2 * r;
  z.nrc = z.gx + 2 * r + D - 1;
  z.nrs = z.gx + D - 1;
  size_t o = 0;
  z.off_sl = o; o = align16(o + sizeof(uint16_t) * (TY + 2 * r) * z.nlc);
  z.off_sr = o; o = align16(o + sizeof(uint16_t) * (TY + 2 * r) * z.nrc);
  z.off_suml = o; o = align16(o + sizeof(int) * TY * z.gx);
  z.off_invl = o; o = align16(o + sizeof(float) * TY * z.gx);
  z.off_statr = o; o = align16(o + 2 * sizeof(int) * TY * z.nrs);  // {sum, 1/sigma} per right window
  z.off_cs = o; o = align16(o + sizeof(int) * TY * z.nrc);
  z.off_cs2 = o; o = align16(o + sizeof(unsigned) * TY * z.nrc);
  z.total = o;
  return z;
}
inline size_t zncc_smem_bytes(int r, int D) { return zlayout(r, D, zncc_tx(zncc_kd(D))).total; }

// Fused downsample + ZNCC + WTA over the given jobs, one entry per window radius
// r = 1..7 (each compiled in its own translation unit).
// mode 0: disparities only; 1: also the best / second scores of the pairs that ask for them;
// 2: also the cost volume (the pairs' cost pointers are set).
#define SV_ZNCC_DECL(r)                                                                              \
  cudaError_t launch_zncc_wta_r##r(const ZPair* d_pairs, const ZJob* d_jobs, int n_jobs, int maxD, \
                                   int mode, cudaStream_t st);
SV_ZNCC_DECL(1) SV_ZNCC_DECL(2) SV_ZNCC_DECL(3) SV_ZNCC_DECL(4) SV_ZNCC_DECL(5) SV_ZNCC_DECL(6) SV_ZNCC_DECL(7)
inline cudaError_t launch_zncc_wta(const ZPair* p, const ZJob* j, int n, int r, int maxD, cudaStream_t st,
                                   int mode) {
  switch (r) {
    case 1: return launch_zncc_wta_r1(p, j, n, maxD, mode, st);
    case 2: return launch_zncc_wta_r2(p, j, n, maxD, mode, st);
    case 3: return launch_zncc_wta_r3(p, j, n, maxD, mode, st);
    case 4: return launch_zncc_wta_r4(p, j, n, maxD, mode, st);
    case 5: return launch_zncc_wta_r5(p, j, n, maxD, mode, st);
    case 6: return launch_zncc_wta_r6(p, j, n, maxD, mode, st);
    case 7: return launch_zncc_wta_r7(p, j, n, maxD, mode, st);
  }
  return cudaErrorInvalidValue;
}

// ------------------------------------------------------------------ refinement
enum Layer { L_ENC1 = 0, L_ENC2, L_ENC3, L_MU, L_LV, L_DEC1, L_DEC2, L_DEC3, L_FINAL, L_COUNT };

struct NetDims {
  int enc[3], lat, dec[3];
  int cout(int l) const;
  int cin(int l) const;
  int ks(int l) const;
  size_t w_off(int l) const;   // offset of W of layer l in the flat vector
  size_t b_off(int l) const;   // offset of b
  size_t count() const;
};

// Spatial sizes of the four levels of a W x H input.
struct Levels {
  int H[4], W[4];
  explicit Levels(int H0 = 0, int W0 = 0) {
    H[0] = H0; W[0] = W0;
    for (int i = 1; i < 4; ++i) { H[i] = (H[i - 1] + 1) / 2; W[i] = (W[i - 1] + 1) / 2; }
  }
};

// Direct (CUDA-core) convolution arguments, element type T (float or double).
// Activations NHWC; weights canonical [cout][ks][ks][cin].
enum ConvMode { CM_S1 = 0, CM_S2 = 1, CM_UP2 = 2 };
template <typename T>
struct DirectConvArgs {
  const T* in; int Hi, Wi, Ci;
  const T* wt; const T* bias; int Co;
  int Ho, Wo;
  int relu;
  T* out;
};

template <typename T>
cudaError_t launch_conv_direct(const DirectConvArgs<T>& a, int mode, int ks, cudaStream_t st);

// enc1 with the network input built on the fly: x0 = (L / 256, U / 256), U = 4 *
// bilinear(coarse).  CoarseT = int16_t (inference) or T (training).
template <typename T, typename CoarseT>
cudaError_t launch_enc1(const uint8_t* L, int pitch, int W, int H, const CoarseT* coarse, int w, int h,
                        const T* wt, const T* bias, int Co, T* out, cudaStream_t st);

// final 3x3 conv (cin -> 1) + bias + U (recomputed bilinear) -> Y
template <typename T, typename CoarseT, typename OutT>
cudaError_t launch_final(const T* in, int W, int H, int Ci, const T* wt, const T* bias, const CoarseT* coarse,
                         int w, int h, OutT* Y, cudaStream_t st);

// Per-pair descriptors of the batched CUDA-core layers of the tensor-core form.
struct alignas(128) EdgePair {
  const uint8_t* L;
  int pitch, W, H, w, h;
  const int16_t* coarse;    // integer coarse map (inference), or
  const float* coarse_f;    // real-valued coarse map (training) when non-null
  __nv_bfloat16* e1;        // enc1 output [H1][W1][C1]
  const __nv_bfloat16* d3;  // last decoder output [H][W][C]
  float* Y;                 // refined disparity [H][W]
  uint8_t* e1q;             // FP8 form: the tensor-core enc1 writes E4M3 codes of e1 here instead
  CUtensorMap d3_map;       // TMA view of d3 for the final conv (final_staged_by_tma(C))
};
// Row copy between device-accessible buffers (host_io.cu): `height` rows of `width`
// elements of elem_bytes bytes.
struct HostRowCopy {
  const unsigned char* src;
  unsigned char* dst;
  int spitch, dpitch, width, height;  // pitches in bytes
};
cudaError_t launch_copy_rows(const HostRowCopy* jobs, int njobs, int max_rows, int elem_bytes, cudaStream_t st);

// U = 4 x bilinear(coarse) at full-resolution pixel (X, Y), half-pixel centres, source
// clamped to the coarse map (Sec. IV-C "linear scaling", reading N1), FP32.
template <typename CT>
__device__ __forceinline__ float upsample4_f(const CT* __restrict__ c, int w, int h, int X, int Y) {
  float sx = (float)X * 0.25f - 0.375f, sy = (float)Y * 0.25f - 0.375f;
  sx = fminf(fmaxf(sx, 0.f), (float)(w - 1));
  sy = fminf(fmaxf(sy, 0.f), (float)(h - 1));
  const int x0 = (int)sx, y0 = (int)sy;
  const int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
  const float fx = sx - (float)x0, fy = sy - (float)y0;
  const float top = (1.f - fx) * (float)c[(size_t)y0 * w + x0] + fx * (float)c[(size_t)y0 * w + x1];
  const float bot = (1.f - fx) * (float)c[(size_t)y1 * w + x0] + fx * (float)c[(size_t)y1 * w + x1];
  return 4.f * ((1.f - fy) * top + fy * bot);
}

// Final conv of the tensor-core form: widths with the register-blocked kernel stage their
// (rows + 2) x 34 x C input tile with one TMA box; its height in output rows per block.
inline bool final_staged_by_tma(int C) { return C == 16 || C == 32 || C == 64 || C == 128; }
inline int final_tile_rows(int C) { return 16 * (C / 8 >= 8 ? 1 : 8 / (C / 8)); }
struct UpFixPair {          // one decoder layer of one pair (input, output, sizes)
  const __nv_bfloat16* in;
  __nv_bfloat16* out;
  int Hi, Wi, Ho, Wo, Hu, Wu;
};
// enc1 for every pair of a call; `tensor`: the tensor-core kernel where C1 allows (16, 32,
// 64), whose bounded wait records code 7 in `err`.
cudaError_t launch_edge_enc1(const EdgePair* pairs, int n, int maxW1, int maxH1, const float* W, const float* B, int C1,
                             int* err, long long spin, bool tensor, cudaStream_t st);
cudaError_t launch_edge_final(const EdgePair* pairs, int n, int maxW, int maxH, const float* W, const float* B, int C,
                              int* err, long long spin, cudaStream_t st);
// Border pixels of a cropped nearest-x2 + 3x3 conv output that the 4-phase form folds
// wrongly: the last row when Ho is odd, the last column (above that row) when Wo is odd.
// The fix kernel takes them in segments of kUpFixSeg pixels, one block per segment.
constexpr int kUpFixSeg = 64;
inline int upfix_segments(int Ho, int Wo) {
  const int nrow = (Ho & 1) ? Wo : 0, ncol = (Wo & 1) ? Ho - (Ho & 1) : 0;
  return (nrow + kUpFixSeg - 1) / kUpFixSeg + (ncol + kUpFixSeg - 1) / kUpFixSeg;
}
cudaError_t launch_edge_up2fix(const UpFixPair* pairs, int n, int max_segments, const __nv_bfloat16* Wb,
                               const float* bias, int cin, int cout, int relu, cudaStream_t st);

// FP8 form: border recompute on E4M3 input codes with E4M3 unfolded weights and their
// per-output-channel scale (output E4M3 codes, or BF16 when out_f8 = 0); E4M3 codes of a
// BF16 tensor.
cudaError_t launch_edge_up2fix_f8(const UpFixPair* pairs, int n, int max_segments, const uint8_t* Wq,
                                  const float* wscale, const float* bias, int cin, int cout, int relu, int out_f8,
                                  cudaStream_t st);
cudaError_t launch_bf16_to_e4m3(const __nv_bfloat16* a, uint8_t* b, size_t n, cudaStream_t st);

// Training latent of the tensor-core form: mu, logvar (FP32, caller's buffers) from BF16
// e3 with FP32 weights, z = mu + eps exp(logvar / 2) stored as BF16 for the decoder.
cudaError_t launch_train_latent_bf16(const __nv_bfloat16* e3, int P, int Ci, const float* wmu, const float* bmu,
                                     const float* wlv, const float* blv, int lat, const float* eps, float* mu,
                                     float* lv, __nv_bfloat16* z, cudaStream_t st);
cudaError_t launch_bf16_to_f32(const __nv_bfloat16* a, float* b, size_t n, cudaStream_t st);

// FP32 gradients of a conv read through its input view (bwd_tiled.cu): dgrad writes (or adds
// to) the input gradient, masked by the input activation's ReLU; wgrad adds the weight and
// bias gradients, reducing per-CTA partial sums (slots, wgrad_slot_floats floats) in a fixed
// order.
cudaError_t launch_dgrad_tiled(const float* gout, int Ho, int Wo, int Co, const float* w, int ks, int mode,
                               const float* mask_act, int Hi, int Wi, int Ci, int accumulate, float* gin,
                               cudaStream_t st);
cudaError_t launch_wgrad_tiled(const float* gout, int Ho, int Wo, int Co, const float* in, int Hi, int Wi, int Ci,
                               int ks, int mode, float* gw, float* gb, float* slots, size_t slot_cap,
                               cudaStream_t st);
size_t wgrad_slot_floats(int Ho, int Wo, int Co, int Ci, int ks);

// latent heads on the H3 x W3 grid: mu = 1x1(e3) + b; optionally logvar and z = mu + eps * exp(lv / 2).
template <typename T>
cudaError_t launch_latent(const T* e3, int H3, int W3, int Ci, const T* wmu, const T* bmu, const T* wlv, const T* blv,
                          int lat, const T* eps, T* mu, T* lv, T* z, cudaStream_t st);

}  // namespace sv
