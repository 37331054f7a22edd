// bwd_tiled.cu -- weight and input gradients of the refinement convolutions in FP32, tiled
// through shared memory (the differentiation form's hot kernels).
//
// Both read the forward convolution through its input view V (conv_direct.cu): stride 1,
// stride 2, or nearest x2 upsampling cropped to the output size, zero outside.
//
//   wgrad_tiled   dW[co][ky][kx][ci] = sum over output pixels p of dY(p, co) V(p S + k - pad, ci)
//                 and db[co] = sum_p dY(p, co): a GEMM whose reduction runs over the pixels.
//                 A CTA owns a block of COB output x CIB input channels and walks a fixed
//                 set of 8 x 16 output tiles, staging dY of the tile and the view patch the
//                 tile's taps read; a thread accumulates 4 output x 2 input channels for
//                 every tap in registers.  Each CTA writes its partial sums to its own slot;
//                 wgrad_reduce adds the slots in CTA order to the gradient (deterministic,
//                 no atomics).
//   dgrad_tiled   dX(i, ci) = sum over the view positions v of input pixel i (one, or the
//                 two-by-two block of the upsampled grid, cropped) and the taps k with
//                 o = (v + pad - k) / S an output pixel: dY(o, co) W[co][k][ci]; times the
//                 ReLU mask of the input.  A CTA owns 8 x 16 input pixels and CIT input
//                 channels and stages dY of the output region they reach (zero outside
//                 the output) and the weights, eight output channels at a time.
#include <algorithm>

#include "sv_internal.cuh"

namespace sv {

namespace {

constexpr int kWTH = 8, kWTW = 16;  // output pixels per wgrad tile
constexpr int kDTH = 8, kDTW = 16;  // input pixels per dgrad tile

__host__ __device__ constexpr int view_stride(int mode) { return mode == CM_S2 ? 2 : 1; }

__device__ __forceinline__ int floor_div(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

template <int MODE, int KS>
struct WgradGeo {
  static constexpr int S = view_stride(MODE), PAD = KS / 2;
  static constexpr int PR = (kWTH - 1) * S + KS, PC = (kWTW - 1) * S + KS;
};

template <int MODE, int KS, int COB, int CIB>
__global__ void __launch_bounds__(COB / 4 * CIB / 2)
wgrad_tiled(const float* __restrict__ gout, int Ho, int Wo, int Co, const float* __restrict__ in, int Hi, int Wi, int Ci,
            float* __restrict__ slots, int nW) {
  using G = WgradGeo<MODE, KS>;
  constexpr int S = G::S, PAD = G::PAD, PR = G::PR, PC = G::PC, NT = COB / 4 * CIB / 2, NP = kWTH * kWTW;
  extern __shared__ __align__(16) float wg_sm[];
  float* gs = wg_sm;               // [NP][COB]
  float* xs = wg_sm + NP * COB;    // [PR * PC][CIB]
  const int co0 = blockIdx.z * COB, ci0 = blockIdx.y * CIB;
  const int tid = threadIdx.x, cg = tid / (CIB / 2), ig = tid % (CIB / 2);
  const int Hv = MODE == CM_UP2 ? Ho : Hi, Wv = MODE == CM_UP2 ? Wo : Wi;
  const int tiles_x = (Wo + kWTW - 1) / kWTW, ntiles = tiles_x * ((Ho + kWTH - 1) / kWTH);
  float acc[KS * KS][4][2];
  float bacc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int t = 0; t < KS * KS; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[t][j][0] = acc[t][j][1] = 0.f;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int Y0 = (tile / tiles_x) * kWTH, X0 = (tile % tiles_x) * kWTW;
    __syncthreads();  // the previous tile's reads are done
    for (int e = tid; e < NP * COB; e += NT) {
      const int p = e / COB, c = e - p * COB;
      const int oy = Y0 + p / kWTW, ox = X0 + p % kWTW;
      gs[e] = (oy < Ho && ox < Wo && co0 + c < Co) ? gout[((size_t)oy * Wo + ox) * Co + co0 + c] : 0.f;
    }
    for (int e = tid; e < PR * PC * CIB; e += NT) {
      const int q = e / CIB, c = e - q * CIB;
      const int vy = Y0 * S - PAD + q / PC, vx = X0 * S - PAD + q % PC;
      float v = 0.f;
      if (vy >= 0 && vx >= 0 && vy < Hv && vx < Wv && ci0 + c < Ci) {
        const int iy = MODE == CM_UP2 ? vy >> 1 : vy, ix = MODE == CM_UP2 ? vx >> 1 : vx;
        v = in[((size_t)iy * Wi + ix) * Ci + ci0 + c];
      }
      xs[e] = v;
    }
    __syncthreads();
    for (int p = 0; p < NP; ++p) {
      const float4 g = *reinterpret_cast<const float4*>(gs + p * COB + cg * 4);
      bacc[0] += g.x;
      bacc[1] += g.y;
      bacc[2] += g.z;
      bacc[3] += g.w;
      const int py = p / kWTW, px = p - py * kWTW;
#pragma unroll
      for (int ky = 0; ky < KS; ++ky)
#pragma unroll
        for (int kx = 0; kx < KS; ++kx) {
          const float2 x = *reinterpret_cast<const float2*>(xs + ((py * S + ky) * PC + px * S + kx) * CIB + ig * 2);
          float* a = acc[ky * KS + kx][0];
          a[0] = fmaf(g.x, x.x, a[0]);
          a[1] = fmaf(g.x, x.y, a[1]);
          a[2] = fmaf(g.y, x.x, a[2]);
          a[3] = fmaf(g.y, x.y, a[3]);
          a[4] = fmaf(g.z, x.x, a[4]);
          a[5] = fmaf(g.z, x.y, a[5]);
          a[6] = fmaf(g.w, x.x, a[6]);
          a[7] = fmaf(g.w, x.y, a[7]);
        }
    }
  }
  float* out = slots + (size_t)blockIdx.x * nW;
#pragma unroll
  for (int t = 0; t < KS * KS; ++t)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int co = co0 + cg * 4 + j, ci = ci0 + ig * 2 + h;
        if (co < Co && ci < Ci) out[((size_t)co * KS * KS + t) * Ci + ci] = acc[t][j][h];
      }
  if (blockIdx.y == 0 && ig == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int co = co0 + cg * 4 + j;
      if (co < Co) out[(size_t)Co * KS * KS * Ci + co] = bacc[j];
    }
}

// The same for layers with few weights (Co KS^2 Ci <= 512: the one-channel final conv, the
// two-channel first encoder layer): one thread per weight, the tile's pixels summed in order.
template <int MODE, int KS>
__global__ void __launch_bounds__(512)
wgrad_small(const float* __restrict__ gout, int Ho, int Wo, int Co, const float* __restrict__ in, int Hi, int Wi, int Ci,
            float* __restrict__ slots, int nW) {
  using G = WgradGeo<MODE, KS>;
  constexpr int S = G::S, PAD = G::PAD, PR = G::PR, PC = G::PC, NP = kWTH * kWTW;
  extern __shared__ __align__(16) float ws_sm[];
  float* gs = ws_sm;              // [NP][Co]
  float* xs = ws_sm + NP * Co;    // [PR * PC][Ci]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nWw = Co * KS * KS * Ci;
  const int ci = tid % Ci, tap = (tid / Ci) % (KS * KS), co = tid / (Ci * KS * KS);
  const int ky = tap / KS, kx = tap % KS;
  const bool wt_thread = tid < nWw, b_thread = tid >= nWw && tid < nWw + Co;
  const int bco = tid - nWw;
  const int Hv = MODE == CM_UP2 ? Ho : Hi, Wv = MODE == CM_UP2 ? Wo : Wi;
  const int tiles_x = (Wo + kWTW - 1) / kWTW, ntiles = tiles_x * ((Ho + kWTH - 1) / kWTH);
  float acc = 0.f;
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int Y0 = (tile / tiles_x) * kWTH, X0 = (tile % tiles_x) * kWTW;
    __syncthreads();
    for (int e = tid; e < NP * Co; e += nt) {
      const int p = e / Co, c = e - p * Co;
      const int oy = Y0 + p / kWTW, ox = X0 + p % kWTW;
      gs[e] = (oy < Ho && ox < Wo) ? gout[((size_t)oy * Wo + ox) * Co + c] : 0.f;
    }
    for (int e = tid; e < PR * PC * Ci; e += nt) {
      const int q = e / Ci, c = e - q * Ci;
      const int vy = Y0 * S - PAD + q / PC, vx = X0 * S - PAD + q % PC;
      float v = 0.f;
      if (vy >= 0 && vx >= 0 && vy < Hv && vx < Wv) {
        const int iy = MODE == CM_UP2 ? vy >> 1 : vy, ix = MODE == CM_UP2 ? vx >> 1 : vx;
        v = in[((size_t)iy * Wi + ix) * Ci + c];
      }
      xs[e] = v;
    }
    __syncthreads();
    if (wt_thread) {
      for (int p = 0; p < NP; ++p) {
        const int py = p / kWTW, px = p - py * kWTW;
        acc = fmaf(gs[p * Co + co], xs[((py * S + ky) * PC + px * S + kx) * Ci + ci], acc);
      }
    } else if (b_thread) {
      for (int p = 0; p < NP; ++p) acc += gs[p * Co + bco];
    }
  }
  if (wt_thread) slots[(size_t)blockIdx.x * nW + ((size_t)co * KS * KS + tap) * Ci + ci] = acc;
  else if (b_thread) slots[(size_t)blockIdx.x * nW + nWw + bco] = acc;
}

// gw[e] += sum over the nb slots of slots[b][e] (e < nWw), gb[e - nWw] likewise after, in
// slot order.
__global__ void wgrad_reduce(const float* __restrict__ slots, int nb, int nW, int nWw, float* __restrict__ gw,
                             float* __restrict__ gb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nW) return;
  float s = 0.f;
  for (int b = 0; b < nb; ++b) s += slots[(size_t)b * nW + e];
  if (e < nWw)
    gw[e] += s;
  else
    gb[e - nWw] += s;
}

template <int MODE, int KS>
struct DgradGeo {
  static constexpr int S = view_stride(MODE), PAD = KS / 2;
  static constexpr int NV = MODE == CM_UP2 ? 2 : 1;  // view positions per input pixel along an axis
  // output rows / columns the tile's view positions reach
  static constexpr int GR = (NV * kDTH - 1 + KS - 1) / S + 2, GC = (NV * kDTW - 1 + KS - 1) / S + 2;
};

template <int MODE, int KS, int CIT>
__global__ void __launch_bounds__(kDTH * kDTW)
dgrad_tiled(const float* __restrict__ gout, int Ho, int Wo, int Co, const float* __restrict__ w,
            const float* __restrict__ mask_act, int Hi, int Wi, int Ci, int accumulate, float* __restrict__ gin) {
  using G = DgradGeo<MODE, KS>;
  constexpr int S = G::S, PAD = G::PAD, NV = G::NV, GR = G::GR, GC = G::GC, COC = 8;
  __shared__ float gp[GR][GC][COC];
  __shared__ __align__(16) float wsm[KS * KS][COC][CIT];
  const int tid = threadIdx.x, ty = tid / kDTW, tx = tid % kDTW;
  const int I0 = blockIdx.y * kDTH, J0 = blockIdx.x * kDTW, ci0 = blockIdx.z * CIT;
  const int iy = I0 + ty, ix = J0 + tx;
  const int Hv = MODE == CM_UP2 ? Ho : Hi, Wv = MODE == CM_UP2 ? Wo : Wi;
  // output region: view rows NV I0 .. NV (I0 + kDTH) - 1 reach o = (v + PAD - k) / S
  const int oy0 = floor_div(NV * I0 + PAD - (KS - 1), S), ox0 = floor_div(NV * J0 + PAD - (KS - 1), S);
  float acc[CIT];
#pragma unroll
  for (int c = 0; c < CIT; ++c) acc[c] = 0.f;
  for (int c0 = 0; c0 < Co; c0 += COC) {
    __syncthreads();
    for (int e = tid; e < GR * GC * COC; e += kDTH * kDTW) {
      const int c = e % COC, q = e / COC;
      const int oy = oy0 + q / GC, ox = ox0 + q % GC;
      gp[q / GC][q % GC][c] =
          (oy >= 0 && ox >= 0 && oy < Ho && ox < Wo && c0 + c < Co) ? gout[((size_t)oy * Wo + ox) * Co + c0 + c] : 0.f;
    }
    for (int e = tid; e < KS * KS * COC * CIT; e += kDTH * kDTW) {
      const int ci = e % CIT, t = e / CIT;
      const int co = t % COC, tap = t / COC;
      wsm[tap][co][ci] = (c0 + co < Co && ci0 + ci < Ci) ? w[((size_t)(c0 + co) * KS * KS + tap) * Ci + ci0 + ci] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int a = 0; a < NV; ++a)
#pragma unroll
      for (int b = 0; b < NV; ++b) {
        const int vy = NV * iy + a, vx = NV * ix + b;
        if (vy >= Hv || vx >= Wv) continue;  // cropped away (or beyond the input)
#pragma unroll
        for (int ky = 0; ky < KS; ++ky) {
          const int ny = vy + PAD - ky;
          if (S == 2 && (ny & 1)) continue;
          const int ry = floor_div(ny, S) - oy0;
#pragma unroll
          for (int kx = 0; kx < KS; ++kx) {
            const int nx = vx + PAD - kx;
            if (S == 2 && (nx & 1)) continue;
            const int rx = floor_div(nx, S) - ox0;
#pragma unroll
            for (int co = 0; co < COC; ++co) {
              const float g = gp[ry][rx][co];
              const float* wp = wsm[ky * KS + kx][co];
#pragma unroll
              for (int c = 0; c < CIT; ++c) acc[c] = fmaf(g, wp[c], acc[c]);
            }
          }
        }
      }
  }
  if (iy >= Hi || ix >= Wi) return;
  const size_t base = ((size_t)iy * Wi + ix) * Ci + ci0;
#pragma unroll
  for (int c = 0; c < CIT; ++c) {
    if (ci0 + c >= Ci) break;
    float v = acc[c];
    if (mask_act && !(mask_act[base + c] > 0.f)) v = 0.f;
    gin[base + c] = accumulate ? gin[base + c] + v : v;
  }
}

template <int MODE, int KS, int COB, int CIB>
cudaError_t run_wgrad(const float* gout, int Ho, int Wo, int Co, const float* in, int Hi, int Wi, int Ci, float* gw,
                      float* gb, float* slots, size_t slot_cap, cudaStream_t st) {
  using G = WgradGeo<MODE, KS>;
  const int nW = Co * KS * KS * Ci + Co;
  const int ntiles = ((Wo + kWTW - 1) / kWTW) * ((Ho + kWTH - 1) / kWTH);
  int nb = std::min(ntiles, 304);
  if ((size_t)nb * nW > slot_cap) nb = (int)std::max<size_t>(1, slot_cap / nW);
  const size_t smem = sizeof(float) * (kWTH * kWTW * COB + G::PR * G::PC * CIB);
  auto kern = wgrad_tiled<MODE, KS, COB, CIB>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<dim3(nb, (Ci + CIB - 1) / CIB, (Co + COB - 1) / COB), COB / 4 * CIB / 2, smem, st>>>(gout, Ho, Wo, Co, in, Hi,
                                                                                             Wi, Ci, slots, nW);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  wgrad_reduce<<<(nW + 255) / 256, 256, 0, st>>>(slots, nb, nW, Co * KS * KS * Ci, gw, gb);
  return cudaGetLastError();
}

template <int MODE, int KS>
cudaError_t run_wgrad_small(const float* gout, int Ho, int Wo, int Co, const float* in, int Hi, int Wi, int Ci,
                            float* gw, float* gb, float* slots, size_t slot_cap, cudaStream_t st) {
  using G = WgradGeo<MODE, KS>;
  const int nW = Co * KS * KS * Ci + Co;
  const int ntiles = ((Wo + kWTW - 1) / kWTW) * ((Ho + kWTH - 1) / kWTH);
  int nb = std::min(ntiles, 4 * 152);
  if ((size_t)nb * nW > slot_cap) nb = (int)std::max<size_t>(1, slot_cap / nW);
  const size_t smem = sizeof(float) * (kWTH * kWTW * Co + G::PR * G::PC * Ci);
  auto kern = wgrad_small<MODE, KS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<nb, (nW + 31) / 32 * 32, smem, st>>>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, slots, nW);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  wgrad_reduce<<<(nW + 255) / 256, 256, 0, st>>>(slots, nb, nW, Co * KS * KS * Ci, gw, gb);
  return cudaGetLastError();
}

template <int MODE, int KS>
cudaError_t wgrad_mode(const float* gout, int Ho, int Wo, int Co, const float* in, int Hi, int Wi, int Ci, float* gw,
                       float* gb, float* slots, size_t cap, cudaStream_t st) {
  if (Co * KS * KS * Ci + Co <= 512 && (Co < 16 || Ci < 16))
    return run_wgrad_small<MODE, KS>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, gw, gb, slots, cap, st);
  if (Co >= 64 && Ci >= 32) return run_wgrad<MODE, KS, 64, 32>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, gw, gb, slots, cap, st);
  if (Co >= 32) return run_wgrad<MODE, KS, 32, 32>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, gw, gb, slots, cap, st);
  if (Co >= 16) return run_wgrad<MODE, KS, 16, 32>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, gw, gb, slots, cap, st);
  return run_wgrad<MODE, KS, 4, 32>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, gw, gb, slots, cap, st);
}

template <int MODE, int KS>
cudaError_t dgrad_mode(const float* gout, int Ho, int Wo, int Co, const float* w, const float* mask, int Hi, int Wi,
                       int Ci, int accumulate, float* gin, cudaStream_t st) {
  constexpr int CIT = 16;
  dgrad_tiled<MODE, KS, CIT><<<dim3((Wi + kDTW - 1) / kDTW, (Hi + kDTH - 1) / kDTH, (Ci + CIT - 1) / CIT),
                               kDTH * kDTW, 0, st>>>(gout, Ho, Wo, Co, w, mask, Hi, Wi, Ci, accumulate, gin);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_wgrad_tiled(const float* gout, int Ho, int Wo, int Co, const float* in, int Hi, int Wi, int Ci,
                               int ks, int mode, float* gw, float* gb, float* slots, size_t slot_cap,
                               cudaStream_t st) {
  if (ks == 1 && mode == CM_S1) return wgrad_mode<CM_S1, 1>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, gw, gb, slots, slot_cap, st);
  if (ks != 3) return cudaErrorInvalidValue;
  switch (mode) {
    case CM_S1: return wgrad_mode<CM_S1, 3>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, gw, gb, slots, slot_cap, st);
    case CM_S2: return wgrad_mode<CM_S2, 3>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, gw, gb, slots, slot_cap, st);
    case CM_UP2: return wgrad_mode<CM_UP2, 3>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, gw, gb, slots, slot_cap, st);
  }
  return cudaErrorInvalidValue;
}

size_t wgrad_slot_floats(int Ho, int Wo, int Co, int Ci, int ks) {
  const int ntiles = ((Wo + kWTW - 1) / kWTW) * ((Ho + kWTH - 1) / kWTH);
  return (size_t)std::min(ntiles, 4 * 152) * (size_t)(Co * ks * ks * Ci + Co);
}

cudaError_t launch_dgrad_tiled(const float* gout, int Ho, int Wo, int Co, const float* w, int ks, int mode,
                               const float* mask_act, int Hi, int Wi, int Ci, int accumulate, float* gin,
                               cudaStream_t st) {
  if (ks == 1 && mode == CM_S1) return dgrad_mode<CM_S1, 1>(gout, Ho, Wo, Co, w, mask_act, Hi, Wi, Ci, accumulate, gin, st);
  if (ks != 3) return cudaErrorInvalidValue;
  switch (mode) {
    case CM_S1: return dgrad_mode<CM_S1, 3>(gout, Ho, Wo, Co, w, mask_act, Hi, Wi, Ci, accumulate, gin, st);
    case CM_S2: return dgrad_mode<CM_S2, 3>(gout, Ho, Wo, Co, w, mask_act, Hi, Wi, Ci, accumulate, gin, st);
    case CM_UP2: return dgrad_mode<CM_UP2, 3>(gout, Ho, Wo, Co, w, mask_act, Hi, Wi, Ci, accumulate, gin, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sv
