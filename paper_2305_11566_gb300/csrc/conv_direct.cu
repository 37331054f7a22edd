// conv_direct.cu -- plain refinement layers on CUDA cores, FP32 (the plain method) and
// FP64 (gradient-check form).  Activations NHWC, weights [cout][ks][ks][cin].
//
//   conv_direct_kernel  3x3 / 1x1 convolution with the input read through a view:
//                       stride 1, stride 2, or nearest x2 upsampling cropped to the
//                       output size (decoder); bias + optional ReLU epilogue.
//   enc1 source         the network input x0 = (L / 256, U / 256) built while staging:
//                       U = 4 * bilinear(coarse) (upsampling fused into the first conv).
//   final_tiled_kernel  3x3 conv to one channel + bias + U recomputed (the residual).
//   latent heads        1x1 convolutions (conv_direct_kernel); reparam_kernel z = mu + eps exp(lv / 2)
//                       (latent_kernel computes both heads per thread where an output is absent).
#include "sv_internal.cuh"

namespace sv {

namespace {

constexpr int TW = 16, TH = 8;  // output tile (threads)

// U(X, Y) = 4 * bilinear sample of the coarse map at s = (X + 1/2) / 4 - 1/2,
// clamped to [0, w-1] x [0, h-1]  (half-pixel centres, factor 4).
template <typename T, typename CoarseT>
__device__ __forceinline__ T upsample4_at(const CoarseT* __restrict__ c, int w, int h, int X, int Y) {
  T sx = (T)X * (T)0.25 - (T)0.375;
  T sy = (T)Y * (T)0.25 - (T)0.375;
  sx = sx < (T)0 ? (T)0 : (sx > (T)(w - 1) ? (T)(w - 1) : sx);
  sy = sy < (T)0 ? (T)0 : (sy > (T)(h - 1) ? (T)(h - 1) : sy);
  int x0 = (int)sx, y0 = (int)sy;  // sx, sy >= 0: truncation == floor
  int x1 = min(x0 + 1, w - 1), y1 = min(y0 + 1, h - 1);
  T fx = sx - (T)x0, fy = sy - (T)y0;
  T d00 = (T)c[(size_t)y0 * w + x0], d01 = (T)c[(size_t)y0 * w + x1];
  T d10 = (T)c[(size_t)y1 * w + x0], d11 = (T)c[(size_t)y1 * w + x1];
  T top = ((T)1 - fx) * d00 + fx * d01;
  T bot = ((T)1 - fx) * d10 + fx * d11;
  return (T)4 * (((T)1 - fy) * top + fy * bot);
}

// Input view of an NHWC tensor.  Returns V(vy, vx, ci) with zero padding.
template <typename T, int MODE>
struct SrcNHWC {
  const T* in;
  int Hi, Wi, Ci, Hv, Wv;
  __device__ __forceinline__ T operator()(int vy, int vx, int ci) const {
    if (vy < 0 || vx < 0 || vy >= Hv || vx >= Wv || ci >= Ci) return (T)0;
    int iy = MODE == CM_UP2 ? (vy >> 1) : vy;
    int ix = MODE == CM_UP2 ? (vx >> 1) : vx;
    return in[((size_t)iy * Wi + ix) * Ci + ci];
  }
};

// Network input x0 = (L / 256, U / 256) at full resolution.
template <typename T, typename CoarseT>
struct SrcEnc1 {
  const uint8_t* L;
  int pitch, W, H;
  const CoarseT* coarse;
  int w, h;
  __device__ __forceinline__ T operator()(int vy, int vx, int ci) const {
    if (vy < 0 || vx < 0 || vy >= H || vx >= W || ci >= 2) return (T)0;
    if (ci == 0) return (T)L[(size_t)vy * pitch + vx] * (T)(1.0 / 256.0);
    return upsample4_at<T, CoarseT>(coarse, w, h, vx, vy) * (T)(1.0 / 256.0);
  }
};

template <typename OutT, typename T> __device__ __forceinline__ OutT to_out(T v) { return (OutT)v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_out<__nv_bfloat16, float>(float v) {
  return __float2bfloat16_rn(v);
}

// One CTA: TH x TW output pixels x COT output channels; input channels in chunks of CIC
// staged channel-planar in shared memory ([ci][row][col]) with the weights [tap][ci][co].
template <typename T, typename Src, int S, int KS, int COT, int CIC, typename OutT>
__global__ void __launch_bounds__(TW * TH)
conv_direct_kernel(Src src, int Ci, const T* __restrict__ wt, const T* __restrict__ bias, int Co, int Ho, int Wo,
                   int relu, OutT* __restrict__ out) {
  constexpr int PAD = KS / 2;
  constexpr int TR = (TH - 1) * S + KS, TC = (TW - 1) * S + KS;
  __shared__ T tile[CIC][TR][TC];
  __shared__ __align__(16) T wsm[KS * KS][CIC][COT];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * TW + tx;
  const int X0 = blockIdx.x * TW, Y0 = blockIdx.y * TH, co0 = blockIdx.z * COT;
  const int X = X0 + tx, Y = Y0 + ty;
  T acc[COT];
#pragma unroll
  for (int c = 0; c < COT; ++c) acc[c] = (T)0;
  for (int ci0 = 0; ci0 < Ci; ci0 += CIC) {
    for (int e = tid; e < TR * TC * CIC; e += TW * TH) {
      int ci = e % CIC, rc = e / CIC;
      int r = rc / TC, c = rc - r * TC;
      tile[ci][r][c] = src(Y0 * S - PAD + r, X0 * S - PAD + c, ci0 + ci);
    }
    for (int e = tid; e < KS * KS * CIC * COT; e += TW * TH) {
      int co = e % COT, t = e / COT;
      int ci = t % CIC, tap = t / CIC;
      int gco = co0 + co, gci = ci0 + ci;
      wsm[tap][ci][co] = (gco < Co && gci < Ci) ? wt[((size_t)gco * KS * KS + tap) * Ci + gci] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int ky = 0; ky < KS; ++ky)
#pragma unroll
      for (int kx = 0; kx < KS; ++kx)
#pragma unroll 4
        for (int ci = 0; ci < CIC; ++ci) {
          const T v = tile[ci][ty * S + ky][tx * S + kx];
          const T* wp = wsm[ky * KS + kx][ci];
#pragma unroll
          for (int c = 0; c < COT; ++c) acc[c] = fma(v, wp[c], acc[c]);
        }
    __syncthreads();
  }
  if (X < Wo && Y < Ho) {
    OutT* op = out + ((size_t)Y * Wo + X) * Co + co0;
#pragma unroll
    for (int c = 0; c < COT; ++c) {
      if (co0 + c < Co) {
        T v = acc[c] + bias[co0 + c];
        if (relu && v < (T)0) v = (T)0;
        op[c] = to_out<OutT, T>(v);
      }
    }
  }
}

template <typename T> struct Cfg;
template <> struct Cfg<float> { static constexpr int COT = 32, CIC = 8; };
template <> struct Cfg<double> { static constexpr int COT = 16, CIC = 8; };

template <typename T, typename Src, int S, int KS, int CIC = Cfg<T>::CIC, typename OutT = T>
cudaError_t run_conv(const Src& src, int Ci, const T* wt, const T* bias, int Co, int Ho, int Wo, int relu, OutT* out,
                     cudaStream_t st) {
  constexpr int COT = Cfg<T>::COT;
  dim3 grid((Wo + TW - 1) / TW, (Ho + TH - 1) / TH, (Co + COT - 1) / COT);
  conv_direct_kernel<T, Src, S, KS, COT, CIC, OutT>
      <<<grid, dim3(TW, TH), 0, st>>>(src, Ci, wt, bias, Co, Ho, Wo, relu, out);
  return cudaGetLastError();
}

// final layer, tiled: a CTA computes an FH x FW output tile; the (FH + 2) x (FW + 2) input
// window is staged channel-planar in shared memory, FCIC channels at a time (zero outside the
// image), with the chunk's weights; one output pixel per thread.
constexpr int FW = 32, FH = 8, FCIC = 8;
template <typename T, typename CoarseT, typename OutT>
__global__ void __launch_bounds__(FW * FH)
final_tiled_kernel(const T* __restrict__ in, int W, int H, int Ci, const T* __restrict__ wt, const T* __restrict__ bias,
                   const CoarseT* __restrict__ coarse, int w, int h, OutT* __restrict__ Y) {
  __shared__ T tile[FCIC][FH + 2][FW + 2];
  __shared__ T ws[9][FCIC];
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * FW + tx;
  const int X0 = blockIdx.x * FW, Y0 = blockIdx.y * FH;
  T acc = (T)0;
  for (int ci0 = 0; ci0 < Ci; ci0 += FCIC) {
    for (int e = tid; e < (FH + 2) * (FW + 2) * FCIC; e += FW * FH) {
      const int ci = e % FCIC, px = e / FCIC;
      const int r = px / (FW + 2), c = px - r * (FW + 2);
      const int vy = Y0 - 1 + r, vx = X0 - 1 + c;
      const bool ok = vy >= 0 && vy < H && vx >= 0 && vx < W && ci0 + ci < Ci;
      tile[ci][r][c] = ok ? in[((size_t)vy * W + vx) * Ci + ci0 + ci] : (T)0;
    }
    for (int e = tid; e < 9 * FCIC; e += FW * FH) {
      const int ci = e % FCIC, tap = e / FCIC;
      ws[tap][ci] = ci0 + ci < Ci ? wt[(size_t)tap * Ci + ci0 + ci] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx)
#pragma unroll
        for (int ci = 0; ci < FCIC; ++ci) acc = fma(ws[ky * 3 + kx][ci], tile[ci][ty + ky][tx + kx], acc);
    __syncthreads();
  }
  const int X = X0 + tx, Yy = Y0 + ty;
  if (X < W && Yy < H) Y[(size_t)Yy * W + X] = (OutT)(upsample4_at<T, CoarseT>(coarse, w, h, X, Yy) + (bias[0] + acc));
}

// z = mu + eps exp(lv / 2) (training form of the latent, after the two 1x1 heads)
template <typename T>
__global__ void reparam_kernel(const T* __restrict__ mu, const T* __restrict__ lv, const T* __restrict__ eps, size_t n,
                               T* __restrict__ z) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = mu[i] + eps[i] * exp((T)0.5 * lv[i]);
}

template <typename T>
__global__ void latent_kernel(const T* __restrict__ e3, int P, int Ci, const T* __restrict__ wmu,
                              const T* __restrict__ bmu, const T* __restrict__ wlv, const T* __restrict__ blv, int lat,
                              const T* __restrict__ eps, T* __restrict__ mu, T* __restrict__ lv, T* __restrict__ z) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)P * lat) return;
  const int co = (int)(i % lat);
  const size_t p = i / lat;
  const T* x = e3 + p * Ci;
  T m = bmu[co];
  for (int ci = 0; ci < Ci; ++ci) m = fma(wmu[(size_t)co * Ci + ci], x[ci], m);
  if (mu) mu[i] = m;
  T zz = m;
  if (lv || eps) {
    T l = blv[co];
    for (int ci = 0; ci < Ci; ++ci) l = fma(wlv[(size_t)co * Ci + ci], x[ci], l);
    if (lv) lv[i] = l;
    if (eps) zz = m + eps[i] * exp((T)0.5 * l);
  }
  if (z) z[i] = zz;
}

}  // namespace

template <typename T>
cudaError_t launch_conv_direct(const DirectConvArgs<T>& a, int mode, int ks, cudaStream_t st) {
  if (ks == 1) {
    SrcNHWC<T, CM_S1> s{a.in, a.Hi, a.Wi, a.Ci, a.Hi, a.Wi};
    return run_conv<T, SrcNHWC<T, CM_S1>, 1, 1>(s, a.Ci, a.wt, a.bias, a.Co, a.Ho, a.Wo, a.relu, a.out, st);
  }
  switch (mode) {
    case CM_S1: {
      SrcNHWC<T, CM_S1> s{a.in, a.Hi, a.Wi, a.Ci, a.Hi, a.Wi};
      return run_conv<T, SrcNHWC<T, CM_S1>, 1, 3>(s, a.Ci, a.wt, a.bias, a.Co, a.Ho, a.Wo, a.relu, a.out, st);
    }
    case CM_S2: {
      SrcNHWC<T, CM_S2> s{a.in, a.Hi, a.Wi, a.Ci, a.Hi, a.Wi};
      return run_conv<T, SrcNHWC<T, CM_S2>, 2, 3>(s, a.Ci, a.wt, a.bias, a.Co, a.Ho, a.Wo, a.relu, a.out, st);
    }
    case CM_UP2: {
      SrcNHWC<T, CM_UP2> s{a.in, a.Hi, a.Wi, a.Ci, a.Ho, a.Wo};
      return run_conv<T, SrcNHWC<T, CM_UP2>, 1, 3>(s, a.Ci, a.wt, a.bias, a.Co, a.Ho, a.Wo, a.relu, a.out, st);
    }
  }
  return cudaErrorInvalidValue;
}

template <typename T, typename CoarseT>
cudaError_t launch_enc1(const uint8_t* L, int pitch, int W, int H, const CoarseT* coarse, int w, int h, const T* wt,
                        const T* bias, int Co, T* out, cudaStream_t st) {
  SrcEnc1<T, CoarseT> s{L, pitch, W, H, coarse, w, h};
  Levels lv(H, W);
  return run_conv<T, SrcEnc1<T, CoarseT>, 2, 3, 2>(s, 2, wt, bias, Co, lv.H[1], lv.W[1], 1, out, st);
}

template <typename T, typename CoarseT, typename OutT>
cudaError_t launch_final(const T* in, int W, int H, int Ci, const T* wt, const T* bias, const CoarseT* coarse, int w,
                         int h, OutT* Y, cudaStream_t st) {
  dim3 grid((W + FW - 1) / FW, (H + FH - 1) / FH);
  final_tiled_kernel<T, CoarseT, OutT><<<grid, dim3(FW, FH), 0, st>>>(in, W, H, Ci, wt, bias, coarse, w, h, Y);
  return cudaGetLastError();
}

// Latent heads on the [H3][W3] grid.  Inference (no eps): z = the mean head, a 1x1
// convolution.  Training with both head outputs given: the two heads as 1x1 convolutions
// into mu and lv, then the reparameterisation; otherwise one thread per (pixel, channel)
// computing both heads.
template <typename T>
cudaError_t launch_latent(const T* e3, int H3, int W3, int Ci, const T* wmu, const T* bmu, const T* wlv, const T* blv,
                          int lat, const T* eps, T* mu, T* lv, T* z, cudaStream_t st) {
  const int P = H3 * W3;
  const size_t n = (size_t)P * lat;
  if (!eps && !lv && !mu && z) {
    DirectConvArgs<T> a{e3, H3, W3, Ci, wmu, bmu, lat, H3, W3, 0, z};
    return launch_conv_direct<T>(a, CM_S1, 1, st);
  }
  if (eps && mu && lv && z) {
    DirectConvArgs<T> a{e3, H3, W3, Ci, wmu, bmu, lat, H3, W3, 0, mu};
    cudaError_t e = launch_conv_direct<T>(a, CM_S1, 1, st);
    if (e != cudaSuccess) return e;
    a = {e3, H3, W3, Ci, wlv, blv, lat, H3, W3, 0, lv};
    if ((e = launch_conv_direct<T>(a, CM_S1, 1, st)) != cudaSuccess) return e;
    reparam_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mu, lv, eps, n, z);
    return cudaGetLastError();
  }
  latent_kernel<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(e3, P, Ci, wmu, bmu, wlv, blv, lat, eps, mu, lv, z);
  return cudaGetLastError();
}

template cudaError_t launch_conv_direct<float>(const DirectConvArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_conv_direct<double>(const DirectConvArgs<double>&, int, int, cudaStream_t);
template cudaError_t launch_enc1<float, int16_t>(const uint8_t*, int, int, int, const int16_t*, int, int, const float*,
                                                 const float*, int, float*, cudaStream_t);
template cudaError_t launch_enc1<float, float>(const uint8_t*, int, int, int, const float*, int, int, const float*,
                                               const float*, int, float*, cudaStream_t);
template cudaError_t launch_enc1<double, double>(const uint8_t*, int, int, int, const double*, int, int, const double*,
                                                 const double*, int, double*, cudaStream_t);
template cudaError_t launch_enc1<double, int16_t>(const uint8_t*, int, int, int, const int16_t*, int, int,
                                                  const double*, const double*, int, double*, cudaStream_t);
template cudaError_t launch_final<double, int16_t, double>(const double*, int, int, int, const double*, const double*,
                                                           const int16_t*, int, int, double*, cudaStream_t);
template cudaError_t launch_final<float, int16_t, float>(const float*, int, int, int, const float*, const float*,
                                                         const int16_t*, int, int, float*, cudaStream_t);
template cudaError_t launch_final<float, float, float>(const float*, int, int, int, const float*, const float*,
                                                       const float*, int, int, float*, cudaStream_t);
template cudaError_t launch_final<double, double, double>(const double*, int, int, int, const double*, const double*,
                                                          const double*, int, int, double*, cudaStream_t);
template cudaError_t launch_latent<float>(const float*, int, int, int, const float*, const float*, const float*,
                                          const float*, int, const float*, float*, float*, float*, cudaStream_t);
template cudaError_t launch_latent<double>(const double*, int, int, int, const double*, const double*, const double*,
                                           const double*, int, const double*, double*, double*, double*, cudaStream_t);

}  // namespace sv
