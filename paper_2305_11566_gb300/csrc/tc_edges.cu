// tc_edges.cu -- the CUDA-core layers around the tensor-core convolutions of the BF16
// form, each one launch for all pairs of a call (blockIdx.z = pair):
//
//   edge_enc1    first conv (3x3 stride 2, 2 -> C1, ReLU) with its input built while
//                staging: x0 = (L / 256, U / 256), U = 4 * bilinear(coarse) (a5, a6, a7).
//                FP32 arithmetic, BF16 NHWC output.
//   edge_final   last conv (3x3, C -> 1) + bias + U (residual), BF16 input, FP32 output (a11).
//   edge_up2fix  exact recomputation of the last row / column of an odd-sized (cropped)
//                nearest-x2 + 3x3 conv output, which the 4-phase tensor-core form folds wrongly.
#include "sv_ctx.cuh"

namespace sv {

namespace {

using bf16 = __nv_bfloat16;

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

constexpr int ETW = 32, ETH = 8;  // output tile of the edge kernels (256 threads)

// enc1: 17 x 65 x 2 input tile in shared memory, weights [18][C1] (broadcast), one output
// pixel and all C1 channels per thread.
__global__ void __launch_bounds__(256) edge_enc1(const EdgePair* __restrict__ pairs, const float* __restrict__ W,
                                                 const float* __restrict__ B, int C1) {
  constexpr int TR = 2 * ETH + 1, TC = 2 * ETW + 1;
  __shared__ float x0[TR][TC][2];
  extern __shared__ __align__(16) float wsm[];  // [18][C1] then bias[C1]
  const EdgePair P = pairs[blockIdx.z];
  const int H1 = (P.H + 1) / 2, W1 = (P.W + 1) / 2;
  const int X0 = blockIdx.x * ETW, Y0 = blockIdx.y * ETH;
  if (X0 >= W1 || Y0 >= H1) return;
  const int tid = threadIdx.y * ETW + threadIdx.x;
  for (int e = tid; e < 18 * C1; e += 256) {
    const int co = e % C1, k = e / C1;  // k = tap * 2 + channel
    wsm[e] = W[(size_t)co * 18 + k];
  }
  for (int e = tid; e < C1; e += 256) wsm[18 * C1 + e] = B[e];
  for (int e = tid; e < TR * TC; e += 256) {
    const int r = e / TC, c = e - r * TC;
    const int vy = 2 * Y0 - 1 + r, vx = 2 * X0 - 1 + c;
    float l = 0.f, u = 0.f;
    if (vy >= 0 && vy < P.H && vx >= 0 && vx < P.W) {
      l = (float)P.L[(size_t)vy * P.pitch + vx] * (1.f / 256.f);
      u = (P.coarse_f ? upsample4_f(P.coarse_f, P.w, P.h, vx, vy) : upsample4_f(P.coarse, P.w, P.h, vx, vy)) *
          (1.f / 256.f);
    }
    x0[r][c][0] = l;
    x0[r][c][1] = u;
  }
  __syncthreads();
  const int X = X0 + threadIdx.x, Y = Y0 + threadIdx.y;
  if (X >= W1 || Y >= H1) return;
  float xin[18];
#pragma unroll
  for (int ky = 0; ky < 3; ++ky)
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      xin[(ky * 3 + kx) * 2] = x0[2 * threadIdx.y + ky][2 * threadIdx.x + kx][0];
      xin[(ky * 3 + kx) * 2 + 1] = x0[2 * threadIdx.y + ky][2 * threadIdx.x + kx][1];
    }
  bf16* out = P.e1 + ((size_t)Y * W1 + X) * C1;
  for (int c0 = 0; c0 < C1; c0 += 8) {
    float acc[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = wsm[18 * C1 + c0 + j];
#pragma unroll
    for (int k = 0; k < 18; ++k) {
      const float4 a = *reinterpret_cast<const float4*>(&wsm[k * C1 + c0]);
      const float4 b = *reinterpret_cast<const float4*>(&wsm[k * C1 + c0 + 4]);
      acc[0] = fmaf(a.x, xin[k], acc[0]); acc[1] = fmaf(a.y, xin[k], acc[1]);
      acc[2] = fmaf(a.z, xin[k], acc[2]); acc[3] = fmaf(a.w, xin[k], acc[3]);
      acc[4] = fmaf(b.x, xin[k], acc[4]); acc[5] = fmaf(b.y, xin[k], acc[5]);
      acc[6] = fmaf(b.z, xin[k], acc[6]); acc[7] = fmaf(b.w, xin[k], acc[7]);
    }
    uint32_t pk[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(acc[2 * j], 0.f), fmaxf(acc[2 * j + 1], 0.f));
      pk[j] = *reinterpret_cast<uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(out + c0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// final: (ETH + 2) x (ETW + 2) x C BF16 tile in shared memory with an 80-byte-per-32-channel
// pixel stride (conflict-free 16-byte reads), weights [9][C] FP32.
template <int C>
__global__ void __launch_bounds__(256) edge_final(const EdgePair* __restrict__ pairs, const float* __restrict__ W,
                                                  const float* __restrict__ B) {
  extern __shared__ __align__(16) unsigned char fsm[];
  const EdgePair P = pairs[blockIdx.z];
  const int X0 = blockIdx.x * ETW, Y0 = blockIdx.y * ETH;
  if (X0 >= P.W || Y0 >= P.H) return;
  constexpr int cpx = C / 8;             // 16-byte chunks per pixel
  constexpr int pstride = cpx + 1;       // padded pixel stride in chunks
  uint4* tile = reinterpret_cast<uint4*>(fsm);
  float* ws = reinterpret_cast<float*>(fsm + sizeof(uint4) * (ETH + 2) * (ETW + 2) * pstride);
  const int tid = threadIdx.y * ETW + threadIdx.x;
  for (int e = tid; e < 9 * C; e += 256) ws[e] = W[e];
  for (int e = tid; e < (ETH + 2) * (ETW + 2) * cpx; e += 256) {
    const int q = e % cpx, pix = e / cpx;
    const int r = pix / (ETW + 2), c = pix - r * (ETW + 2);
    const int vy = Y0 - 1 + r, vx = X0 - 1 + c;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (vy >= 0 && vy < P.H && vx >= 0 && vx < P.W)
      v = *reinterpret_cast<const uint4*>(P.d3 + ((size_t)vy * P.W + vx) * C + q * 8);
    tile[pix * pstride + q] = v;
  }
  __syncthreads();
  const int X = X0 + threadIdx.x, Y = Y0 + threadIdx.y;
  if (X >= P.W || Y >= P.H) return;
  float acc = B[0];
#pragma unroll
  for (int ky = 0; ky < 3; ++ky)
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      const uint4* src = tile + ((threadIdx.y + ky) * (ETW + 2) + threadIdx.x + kx) * pstride;
      const float* wp = ws + (ky * 3 + kx) * C;
#pragma unroll
      for (int q = 0; q < cpx; ++q) {
        const uint4 v = src[q];
        const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 f = __bfloat1622float2(h[j]);
          acc = fmaf(wp[q * 8 + 2 * j], f.x, acc);
          acc = fmaf(wp[q * 8 + 2 * j + 1], f.y, acc);
        }
      }
    }
  const float U = P.coarse_f ? upsample4_f(P.coarse_f, P.w, P.h, X, Y) : upsample4_f(P.coarse, P.w, P.h, X, Y);
  P.Y[(size_t)Y * P.W + X] = U + acc;
}

// Exact last row / column of a nearest-x2 + 3x3 conv with an odd output size.  One block
// per border pixel: the block stages the pixel's 3x3 input neighbourhood (BF16) in shared
// memory, thread t computes output channel t (and t + blockDim, ...) from the BF16-rounded
// unfolded weights Wb[co][ky][kx][ci], FP32 accumulation, 8 independent 16-byte weight
// loads in flight per thread.
__global__ void __launch_bounds__(128) edge_up2fix(const UpFixPair* __restrict__ pairs, const bf16* __restrict__ Wb,
                                                   const float* __restrict__ bias, int cin, int cout, int relu) {
  extern __shared__ __align__(16) uint4 patch[];  // [9][cin / 8]
  const UpFixPair L = pairs[blockIdx.y];
  const int nrow = (L.Ho & 1) ? L.Wo : 0;
  const int ncol = (L.Wo & 1) ? L.Ho : 0;
  const int pix = blockIdx.x;
  if (pix >= nrow + ncol) return;
  int Y, X;
  if (pix < nrow) {
    Y = L.Ho - 1;
    X = pix;
  } else {
    Y = pix - nrow;
    X = L.Wo - 1;
  }
  const int q8 = cin / 8, n = 9 * q8;
  for (int e = threadIdx.x; e < n; e += blockDim.x) {
    const int t = e / q8, q = e - t * q8;
    const int vy = Y + t / 3 - 1, vx = X + t % 3 - 1;
    uint4 v = make_uint4(0, 0, 0, 0);
    if (vy >= 0 && vy < L.Ho && vx >= 0 && vx < L.Wo)
      v = reinterpret_cast<const uint4*>(L.in + ((size_t)(vy >> 1) * L.Wi + (vx >> 1)) * cin)[q];
    patch[e] = v;
  }
  __syncthreads();
  for (int co = threadIdx.x; co < cout; co += blockDim.x) {
    const uint4* wp = reinterpret_cast<const uint4*>(Wb + (size_t)co * 9 * cin);
    float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int e0 = 0; e0 < n; e0 += 8) {  // n = 9 * cin / 8 is a multiple of 8 (cin % 64 == 0) or handled below
      uint4 w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) w[u] = e0 + u < n ? wp[e0 + u] : make_uint4(0, 0, 0, 0);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (e0 + u >= n) break;
        const uint4 x = patch[e0 + u];
        const __nv_bfloat162* wh = reinterpret_cast<const __nv_bfloat162*>(&w[u]);
        const __nv_bfloat162* xh = reinterpret_cast<const __nv_bfloat162*>(&x);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const float2 wf = __bfloat1622float2(wh[j]), xf = __bfloat1622float2(xh[j]);
          acc[u] = fmaf(wf.x, xf.x, acc[u]);
          acc[u] = fmaf(wf.y, xf.y, acc[u]);
        }
      }
    }
    float v = bias[co] + ((acc[0] + acc[1]) + (acc[2] + acc[3])) + ((acc[4] + acc[5]) + (acc[6] + acc[7]));
    if (relu) v = fmaxf(v, 0.f);
    L.out[((size_t)Y * L.Wo + X) * cout + co] = __float2bfloat16_rn(v);
  }
}

// Training latent: one thread per (latent pixel, channel).
__global__ void train_latent_bf16(const bf16* __restrict__ e3, int P, int Ci, const float* __restrict__ wmu,
                                  const float* __restrict__ bmu, const float* __restrict__ wlv,
                                  const float* __restrict__ blv, int lat, const float* __restrict__ eps,
                                  float* __restrict__ mu, float* __restrict__ lv, bf16* __restrict__ z) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)P * lat) return;
  const int co = (int)(i % lat);
  const bf16* x = e3 + (i / lat) * Ci;
  float m = bmu[co], l = blv[co];
  for (int ci = 0; ci < Ci; ++ci) {
    const float xv = __bfloat162float(x[ci]);
    m = fmaf(wmu[(size_t)co * Ci + ci], xv, m);
    l = fmaf(wlv[(size_t)co * Ci + ci], xv, l);
  }
  mu[i] = m;
  lv[i] = l;
  z[i] = __float2bfloat16_rn(m + eps[i] * expf(0.5f * l));
}

__global__ void bf16_to_f32(const bf16* __restrict__ a, float* __restrict__ b, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __bfloat162float(a[i]);
}

}  // namespace

cudaError_t launch_train_latent_bf16(const bf16* e3, int P, int Ci, const float* wmu, const float* bmu,
                                     const float* wlv, const float* blv, int lat, const float* eps, float* mu,
                                     float* lv, bf16* z, cudaStream_t st) {
  const size_t n = (size_t)P * lat;
  train_latent_bf16<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(e3, P, Ci, wmu, bmu, wlv, blv, lat, eps, mu, lv, z);
  return cudaGetLastError();
}

cudaError_t launch_bf16_to_f32(const bf16* a, float* b, size_t n, cudaStream_t st) {
  bf16_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_edge_enc1(const EdgePair* pairs, int n, int maxW1, int maxH1, const float* W, const float* B, int C1,
                             cudaStream_t st) {
  dim3 grid((maxW1 + ETW - 1) / ETW, (maxH1 + ETH - 1) / ETH, n);
  edge_enc1<<<grid, dim3(ETW, ETH), sizeof(float) * 19 * C1, st>>>(pairs, W, B, C1);
  return cudaGetLastError();
}

template <int C>
static cudaError_t run_final(const EdgePair* pairs, int n, int maxW, int maxH, const float* W, const float* B,
                             cudaStream_t st) {
  dim3 grid((maxW + ETW - 1) / ETW, (maxH + ETH - 1) / ETH, n);
  const size_t smem = sizeof(uint4) * (ETH + 2) * (ETW + 2) * (C / 8 + 1) + sizeof(float) * 9 * C;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(edge_final<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  edge_final<C><<<grid, dim3(ETW, ETH), smem, st>>>(pairs, W, B);
  return cudaGetLastError();
}

cudaError_t launch_edge_final(const EdgePair* pairs, int n, int maxW, int maxH, const float* W, const float* B, int C,
                              cudaStream_t st) {
  switch (C) {  // decoder widths are multiples of 16 up to 256
#define SV_FINAL_CASE(c) \
  case c: return run_final<c>(pairs, n, maxW, maxH, W, B, st);
    SV_FINAL_CASE(16) SV_FINAL_CASE(32) SV_FINAL_CASE(48) SV_FINAL_CASE(64) SV_FINAL_CASE(80) SV_FINAL_CASE(96)
    SV_FINAL_CASE(112) SV_FINAL_CASE(128) SV_FINAL_CASE(144) SV_FINAL_CASE(160) SV_FINAL_CASE(176) SV_FINAL_CASE(192)
    SV_FINAL_CASE(208) SV_FINAL_CASE(224) SV_FINAL_CASE(240) SV_FINAL_CASE(256)
#undef SV_FINAL_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_edge_up2fix(const UpFixPair* pairs, int n, int max_border, const bf16* Wb, const float* bias,
                               int cin, int cout, int relu, cudaStream_t st) {
  dim3 grid((unsigned)std::max(1, max_border), n);
  const size_t smem = sizeof(uint4) * 9 * (cin / 8);
  edge_up2fix<<<grid, std::min(128, std::max(32, cout)), smem, st>>>(pairs, Wb, bias, cin, cout, relu);
  return cudaGetLastError();
}

}  // namespace sv
