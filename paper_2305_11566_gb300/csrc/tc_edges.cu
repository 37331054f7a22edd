// tc_edges.cu -- the CUDA-core layers around the tensor-core convolutions of the BF16
// form, each one launch for all pairs of a call (blockIdx.z = pair):
//
//   edge_enc1    first conv (3x3 stride 2, 2 -> C1, ReLU) with its input built while
//                staging: x0 = (L / 256, U / 256), U = 4 * bilinear(coarse).  FP32
//                arithmetic, BF16 NHWC output; 4 output rows per thread.
//   enc1_tc      the same layer with the 2 -> C1 products on the tensor cores (C1 = 16, 32,
//                64): the staged input becomes an im2col A tile in shared memory; a
//                persistent grid whose blocks walk the (pair, tile) list.
//   edge_final   last conv (3x3, C -> 1) + bias + U (residual), BF16 input, FP32 output;
//                register-blocked packed-FP32 form for C = 16, 32, 64, 128.
//   edge_up2fix  exact recomputation of the last row / column of an odd-sized (cropped)
//                nearest-x2 + 3x3 conv output, which the 4-phase tensor-core form folds
//                wrongly: segments of 64 border pixels x 32 channels per block.
#include <cuda_fp8.h>

#include "sv_ctx.cuh"

namespace sv {

namespace {

using bf16 = __nv_bfloat16;

// 16-byte asynchronous global -> shared copy (zero fill when !valid: no bytes are read,
// `src` is only a placeholder then); every copy of a staging loop is in flight at once.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ bool mbar_try_e(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ bool mbar_wait_e(uint32_t bar, uint32_t parity, long long spin) {
  if (mbar_try_e(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_e(bar, parity))
    if (clock64() - t0 > spin) return false;
  return true;
}

constexpr int ETW = 32, ETH = 8;  // output tile of the edge kernels (256 threads)

// enc1, register-blocked: a block computes 32 output columns x 32 output rows; thread
// (cx, g) computes rows 4g .. 4g + 3 of column cx for 8 channels at a time, so each
// broadcast weight read feeds four pixels.  Its input, x0 = (L / 256, U / 256) on the
// 65 x 65 positions the tile reads, is staged in shared memory; U (bilinear x4 of the
// coarse map) is separable: the coarse rows the tile touches are interpolated along x
// once (T), then every position interpolates T along y.  The four rows' overlapping
// 9 x 3 x 2 input window sits in registers.
constexpr int E1W = 32, E1H = 32, E1R = 2 * E1H + 1, E1C = 2 * E1W + 1, E1CR = 20;

template <typename CT>
__device__ __forceinline__ void coarse_axis(float v, int n, int& i0, int& i1, float& f) {
  float s = v * 0.25f - 0.375f;
  s = fminf(fmaxf(s, 0.f), (float)(n - 1));
  i0 = (int)s;
  i1 = min(i0 + 1, n - 1);
  f = s - (float)i0;
}

// The window's global loads (image bytes and the coarse values of T), all issued in one pass
// before any is used, so that their latency overlaps whatever the kernel does next.
// Window of a block of BH e1 rows (x 32 columns): R staged full-resolution rows, CR coarse rows
// of T (with a margin), NTT / NXS loads per thread of the two passes.
template <int BH>
struct E1Geo {
  static constexpr int R = 2 * BH + 1, CR = BH == E1H ? E1CR : BH / 2 + 4;
  static constexpr int NTT = (CR * E1C + 255) / 256, NXS = (R * E1C + 255) / 256;
};
template <int BH>
struct E1Loads {
  uint32_t lv[E1Geo<BH>::NXS];
  float c0v[E1Geo<BH>::NTT], c1v[E1Geo<BH>::NTT], fxv[E1Geo<BH>::NTT];
  int cy_lo;
};
template <typename CT, int BH>
__device__ __forceinline__ void enc1_stage_load(const EdgePair* P, const CT* __restrict__ cmap, int X0, int Y0,
                                                E1Loads<BH>& ld) {
  using G = E1Geo<BH>;
  const int Wd = P->W, Hd = P->H, w4 = P->w, h4 = P->h, pitch = P->pitch;
  const uint8_t* Lp = P->L;
  int dummy;
  float fdummy;
  coarse_axis<CT>((float)max(0, 2 * Y0 - 1), h4, ld.cy_lo, dummy, fdummy);
#pragma unroll
  for (int i = 0; i < G::NXS; ++i) {
    const int e = (int)threadIdx.x + 256 * i;
    const int r = e / E1C, c = e - r * E1C;
    const int vy = 2 * Y0 - 1 + r, vx = 2 * X0 - 1 + c;
    ld.lv[i] = (e < G::R * E1C && vy >= 0 && vy < Hd && vx >= 0 && vx < Wd) ? (uint32_t)Lp[(size_t)vy * pitch + vx] : 256u;
  }
#pragma unroll
  for (int i = 0; i < G::NTT; ++i) {
    const int e = min((int)threadIdx.x + 256 * i, G::CR * E1C - 1);
    const int ry = e / E1C, c = e - ry * E1C;
    const int cy = min(ld.cy_lo + ry, h4 - 1);
    const int vx = min(max(2 * X0 - 1 + c, 0), Wd - 1);
    int x0, x1;
    coarse_axis<CT>((float)vx, w4, x0, x1, ld.fxv[i]);
    ld.c0v[i] = (float)cmap[(size_t)cy * w4 + x0];
    ld.c1v[i] = (float)cmap[(size_t)cy * w4 + x1];
  }
}
// x0 = (L / 256, U / 256) on the window from the loaded values: the coarse rows
// interpolated along x (T), then every position along y.  Ends with the block synchronised.
template <typename CT, int BH>
__device__ __forceinline__ void enc1_stage_finish(const EdgePair* P, int Y0, const E1Loads<BH>& ld,
                                                  float (*xs)[E1C][2], float (*T)[E1C]) {
  using G = E1Geo<BH>;
  const int h4 = P->h;
#pragma unroll
  for (int i = 0; i < G::NTT; ++i) {
    const int e = (int)threadIdx.x + 256 * i;
    if (e < G::CR * E1C) T[e / E1C][e % E1C] = (1.f - ld.fxv[i]) * ld.c0v[i] + ld.fxv[i] * ld.c1v[i];
  }
  __syncthreads();  // T complete
#pragma unroll
  for (int i = 0; i < G::NXS; ++i) {
    const int e = (int)threadIdx.x + 256 * i;
    if (e >= G::R * E1C) break;
    const int r = e / E1C, c = e - r * E1C;
    const int vy = 2 * Y0 - 1 + r;
    float l = 0.f, u = 0.f;
    if (ld.lv[i] != 256u) {  // inside the image
      int y0, y1;
      float fy;
      coarse_axis<CT>((float)vy, h4, y0, y1, fy);
      l = (float)ld.lv[i] * (1.f / 256.f);
      u = 4.f * ((1.f - fy) * T[y0 - ld.cy_lo][c] + fy * T[y1 - ld.cy_lo][c]) * (1.f / 256.f);
    }
    xs[r][c][0] = l;
    xs[r][c][1] = u;
  }
  __syncthreads();
}
template <typename CT>
__device__ __forceinline__ void enc1_stage(const EdgePair* P, const CT* __restrict__ cmap, int X0, int Y0,
                                           float (*xs)[E1C][2], float (*T)[E1C]) {
  E1Loads<E1H> ld;
  enc1_stage_load<CT, E1H>(P, cmap, X0, Y0, ld);
  enc1_stage_finish<CT, E1H>(P, Y0, ld, xs, T);
}

__global__ void __launch_bounds__(256) edge_enc1(const EdgePair* __restrict__ pairs, const float* __restrict__ W,
                                                 const float* __restrict__ B, int C1) {
  // blockDim.x must be 256 (the staging passes are unrolled for it)
  __shared__ float xs[E1Geo<E1H>::R][E1C][2];
  __shared__ float T[E1Geo<E1H>::CR][E1C];
  extern __shared__ __align__(16) float wsm[];  // [18][C1] then bias[C1]
  const EdgePair* P = pairs + blockIdx.z;
  const int H1 = (P->H + 1) / 2, W1 = (P->W + 1) / 2;
  const int X0 = blockIdx.x * E1W, Y0 = blockIdx.y * E1H;
  if (X0 >= W1 || Y0 >= H1) return;
  const int tid = threadIdx.x;
  for (int e = tid; e < 18 * C1; e += blockDim.x) {
    const int co = e % C1, k = e / C1;  // k = tap * 2 + channel
    wsm[e] = W[(size_t)co * 18 + k];
  }
  for (int e = tid; e < C1; e += blockDim.x) wsm[18 * C1 + e] = B[e];
  if (P->coarse_f) enc1_stage(P, P->coarse_f, X0, Y0, xs, T);
  else enc1_stage(P, P->coarse, X0, Y0, xs, T);
  __syncthreads();
  const int cx = tid & 31, g = tid >> 5;
  const int X = X0 + cx;
  // input window of rows 4g .. 4g + 3: staged rows 8g .. 8g + 8, columns 2cx .. 2cx + 2
  float xv[9][3][2];
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int kx = 0; kx < 3; ++kx) {
      const float2 v = *reinterpret_cast<const float2*>(&xs[8 * g + r][2 * cx + kx][0]);
      xv[r][kx][0] = v.x;
      xv[r][kx][1] = v.y;
    }
  for (int c0 = 0; c0 < C1; c0 += 8) {
    // packed FP32 FMA: channel pairs (c, c + 1) of one pixel share the input value
    float2 acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 bj = make_float2(wsm[18 * C1 + c0 + 2 * j], wsm[18 * C1 + c0 + 2 * j + 1]);
#pragma unroll
      for (int k = 0; k < 4; ++k) acc[k][j] = bj;
    }
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx)
#pragma unroll
        for (int ch = 0; ch < 2; ++ch) {
          const int kk = (ky * 3 + kx) * 2 + ch;
          const float4 a = *reinterpret_cast<const float4*>(&wsm[kk * C1 + c0]);
          const float4 b = *reinterpret_cast<const float4*>(&wsm[kk * C1 + c0 + 4]);
          const float2 w2[4] = {make_float2(a.x, a.y), make_float2(a.z, a.w), make_float2(b.x, b.y),
                                make_float2(b.z, b.w)};
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const float x = xv[2 * k + ky][kx][ch];
            const float2 xx = make_float2(x, x);
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[k][j] = __ffma2_rn(w2[j], xx, acc[k][j]);
          }
        }
    if (X < W1) {
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int Y = Y0 + 4 * g + k;
        if (Y >= H1) break;
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(acc[k][j].x, 0.f), fmaxf(acc[k][j].y, 0.f));
          pk[j] = *reinterpret_cast<uint32_t*>(&h);
        }
        *reinterpret_cast<uint4*>(P->e1 + ((size_t)Y * W1 + X) * C1 + c0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
    }
  }
}

// ------------------------------------------------------------------ enc1 on the tensor cores
// The block's 32 x 32 output pixels are eight M = 128 tiles (tile t: output rows 4t .. 4t + 3,
// pixel m = 32 j + column of row 4t + j).  A pixel's A row holds its 27 inputs, the 9 taps x
// (L / 256, and U / 256 split into BF16 high and low parts), then 5 zeros: K = 32, in the
// no-swizzle K-major core-matrix layout (8 rows x 16 bytes per core matrix; K neighbours 128 B
// apart, 8-row groups 512 B apart).  B holds the C1 x 32 weights (the same U weight for both
// U parts) split into BF16 high and low parts, two MMA passes into the same accumulator, so
// that the result keeps FP32 accuracy to about 2^-16 (L / 256 is exact in BF16).  One TMEM
// accumulator of C1 columns per tile; the epilogue adds the bias, applies ReLU and stores
// BF16 NHWC.
__device__ __forceinline__ uint32_t smem_u32_e(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mma_bf16_e(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// descriptor of a no-swizzle K-major operand: start, LBO = 128 B (next 8 K), SBO (next 8 rows)
__device__ __forceinline__ uint64_t desc_ns_e(uint32_t addr, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         (1ull << 46);
}
__device__ __forceinline__ void tmem_ld32_e(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
      "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16_e(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&h);
}

constexpr uint32_t kE1Tile = 128 * 32 * 2;  // one A tile (128 pixels x K = 32, BF16)
constexpr int kE1TcBH = 16;                  // e1 rows per block of the tensor-core kernel
constexpr int kE1Tiles = kE1TcBH / 4;        // its MMA tiles (4 rows x 32 columns each)
constexpr int kE1BlocksPerSm = 3;            // resident blocks of the persistent kernel
__host__ __device__ constexpr size_t enc1_tc_smem(int C1) {
  return 128 + kE1Tiles * (size_t)kE1Tile + 2 * (size_t)C1 * 64 + (size_t)C1 * 4 + 16;
}

// Tiles of 16 x 32 e1 pixels (4 MMA tiles of 128 pixels), walked persistently: a block keeps
// its tensor memory, split weights and mbarrier for all its tiles, and issues the next tile's
// window loads before it waits for the current tile's MMAs, so that their latency hides behind
// the wait and the epilogue's stores.  Tile t of the launch is pair t / (gx gy), block row
// (t mod gx gy) / gx, block column t mod gx; a block takes tiles blockIdx.x, + gridDim.x, ...,
// skipping those outside their pair (ragged batches).
__device__ __forceinline__ int enc1_next_tile(const EdgePair* __restrict__ pairs, int t, int gx, int per, int ntiles,
                                              int BH, int& X0, int& Y0) {
  for (; t < ntiles; t += (int)gridDim.x) {
    const int z = t / per, rem = t - z * per, by = rem / gx;
    const EdgePair* P = pairs + z;
    X0 = (rem - by * gx) * E1W;
    Y0 = by * BH;
    if (X0 < (P->W + 1) / 2 && Y0 < (P->H + 1) / 2) return t;
  }
  return ntiles;
}

template <int C1>
__global__ void __launch_bounds__(256, kE1BlocksPerSm)
    enc1_tc(const EdgePair* __restrict__ pairs, int gx, int gy, int ntiles, const float* __restrict__ W,
            const float* __restrict__ B, int* err, long long spin) {
  static_assert(C1 == 16 || C1 == 32 || C1 == 64, "enc1 widths");
  constexpr int BH = kE1TcBH, NTILE = kE1Tiles, RPW = BH / 8;  // e1 rows per warp in the A build
  __shared__ float xs[E1Geo<BH>::R][E1C][2];
  __shared__ float T[E1Geo<BH>::CR][E1C];
  extern __shared__ unsigned char e1dyn[];
  const int per = gx * gy;
  int X0, Y0;
  int t = enc1_next_tile(pairs, (int)blockIdx.x, gx, per, ntiles, BH, X0, Y0);
  if (t >= ntiles) return;  // (uniform over the block)
  const EdgePair* P = pairs + t / per;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  E1Loads<BH> ld;  // the first window's loads go out first: their latency overlaps the set-up below
  if (P->coarse_f) enc1_stage_load<float, BH>(P, P->coarse_f, X0, Y0, ld);
  else enc1_stage_load<int16_t, BH>(P, P->coarse, X0, Y0, ld);
  const uint32_t raw = smem_u32_e(e1dyn), base = (raw + 127u) & ~127u;
  unsigned char* g = e1dyn + (base - raw);
  const uint32_t sA = base, sBh = base + NTILE * kE1Tile, sBl = sBh + C1 * 64;
  float* bias_s = reinterpret_cast<float*>(g + NTILE * kE1Tile + 2 * C1 * 64);
  const uint32_t mbar = smem_u32_e(bias_s + C1);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bias_s + C1 + 2);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32_e(tslot)),
                 "r"(NTILE * C1));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // B (high, low): element (n, k), k = 3 tap + part (0: L, 1 and 2: the two U parts)
  for (int e = tid; e < C1 * 32; e += 256) {
    const int n = e >> 5, k = e & 31;
    float w = 0.f;
    if (k < 27) w = W[(size_t)n * 18 + (k / 3) * 2 + (k % 3 == 0 ? 0 : 1)];
    const __nv_bfloat16 hi = __float2bfloat16_rn(w);
    const uint32_t off = (uint32_t)((n & 7) * 8 + (n >> 3) * 256 + (k & 7) + (k >> 3) * 64) * 2;
    *reinterpret_cast<__nv_bfloat16*>(g + NTILE * kE1Tile + off) = hi;
    *reinterpret_cast<__nv_bfloat16*>(g + NTILE * kE1Tile + C1 * 64 + off) =
        __float2bfloat16_rn(w - __bfloat162float(hi));
  }
  for (int e = tid; e < C1; e += 256) bias_s[e] = B[e];
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  uint32_t tmem = 0, phase = 0;
#pragma unroll 1
  for (;;) {
    // (the previous tile's epilogue has left the A tiles and tensor memory: block barrier below)
    if (P->coarse_f) enc1_stage_finish<float, BH>(P, Y0, ld, xs, T);
    else enc1_stage_finish<int16_t, BH>(P, Y0, ld, xs, T);
    // A rows: warp w builds block rows RPW w .. RPW w + RPW - 1 (tile oy / 4, row j = oy % 4);
    // lane = output column
#pragma unroll 1
    for (int jj = 0; jj < RPW; ++jj) {
      const int oy = RPW * warp + jj, j = oy & 3, tile = oy >> 2;
      float v[32];
#pragma unroll
      for (int ky = 0; ky < 3; ++ky)
#pragma unroll
        for (int kx = 0; kx < 3; ++kx) {
          const float2 tv = *reinterpret_cast<const float2*>(&xs[2 * oy + ky][2 * lane + kx][0]);
          const float uh = __bfloat162float(__float2bfloat16_rn(tv.y));
          const int k = 3 * (ky * 3 + kx);
          v[k] = tv.x;
          v[k + 1] = uh;
          v[k + 2] = tv.y - uh;
        }
#pragma unroll
      for (int k = 27; k < 32; ++k) v[k] = 0.f;
      const int m = 32 * j + lane;
      unsigned char* row = g + (size_t)tile * kE1Tile + (m & 7) * 16 + (m >> 3) * 512;
#pragma unroll
      for (int kc = 0; kc < 4; ++kc)
        *reinterpret_cast<uint4*>(row + kc * 128) =
            make_uint4(pack_bf16x2(v[8 * kc], v[8 * kc + 1]), pack_bf16x2(v[8 * kc + 2], v[8 * kc + 3]),
                       pack_bf16x2(v[8 * kc + 4], v[8 * kc + 5]), pack_bf16x2(v[8 * kc + 6], v[8 * kc + 7]));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    tmem = *tslot;
    if (tid == 0) {
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(C1 >> 3) << 17) | ((128u >> 4) << 24);
#pragma unroll
      for (int tt = 0; tt < NTILE; ++tt) {
        const uint64_t a = desc_ns_e(sA + tt * kE1Tile, 512);
        const uint32_t d = tmem + tt * C1;
        // K step of 16 = two core matrices along K = +256 B (+16 in the start field)
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) mma_bf16_e(d, a + 16 * ks, desc_ns_e(sBh, 256 * 2) + 16 * ks, idesc, ks);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) mma_bf16_e(d, a + 16 * ks, desc_ns_e(sBl, 256 * 2) + 16 * ks, idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                   : "memory");
    }
    __syncwarp();
    // the next tile's window loads go out now, ahead of the wait and the stores below
    int nX0 = 0, nY0 = 0;
    const int nt = enc1_next_tile(pairs, t + (int)gridDim.x, gx, per, ntiles, BH, nX0, nY0);
    const EdgePair* nP = pairs + (nt < ntiles ? nt / per : 0);
    if (nt < ntiles) {
      if (nP->coarse_f) enc1_stage_load<float, BH>(nP, nP->coarse_f, nX0, nY0, ld);
      else enc1_stage_load<int16_t, BH>(nP, nP->coarse, nX0, nY0, ld);
    }
    // lane 0 of each warp waits for the accumulators and tells the warp
    bool got = lane != 0 || mbar_wait_e(mbar, phase, spin);
    got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
    if (!got) {
      if (lane == 0) atomicCAS(err, 0, 7);
      // the MMAs may still be running: wait (bounded) before the allocation is released
      if (lane == 0) mbar_wait_e(mbar, phase, spin > 2000000000LL ? spin : 2000000000LL);
      __syncwarp();
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (got) {
      const int q = warp & 3;
      const int H1 = (P->H + 1) / 2, W1 = (P->W + 1) / 2;
      // 16 accumulator columns per tensor-memory load, which keeps the registers of the
      // epilogue low enough for the next window's loads to stay in flight beside it
#pragma unroll 1
      for (int tt = warp >> 2; tt < NTILE; tt += 2) {
        const int Y = Y0 + 4 * tt + q, X = X0 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(tt * C1);
        uint4* sw = reinterpret_cast<uint4*>(g) + warp * 128;
#pragma unroll
        for (int c0 = 0; c0 < C1; c0 += 16) {
          uint32_t r[32];
          tmem_ld16_e(taddr + c0, r);
          if (P->e1q) {
            // FP8 form: E4M3 codes of the BF16-rounded output (16 per 16-byte store)
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 16; e += 4) {
              float qv[4];
#pragma unroll
              for (int u = 0; u < 4; ++u)
                qv[u] = __bfloat162float(
                    __float2bfloat16_rn(fmaxf(__uint_as_float(r[e + u]) + bias_s[c0 + e + u], 0.f)));
              pk[e / 4] = (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(qv[0], qv[1]), __NV_SATFINITE, __NV_E4M3) |
                          ((uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(qv[2], qv[3]), __NV_SATFINITE, __NV_E4M3)
                           << 16);
            }
            if (X < W1 && Y < H1)
              *reinterpret_cast<uint4*>(P->e1q + ((size_t)Y * W1 + X) * C1 + c0) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
            continue;
          }
          uint32_t pk[8];
#pragma unroll
          for (int e = 0; e < 16; e += 2) {
            const float2 v = __fadd2_rn(make_float2(__uint_as_float(r[e]), __uint_as_float(r[e + 1])),
                                        make_float2(bias_s[c0 + e], bias_s[c0 + e + 1]));
            const __nv_bfloat162 h = __hmax2(__floats2bfloat162_rn(v.x, v.y), __float2bfloat162_rn(0.f));
            pk[e / 2] = *reinterpret_cast<const uint32_t*>(&h);
          }
          if (C1 == 16) {
            if (X < W1 && Y < H1) {
              uint4* dst = reinterpret_cast<uint4*>(P->e1 + ((size_t)Y * W1 + X) * C1);
              dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
              dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
            }
            continue;
          }
          // through a 2 KB stage per warp in the (now free) A tiles: lane = pixel writes the
          // four 16-byte pieces of a 32-channel group (piece qq at slot qq ^ ((pixel >> 1) & 3):
          // conflict-free), two per 16-column load; then four lanes per pixel store its
          // 64 bytes, eight pixels (512 bytes) per instruction
          const int h = (c0 >> 4) & 1;
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const int qq = 2 * h + u;
            sw[lane * 4 + (qq ^ ((lane >> 1) & 3))] = make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
          }
          if (h == 1) {
            __syncwarp();
            const int cg = c0 - 16;
#pragma unroll
            for (int s8 = 0; s8 < 4; ++s8) {
              const int pp = 8 * s8 + (lane >> 2), qq = lane & 3;
              const uint4 v = sw[pp * 4 + (qq ^ ((pp >> 1) & 3))];
              if (X0 + pp < W1 && Y < H1)
                *reinterpret_cast<uint4*>(P->e1 + ((size_t)Y * W1 + X0 + pp) * C1 + cg + 8 * qq) = v;
            }
            __syncwarp();
          }
        }
      }
    }
    // tensor memory read and the stage drained before the next tile's A build and MMAs
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    const int failed = __syncthreads_or(got ? 0 : 1);
    phase ^= 1u;
    if (failed || nt >= ntiles) break;
    t = nt;
    P = nP;
    X0 = nX0;
    Y0 = nY0;
  }
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NTILE * C1));
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
    const bool in = vy >= 0 && vy < P.H && vx >= 0 && vx < P.W;
    cp_async16(tile + pix * pstride + q, in ? P.d3 + ((size_t)vy * P.W + vx) * C + q * 8 : P.d3, in);
  }
  cp_async_wait_all();
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

// final, register-blocked form for C in {16, 32, 64, 128}: TPP = C / 8 threads per output
// column, each holding the 9 x 8 weights of its 8 channels in registers and computing RPT
// consecutive output rows of its column, so each staged 8-channel load serves up to three
// output rows.  Packed FP32 FMA (two channels per instruction); the TPP partial sums of a
// pixel are added with xor shuffles.  Tile: 32 columns x TH rows; its (TH + 2) x 34 x C
// BF16 input (pixels contiguous: the 16-byte reads of 8 consecutive lanes hit 8 distinct
// bank groups) arrives by one TMA box, zero-filled outside the map.
template <int C>
struct FinalGeo {
  static constexpr int TPP = C / 8, RPT = 16, RGN = TPP >= 8 ? 1 : 8 / TPP;
  static constexpr int NTH = 32 * TPP * RGN, TW = 32, TH = RPT * RGN, SR = TH + 2, SC = TW + 2;
  static constexpr uint32_t tile_bytes = (uint32_t)SR * SC * C * 2;
  static constexpr size_t smem = tile_bytes + 128 + 9 * C * 4;  // tile (+ alignment slack), FP32 weights
};

template <int C>
__global__ void __launch_bounds__(FinalGeo<C>::NTH) edge_final_rb(const EdgePair* __restrict__ pairs,
                                                                 const float* __restrict__ W,
                                                                 const float* __restrict__ B, int* err,
                                                                 long long spin) {
  using G = FinalGeo<C>;
  constexpr int TPP = G::TPP, RPT = G::RPT, TW = G::TW, TH = G::TH, SC = G::SC;
  extern __shared__ unsigned char fraw[];
  __shared__ __align__(8) uint64_t fbar;
  const EdgePair* P = pairs + blockIdx.z;
  const int Wd = P->W, Hd = P->H;
  const int X0 = blockIdx.x * TW, Y0 = blockIdx.y * TH;
  if (X0 >= Wd || Y0 >= Hd) return;
  const uint32_t tile_s = ((uint32_t)__cvta_generic_to_shared(fraw) + 127u) & ~127u;
  const uint4* ftile = reinterpret_cast<const uint4*>(fraw + (tile_s - (uint32_t)__cvta_generic_to_shared(fraw)));
  const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&fbar);
  const int tid = threadIdx.x;
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(&P->d3_map))
                 : "memory");
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar),
                 "r"(G::tile_bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
            tile_s),
        "l"(reinterpret_cast<uint64_t>(&P->d3_map)), "r"(0), "r"(X0 - 1), "r"(Y0 - 1), "r"(bar)
        : "memory");
  }
  const int rg = tid / (32 * TPP), rem = tid - rg * 32 * TPP, cx = rem / TPP, q = rem - cx * TPP;
  float* ws = reinterpret_cast<float*>(fraw + 128 + G::tile_bytes);  // [9][C]
  for (int e = tid; e < 9 * C; e += G::NTH) ws[e] = W[e];
  // residual U (bilinear x4 of the coarse map) of the rows this lane writes, k = q + e TPP:
  // its global loads overlap the tile copy
  constexpr int NE = (RPT + TPP - 1) / TPP;
  const int X = X0 + cx;
  float Ue[NE];
  {
    const int16_t* coarse = P->coarse;
    const float* coarse_f = P->coarse_f;
    const int w4 = P->w, h4 = P->h;
    const int Xc = min(X, Wd - 1);
#pragma unroll
    for (int e = 0; e < NE; ++e) {
      const int Yr = min(Y0 + rg * RPT + q + e * TPP, Hd - 1);
      Ue[e] = coarse_f ? upsample4_f(coarse_f, w4, h4, Xc, Yr) : upsample4_f(coarse, w4, h4, Xc, Yr);
    }
  }
  __syncthreads();  // barrier initialised
  if (!mbar_wait_e(bar, 0, spin)) {
    atomicCAS(err, 0, 6);
    // the copy may still land: no thread leaves while it can write this block's memory
    mbar_wait_e(bar, 0, spin > 2000000000LL ? spin : 2000000000LL);
    return;
  }
  float2 acc[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) acc[k] = make_float2(0.f, 0.f);
#pragma unroll
  for (int kx = 0; kx < 3; ++kx) {
    // this lane's 8 channels of the three taps of column kx (broadcast reads)
    float2 w[3][4];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky) {
      const float4 lo = *reinterpret_cast<const float4*>(ws + (ky * 3 + kx) * C + q * 8);
      const float4 hi = *reinterpret_cast<const float4*>(ws + (ky * 3 + kx) * C + q * 8 + 4);
      w[ky][0] = make_float2(lo.x, lo.y);
      w[ky][1] = make_float2(lo.z, lo.w);
      w[ky][2] = make_float2(hi.x, hi.y);
      w[ky][3] = make_float2(hi.z, hi.w);
    }
#pragma unroll
    for (int r = 0; r < RPT + 2; ++r) {
      const uint4 v = ftile[((rg * RPT + r) * SC + cx + kx) * TPP + q];
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
      float2 a[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) a[j] = __bfloat1622float2(h[j]);
      // staged row r feeds output row k = r - ky of this thread's column
#pragma unroll
      for (int ky = 0; ky < 3; ++ky) {
        const int k = r - ky;
        if (k >= 0 && k < RPT) {
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[k] = __ffma2_rn(a[j], w[ky][j], acc[k]);
        }
      }
    }
  }
  float sum[RPT];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    sum[k] = acc[k].x + acc[k].y;
#pragma unroll
    for (int o = TPP / 2; o > 0; o >>= 1) sum[k] += __shfl_xor_sync(0xffffffffu, sum[k], o);
  }
  if (X >= Wd) return;
  const float b = B[0];
  float* Y = P->Y;
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    if (k % TPP != q) continue;  // the TPP lanes of a column share the rows' epilogue
    const int Yr = Y0 + rg * RPT + k;
    if (Yr >= Hd) break;
    Y[(size_t)Yr * Wd + X] = Ue[k / TPP] + (b + sum[k]);
  }
}

// Exact last row / column of a nearest-x2 + 3x3 conv with an odd (cropped) output size.
// At those pixels one tap row (column) of the 3x3 window falls on the cropped-away part of
// the up-sampled map and must read zero, which the 4-phase form cannot express; only the
// six other taps contribute.  One block per (segment of kUpFixSeg border pixels, 32 output
// channels, pair), chunks of kFixCk input channels at a time:
//   S[a][q][c]   the two up-sampled rows (row fix) or columns (column fix) that can be
//                non-zero, positions p0 - 1 + q along the border, FP32, zero outside the crop
//   Wf[t][c][o]  the six live taps t = 3a + b of the BF16-rounded weights, FP32
// Lane = output channel (conflict-free weight reads), warp = 8 consecutive border pixels
// (broadcast S reads); FP32 accumulation as in the tensor-core form.
constexpr int kFixCk = 64;
constexpr int kFixQ = kUpFixSeg + 2;
constexpr size_t kFixSmem = sizeof(float) * (2 * kFixQ * kFixCk + 6 * kFixCk * 32);

__device__ __forceinline__ void bf16x8_to_f32(const uint4& v, float* d) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&v);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float2 f = __bfloat1622float2(h[j]);
    d[2 * j] = f.x;
    d[2 * j + 1] = f.y;
  }
}

__global__ void __launch_bounds__(256) edge_up2fix(const UpFixPair* __restrict__ pairs, const bf16* __restrict__ Wb,
                                                   const float* __restrict__ bias, int cin, int cout, int relu) {
  extern __shared__ __align__(16) float xsm[];
  float* S = xsm;                          // [2][kFixQ][kFixCk]
  float* Wf = xsm + 2 * kFixQ * kFixCk;    // [6][kFixCk][32]
  const UpFixPair L = pairs[blockIdx.z];
  const int nrow = (L.Ho & 1) ? L.Wo : 0;               // last row, every column
  const int ncol = (L.Wo & 1) ? L.Ho - (L.Ho & 1) : 0;  // last column, rows above a fixed last row
  const int segr = (nrow + kUpFixSeg - 1) / kUpFixSeg, segc = (ncol + kUpFixSeg - 1) / kUpFixSeg;
  int seg = blockIdx.x;
  if (seg >= segr + segc) return;
  const bool rowfix = seg < segr;
  if (!rowfix) seg -= segr;
  const int p0 = seg * kUpFixSeg;
  const int npix = min(kUpFixSeg, (rowfix ? nrow : ncol) - p0);
  const int cb = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.f;
  for (int c0 = 0; c0 < cin; c0 += kFixCk) {
    const int ck = min(kFixCk, cin - c0), c8 = ck / 8;
    __syncthreads();  // the previous chunk has been consumed
    // row fix: up rows Ho-2, Ho-1 (a = ky) x up columns p0-1+q; column fix: up columns
    // Wo-2, Wo-1 (a = kx) x up rows p0-1+q
    // loads of 4 elements per thread are issued before any is converted and stored
    constexpr int U = 4;
    for (int e0 = threadIdx.x; e0 < 2 * kFixQ * c8; e0 += U * blockDim.x) {
      uint4 v[U];
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int e = e0 + i * (int)blockDim.x;
        const int a = e / (kFixQ * c8), r = e - a * kFixQ * c8, q = r / c8, u = r - q * c8;
        const int uy = rowfix ? L.Ho - 2 + a : p0 - 1 + q;
        const int ux = rowfix ? p0 - 1 + q : L.Wo - 2 + a;
        v[i] = make_uint4(0, 0, 0, 0);
        if (e < 2 * kFixQ * c8 && uy >= 0 && uy < L.Ho && ux >= 0 && ux < L.Wo)
          v[i] = *reinterpret_cast<const uint4*>(L.in + ((size_t)(uy >> 1) * L.Wi + (ux >> 1)) * cin + c0 + u * 8);
      }
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int e = e0 + i * (int)blockDim.x;
        if (e >= 2 * kFixQ * c8) break;
        const int a = e / (kFixQ * c8), r = e - a * kFixQ * c8, q = r / c8, u = r - q * c8;
        bf16x8_to_f32(v[i], S + ((size_t)a * kFixQ + q) * kFixCk + u * 8);
      }
    }
    // tap t = 3a + b: (ky, kx) = (a, b) for the row fix, (b, a) for the column fix
    for (int e0 = threadIdx.x; e0 < 6 * c8 * 32; e0 += U * blockDim.x) {
      uint4 v[U];
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int e = e0 + i * (int)blockDim.x;
        const int o = e & 31, r = e >> 5, t = r / c8, u = r - t * c8;
        const int a = t / 3, b = t - 3 * a, ky = rowfix ? a : b, kx = rowfix ? b : a;
        v[i] = make_uint4(0, 0, 0, 0);
        if (e < 6 * c8 * 32 && cb + o < cout)
          v[i] = *reinterpret_cast<const uint4*>(Wb + ((size_t)((cb + o) * 3 + ky) * 3 + kx) * cin + c0 + u * 8);
      }
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int e = e0 + i * (int)blockDim.x;
        if (e >= 6 * c8 * 32) break;
        const int o = e & 31, r = e >> 5, t = r / c8, u = r - t * c8;
        float f[8];
        bf16x8_to_f32(v[i], f);
        float* d = Wf + ((size_t)t * kFixCk + u * 8) * 32 + o;
#pragma unroll
        for (int j = 0; j < 8; ++j) d[j * 32] = f[j];
      }
    }
    __syncthreads();
    for (int t = 0; t < 6; ++t) {
      const int a = t / 3, b = t - 3 * a;
      const float* sp = S + ((size_t)a * kFixQ + warp * 8 + b) * kFixCk;
      const float* wp = Wf + (size_t)t * kFixCk * 32 + lane;
      for (int c = 0; c < ck; c += 4) {
        const float w0 = wp[(c + 0) * 32], w1 = wp[(c + 1) * 32], w2 = wp[(c + 2) * 32], w3 = wp[(c + 3) * 32];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 x = *reinterpret_cast<const float4*>(sp + j * kFixCk + c);
          acc[j] = fmaf(w0, x.x, acc[j]);
          acc[j] = fmaf(w1, x.y, acc[j]);
          acc[j] = fmaf(w2, x.z, acc[j]);
          acc[j] = fmaf(w3, x.w, acc[j]);
        }
      }
    }
  }
  const int co = cb + lane;
  if (co >= cout) return;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = warp * 8 + j;
    if (p >= npix) break;
    const int Y = rowfix ? L.Ho - 1 : p0 + p, X = rowfix ? p0 + p : L.Wo - 1;
    float v = bias[co] + acc[j];
    if (relu) v = fmaxf(v, 0.f);
    L.out[((size_t)Y * L.Wo + X) * cout + co] = __float2bfloat16_rn(v);
  }
}

// The border recompute of the FP8 form: the same geometry and pixel / channel mapping, on
// E4M3 input codes (`in` holds bytes) and the E4M3 codes of the unfolded 3 x 3 weights with
// their per-output-channel scale: relu(scale * sum(code * code) + bias), stored as E4M3
// codes (out_f8) or BF16 (the last decoder layer, whose output feeds the BF16 final conv).
__device__ __forceinline__ float e4m3_value(uint8_t c) {
  __nv_fp8_e4m3 x;
  x.__x = c;
  return static_cast<float>(x);
}

// sixteen E4M3 codes (one 16-byte word) to FP32, two at a time through the paired conversion
__device__ __forceinline__ void e4m3x16_to_f32(const uint4& v, float* d) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const __half2_raw hr = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)((w[k] >> (16 * h)) & 0xFFFFu), __NV_E4M3);
      const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&hr));
      d[4 * k + 2 * h] = f.x;
      d[4 * k + 2 * h + 1] = f.y;
    }
}

__global__ void __launch_bounds__(256) edge_up2fix_f8(const UpFixPair* __restrict__ pairs, const uint8_t* __restrict__ Wq,
                                                      const float* __restrict__ wscale, const float* __restrict__ bias,
                                                      int cin, int cout, int relu, int out_f8) {
  extern __shared__ __align__(16) float xsm8[];
  float* S = xsm8;                          // [2][kFixQ][kFixCk]
  float* Wf = xsm8 + 2 * kFixQ * kFixCk;    // [6][kFixCk][32]
  const UpFixPair L = pairs[blockIdx.z];
  const uint8_t* in = reinterpret_cast<const uint8_t*>(L.in);
  const int nrow = (L.Ho & 1) ? L.Wo : 0;
  const int ncol = (L.Wo & 1) ? L.Ho - (L.Ho & 1) : 0;
  const int segr = (nrow + kUpFixSeg - 1) / kUpFixSeg, segc = (ncol + kUpFixSeg - 1) / kUpFixSeg;
  int seg = blockIdx.x;
  if (seg >= segr + segc) return;
  const bool rowfix = seg < segr;
  if (!rowfix) seg -= segr;
  const int p0 = seg * kUpFixSeg;
  const int npix = min(kUpFixSeg, (rowfix ? nrow : ncol) - p0);
  const int cb = blockIdx.y * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float acc[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) acc[j] = 0.f;
  for (int c0 = 0; c0 < cin; c0 += kFixCk) {
    const int ck = min(kFixCk, cin - c0);
    __syncthreads();
    // 16 codes per 16-byte load (cin is a multiple of 32); a thread's loads are all issued
    // before any is decoded
    const int c16 = ck / 16;
    constexpr int U = 4;
    for (int e0 = threadIdx.x; e0 < 2 * kFixQ * c16; e0 += U * blockDim.x) {
      uint4 v[U];
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int e = e0 + i * (int)blockDim.x;
        const int a = e / (kFixQ * c16), r = e - a * kFixQ * c16, q = r / c16, u = r - q * c16;
        const int uy = rowfix ? L.Ho - 2 + a : p0 - 1 + q;
        const int ux = rowfix ? p0 - 1 + q : L.Wo - 2 + a;
        v[i] = make_uint4(0, 0, 0, 0);
        if (e < 2 * kFixQ * c16 && uy >= 0 && uy < L.Ho && ux >= 0 && ux < L.Wo)
          v[i] = *reinterpret_cast<const uint4*>(in + ((size_t)(uy >> 1) * L.Wi + (ux >> 1)) * cin + c0 + u * 16);
      }
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int e = e0 + i * (int)blockDim.x;
        if (e >= 2 * kFixQ * c16) break;
        const int a = e / (kFixQ * c16), r = e - a * kFixQ * c16, q = r / c16, u = r - q * c16;
        e4m3x16_to_f32(v[i], S + ((size_t)a * kFixQ + q) * kFixCk + u * 16);
      }
    }
    for (int e0 = threadIdx.x; e0 < 6 * c16 * 32; e0 += U * blockDim.x) {
      uint4 v[U];
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int e = e0 + i * (int)blockDim.x;
        const int o = e & 31, r = e >> 5, t = r / c16, u = r - t * c16;
        const int a = t / 3, b = t - 3 * a, ky = rowfix ? a : b, kx = rowfix ? b : a;
        v[i] = make_uint4(0, 0, 0, 0);
        if (e < 6 * c16 * 32 && cb + o < cout)
          v[i] = *reinterpret_cast<const uint4*>(Wq + ((size_t)((cb + o) * 3 + ky) * 3 + kx) * cin + c0 + u * 16);
      }
#pragma unroll
      for (int i = 0; i < U; ++i) {
        const int e = e0 + i * (int)blockDim.x;
        if (e >= 6 * c16 * 32) break;
        const int o = e & 31, r = e >> 5, t = r / c16, u = r - t * c16;
        float f[16];
        e4m3x16_to_f32(v[i], f);
        float* d = Wf + ((size_t)t * kFixCk + u * 16) * 32 + o;
#pragma unroll
        for (int j = 0; j < 16; ++j) d[j * 32] = f[j];
      }
    }
    __syncthreads();
    for (int t = 0; t < 6; ++t) {
      const int a = t / 3, b = t - 3 * a;
      const float* sp = S + ((size_t)a * kFixQ + warp * 8 + b) * kFixCk;
      const float* wp = Wf + (size_t)t * kFixCk * 32 + lane;
      for (int c = 0; c < ck; ++c) {
        const float wv = wp[c * 32];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = fmaf(wv, sp[j * kFixCk + c], acc[j]);
      }
    }
  }
  const int co = cb + lane;
  if (co >= cout) return;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int p = warp * 8 + j;
    if (p >= npix) break;
    const int Y = rowfix ? L.Ho - 1 : p0 + p, X = rowfix ? p0 + p : L.Wo - 1;
    float v = fmaf(acc[j], wscale[co], bias[co]);
    if (relu) v = fmaxf(v, 0.f);
    const size_t o = ((size_t)Y * L.Wo + X) * cout + co;
    if (out_f8)
      reinterpret_cast<uint8_t*>(L.out)[o] = (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3);
    else
      L.out[o] = __float2bfloat16_rn(v);
  }
}

// E4M3 codes of a BF16 activation (the first layer's output in the FP8 form).
__global__ void bf16_to_e4m3(const bf16* __restrict__ a, uint8_t* __restrict__ b, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (uint8_t)__nv_cvt_float_to_fp8(__bfloat162float(a[i]), __NV_SATFINITE, __NV_E4M3);
}

// Training latent heads: a thread per (pixel, output channel).  staged: the weights of both heads are staged
// transposed in shared memory ([ci][co]: consecutive threads read consecutive output
// channels); else (widths whose weights do not fit) read from global memory.
__global__ void train_latent_bf16(const bf16* __restrict__ e3, int P, int Ci, const float* __restrict__ wmu,
                                  const float* __restrict__ bmu, const float* __restrict__ wlv,
                                  const float* __restrict__ blv, int lat, const float* __restrict__ eps,
                                  float* __restrict__ mu, float* __restrict__ lv, bf16* __restrict__ z, int staged) {
  extern __shared__ float tl_sm[];
  float* wm = tl_sm;              // [Ci][lat]
  float* wl = tl_sm + Ci * lat;   // [Ci][lat]
  for (int e = threadIdx.x; staged && e < Ci * lat; e += blockDim.x) {
    const int ci = e / lat, co = e - ci * lat;
    wm[e] = wmu[(size_t)co * Ci + ci];
    wl[e] = wlv[(size_t)co * Ci + ci];
  }
  __syncthreads();
  const size_t n = (size_t)P * lat;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int co = (int)(i % lat);
    const bf16* x = e3 + (i / lat) * Ci;
    float m = bmu[co], l = blv[co];
    for (int ci = 0; ci < Ci; ++ci) {
      const float xv = __bfloat162float(x[ci]);
      m = fmaf(staged ? wm[ci * lat + co] : wmu[(size_t)co * Ci + ci], xv, m);
      l = fmaf(staged ? wl[ci * lat + co] : wlv[(size_t)co * Ci + ci], xv, l);
    }
    mu[i] = m;
    lv[i] = l;
    z[i] = __float2bfloat16_rn(m + eps[i] * expf(0.5f * l));
  }
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
  const bool staged = 2 * sizeof(float) * Ci * lat <= 160 * 1024;
  const size_t smem = staged ? 2 * sizeof(float) * Ci * lat : 0;
  cudaError_t e = cudaFuncSetAttribute(train_latent_bf16, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const unsigned grid = (unsigned)std::min<size_t>((n + 255) / 256, 4 * 152);
  train_latent_bf16<<<grid, 256, smem, st>>>(e3, P, Ci, wmu, bmu, wlv, blv, lat, eps, mu, lv, z, staged ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_edge_up2fix_f8(const UpFixPair* pairs, int n, int max_segments, const uint8_t* Wq,
                                  const float* wscale, const float* bias, int cin, int cout, int relu, int out_f8,
                                  cudaStream_t st) {
  if (n <= 0 || max_segments <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(edge_up2fix_f8, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixSmem);
  if (e != cudaSuccess) return e;
  edge_up2fix_f8<<<dim3(max_segments, (cout + 31) / 32, n), 256, kFixSmem, st>>>(pairs, Wq, wscale, bias, cin, cout,
                                                                                  relu, out_f8);
  return cudaGetLastError();
}

cudaError_t launch_bf16_to_e4m3(const bf16* a, uint8_t* b, size_t n, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  bf16_to_e4m3<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

cudaError_t launch_bf16_to_f32(const bf16* a, float* b, size_t n, cudaStream_t st) {
  bf16_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

// Persistent launch: three blocks per SM (the register bound of the kernel and its shared
// memory under the largest carveout allow three; the occupancy query, which takes the default
// carveout, reports one), two for C1 = 64 (the 512 tensor-memory columns of an SM), never more
// blocks than tiles.
constexpr size_t kE1StaticSmem = sizeof(float) * (E1Geo<kE1TcBH>::R * E1C * 2 + E1Geo<kE1TcBH>::CR * E1C);
static_assert(kE1BlocksPerSm * (enc1_tc_smem(64) + kE1StaticSmem + 1024) <= 228 * 1024,
              "three enc1 blocks must fit the shared memory of an SM");
template <int C1>
static cudaError_t run_enc1_tc(const EdgePair* pairs, int n, int maxW1, int maxH1, const float* W, const float* B,
                               int* err, long long spin, cudaStream_t st) {
  const size_t smem = enc1_tc_smem(C1);
  cudaError_t e = cudaFuncSetAttribute(enc1_tc<C1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(enc1_tc<C1>, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int per_sm = std::min(kE1BlocksPerSm, 512 / (kE1Tiles * C1));
  const int gx = (maxW1 + E1W - 1) / E1W, gy = (maxH1 + kE1TcBH - 1) / kE1TcBH;
  const long long tiles = (long long)gx * gy * n;
  if (tiles <= 0) return cudaSuccess;
  if (tiles > INT_MAX) return cudaErrorInvalidValue;
  const int grid = (int)std::min<long long>(tiles, (long long)nsm * per_sm);
  enc1_tc<C1><<<grid, 256, smem, st>>>(pairs, gx, gy, (int)tiles, W, B, err, spin);
  return cudaGetLastError();
}

cudaError_t launch_edge_enc1(const EdgePair* pairs, int n, int maxW1, int maxH1, const float* W, const float* B, int C1,
                             int* err, long long spin, bool tensor, cudaStream_t st) {
  if (tensor && C1 == 32) return run_enc1_tc<32>(pairs, n, maxW1, maxH1, W, B, err, spin, st);
  if (tensor && C1 == 16) return run_enc1_tc<16>(pairs, n, maxW1, maxH1, W, B, err, spin, st);
  if (tensor && C1 == 64) return run_enc1_tc<64>(pairs, n, maxW1, maxH1, W, B, err, spin, st);
  dim3 grid((maxW1 + E1W - 1) / E1W, (maxH1 + E1H - 1) / E1H, n);
  edge_enc1<<<grid, 256, sizeof(float) * 19 * C1, st>>>(pairs, W, B, C1);
  return cudaGetLastError();
}

template <int C>
static cudaError_t run_final_rb(const EdgePair* pairs, int n, int maxW, int maxH, const float* W, const float* B,
                                int* err, long long spin, cudaStream_t st) {
  using G = FinalGeo<C>;
  static_assert(G::TH == 16 * (C / 8 >= 8 ? 1 : 8 / (C / 8)), "tile height must match final_tile_rows()");
  dim3 grid((maxW + G::TW - 1) / G::TW, (maxH + G::TH - 1) / G::TH, n);
  if (G::smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(edge_final_rb<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)G::smem);
    if (e != cudaSuccess) return e;
  }
  edge_final_rb<C><<<grid, G::NTH, G::smem, st>>>(pairs, W, B, err, spin);
  return cudaGetLastError();
}

template <int C>
static cudaError_t run_final(const EdgePair* pairs, int n, int maxW, int maxH, const float* W, const float* B,
                             int* err, long long spin, cudaStream_t st) {
  if constexpr (C == 16 || C == 32 || C == 64 || C == 128)
    return run_final_rb<C>(pairs, n, maxW, maxH, W, B, err, spin, st);
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
                              int* err, long long spin, cudaStream_t st) {
  switch (C) {  // decoder widths are multiples of 16 up to 256
#define SV_FINAL_CASE(c) \
  case c: return run_final<c>(pairs, n, maxW, maxH, W, B, err, spin, st);
    SV_FINAL_CASE(16) SV_FINAL_CASE(32) SV_FINAL_CASE(48) SV_FINAL_CASE(64) SV_FINAL_CASE(80) SV_FINAL_CASE(96)
    SV_FINAL_CASE(112) SV_FINAL_CASE(128) SV_FINAL_CASE(144) SV_FINAL_CASE(160) SV_FINAL_CASE(176) SV_FINAL_CASE(192)
    SV_FINAL_CASE(208) SV_FINAL_CASE(224) SV_FINAL_CASE(240) SV_FINAL_CASE(256)
#undef SV_FINAL_CASE
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_edge_up2fix(const UpFixPair* pairs, int n, int max_segments, const bf16* Wb, const float* bias,
                               int cin, int cout, int relu, cudaStream_t st) {
  if (cin % 8 != 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(edge_up2fix, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFixSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)std::max(1, max_segments), (unsigned)((cout + 31) / 32), (unsigned)n);
  edge_up2fix<<<grid, 256, kFixSmem, st>>>(pairs, Wb, bias, cin, cout, relu);
  return cudaGetLastError();
}

}  // namespace sv
