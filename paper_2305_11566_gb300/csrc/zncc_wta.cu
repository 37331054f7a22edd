// zncc_wta.cu -- K1: fused quarter-size downsample + ZNCC (Eq. 1-3) + winner-take-all
// (Eq. 6) for many pairs in one launch.
//
// One CTA job = one pair, kZnccTY coarse rows, kZnccWarps * TX coarse columns.
//  stage 1  4x4 box sums S (uint16, exact) of the rows/columns the job touches,
//           window positions outside the image clamped to the edge;
//  stage 2  per-window sums sum(S) and exact variance v = N sum(S^2) - sum(S)^2 for every
//           left window of the job and every right window any candidate can reach
//           (right windows are shared across disparities); 1/sigma = rsqrt(v), 0 if v == 0;
//  stage 3  each warp owns TX output columns, lane l the disparities d = l + 32 kd.
//           Column sums of L(u, .) * R(u - d, .) over the window rows live in registers
//           and slide down the rows (add the entering row, drop the leaving one); the
//           window sum slides along x.  All sums are exact integers; the numerator
//           n = N sum(LR) - sum(L) sum(R) is exact in int64, and
//           rho = float(n) * (1/sigma_L) * (1/sigma_R).  The argmax over d is two warp
//           reductions (__reduce_max_sync on an order-preserving integer key, then
//           __reduce_min_sync on d among the maxima: lowest d wins ties).
//           MODE 2 (cost volume): every lane also stores the cost 1 - rho of its candidates (Eq. 1; 2,
//           the largest value, where x - d < 0) into the pair's volume [h][w][D]: lanes hold
//           consecutive d, so a warp's stores of one pixel are contiguous.
#include "sv_internal.cuh"

namespace sv {

namespace {

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Order-preserving map float -> int (for finite values): larger float, larger int.
__device__ __forceinline__ int order_key(float f) {
  int i = __float_as_int(f + 0.0f);  // -0 -> +0
  return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}
__device__ __forceinline__ float key_value(int k) {
  if (k == INT_MIN) return -2.0f;
  return __int_as_float(k >= 0 ? k : (k ^ 0x7FFFFFFF));
}

// Stage 4x4 box sums of rows y0 - R .. y0 + TY + R - 1 (clamped) and columns base_c ..
// base_c + ncols - 1 (clamped) into dst[row][col]; the loads of 8 elements per thread are
// all issued before any is summed (one memory round trip per 8 elements, not per element).
template <int R>
__device__ __forceinline__ void stage_box(const uint8_t* __restrict__ img, int pitch, int w, int h, int base_c,
                                          int y0, int ncols, uint16_t* dst) {
  const int n = (kZnccTY + 2 * R) * ncols;
  constexpr int U = 8;
  for (int e0 = threadIdx.x; e0 < n; e0 += U * blockDim.x) {
    unsigned v[U][4];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = min(e0 + u * (int)blockDim.x, n - 1);
      const int ry = e / ncols, c = e - ry * ncols;
      const uint8_t* p = img + (size_t)(4 * clampi(y0 - R + ry, 0, h - 1)) * pitch + 4 * clampi(base_c + c, 0, w - 1);
#pragma unroll
      for (int j = 0; j < 4; ++j) v[u][j] = *reinterpret_cast<const unsigned*>(p + (size_t)j * pitch);  // 4u: aligned
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int e = e0 + u * (int)blockDim.x;
      if (e < n) {
        unsigned t = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
          t += (v[u][j] & 0xFFu) + ((v[u][j] >> 8) & 0xFFu) + ((v[u][j] >> 16) & 0xFFu) + (v[u][j] >> 24);
        dst[e] = (uint16_t)t;
      }
    }
  }
}

// Vertical then horizontal window sums of S over rows [yi, yi + 2r] for each of the
// TY output rows; writes sum and 1/sigma for `ncols_out` windows starting at column
// `c0` of the staged array (staged column c0 + t is the window's left edge), either to
// sum_out / inv_out or, packed as {sum, bits of 1/sigma}, to packed.
template <int R>
__device__ void window_stats(const uint16_t* s, int ncols, int* cs, unsigned* cs2, int* sum_out, float* inv_out,
                             int2* packed, int ncols_out) {
  const int TY = kZnccTY;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    int a = 0;
    unsigned a2 = 0;
#pragma unroll
    for (int j = 0; j <= 2 * R; ++j) {
      unsigned v = s[j * ncols + c];
      a += (int)v;
      a2 += v * v;
    }
    cs[c] = a;
    cs2[c] = a2;
    for (int yi = 1; yi < TY; ++yi) {
      unsigned vin = s[(yi + 2 * R) * ncols + c], vout = s[(yi - 1) * ncols + c];
      a += (int)vin - (int)vout;
      a2 += vin * vin - vout * vout;  // exact modulo 2^32, true value < 2^32
      cs[yi * ncols + c] = a;
      cs2[yi * ncols + c] = a2;
    }
  }
  __syncthreads();
  const long long N = (long long)(2 * R + 1) * (2 * R + 1);
  for (int e = threadIdx.x; e < TY * ncols_out; e += blockDim.x) {
    int yi = e / ncols_out, t = e - yi * ncols_out;
    int a = 0;
    unsigned a2 = 0;
#pragma unroll
    for (int i = 0; i <= 2 * R; ++i) {
      a += cs[yi * ncols + t + i];
      a2 += cs2[yi * ncols + t + i];
    }
    long long v = N * (long long)a2 - (long long)a * a;
    const float inv = v > 0 ? __frsqrt_rn((float)v) : 0.0f;
    if (packed) {
      packed[e] = make_int2(a, __float_as_int(inv));
    } else {
      sum_out[e] = a;
      inv_out[e] = inv;
    }
  }
  __syncthreads();
}

// MODE 0: disparity only; 1: also best / second scores; 2: also the cost volume.
template <int R, int KD, int TX, int MODE>
__global__ void __launch_bounds__(kZnccWarps * 32, (KD == 1 || (KD == 2 && R <= 5)) ? 2 : 1)
zncc_wta_kernel(const ZPair* __restrict__ pairs, const ZJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int TY = kZnccTY;
  const ZJob job = jobs[blockIdx.x];
  const ZPair P = pairs[job.pair];
  const int D = P.D, w = P.w, h = P.h;
  const ZLayout Z = zlayout(R, D, TX);
  uint16_t* sL = reinterpret_cast<uint16_t*>(smem + Z.off_sl);
  uint16_t* sR = reinterpret_cast<uint16_t*>(smem + Z.off_sr);
  int* sumL = reinterpret_cast<int*>(smem + Z.off_suml);
  float* invL = reinterpret_cast<float*>(smem + Z.off_invl);
  int2* statR = reinterpret_cast<int2*>(smem + Z.off_statr);  // {sum, 1/sigma bits} of each right window
  int* cs = reinterpret_cast<int*>(smem + Z.off_cs);
  unsigned* cs2 = reinterpret_cast<unsigned*>(smem + Z.off_cs2);
  const int y0 = job.y0, x0 = job.x0;
  const int lbase = x0 - R;               // coarse column of staged left column 0
  const int rbase = x0 - R - (D - 1);     // coarse column of staged right column 0

  // ---- stage 1: box sums, clamped rows / columns
  stage_box<R>(P.L, P.pitch, w, h, lbase, y0, Z.nlc, sL);
  stage_box<R>(P.R, P.pitch, w, h, rbase, y0, Z.nrc, sR);
  __syncthreads();
  // ---- stage 2: window statistics (left windows at x0 + t; right windows at rbase + R + t)
  window_stats<R>(sL, Z.nlc, cs, cs2, sumL, invL, nullptr, Z.gx);
  window_stats<R>(sR, Z.nrc, cs, cs2, nullptr, nullptr, statR, Z.nrs);

  // ---- stage 3: sliding ZNCC + WTA
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int xw = x0 + warp * TX;          // first output column of this warp
  if (xw >= w) return;                    // all of this warp's columns lie beyond the image
  const int lc0 = warp * TX;              // staged left column of u = xw - R
  const long long N = (long long)(2 * R + 1) * (2 * R + 1);
  int dd[KD], rc0[KD];
#pragma unroll
  for (int k = 0; k < KD; ++k) {
    int d = lane + 32 * k;
    dd[k] = d < D ? d : D - 1;            // reads stay in the staged range; masked below
    rc0[k] = lc0 - dd[k] + (D - 1);       // staged right column of u - d for u = xw - R
  }
  unsigned colsum[KD][TX + 2 * R];
#pragma unroll
  for (int c = 0; c < TX + 2 * R; ++c) {
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      unsigned a = 0;
#pragma unroll
      for (int j = 0; j <= 2 * R; ++j) a += (unsigned)sL[j * Z.nlc + lc0 + c] * (unsigned)sR[j * Z.nrc + rc0[k] + c];
      colsum[k][c] = a;
    }
  }
  for (int yi = 0; yi < TY; ++yi) {
    const int y = y0 + yi;
    if (yi > 0) {
      const int rin = yi + 2 * R, rout = yi - 1;
#pragma unroll
      for (int c = 0; c < TX + 2 * R; ++c) {
        unsigned lin = sL[rin * Z.nlc + lc0 + c], lout = sL[rout * Z.nlc + lc0 + c];
#pragma unroll
        for (int k = 0; k < KD; ++k)
          colsum[k][c] += lin * (unsigned)sR[rin * Z.nrc + rc0[k] + c] - lout * (unsigned)sR[rout * Z.nrc + rc0[k] + c];
      }
    }
    unsigned run[KD];
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      unsigned a = 0;
#pragma unroll
      for (int i = 0; i <= 2 * R; ++i) a += colsum[k][i];
      run[k] = a;
    }
    int my_d = 0, my_b = INT_MIN, my_s = INT_MIN;
#pragma unroll
    for (int t = 0; t < TX; ++t) {
      if (t > 0) {
#pragma unroll
        for (int k = 0; k < KD; ++k) run[k] += colsum[k][t + 2 * R] - colsum[k][t - 1];
      }
      const int x = xw + t;
      const int sl = sumL[yi * Z.gx + lc0 + t];
      const float il = invL[yi * Z.gx + lc0 + t];
      // the lane's best (and second) candidate, compared as floats: ties keep the lower k,
      // i.e. the lower d; -4 marks "none" (every score lies in [-1, 1])
      float bv = -4.0f, sv = -4.0f;
      int bd = 0x7FFFFFFF;
#pragma unroll
      for (int k = 0; k < KD; ++k) {
        const int d = lane + 32 * k;
        const int2 sr = statR[yi * Z.nrs + lc0 + t - dd[k] + (D - 1)];  // right window at x - d
        const long long n = N * (long long)run[k] - (long long)sl * (long long)sr.x;
        const float rho = (float)n * il * __int_as_float(sr.y);
        const bool valid = d < D && d <= x && x < w;
        if constexpr (MODE == 2) {
          if (d < D && x < w && y < h) P.cost[((size_t)y * w + x) * D + d] = d <= x ? 1.0f - rho : 2.0f;
        }
        if (valid && rho > bv) {
          if constexpr (MODE == 1) sv = bv;
          bv = rho;
          bd = d;
        } else if (MODE == 1 && valid && rho > sv) {
          sv = rho;
        }
      }
      const int bk = bv > -3.0f ? order_key(bv) : INT_MIN;
      const int gbest = __reduce_max_sync(0xFFFFFFFFu, bk);
      const unsigned dstar = __reduce_min_sync(0xFFFFFFFFu, (bk == gbest) ? (unsigned)bd : 0x7FFFFFFFu);
      int gsec = INT_MIN;
      if constexpr (MODE == 1) {
        const int sk = sv > -3.0f ? order_key(sv) : INT_MIN;
        gsec = __reduce_max_sync(0xFFFFFFFFu, ((unsigned)bd == dstar) ? sk : bk);
      }
      if (lane == t) { my_d = (int)dstar; my_b = gbest; my_s = gsec; }
    }
    const int x = xw + lane;
    if (lane < TX && x < w && y < h) {
      const size_t o = (size_t)y * w + x;
      P.disp[o] = (int16_t)my_d;
      if constexpr (MODE == 1) {
        if (P.best) P.best[o] = key_value(my_b);
        if (P.second) P.second[o] = key_value(my_s);
      }
    }
  }
}

// Disparity ranges of 33-48 (MODE 0, disparities only): the two half-warps own TXH output
// columns each (half h: columns xw + h TXH + t) and lane l = lane % 16 the disparities d = l +
// 16 k, k < 3, so that all 48 candidates of a pixel fill the half's 48 slots (the full-warp
// layout uses 64 slots for them).  A lane keeps its best candidate as a float (strict ">"
// over ascending k: lowest d on exact ties); the half's argmax is one max reduction over a
// 64-bit key, the lane's order key above 63 - d, so that the lowest d wins exact ties, as in
// the full-warp kernel.  Stages 1 and 2 as in zncc_wta_kernel.
template <int R, int TXH>
__global__ void __launch_bounds__(kZnccWarps * 32, 2)
zncc_wta_hw_kernel(const ZPair* __restrict__ pairs, const ZJob* __restrict__ jobs) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int KH = 3, TX = 2 * TXH;
  const int TY = kZnccTY;
  const ZJob job = jobs[blockIdx.x];
  const ZPair P = pairs[job.pair];
  const int D = P.D, w = P.w, h = P.h;
  const ZLayout Z = zlayout(R, D, TX);
  uint16_t* sL = reinterpret_cast<uint16_t*>(smem + Z.off_sl);
  uint16_t* sR = reinterpret_cast<uint16_t*>(smem + Z.off_sr);
  int* sumL = reinterpret_cast<int*>(smem + Z.off_suml);
  float* invL = reinterpret_cast<float*>(smem + Z.off_invl);
  int2* statR = reinterpret_cast<int2*>(smem + Z.off_statr);
  int* cs = reinterpret_cast<int*>(smem + Z.off_cs);
  unsigned* cs2 = reinterpret_cast<unsigned*>(smem + Z.off_cs2);
  const int y0 = job.y0, x0 = job.x0;
  const int lbase = x0 - R;
  const int rbase = x0 - R - (D - 1);
  stage_box<R>(P.L, P.pitch, w, h, lbase, y0, Z.nlc, sL);
  stage_box<R>(P.R, P.pitch, w, h, rbase, y0, Z.nrc, sR);
  __syncthreads();
  window_stats<R>(sL, Z.nlc, cs, cs2, sumL, invL, nullptr, Z.gx);
  window_stats<R>(sR, Z.nrc, cs, cs2, nullptr, nullptr, statR, Z.nrs);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, hf = lane >> 4, l = lane & 15;
  const int xw = x0 + warp * TX;
  if (xw >= w) return;                     // all of this warp's columns lie beyond the image
  const int xh = xw + hf * TXH;            // this half's first output column
  const int lc0 = warp * TX + hf * TXH;    // staged left column of u = xh - R
  const long long N = (long long)(2 * R + 1) * (2 * R + 1);
  int dd[KH], rc0[KH];
#pragma unroll
  for (int k = 0; k < KH; ++k) {
    const int d = l + 16 * k;
    dd[k] = d < D ? d : D - 1;             // reads stay in the staged range; masked below
    rc0[k] = lc0 - dd[k] + (D - 1);
  }
  unsigned colsum[KH][TXH + 2 * R];
#pragma unroll
  for (int c = 0; c < TXH + 2 * R; ++c) {
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      unsigned a = 0;
#pragma unroll
      for (int j = 0; j <= 2 * R; ++j) a += (unsigned)sL[j * Z.nlc + lc0 + c] * (unsigned)sR[j * Z.nrc + rc0[k] + c];
      colsum[k][c] = a;
    }
  }
  for (int yi = 0; yi < TY; ++yi) {
    const int y = y0 + yi;
    if (yi > 0) {
      const int rin = yi + 2 * R, rout = yi - 1;
#pragma unroll
      for (int c = 0; c < TXH + 2 * R; ++c) {
        const unsigned lin = sL[rin * Z.nlc + lc0 + c], lout = sL[rout * Z.nlc + lc0 + c];
#pragma unroll
        for (int k = 0; k < KH; ++k)
          colsum[k][c] += lin * (unsigned)sR[rin * Z.nrc + rc0[k] + c] - lout * (unsigned)sR[rout * Z.nrc + rc0[k] + c];
      }
    }
    unsigned run[KH];
#pragma unroll
    for (int k = 0; k < KH; ++k) {
      unsigned a = 0;
#pragma unroll
      for (int i = 0; i <= 2 * R; ++i) a += colsum[k][i];
      run[k] = a;
    }
    long long my_key = LLONG_MIN;
#pragma unroll
    for (int t = 0; t < TXH; ++t) {
      if (t > 0) {
#pragma unroll
        for (int k = 0; k < KH; ++k) run[k] += colsum[k][t + 2 * R] - colsum[k][t - 1];
      }
      const int x = xh + t;
      const int sl = sumL[yi * Z.gx + lc0 + t];
      const float il = invL[yi * Z.gx + lc0 + t];
      float bv = -4.0f;
      int bd = 0;
#pragma unroll
      for (int k = 0; k < KH; ++k) {
        const int d = l + 16 * k;
        const int2 sr = statR[yi * Z.nrs + lc0 + t - dd[k] + (D - 1)];  // right window at x - d
        const long long n = N * (long long)run[k] - (long long)sl * (long long)sr.x;
        const float rho = (float)n * il * __int_as_float(sr.y);
        if (d < D && d <= x && x < w && rho > bv) {
          bv = rho;
          bd = d;
        }
      }
      long long key = bv > -3.0f ? (long long)order_key(bv) * 4294967296LL + (63 - bd) : LLONG_MIN;
#pragma unroll
      for (int off = 8; off >= 1; off >>= 1) key = max(key, __shfl_xor_sync(0xFFFFFFFFu, key, off));
      if (l == t) my_key = key;
    }
    const int x = xh + l;
    if (l < TXH && x < w && y < h) P.disp[(size_t)y * w + x] = (int16_t)(my_key == LLONG_MIN ? 0 : 63 - (int)(my_key & 63));
  }
}

template <int R, int KD, int MODE>
cudaError_t launch_rk(const ZPair* p, const ZJob* j, int n, int maxD, cudaStream_t st) {
  constexpr int TX = KD == 1 ? 32 : KD == 2 ? 20 : KD == 3 ? 16 : 12;  // == zncc_tx(KD)
  if constexpr (MODE == 0 && KD == 2) {
    if (maxD <= 48) {  // half-warp layout: 48 candidate slots per pixel, the same job geometry
      auto kern = zncc_wta_hw_kernel<R, TX / 2>;
      const size_t smem = zlayout(R, maxD, TX).total;
      cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      kern<<<n, kZnccWarps * 32, smem, st>>>(p, j);
      return cudaGetLastError();
    }
  }
  auto kern = zncc_wta_kernel<R, KD, TX, MODE>;
  const size_t smem = zlayout(R, maxD, TX).total;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<n, kZnccWarps * 32, smem, st>>>(p, j);
  return cudaGetLastError();
}

}  // namespace

#ifndef SV_ZNCC_R
#error "compile this file once per window radius with -DSV_ZNCC_R=<r>"
#endif

#define SV_CAT2(a, b) a##b
#define SV_CAT(a, b) SV_CAT2(a, b)
// Internal linkage: every radius has its own translation unit, and a template with external
// linkage instantiated in all of them would be merged by the linker into one radius's copy.
namespace {
template <int MODE>
cudaError_t launch_r(const ZPair* p, const ZJob* j, int n, int maxD, cudaStream_t st) {
  switch (zncc_kd(maxD)) {
    case 1: return launch_rk<SV_ZNCC_R, 1, MODE>(p, j, n, maxD, st);
    case 2: return launch_rk<SV_ZNCC_R, 2, MODE>(p, j, n, maxD, st);
    case 3: return launch_rk<SV_ZNCC_R, 3, MODE>(p, j, n, maxD, st);
    case 4: return launch_rk<SV_ZNCC_R, 4, MODE>(p, j, n, maxD, st);
  }
  return cudaErrorInvalidValue;
}
}  // namespace

cudaError_t SV_CAT(launch_zncc_wta_r, SV_ZNCC_R)(const ZPair* p, const ZJob* j, int n, int maxD, int mode,
                                                  cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  switch (mode) {
    case 0: return launch_r<0>(p, j, n, maxD, st);
    case 1: return launch_r<1>(p, j, n, maxD, st);
    case 2: return launch_r<2>(p, j, n, maxD, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace sv
