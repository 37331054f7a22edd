// coarse_ext.cu -- variants of the coarse stage (Sec. III-A and the robustness study of
// Sec. IV-C): a matching cost, an aggregation, winner-take-all and post-processing, for
// every pair of a call.
//
//   cost volume C [h][w][D]
//     ZNCC     1 - rho of Eq. 1-3, written by the coarse matcher itself (zncc_wta.cu, the
//              cost-writing instance) while it computes its own winner-take-all;
//     census   box4 (4 x 4 box sums of L and R), census_codes (kc x kc census bit strings of
//              the box sums, clamped windows), census_cost (Hamming distance of the codes of
//              (x, y) and (x - d, y); kc^2 - 1 where x - d < 0)
//   aggregation A [h][w][D]
//     SGM      sgm_path: Eq. 4 along one direction per launch, one warp per path line, the
//              lanes holding consecutive disparities (d = lane + 32 k) so that the d - 1 and
//              d + 1 terms are register shuffles and the minimum over d a warp reduction;
//              the directions add into A in launch order (Eq. 5, deterministic); the last
//              direction also takes the winner-take-all of the sum (Eq. 6)
//     DT       dt_rows / dt_cols: the recursive domain-transform filter on every disparity
//              slice, guided by the left box sums, one thread per (row, d) or (column, d)
//   wta        Eq. 6 on a volume: one warp per pixel, argmin over d, lowest d on ties
//   smp        single-matching-phase check (Eq. 7, read as uniqueness of the target column),
//              one block per row; median3: 3 x 3 median filter, one thread per pixel
#include "sv_ctx.cuh"

namespace sv {

namespace {

struct XPair {
  const uint8_t* L;
  const uint8_t* R;
  int pitch, w, h, D;
  int32_t* SL;      // [h][w] box sums of L
  int32_t* SR;      // [h][w] box sums of R
  uint64_t* CL;     // [h][w] census codes of L
  uint64_t* CR;     // [h][w] census codes of R
  float* C;         // [h][w][D] cost
  float* A;         // [h][w][D] aggregated cost
  int16_t* wta;     // [h][w] winner-take-all map
  int16_t* mid;     // [h][w] after the occlusion check, when the median filter follows
  int16_t* disp;    // [h][w] result
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Order-preserving float -> int key (finite values): smaller float, smaller key.
__device__ __forceinline__ int fkey(float f) {
  int i = __float_as_int(f + 0.0f);
  return i >= 0 ? i : (i ^ 0x7FFFFFFF);
}

__global__ void box4_kernel(const XPair* __restrict__ P) {
  const XPair& p = P[blockIdx.z];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (y >= p.h || x >= p.w) return;
  int32_t sl = 0, sr = 0;
  for (int j = 0; j < 4; ++j) {
    const unsigned a = *reinterpret_cast<const unsigned*>(p.L + (size_t)(4 * y + j) * p.pitch + 4 * x);
    const unsigned b = *reinterpret_cast<const unsigned*>(p.R + (size_t)(4 * y + j) * p.pitch + 4 * x);
    sl += (a & 0xFF) + ((a >> 8) & 0xFF) + ((a >> 16) & 0xFF) + (a >> 24);
    sr += (b & 0xFF) + ((b >> 8) & 0xFF) + ((b >> 16) & 0xFF) + (b >> 24);
  }
  p.SL[(size_t)y * p.w + x] = sl;
  p.SR[(size_t)y * p.w + x] = sr;
}

// Census bit strings: bit b (window offsets in raster order, the centre skipped) is set
// where the neighbour's box sum is below the centre's.
template <int RC>
__global__ void census_codes_kernel(const XPair* __restrict__ P) {
  const XPair& p = P[blockIdx.z];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (y >= p.h || x >= p.w) return;
  const int w = p.w, h = p.h;
  const int32_t cl = p.SL[(size_t)y * w + x], cr = p.SR[(size_t)y * w + x];
  uint64_t ml = 0, mr = 0;
  int bit = 0;
#pragma unroll
  for (int j = -RC; j <= RC; ++j) {
    const size_t row = (size_t)clampi(y + j, 0, h - 1) * w;
#pragma unroll
    for (int i = -RC; i <= RC; ++i) {
      if (i == 0 && j == 0) continue;
      const int xx = clampi(x + i, 0, w - 1);
      if (p.SL[row + xx] < cl) ml |= 1ull << bit;
      if (p.SR[row + xx] < cr) mr |= 1ull << bit;
      ++bit;
    }
  }
  p.CL[(size_t)y * w + x] = ml;
  p.CR[(size_t)y * w + x] = mr;
}

__global__ void census_cost_kernel(const XPair* __restrict__ P, int kc2m1) {
  const XPair& p = P[blockIdx.y];
  const size_t n = (size_t)p.w * p.h * p.D;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const size_t q = i / p.D;
    const int d = (int)(i - q * p.D);
    const int x = (int)(q % p.w);
    p.C[i] = x - d >= 0 ? (float)__popcll(p.CL[q] ^ p.CR[q - d]) : (float)kc2m1;
  }
}

// Eq. 4 along direction dir (0: left to right along rows, 1: right to left, 2: top to
// bottom along columns, 3: bottom to top), one warp per line.  first: write A, else add.
// last: also the winner-take-all of A into wta; keep: store A (else only the map).
template <int KD>
__global__ void __launch_bounds__(256) sgm_path_kernel(const XPair* __restrict__ P, int dir, int first, int last,
                                                       int keep, float P1, float P2) {
  const XPair& p = P[blockIdx.y];
  const int w = p.w, h = p.h, D = p.D;
  const int dx = dir == 0 ? 1 : dir == 1 ? -1 : 0;
  const int dy = dir == 2 ? 1 : dir == 3 ? -1 : 0;
  const int nlines = dy == 0 ? h : w, len = dy == 0 ? w : h;
  const int line = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (line >= nlines) return;  // whole warp
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const float INF = __int_as_float(0x7f800000);
  auto at = [&](int s) {
    const int x = dx == 0 ? line : dx > 0 ? s : w - 1 - s;
    const int y = dy == 0 ? line : dy > 0 ? s : h - 1 - s;
    return ((size_t)y * w + x) * D;
  };
  float prev[KD], cur[KD], cn[KD], an[KD];
  float m = 0.f;
  size_t o = at(0);
#pragma unroll
  for (int k = 0; k < KD; ++k) {
    const int d = lane + 32 * k;
    cn[k] = d < D ? p.C[o + d] : INF;
    an[k] = (!first && d < D) ? p.A[o + d] : 0.f;
  }
  for (int s = 0; s < len; ++s) {
    float c[KD], a[KD];
#pragma unroll
    for (int k = 0; k < KD; ++k) { c[k] = cn[k]; a[k] = an[k]; }
    const size_t on = s + 1 < len ? at(s + 1) : o;
    if (s + 1 < len) {  // the next pixel's loads go out before this pixel's arithmetic
#pragma unroll
      for (int k = 0; k < KD; ++k) {
        const int d = lane + 32 * k;
        cn[k] = d < D ? p.C[on + d] : INF;
        an[k] = (!first && d < D) ? p.A[on + d] : 0.f;
      }
    }
    if (s == 0) {
#pragma unroll
      for (int k = 0; k < KD; ++k) cur[k] = c[k];
    } else {
#pragma unroll
      for (int k = 0; k < KD; ++k) {
        float lo = __shfl_up_sync(FULL, prev[k], 1);                 // d - 1
        const float lo_wrap = __shfl_sync(FULL, prev[k > 0 ? k - 1 : 0], 31);
        float hi = __shfl_down_sync(FULL, prev[k], 1);               // d + 1
        const float hi_wrap = __shfl_sync(FULL, prev[k + 1 < KD ? k + 1 : k], 0);
        if (lane == 0) lo = k > 0 ? lo_wrap : INF;
        if (lane == 31) hi = k + 1 < KD ? hi_wrap : INF;
        const int d = lane + 32 * k;
        float best = fminf(prev[k], fminf(lo, hi) + P1);
        best = fminf(best, m + P2);
        cur[k] = d < D ? c[k] + (best - m) : INF;
      }
    }
    float mn = cur[0];
#pragma unroll
    for (int k = 1; k < KD; ++k) mn = fminf(mn, cur[k]);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) mn = fminf(mn, __shfl_xor_sync(FULL, mn, off));
    m = mn;
    float tot[KD];
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      prev[k] = cur[k];
      tot[k] = first ? cur[k] : a[k] + cur[k];
      const int d = lane + 32 * k;
      if (d < D && (keep || !last)) p.A[o + d] = tot[k];
    }
    if (last) {
      int key = INT_MAX, bd = 0x7FFFFFFF;
#pragma unroll
      for (int k = 0; k < KD; ++k) {
        const int d = lane + 32 * k;
        const int kk = d < D ? fkey(tot[k]) : INT_MAX;
        if (kk < key) { key = kk; bd = d; }
      }
      const int gk = __reduce_min_sync(FULL, key);
      const unsigned gd = __reduce_min_sync(FULL, key == gk ? (unsigned)bd : 0x7FFFFFFFu);
      if (lane == 0) p.wta[o / D] = (int16_t)gd;
    }
    o = on;
  }
}

// One domain-transform pass along rows (both ways) for every (row, d) of a pair; src is
// read once (the first pass reads C), dst written (the aggregated volume).
__global__ void dt_rows_kernel(const XPair* __restrict__ P, int from_cost, float lna, float ratio) {
  const XPair& p = P[blockIdx.y];
  const int w = p.w, h = p.h, D = p.D;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= h * D) return;
  const int y = t / D, d = t - y * D;
  const float* src = from_cost ? p.C : p.A;
  float* dst = p.A;
  const int32_t* g = p.SL + (size_t)y * w;
  const size_t base = (size_t)y * w * D + d;
  constexpr int U = 8;
  float J = src[base];
  dst[base] = J;
  for (int x0 = 1; x0 < w; x0 += U) {
    float c[U], wt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int x = x0 + u;
      if (x < w) {
        c[u] = src[base + (size_t)x * D];
        wt[u] = expf(lna * (1.0f + ratio * fabsf((float)(g[x] - g[x - 1]) * 0.0625f)));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int x = x0 + u;
      if (x < w) {
        J = c[u] + wt[u] * (J - c[u]);
        dst[base + (size_t)x * D] = J;
      }
    }
  }
  for (int x0 = w - 2; x0 >= 0; x0 -= U) {
    float c[U], wt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int x = x0 - u;
      if (x >= 0) {
        c[u] = dst[base + (size_t)x * D];
        wt[u] = expf(lna * (1.0f + ratio * fabsf((float)(g[x + 1] - g[x]) * 0.0625f)));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int x = x0 - u;
      if (x >= 0) {
        J = c[u] + wt[u] * (J - c[u]);
        dst[base + (size_t)x * D] = J;
      }
    }
  }
}

// The same along columns, in place on A, one thread per (column, d): consecutive threads
// touch consecutive addresses of a row.
__global__ void dt_cols_kernel(const XPair* __restrict__ P, float lna, float ratio) {
  const XPair& p = P[blockIdx.y];
  const int w = p.w, h = p.h, D = p.D;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= w * D) return;
  const int x = t / D;
  float* A = p.A + t;
  const size_t row = (size_t)w * D;
  const int32_t* g = p.SL + x;
  constexpr int U = 8;
  float J = A[0];
  for (int y0 = 1; y0 < h; y0 += U) {
    float c[U], wt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int y = y0 + u;
      if (y < h) {
        c[u] = A[(size_t)y * row];
        wt[u] = expf(lna * (1.0f + ratio * fabsf((float)(g[(size_t)y * w] - g[(size_t)(y - 1) * w]) * 0.0625f)));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int y = y0 + u;
      if (y < h) {
        J = c[u] + wt[u] * (J - c[u]);
        A[(size_t)y * row] = J;
      }
    }
  }
  for (int y0 = h - 2; y0 >= 0; y0 -= U) {
    float c[U], wt[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int y = y0 - u;
      if (y >= 0) {
        c[u] = A[(size_t)y * row];
        wt[u] = expf(lna * (1.0f + ratio * fabsf((float)(g[(size_t)(y + 1) * w] - g[(size_t)y * w]) * 0.0625f)));
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int y = y0 - u;
      if (y >= 0) {
        J = c[u] + wt[u] * (J - c[u]);
        A[(size_t)y * row] = J;
      }
    }
  }
}

// Eq. 6 on a volume (vol_sel 0: C, 1: A): one warp per pixel, lowest d among the minima.
template <int KD>
__global__ void vol_wta_kernel(const XPair* __restrict__ P, int vol_sel) {
  const XPair& p = P[blockIdx.y];
  const int D = p.D;
  const float* V = vol_sel ? p.A : p.C;
  const int lane = threadIdx.x & 31;
  const int npix = p.w * p.h;
  for (int q = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); q < npix; q += gridDim.x * (blockDim.x >> 5)) {
    int key = INT_MAX, bd = 0x7FFFFFFF;
#pragma unroll
    for (int k = 0; k < KD; ++k) {
      const int d = lane + 32 * k;
      if (d < D) {
        const int kk = fkey(V[(size_t)q * D + d]);
        if (kk < key) { key = kk; bd = d; }
      }
    }
    const int gk = __reduce_min_sync(0xffffffffu, key);
    const unsigned gd = __reduce_min_sync(0xffffffffu, key == gk ? (unsigned)bd : 0x7FFFFFFFu);
    if (lane == 0) p.wta[q] = (int16_t)gd;
  }
}

// Single-matching-phase check of one row: pixel x keeps its disparity unless a pixel x - k
// (0 < k < D) of the row has the same target column x - disp; the others take the
// disparity of the nearest kept pixel of the row (left first at equal distance).  A row
// without a kept pixel is copied.  in / out: the pair's maps selected by sel_in / sel_out
// (0: wta, 1: mid, 2: disp).
__global__ void smp_kernel(const XPair* __restrict__ P, int sel_in, int sel_out) {
  extern __shared__ int smp_sm[];
  const XPair& p = P[blockIdx.y];
  const int y = blockIdx.x, w = p.w, D = p.D;
  if (y >= p.h) return;
  const int16_t* in = (sel_in == 0 ? p.wta : sel_in == 1 ? p.mid : p.disp) + (size_t)y * w;
  int16_t* out = (sel_out == 0 ? p.wta : sel_out == 1 ? p.mid : p.disp) + (size_t)y * w;
  int* tgt = smp_sm;                                               // [w] target columns
  unsigned char* ok = reinterpret_cast<unsigned char*>(smp_sm + w);  // [w] kept
  int* val = smp_sm + w + (w + 3) / 4;                             // [w] disparities
  for (int x = threadIdx.x; x < w; x += blockDim.x) {
    val[x] = in[x];
    tgt[x] = x - val[x];
  }
  __syncthreads();
  int any = 0;
  for (int x = threadIdx.x; x < w; x += blockDim.x) {
    int keep = 1;
    const int lo = max(0, x - D + 1);
    for (int u = x - 1; u >= lo; --u)
      if (tgt[u] == tgt[x]) { keep = 0; break; }
    ok[x] = (unsigned char)keep;
    any |= keep;
  }
  any = __syncthreads_or(any);
  for (int x = threadIdx.x; x < w; x += blockDim.x) {
    int v = val[x];
    if (!ok[x] && any) {
      for (int dist = 1; dist < w; ++dist) {
        if (x - dist >= 0 && ok[x - dist]) { v = val[x - dist]; break; }
        if (x + dist < w && ok[x + dist]) { v = val[x + dist]; break; }
      }
    }
    out[x] = (int16_t)v;
  }
}

// 3 x 3 median with clamped edges: the 5th smallest of the 9 values (partial selection).
__global__ void median3_kernel(const XPair* __restrict__ P, int sel_in) {
  const XPair& p = P[blockIdx.z];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (y >= p.h || x >= p.w) return;
  const int w = p.w, h = p.h;
  const int16_t* in = sel_in == 0 ? p.wta : p.mid;
  int v[9];
  int n = 0;
#pragma unroll
  for (int j = -1; j <= 1; ++j)
#pragma unroll
    for (int i = -1; i <= 1; ++i) v[n++] = in[(size_t)clampi(y + j, 0, h - 1) * w + clampi(x + i, 0, w - 1)];
#pragma unroll
  for (int a = 0; a < 5; ++a)
#pragma unroll
    for (int b = a + 1; b < 9; ++b) {
      const int lo = min(v[a], v[b]), hi = max(v[a], v[b]);
      v[a] = lo;
      v[b] = hi;
    }
  p.disp[(size_t)y * w + x] = (int16_t)v[4];
}

cudaError_t launch_census_codes(const XPair* T, int kc, int maxw, int maxh, int n, cudaStream_t st) {
  const dim3 g((maxw + 127) / 128, maxh, n);
  switch (kc / 2) {
    case 1: census_codes_kernel<1><<<g, 128, 0, st>>>(T); break;
    case 2: census_codes_kernel<2><<<g, 128, 0, st>>>(T); break;
    case 3: census_codes_kernel<3><<<g, 128, 0, st>>>(T); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_sgm_path(const XPair* T, int kd, int nlines, int n, int dir, int first, int last, int keep,
                            float P1, float P2, cudaStream_t st) {
  const dim3 g((nlines + 7) / 8, n);
  switch (kd) {
    case 1: sgm_path_kernel<1><<<g, 256, 0, st>>>(T, dir, first, last, keep, P1, P2); break;
    case 2: sgm_path_kernel<2><<<g, 256, 0, st>>>(T, dir, first, last, keep, P1, P2); break;
    case 3: sgm_path_kernel<3><<<g, 256, 0, st>>>(T, dir, first, last, keep, P1, P2); break;
    case 4: sgm_path_kernel<4><<<g, 256, 0, st>>>(T, dir, first, last, keep, P1, P2); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_vol_wta(const XPair* T, int kd, int n, int vol_sel, cudaStream_t st) {
  const dim3 g(4 * 152, n);
  switch (kd) {
    case 1: vol_wta_kernel<1><<<g, 256, 0, st>>>(T, vol_sel); break;
    case 2: vol_wta_kernel<2><<<g, 256, 0, st>>>(T, vol_sel); break;
    case 3: vol_wta_kernel<3><<<g, 256, 0, st>>>(T, vol_sel); break;
    case 4: vol_wta_kernel<4><<<g, 256, 0, st>>>(T, vol_sel); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace

// Post-processing launches on a prepared table: SMP (wta -> mid or disp), median (wta or
// mid -> disp).  With neither flag nothing runs (the caller wrote disp directly).
sv_status Ctx::post_launch(const void* table, int n, int maxw, int maxh, int post, cudaStream_t st) {
  const XPair* T = (const XPair*)table;
  sv_status s;
  const bool smp = post & SV_POST_SMP, med = post & SV_POST_MEDIAN;
  if (smp) {
    LaunchScope ls(*this, "smp", st);
    const size_t sm = (size_t)maxw * 2 * sizeof(int) + (maxw + 3) / 4 * sizeof(int);
    if (sm > 48 * 1024 &&
        (s = cuda(cudaFuncSetAttribute(smp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
                  "occlusion check shared memory")))
      return s;
    smp_kernel<<<dim3(maxh, n), 256, sm, st>>>(T, 0, med ? 1 : 2);
    if ((s = cuda(cudaGetLastError(), "occlusion check"))) return s;
  }
  if (med) {
    LaunchScope ls(*this, "median3", st);
    median3_kernel<<<dim3((maxw + 127) / 128, maxh, n), 128, 0, st>>>(T, smp ? 1 : 0);
    if ((s = cuda(cudaGetLastError(), "median filter"))) return s;
  }
  return SV_OK;
}

sv_status Ctx::coarse_ext(const sv_pair* pairs, int n, const sv_coarse_opts& o, int16_t* const* disp,
                          float* const* cost_out, cudaStream_t st) {
  if (n == 0) return SV_OK;
  const bool want_cost = cost_out != nullptr;
  const bool zncc = o.cost == SV_COST_ZNCC;
  const int post = o.post & (SV_POST_SMP | SV_POST_MEDIAN);
  // the plain matcher: its own exact winner-take-all straight into the output (or into the
  // map the post-processing reads)
  const bool plain = zncc && o.aggregation == SV_AGG_NONE;
  int maxw = 0, maxh = 0, maxD = 1;
  size_t nS = 0, nV = 0, nA = 0;
  for (int i = 0; i < n; ++i) {
    const int w = pairs[i].width / 4, h = pairs[i].height / 4, D = pairs[i].max_disp;
    maxw = std::max(maxw, w);
    maxh = std::max(maxh, h);
    maxD = std::max(maxD, D);
    nS += (size_t)w * h;
    if (!(want_cost && cost_out[i] && o.aggregation == SV_AGG_NONE)) nV += (size_t)w * h * D;
    if (o.aggregation != SV_AGG_NONE && !(want_cost && cost_out[i])) nA += (size_t)w * h * D;
  }
  if (plain && !want_cost) nV = 0;
  const bool need_box = !zncc || o.aggregation == SV_AGG_DT;
  sv_status s;
  if (need_box && (s = cuda(sgm_s.ensure(2 * nS * sizeof(int32_t)), "alloc box sums"))) return s;
  if (!zncc && (s = cuda(x_codes.ensure(2 * nS * sizeof(uint64_t)), "alloc census codes"))) return s;
  if (nV && (s = cuda(sgm_c.ensure(nV * sizeof(float)), "alloc cost volume"))) return s;
  if (nA && (s = cuda(sgm_a.ensure(nA * sizeof(float)), "alloc aggregated volume"))) return s;
  if ((s = cuda(x_maps.ensure(2 * nS * sizeof(int16_t)), "alloc coarse maps"))) return s;
  if ((s = cuda(sgm_tab.ensure(sizeof(XPair) * n), "alloc pair table"))) return s;
  std::vector<XPair> tab(n);
  size_t oS = 0, oV = 0, oA = 0;
  for (int i = 0; i < n; ++i) {
    const int w = pairs[i].width / 4, h = pairs[i].height / 4, D = pairs[i].max_disp;
    XPair& q = tab[i];
    q.L = (const uint8_t*)pairs[i].left;
    q.R = (const uint8_t*)pairs[i].right;
    q.pitch = pairs[i].pitch;
    q.w = w;
    q.h = h;
    q.D = D;
    q.SL = need_box ? (int32_t*)sgm_s.p + oS : nullptr;
    q.SR = need_box ? (int32_t*)sgm_s.p + nS + oS : nullptr;
    q.CL = !zncc ? (uint64_t*)x_codes.p + oS : nullptr;
    q.CR = !zncc ? (uint64_t*)x_codes.p + nS + oS : nullptr;
    const bool own_c = !(want_cost && cost_out[i] && o.aggregation == SV_AGG_NONE);
    if (own_c) {
      q.C = nV ? (float*)sgm_c.p + oV : nullptr;
      if (nV) oV += (size_t)w * h * D;
    } else {
      q.C = cost_out[i];
    }
    if (o.aggregation != SV_AGG_NONE) {
      if (want_cost && cost_out[i]) {
        q.A = cost_out[i];
      } else {
        q.A = (float*)sgm_a.p + oA;
        oA += (size_t)w * h * D;
      }
    } else {
      q.A = nullptr;
    }
    q.disp = disp[i];
    q.wta = post ? (int16_t*)x_maps.p + oS : disp[i];
    q.mid = (int16_t*)x_maps.p + nS + oS;
    oS += (size_t)w * h;
  }
  if ((s = cuda(cudaMemcpyAsync(sgm_tab.p, tab.data(), sizeof(XPair) * n, cudaMemcpyHostToDevice, st),
                "upload pair table")))
    return s;
  const XPair* T = (const XPair*)sgm_tab.p;
  const int kd = (maxD + 31) / 32;

  // ---- cost volume (and, for the plain matcher, its winner-take-all)
  if (zncc) {
    std::vector<int16_t*> wta(n);
    for (int i = 0; i < n; ++i) wta[i] = tab[i].wta;
    ZRun z;
    coarse_prepare(pairs, n, wta.data(), nullptr, nullptr, z);
    const bool with_cost = !plain || want_cost;
    if (with_cost)
      for (int i = 0; i < n; ++i) z.pairs[i].cost = tab[i].C;
    if ((s = cuda(zpairs.ensure(sizeof(ZPair) * n), "alloc pair table"))) return s;
    if ((s = cuda(zjobs.ensure(sizeof(ZJob) * z.jobs.size()), "alloc job table"))) return s;
    if ((s = cuda(cudaMemcpyAsync(zpairs.p, z.pairs.data(), sizeof(ZPair) * n, cudaMemcpyHostToDevice, st),
                  "upload pairs")))
      return s;
    if ((s = cuda(cudaMemcpyAsync(zjobs.p, z.jobs.data(), sizeof(ZJob) * z.jobs.size(), cudaMemcpyHostToDevice, st),
                  "upload jobs")))
      return s;
    LaunchScope ls(*this, with_cost ? "zncc_cost" : "zncc_wta", st);
    if ((s = cuda(launch_zncc_wta((const ZPair*)zpairs.p, (const ZJob*)zjobs.p, (int)z.jobs.size(), cfg.window / 2,
                                  z.maxD, st, with_cost ? 2 : 0),
                  "zncc cost")))
      return s;
  }
  if (need_box) {
    LaunchScope ls(*this, "box4", st);
    box4_kernel<<<dim3((maxw + 127) / 128, maxh, n), 128, 0, st>>>(T);
    if ((s = cuda(cudaGetLastError(), "box sums"))) return s;
  }
  if (!zncc) {
    {
      LaunchScope ls(*this, "census_codes", st);
      if ((s = cuda(launch_census_codes(T, o.census_window, maxw, maxh, n, st), "census codes"))) return s;
    }
    LaunchScope ls(*this, "census_cost", st);
    census_cost_kernel<<<dim3(8 * 152 / std::max(1, std::min(n, 8)), n), 256, 0, st>>>(
        T, o.census_window * o.census_window - 1);
    if ((s = cuda(cudaGetLastError(), "census cost"))) return s;
  }

  // ---- aggregation and winner-take-all
  if (o.aggregation == SV_AGG_SGM) {
    for (int dir = 0; dir < o.npaths; ++dir) {
      LaunchScope ls(*this, "sgm_path", st);
      const int nlines = dir < 2 ? maxh : maxw;
      if ((s = cuda(launch_sgm_path(T, kd, nlines, n, dir, dir == 0, dir == o.npaths - 1, want_cost ? 1 : 0, o.P1,
                                    o.P2, st),
                    "SGM path")))
        return s;
    }
  } else if (o.aggregation == SV_AGG_DT) {
    const double N = o.dt_iters;
    const float ratio = (float)((double)o.dt_sigma_s / (double)o.dt_sigma_r);
    for (int it = 1; it <= o.dt_iters; ++it) {
      const double sig = o.dt_sigma_s * std::sqrt(3.0) * std::pow(2.0, N - it) / std::sqrt(std::pow(4.0, N) - 1.0);
      const float lna = (float)(-std::sqrt(2.0) / sig);
      {
        LaunchScope ls(*this, "dt_rows", st);
        dt_rows_kernel<<<dim3((maxh * maxD + 127) / 128, n), 128, 0, st>>>(T, it == 1, lna, ratio);
        if ((s = cuda(cudaGetLastError(), "DT rows"))) return s;
      }
      LaunchScope ls(*this, "dt_cols", st);
      dt_cols_kernel<<<dim3((maxw * maxD + 127) / 128, n), 128, 0, st>>>(T, lna, ratio);
      if ((s = cuda(cudaGetLastError(), "DT columns"))) return s;
    }
    LaunchScope ls(*this, "vol_wta", st);
    if ((s = cuda(launch_vol_wta(T, kd, n, 1, st), "winner-take-all"))) return s;
  } else if (!zncc) {
    LaunchScope ls(*this, "vol_wta", st);
    if ((s = cuda(launch_vol_wta(T, kd, n, 0, st), "winner-take-all"))) return s;
  }

  // ---- post-processing
  return post_launch(T, n, maxw, maxh, post, st);
}

sv_status Ctx::postprocess(const sv_pair* pairs, int n, const int16_t* const* in, int post, int16_t* const* out,
                           cudaStream_t st) {
  if (n == 0) return SV_OK;
  int maxw = 0, maxh = 0;
  size_t nS = 0;
  for (int i = 0; i < n; ++i) {
    maxw = std::max(maxw, pairs[i].width / 4);
    maxh = std::max(maxh, pairs[i].height / 4);
    nS += (size_t)(pairs[i].width / 4) * (pairs[i].height / 4);
  }
  sv_status s;
  if (!(post & (SV_POST_SMP | SV_POST_MEDIAN))) {
    for (int i = 0; i < n; ++i)
      if ((s = cuda(cudaMemcpyAsync(out[i], in[i], sizeof(int16_t) * (pairs[i].width / 4) * (pairs[i].height / 4),
                                    cudaMemcpyDeviceToDevice, st),
                    "copy map")))
        return s;
    return SV_OK;
  }
  if ((s = cuda(x_maps.ensure(2 * nS * sizeof(int16_t)), "alloc coarse maps"))) return s;
  if ((s = cuda(sgm_tab.ensure(sizeof(XPair) * n), "alloc pair table"))) return s;
  std::vector<XPair> tab(n);
  size_t oS = 0;
  for (int i = 0; i < n; ++i) {
    XPair& q = tab[i];
    q = XPair{};
    q.w = pairs[i].width / 4;
    q.h = pairs[i].height / 4;
    q.D = pairs[i].max_disp;
    q.wta = const_cast<int16_t*>(in[i]);  // only read
    q.mid = (int16_t*)x_maps.p + nS + oS;
    q.disp = out[i];
    oS += (size_t)q.w * q.h;
  }
  if ((s = cuda(cudaMemcpyAsync(sgm_tab.p, tab.data(), sizeof(XPair) * n, cudaMemcpyHostToDevice, st),
                "upload pair table")))
    return s;
  return post_launch(sgm_tab.p, n, maxw, maxh, post, st);
}

sv_status Ctx::pipeline_ex(const sv_pair* pairs, int n, const sv_coarse_opts& o, float* const* out, cudaStream_t st) {
  std::vector<size_t> off(n + 1, 0);
  for (int i = 0; i < n; ++i) off[i + 1] = off[i] + (size_t)(pairs[i].width / 4) * (pairs[i].height / 4);
  sv_status s = cuda(coarse_maps.ensure(std::max<size_t>(1, off[n]) * sizeof(int16_t)), "alloc coarse maps");
  if (s) return s;
  std::vector<int16_t*> maps(n);
  for (int i = 0; i < n; ++i) maps[i] = (int16_t*)coarse_maps.p + off[i];
  if ((s = coarse_ext(pairs, n, o, maps.data(), nullptr, st))) return s;
  std::vector<const int16_t*> cm(maps.begin(), maps.end());
  return refine_infer(pairs, cm.data(), n, out, st);
}

}  // namespace sv

namespace {

sv_status check_opts(sv::Ctx* c, const sv_coarse_opts* o) {
  if (!o) return c->fail(SV_ERR_INVALID_ARG, "opts is NULL");
  if (o->cost != SV_COST_ZNCC && o->cost != SV_COST_CENSUS) return c->fail(SV_ERR_INVALID_ARG, "unknown cost %d", o->cost);
  if (o->cost == SV_COST_CENSUS && o->census_window != 3 && o->census_window != 5 && o->census_window != 7)
    return c->fail(SV_ERR_INVALID_ARG, "census_window must be 3, 5 or 7");
  if (o->aggregation == SV_AGG_SGM) {
    if (!(o->P1 >= 0.f) || !(o->P2 >= 0.f)) return c->fail(SV_ERR_INVALID_ARG, "penalties must be >= 0");
    if (o->npaths < 1 || o->npaths > 4) return c->fail(SV_ERR_INVALID_ARG, "npaths must be 1..4");
  } else if (o->aggregation == SV_AGG_DT) {
    if (!(o->dt_sigma_s > 0.f) || !(o->dt_sigma_r > 0.f)) return c->fail(SV_ERR_INVALID_ARG, "DT scales must be > 0");
    if (o->dt_iters < 1 || o->dt_iters > 8) return c->fail(SV_ERR_INVALID_ARG, "dt_iters must be 1..8");
  } else if (o->aggregation != SV_AGG_NONE) {
    return c->fail(SV_ERR_INVALID_ARG, "unknown aggregation %d", o->aggregation);
  }
  if (o->post & ~(SV_POST_SMP | SV_POST_MEDIAN)) return c->fail(SV_ERR_INVALID_ARG, "unknown post-processing flag");
  return SV_OK;
}

sv_status check_outputs(sv::Ctx* c, int n, void* const* out, const char* what) {
  if (n == 0) return SV_OK;
  if (!out) return c->fail(SV_ERR_INVALID_ARG, "%s is NULL", what);
  for (int i = 0; i < n; ++i)
    if (!out[i]) return c->fail(SV_ERR_INVALID_ARG, "%s[%d] is NULL", what, i);
  return SV_OK;
}

}  // namespace

extern "C" sv_status sv_coarse_match_ex(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const sv_coarse_opts* opts,
                                        int16_t* const* disp_out, float* const* cost_out, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  sv::Ctx* c = reinterpret_cast<sv::Ctx*>(ctx);
  c->err.clear();
  sv_status s = c->check_pairs(pairs, n_pairs);
  if (s) return s;
  if ((s = check_opts(c, opts))) return s;
  if ((s = check_outputs(c, n_pairs, (void* const*)disp_out, "disp_out"))) return s;
  if (n_pairs == 0) return SV_OK;
  sv::DeviceGuardInt g(c->device);
  return c->coarse_ext(pairs, n_pairs, *opts, disp_out, cost_out, (cudaStream_t)stream);
}

extern "C" sv_status sv_coarse_match_sgm(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, float P1, float P2, int npaths,
                                         int16_t* const* disp_out, float* const* cost_out, sv_stream stream) {
  sv_coarse_opts o{};
  o.cost = SV_COST_ZNCC;
  o.aggregation = SV_AGG_SGM;
  o.P1 = P1;
  o.P2 = P2;
  o.npaths = npaths;
  return sv_coarse_match_ex(ctx, pairs, n_pairs, &o, disp_out, cost_out, stream);
}

extern "C" sv_status sv_postprocess(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const int16_t* const* disp_in,
                                    int post, int16_t* const* disp_out, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  sv::Ctx* c = reinterpret_cast<sv::Ctx*>(ctx);
  c->err.clear();
  if (n_pairs < 0 || (n_pairs > 0 && !pairs)) return c->fail(SV_ERR_INVALID_ARG, "invalid pair list");
  if (post & ~(SV_POST_SMP | SV_POST_MEDIAN)) return c->fail(SV_ERR_INVALID_ARG, "unknown post-processing flag");
  sv_status s;
  if ((s = check_outputs(c, n_pairs, (void* const*)disp_in, "disp_in"))) return s;
  if ((s = check_outputs(c, n_pairs, (void* const*)disp_out, "disp_out"))) return s;
  for (int i = 0; i < n_pairs; ++i) {
    const sv_pair& p = pairs[i];
    if (p.width < 4 || p.height < 4 || p.width > sv::kMaxSide || p.height > sv::kMaxSide)
      return c->fail(SV_ERR_INVALID_ARG, "pair %d: size %dx%d", i, p.width, p.height);
    if (p.max_disp < 1 || p.max_disp > sv::kMaxDisp || p.max_disp > p.width / 4)
      return c->fail(SV_ERR_INVALID_ARG, "pair %d: max_disp %d", i, p.max_disp);
    const size_t bytes = sizeof(int16_t) * (p.width / 4) * (p.height / 4);
    const char* a = (const char*)disp_in[i];
    const char* b = (const char*)disp_out[i];
    if (a < b + bytes && b < a + bytes) return c->fail(SV_ERR_INVALID_ARG, "pair %d: disp_out overlaps disp_in", i);
  }
  if (n_pairs == 0) return SV_OK;
  sv::DeviceGuardInt g(c->device);
  return c->postprocess(pairs, n_pairs, disp_in, post, disp_out, (cudaStream_t)stream);
}

extern "C" sv_status sv_pipeline_ex(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const sv_coarse_opts* opts,
                                    float* const* disp_out, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  sv::Ctx* c = reinterpret_cast<sv::Ctx*>(ctx);
  c->err.clear();
  sv_status s = c->check_pairs(pairs, n_pairs);
  if (s) return s;
  if ((s = check_opts(c, opts))) return s;
  if ((s = check_outputs(c, n_pairs, (void* const*)disp_out, "disp_out"))) return s;
  if (n_pairs == 0) return SV_OK;
  sv::DeviceGuardInt g(c->device);
  return c->pipeline_ex(pairs, n_pairs, *opts, disp_out, (cudaStream_t)stream);
}
