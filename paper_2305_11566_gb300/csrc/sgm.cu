// sgm.cu -- semi-global matching variant of the coarse stage (Sec. III-A, Eq. 1-6), for
// every pair of a call:
//
//   sgm_box4   quarter-size images: 4 x 4 box sums of L and R (int32; the trailing W mod 4
//              columns and H mod 4 rows are dropped)
//   sgm_cost   cost volume C = 1 - rho (Eq. 1-3: window means, exact integer window sums,
//              clamp-to-edge windows, rho = 0 for a zero-variance window); candidates with
//              x - d < 0 take the largest cost of Eq. 1, 2
//   sgm_path   aggregation along one direction (Eq. 4), one block per path line and one
//              thread per disparity, walked from the image border; the directions run one
//              after another and add into the output volume (Eq. 5)
//   sgm_wta    Eq. 6: argmin over d of the aggregated cost, lowest d on ties
#include "sv_ctx.cuh"

namespace sv {

namespace {

struct SgmPair {
  const uint8_t* L;
  const uint8_t* R;
  int pitch, w, h, D;
  int32_t* SL;    // [h][w] box sums of L
  int32_t* SR;    // [h][w] box sums of R
  float* C;       // [h][w][D] ZNCC cost
  float* A;       // [h][w][D] aggregated cost
  int16_t* disp;  // [h][w]
};

__global__ void sgm_box4(const SgmPair* __restrict__ P) {
  const SgmPair& p = P[blockIdx.z];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (y >= p.h || x >= p.w) return;
  int32_t sl = 0, sr = 0;
  for (int j = 0; j < 4; ++j) {
    const uint8_t* lr = p.L + (size_t)(4 * y + j) * p.pitch + 4 * x;
    const uint8_t* rr = p.R + (size_t)(4 * y + j) * p.pitch + 4 * x;
    for (int i = 0; i < 4; ++i) {
      sl += lr[i];
      sr += rr[i];
    }
  }
  p.SL[(size_t)y * p.w + x] = sl;
  p.SR[(size_t)y * p.w + x] = sr;
}

// One block per (row y, pair): the k box-sum rows of both images around y (clamped) are
// staged in shared memory; a thread takes columns x and every candidate d of each.
__global__ void sgm_cost(const SgmPair* __restrict__ P, int k) {
  extern __shared__ int32_t rows[];  // [k][w] of L, then [k][w] of R
  const SgmPair& p = P[blockIdx.y];
  const int y = blockIdx.x, w = p.w, h = p.h;
  if (y >= h) return;
  const int r = k / 2;
  int32_t* Ls = rows;
  int32_t* Rs = rows + k * w;
  for (int e = threadIdx.x; e < k * w; e += blockDim.x) {
    const int j = e / w, xx = e - j * w;
    const int yy = min(max(y + j - r, 0), h - 1);
    Ls[e] = p.SL[(size_t)yy * w + xx];
    Rs[e] = p.SR[(size_t)yy * w + xx];
  }
  __syncthreads();
  const long long N = (long long)k * k;
  for (int x = threadIdx.x; x < w; x += blockDim.x) {
    long long sl = 0, sll = 0;
    for (int j = 0; j < k; ++j)
      for (int i = -r; i <= r; ++i) {
        const long long a = Ls[j * w + min(max(x + i, 0), w - 1)];
        sl += a;
        sll += a * a;
      }
    const long long vL = N * sll - sl * sl;
    float* out = p.C + ((size_t)y * w + x) * p.D;
    for (int d = 0; d < p.D; ++d) {
      float c = 2.f;
      if (x - d >= 0) {
        long long sr = 0, srr = 0, slr = 0;
        for (int j = 0; j < k; ++j)
          for (int i = -r; i <= r; ++i) {
            const long long a = Ls[j * w + min(max(x + i, 0), w - 1)];
            const long long b = Rs[j * w + min(max(x - d + i, 0), w - 1)];
            sr += b;
            srr += b * b;
            slr += a * b;
          }
        const long long vR = N * srr - sr * sr, num = N * slr - sl * sr;
        const double rho = (vL == 0 || vR == 0) ? 0.0 : (double)num / sqrt((double)vL * (double)vR);
        c = (float)(1.0 - rho);
      }
      out[d] = c;
    }
  }
}

// Eq. 4 along direction dir (0: left to right along rows, 1: right to left, 2: top to bottom
// along columns, 3: bottom to top) for line blockIdx.x of pair blockIdx.y; thread d holds
// disparity d.  first: the direction writes the output volume, later ones add to it.
__global__ void sgm_path(const SgmPair* __restrict__ P, int dir, int first, float P1, float P2) {
  __shared__ float prev[kMaxDisp + 2];  // prev[1 + d]; prev[0], prev[D + 1]: no candidate
  __shared__ float wmin[kMaxDisp / 32];
  const SgmPair& p = P[blockIdx.y];
  const int w = p.w, h = p.h, D = p.D;
  const int dx = dir == 0 ? 1 : dir == 1 ? -1 : 0;
  const int dy = dir == 2 ? 1 : dir == 3 ? -1 : 0;
  const int nlines = dy == 0 ? h : w, len = dy == 0 ? w : h;
  const int line = blockIdx.x;
  if (line >= nlines) return;  // whole block
  const int d = threadIdx.x, nw = blockDim.x >> 5;
  const bool act = d < D;
  const float kNone = __int_as_float(0x7f800000);  // +infinity: a missing neighbour
  if (threadIdx.x == 0) {
    prev[0] = kNone;
    prev[D + 1] = kNone;
  }
  float m = 0.f;  // minimum over d of the previous pixel's C_r
  for (int s = 0; s < len; ++s) {
    const int x = dx == 0 ? line : dx > 0 ? s : w - 1 - s;
    const int y = dy == 0 ? line : dy > 0 ? s : h - 1 - s;
    const size_t at = ((size_t)y * w + x) * D + d;
    float cur = kNone;
    if (act) {
      const float c = p.C[at];
      if (s == 0) {
        cur = c;
      } else {
        float best = prev[1 + d];
        best = fminf(best, prev[d] + P1);      // d - 1
        best = fminf(best, prev[2 + d] + P1);  // d + 1
        best = fminf(best, m + P2);
        cur = c + (best - m);
      }
    }
    __syncthreads();  // every thread has read prev
    if (act) {
      prev[1 + d] = cur;
      p.A[at] = first ? cur : p.A[at] + cur;
    }
    float v = cur;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) wmin[threadIdx.x >> 5] = v;
    __syncthreads();
    m = wmin[0];
    for (int i = 1; i < nw; ++i) m = fminf(m, wmin[i]);
  }
}

__global__ void sgm_wta(const SgmPair* __restrict__ P) {
  const SgmPair& p = P[blockIdx.y];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p.w * p.h) return;
  const float* a = p.A + (size_t)q * p.D;
  int best = 0;
  float bv = a[0];
  for (int d = 1; d < p.D; ++d)
    if (a[d] < bv) {
      bv = a[d];
      best = d;
    }
  p.disp[q] = (int16_t)best;
}

}  // namespace

sv_status Ctx::coarse_sgm(const sv_pair* pairs, int n, float P1, float P2, int npaths, int16_t* const* disp,
                          float* const* cost_out, cudaStream_t st) {
  const int k = cfg.window;
  int maxw = 0, maxh = 0, maxD = 1;
  size_t nS = 0, nV = 0, nA = 0;
  for (int i = 0; i < n; ++i) {
    const int w = pairs[i].width / 4, h = pairs[i].height / 4;
    maxw = std::max(maxw, w);
    maxh = std::max(maxh, h);
    maxD = std::max(maxD, pairs[i].max_disp);
    nS += (size_t)w * h;
    nV += (size_t)w * h * pairs[i].max_disp;
    if (!cost_out || !cost_out[i]) nA += (size_t)w * h * pairs[i].max_disp;
  }
  const size_t cost_smem = (size_t)2 * k * maxw * sizeof(int32_t);
  if (cost_smem > 227 * 1024)
    return fail(SV_ERR_UNSUPPORTED, "SGM cost rows need %zu bytes of shared memory (window %d, coarse width %d)",
                cost_smem, k, maxw);
  sv_status s;
  if ((s = cuda(sgm_s.ensure(2 * nS * sizeof(int32_t)), "alloc SGM box sums"))) return s;
  if ((s = cuda(sgm_c.ensure(nV * sizeof(float)), "alloc SGM cost volume"))) return s;
  if (nA && (s = cuda(sgm_a.ensure(nA * sizeof(float)), "alloc SGM aggregated volume"))) return s;
  if ((s = cuda(sgm_tab.ensure(sizeof(SgmPair) * n), "alloc SGM pair table"))) return s;
  std::vector<SgmPair> tab(n);
  size_t oS = 0, oV = 0, oA = 0;
  for (int i = 0; i < n; ++i) {
    const int w = pairs[i].width / 4, h = pairs[i].height / 4, D = pairs[i].max_disp;
    SgmPair& q = tab[i];
    q.L = (const uint8_t*)pairs[i].left;
    q.R = (const uint8_t*)pairs[i].right;
    q.pitch = pairs[i].pitch;
    q.w = w;
    q.h = h;
    q.D = D;
    q.SL = (int32_t*)sgm_s.p + oS;
    q.SR = (int32_t*)sgm_s.p + nS + oS;
    q.C = (float*)sgm_c.p + oV;
    if (cost_out && cost_out[i]) {
      q.A = cost_out[i];
    } else {
      q.A = (float*)sgm_a.p + oA;
      oA += (size_t)w * h * D;
    }
    q.disp = disp[i];
    oS += (size_t)w * h;
    oV += (size_t)w * h * D;
  }
  if ((s = cuda(cudaMemcpyAsync(sgm_tab.p, tab.data(), sizeof(SgmPair) * n, cudaMemcpyHostToDevice, st),
                "upload SGM pair table")))
    return s;
  const SgmPair* T = (const SgmPair*)sgm_tab.p;
  {
    LaunchScope ls(*this, "sgm_box4", st);
    sgm_box4<<<dim3((maxw + 127) / 128, maxh, n), 128, 0, st>>>(T);
    if ((s = cuda(cudaGetLastError(), "SGM box sums"))) return s;
  }
  {
    LaunchScope ls(*this, "sgm_cost", st);
    if (cost_smem > 48 * 1024 &&
        (s = cuda(cudaFuncSetAttribute(sgm_cost, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cost_smem),
                  "SGM cost shared memory")))
      return s;
    sgm_cost<<<dim3(maxh, n), 256, cost_smem, st>>>(T, k);
    if ((s = cuda(cudaGetLastError(), "SGM cost"))) return s;
  }
  const int threads = 32 * ((maxD + 31) / 32);
  for (int dir = 0; dir < npaths; ++dir) {
    LaunchScope ls(*this, "sgm_path", st);
    sgm_path<<<dim3(std::max(maxw, maxh), n), threads, 0, st>>>(T, dir, dir == 0 ? 1 : 0, P1, P2);
    if ((s = cuda(cudaGetLastError(), "SGM path"))) return s;
  }
  {
    LaunchScope ls(*this, "sgm_wta", st);
    sgm_wta<<<dim3((maxw * maxh + 255) / 256, n), 256, 0, st>>>(T);
    if ((s = cuda(cudaGetLastError(), "SGM winner-take-all"))) return s;
  }
  return SV_OK;
}

}  // namespace sv

extern "C" sv_status sv_coarse_match_sgm(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, float P1, float P2, int npaths,
                                         int16_t* const* disp_out, float* const* cost_out, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  sv::Ctx* c = reinterpret_cast<sv::Ctx*>(ctx);
  c->err.clear();
  sv_status s = c->check_pairs(pairs, n_pairs);
  if (s) return s;
  if (!(P1 >= 0.f) || !(P2 >= 0.f)) return c->fail(SV_ERR_INVALID_ARG, "penalties must be >= 0");
  if (npaths < 1 || npaths > 4) return c->fail(SV_ERR_INVALID_ARG, "npaths must be 1..4");
  if (n_pairs == 0) return SV_OK;
  if (!disp_out) return c->fail(SV_ERR_INVALID_ARG, "disp_out is NULL");
  for (int i = 0; i < n_pairs; ++i)
    if (!disp_out[i]) return c->fail(SV_ERR_INVALID_ARG, "disp_out[%d] is NULL", i);
  sv::DeviceGuardInt g(c->device);
  return c->coarse_sgm(pairs, n_pairs, P1, P2, npaths, disp_out, cost_out, (cudaStream_t)stream);
}
