// t1net.cu -- the paper's Table I network (Sec. III-B1) on CUDA cores, FP32, all pairs of
// a call per launch.
//
//   t1_inputs_kernel   X_1 = 2 x 2 box mean of the left image / 256 and X_0 = 4 x bilinear x2 of
//                      the coarse map / 256, both at half resolution
//   t1_conv_kernel     one layer: 5 x 5 (or 1 x 1) conv, stride 1 or 2, or 5 x 5 stride-2
//                      deconvolution, over the channel concatenation of up to four NHWC
//                      tensors of the same size (the skip connections of Table I are read in
//                      place, never copied); bias, optional leaky ReLU 0.1 and output scale
//   t1_gauss_kernel    mu, sigma from the heads and the decoder input
//                      (mu - 1) + eps exp(sigma - 1) (Eq. 8; eps = 0 at inference)
//
// Every layer is a direct convolution: a CTA stages a tile of the concatenated input for
// CIC channels at a time and the matching weights in shared memory; each thread
// accumulates COT output channels of one output pixel (conv) or of the four output
// phases (2 y + py, 2 x + px) of one input position (deconv: each phase reads its own
// taps ky = py (mod 2), kx = px (mod 2), so a warp's threads share one tap sequence).
#include "sv_ctx.cuh"

namespace sv {

namespace {

constexpr int kTW = 16, kTH = 8;  // thread tile

struct T1Src {
  const float* p[4];
  int c[4];
};

// One layer of one pair.
struct T1Job {
  T1Src src;
  int Hi, Wi;
  float* out;
  int Ho, Wo;
};

// Per-pair inputs of t1_inputs_kernel / t1_gauss_kernel.
struct T1PairIO {
  const uint8_t* L;
  int pitch, W, H, w, h;
  const int16_t* coarse_i;  // integer coarse map, or
  const float* coarse_f;    // real-valued coarse map when non-null
  float* X0;                // [Hh][Wh]
  float* X1;                // [Hh][Wh]
  const float* heads;       // [H8][W8][2]
  const float* eps;         // [H8][W8] or null
  float* g;                 // [H8][W8] decoder input
  float* mu;                // [H8][W8] or null
  float* sigma;             // [H8][W8] or null
  int H8, W8;
};

__device__ __forceinline__ float src_at(const T1Src& s, size_t pix, int ci) {
  if (ci < s.c[0]) return s.p[0][pix * s.c[0] + ci];
  ci -= s.c[0];
  if (ci < s.c[1]) return s.p[1][pix * s.c[1] + ci];
  ci -= s.c[1];
  if (ci < s.c[2]) return s.p[2][pix * s.c[2] + ci];
  ci -= s.c[2];
  if (ci < s.c[3]) return s.p[3][pix * s.c[3] + ci];
  return 0.f;
}

__global__ void t1_inputs_kernel(const T1PairIO* __restrict__ io) {
  const T1PairIO& p = io[blockIdx.z];
  const int Hh = (p.H + 1) / 2, Wh = (p.W + 1) / 2;
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= Wh || y >= Hh) return;
  const int y1 = min(2 * y + 1, p.H - 1), x1 = min(2 * x + 1, p.W - 1);
  const uint8_t* r0 = p.L + (size_t)(2 * y) * p.pitch;
  const uint8_t* r1 = p.L + (size_t)y1 * p.pitch;
  const float s = (float)r0[2 * x] + (float)r0[x1] + (float)r1[2 * x] + (float)r1[x1];
  p.X1[(size_t)y * Wh + x] = s * (1.0f / 1024.0f);
  // bilinear x2 with half-pixel centres: source (x + 1/2) / 2 - 1/2, clamped
  float sx = (float)x * 0.5f - 0.25f, sy = (float)y * 0.5f - 0.25f;
  sx = fminf(fmaxf(sx, 0.f), (float)(p.w - 1));
  sy = fminf(fmaxf(sy, 0.f), (float)(p.h - 1));
  const int a = (int)sx, c = (int)sy;
  const int a1 = min(a + 1, p.w - 1), c1 = min(c + 1, p.h - 1);
  const float fx = sx - (float)a, fy = sy - (float)c;
  auto cm = [&](int yy, int xx) {
    return p.coarse_f ? p.coarse_f[(size_t)yy * p.w + xx] : (float)p.coarse_i[(size_t)yy * p.w + xx];
  };
  const float top = (1.f - fx) * cm(c, a) + fx * cm(c, a1);
  const float bot = (1.f - fx) * cm(c1, a) + fx * cm(c1, a1);
  p.X0[(size_t)y * Wh + x] = ((1.f - fy) * top + fy * bot) * (4.0f / 256.0f);
}

__global__ void t1_gauss_kernel(const T1PairIO* __restrict__ io) {
  const T1PairIO& p = io[blockIdx.y];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= p.H8 * p.W8) return;
  const float m = p.heads[2 * q], s = p.heads[2 * q + 1];
  p.g[q] = (m - 1.0f) + (p.eps ? p.eps[q] * expf(s - 1.0f) : 0.0f);
  if (p.mu) p.mu[q] = m;
  if (p.sigma) p.sigma[q] = s;
}

// MODE 0: conv stride 1, 1: conv stride 2, 2: deconv stride 2 (outputs 2 i + k - 2, cropped).
template <int MODE, int KS, int COT, int CIC>
__global__ void __launch_bounds__(kTW * kTH)
t1_conv_kernel(const T1Job* __restrict__ jobs, int groups, const float* __restrict__ wt, const float* __restrict__ bias,
               int Ci, int Co, int act, float scale) {
  constexpr int PAD = KS / 2;
  constexpr int S = MODE == 1 ? 2 : 1;
  constexpr int TR = MODE == 2 ? kTH + 2 : (kTH - 1) * S + KS;
  constexpr int TC = MODE == 2 ? kTW + 2 : (kTW - 1) * S + KS;
  constexpr int NP = MODE == 2 ? 4 : 1;  // output phases per thread
  __shared__ float tile[CIC][TR][TC];
  __shared__ __align__(16) float wsm[KS * KS][CIC][COT];
  const T1Job& J = jobs[blockIdx.z / groups];
  const int co0 = (blockIdx.z % groups) * COT;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * kTW + tx;
  const int X0 = blockIdx.x * kTW, Y0 = blockIdx.y * kTH;
  // whole-block exit when the tile lies beyond this pair's output
  if (MODE == 2 ? (2 * X0 >= J.Wo || 2 * Y0 >= J.Ho) : (X0 >= J.Wo || Y0 >= J.Ho)) return;
  const int ry0 = MODE == 2 ? Y0 - 1 : Y0 * S - PAD;  // input row / column of tile element 0
  const int rx0 = MODE == 2 ? X0 - 1 : X0 * S - PAD;
  float acc[NP][COT];
#pragma unroll
  for (int q = 0; q < NP; ++q)
#pragma unroll
    for (int c = 0; c < COT; ++c) acc[q][c] = 0.f;
  for (int ci0 = 0; ci0 < Ci; ci0 += CIC) {
    for (int e = tid; e < TR * TC * CIC; e += kTW * kTH) {
      const int ci = e % CIC, rc = e / CIC;
      const int r = rc / TC, c = rc - r * TC;
      const int iy = ry0 + r, ix = rx0 + c;
      float v = 0.f;
      if (iy >= 0 && ix >= 0 && iy < J.Hi && ix < J.Wi && ci0 + ci < Ci) v = src_at(J.src, (size_t)iy * J.Wi + ix, ci0 + ci);
      tile[ci][r][c] = v;
    }
    for (int e = tid; e < KS * KS * CIC * COT; e += kTW * kTH) {
      const int co = e % COT, t = e / COT;
      const int ci = t % CIC, tap = t / CIC;
      const int gco = co0 + co, gci = ci0 + ci;
      wsm[tap][ci][co] = (gco < Co && gci < Ci) ? wt[((size_t)gco * KS * KS + tap) * Ci + gci] : 0.f;
    }
    __syncthreads();
    if constexpr (MODE == 2) {
#pragma unroll
      for (int py = 0; py < 2; ++py)
#pragma unroll
        for (int px = 0; px < 2; ++px)
#pragma unroll
          for (int ky = py; ky < KS; ky += 2)
#pragma unroll
            for (int kx = px; kx < KS; kx += 2) {
              const int r = ty + (py + 2 - ky) / 2 + 1, c = tx + (px + 2 - kx) / 2 + 1;
#pragma unroll
              for (int ci = 0; ci < CIC; ++ci) {
                const float v = tile[ci][r][c];
                const float* wp = wsm[ky * KS + kx][ci];
#pragma unroll
                for (int co = 0; co < COT; ++co) acc[py * 2 + px][co] = fmaf(v, wp[co], acc[py * 2 + px][co]);
              }
            }
    } else {
#pragma unroll
      for (int ky = 0; ky < KS; ++ky)
#pragma unroll
        for (int kx = 0; kx < KS; ++kx)
#pragma unroll
          for (int ci = 0; ci < CIC; ++ci) {
            const float v = tile[ci][ty * S + ky][tx * S + kx];
            const float* wp = wsm[ky * KS + kx][ci];
#pragma unroll
            for (int co = 0; co < COT; ++co) acc[0][co] = fmaf(v, wp[co], acc[0][co]);
          }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NP; ++q) {
    const int oy = MODE == 2 ? 2 * (Y0 + ty) + (q >> 1) : Y0 + ty;
    const int ox = MODE == 2 ? 2 * (X0 + tx) + (q & 1) : X0 + tx;
    if (oy < J.Ho && ox < J.Wo) {
      float* op = J.out + ((size_t)oy * J.Wo + ox) * Co + co0;
#pragma unroll
      for (int co = 0; co < COT; ++co)
        if (co0 + co < Co) {
          float v = acc[q][co] + bias[co0 + co];
          if (act && v < 0.f) v *= 0.1f;
          op[co] = v * scale;
        }
    }
  }
}

// Table I layer table: mode, kernel size, output / input channels.
struct T1Layer {
  int mode, ks, co, ci;
};
constexpr T1Layer kT1[13] = {{0, 5, 32, 1},  {0, 5, 32, 1},  {1, 5, 16, 64}, {0, 5, 8, 16}, {1, 5, 32, 24},
                             {0, 5, 16, 32}, {0, 1, 2, 48},  {0, 1, 32, 1},  {0, 5, 16, 80}, {2, 5, 16, 96},
                             {0, 5, 8, 40},  {2, 5, 16, 48}, {2, 5, 1, 81}};

template <int MODE, int KS, int COT, int CIC>
cudaError_t run_t1(const T1Job* jobs, int n, int gx, int gy, int Ci, int Co, const float* w, const float* b, int act,
                   float scale, cudaStream_t st) {
  const int groups = (Co + COT - 1) / COT;
  t1_conv_kernel<MODE, KS, COT, CIC><<<dim3(gx, gy, n * groups), dim3(kTW, kTH), 0, st>>>(jobs, groups, w, b, Ci, Co,
                                                                                        act, scale);
  return cudaGetLastError();
}

cudaError_t launch_t1_layer(int l, const T1Job* jobs, int n, int maxHo, int maxWo, const float* w, const float* b,
                            cudaStream_t st) {
  const T1Layer L = kT1[l];
  const int gx = L.mode == 2 ? (maxWo + 2 * kTW - 1) / (2 * kTW) : (maxWo + kTW - 1) / kTW;
  const int gy = L.mode == 2 ? (maxHo + 2 * kTH - 1) / (2 * kTH) : (maxHo + kTH - 1) / kTH;
  const int act = l == 6 || l == 12 ? 0 : 1;
  const float scale = l == 12 ? 256.0f : 1.0f;  // the output in pixels (256 Y)
  switch (l) {
    case 0: case 1: return run_t1<0, 5, 16, 1>(jobs, n, gx, gy, L.ci, L.co, w, b, act, scale, st);
    case 2: case 4: return run_t1<1, 5, 16, 8>(jobs, n, gx, gy, L.ci, L.co, w, b, act, scale, st);
    case 3: case 10: return run_t1<0, 5, 8, 8>(jobs, n, gx, gy, L.ci, L.co, w, b, act, scale, st);
    case 5: case 8: return run_t1<0, 5, 16, 8>(jobs, n, gx, gy, L.ci, L.co, w, b, act, scale, st);
    case 6: return run_t1<0, 1, 2, 8>(jobs, n, gx, gy, L.ci, L.co, w, b, act, scale, st);
    case 7: return run_t1<0, 1, 16, 1>(jobs, n, gx, gy, L.ci, L.co, w, b, act, scale, st);
    case 9: case 11: return run_t1<2, 5, 16, 8>(jobs, n, gx, gy, L.ci, L.co, w, b, act, scale, st);
    case 12: return run_t1<2, 5, 1, 8>(jobs, n, gx, gy, L.ci, L.co, w, b, act, scale, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

size_t t1_param_count() {
  size_t o = 0;
  for (const T1Layer& L : kT1) o += (size_t)L.co * L.ks * L.ks * L.ci + L.co;
  return o;
}

static size_t t1_w_off(int l) {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += (size_t)kT1[i].co * kT1[i].ks * kT1[i].ks * kT1[i].ci + kT1[i].co;
  return o;
}

// Forward pass of the Table I network for n pairs.  coarse_i / coarse_f: per pair coarse map
// (one of them); eps (nullable): per pair [H8][W8] noise; Y: per pair H x W disparity in
// pixels; mu / sigma (nullable arrays): per pair [H8][W8].
sv_status Ctx::t1_forward(const sv_pair* pairs, int n, const int16_t* const* coarse_i, const float* const* coarse_f,
                          const float* const* eps, float* const* Y, float* const* mu, float* const* sigma,
                          cudaStream_t st) {
  if (n == 0) return SV_OK;
  // per pair activation sizes (floats): X0, X1, FE1, FE2, EN1, EN1R, EN2, EN2R, heads, g, D1, D1R, D2, D2R, D
  std::vector<std::array<size_t, 15>> off(n);
  size_t total = 0;
  int maxH[4] = {0, 0, 0, 0}, maxW[4] = {0, 0, 0, 0};
  for (int i = 0; i < n; ++i) {
    const Levels lv(pairs[i].height, pairs[i].width);
    for (int k = 0; k < 4; ++k) {
      maxH[k] = std::max(maxH[k], lv.H[k]);
      maxW[k] = std::max(maxW[k], lv.W[k]);
    }
    const size_t P2 = (size_t)lv.H[1] * lv.W[1], P4 = (size_t)lv.H[2] * lv.W[2], P8 = (size_t)lv.H[3] * lv.W[3];
    const size_t sz[15] = {P2, P2, P2 * 32, P2 * 32, P4 * 16, P4 * 8, P8 * 32, P8 * 16, P8 * 2, P8,
                           P8 * 32, P8 * 16, P4 * 16, P4 * 8, P2 * 16};
    for (int k = 0; k < 15; ++k) {
      off[i][k] = total;
      total += (sz[k] + 31) / 32 * 32;  // 128-byte aligned tensors
    }
  }
  sv_status s;
  if ((s = cuda(t1_act.ensure(total * sizeof(float)), "alloc Table I activations"))) return s;
  const size_t io_bytes = sizeof(T1PairIO) * n, job_bytes = sizeof(T1Job) * n * 13;
  if ((s = cuda(t1_tab.ensure(io_bytes + job_bytes), "alloc Table I tables"))) return s;
  std::vector<unsigned char> host(io_bytes + job_bytes);
  T1PairIO* io = reinterpret_cast<T1PairIO*>(host.data());
  T1Job* jobs = reinterpret_cast<T1Job*>(host.data() + io_bytes);
  float* A = (float*)t1_act.p;
  for (int i = 0; i < n; ++i) {
    const sv_pair& p = pairs[i];
    const Levels lv(p.height, p.width);
    auto T = [&](int k) { return A + off[i][k]; };
    T1PairIO& q = io[i];
    q = T1PairIO{};
    q.L = p.left;
    q.pitch = p.pitch;
    q.W = p.width;
    q.H = p.height;
    q.w = p.width / 4;
    q.h = p.height / 4;
    q.coarse_i = coarse_i ? coarse_i[i] : nullptr;
    q.coarse_f = coarse_f ? coarse_f[i] : nullptr;
    q.X0 = T(0);
    q.X1 = T(1);
    q.heads = T(8);
    q.eps = eps ? eps[i] : nullptr;
    q.g = T(9);
    q.mu = mu ? mu[i] : nullptr;
    q.sigma = sigma ? sigma[i] : nullptr;
    q.H8 = lv.H[3];
    q.W8 = lv.W[3];
    // layer l of pair i: sources (concatenated in Table I's order), sizes, output
    auto job = [&](int l, std::initializer_list<std::pair<int, int>> srcs, int lin, int lout, float* out) {
      T1Job& j = jobs[l * n + i];
      j = T1Job{};
      int k = 0;
      for (auto& sc : srcs) {
        j.src.p[k] = T(sc.first);
        j.src.c[k] = sc.second;
        ++k;
      }
      j.Hi = lv.H[lin];
      j.Wi = lv.W[lin];
      j.out = out;
      j.Ho = lv.H[lout];
      j.Wo = lv.W[lout];
    };
    job(0, {{0, 1}}, 1, 1, T(2));                             // FE_1 <- X_0
    job(1, {{1, 1}}, 1, 1, T(3));                             // FE_2 <- X_1
    job(2, {{2, 32}, {3, 32}}, 1, 2, T(4));                   // EN_1 <- FE_1 & FE_2
    job(3, {{4, 16}}, 2, 2, T(5));                            // EN_1_R <- EN_1
    job(4, {{4, 16}, {5, 8}}, 2, 3, T(6));                    // EN_2 <- EN_1 & EN_1_R
    job(5, {{6, 32}}, 3, 3, T(7));                            // EN_2_R <- EN_2
    job(6, {{6, 32}, {7, 16}}, 3, 3, T(8));                   // heads <- EN_2 & EN_2_R
    job(7, {{9, 1}}, 3, 3, T(10));                            // D_1 <- gaussian
    job(8, {{10, 32}, {6, 32}, {7, 16}}, 3, 3, T(11));        // D_1_R <- D_1 & EN_2 & EN_2_R
    job(9, {{10, 32}, {6, 32}, {7, 16}, {11, 16}}, 3, 2, T(12));  // D_2 <- D_1 & EN_2 & EN_2_R & D_1_R
    job(10, {{12, 16}, {4, 16}, {5, 8}}, 2, 2, T(13));        // D_2_R <- D_2 & EN_1 & EN_1_R
    job(11, {{12, 16}, {4, 16}, {5, 8}, {13, 8}}, 2, 1, T(14));  // D <- D_2 & EN_1 & EN_1_R & D_2_R
    job(12, {{14, 16}, {0, 1}, {2, 32}, {3, 32}}, 1, 0, Y[i]);   // Y <- D & X_0 & FE_1 & FE_2
  }
  if ((s = cuda(cudaMemcpyAsync(t1_tab.p, host.data(), host.size(), cudaMemcpyHostToDevice, st),
                "upload Table I tables")))
    return s;
  const T1PairIO* d_io = (const T1PairIO*)t1_tab.p;
  const T1Job* d_jobs = (const T1Job*)((unsigned char*)t1_tab.p + io_bytes);
  const float* W = (const float*)w32.p;
  {
    LaunchScope ls(*this, "t1_inputs", st);
    t1_inputs_kernel<<<dim3((maxW[1] + 127) / 128, maxH[1], n), 128, 0, st>>>(d_io);
    if ((s = cuda(cudaGetLastError(), "Table I inputs"))) return s;
  }
  static const char* names[13] = {"t1_fe1", "t1_fe2", "t1_en1", "t1_en1r", "t1_en2", "t1_en2r", "t1_heads",
                                  "t1_d1", "t1_d1r", "t1_d2", "t1_d2r", "t1_d", "t1_y"};
  static const int out_level[13] = {1, 1, 2, 2, 3, 3, 3, 3, 3, 2, 2, 1, 0};
  for (int l = 0; l < 13; ++l) {
    if (l == 7) {
      LaunchScope ls(*this, "t1_gauss", st);
      t1_gauss_kernel<<<dim3((maxH[3] * maxW[3] + 255) / 256, n), 256, 0, st>>>(d_io);
      if ((s = cuda(cudaGetLastError(), "Table I reparameterisation"))) return s;
    }
    LaunchScope ls(*this, names[l], st);
    const size_t wo = t1_w_off(l);
    const size_t bo = wo + (size_t)kT1[l].co * kT1[l].ks * kT1[l].ks * kT1[l].ci;
    if ((s = cuda(launch_t1_layer(l, d_jobs + (size_t)l * n, n, maxH[out_level[l]], maxW[out_level[l]], W + wo, W + bo,
                                  st),
                  names[l])))
      return s;
  }
  return SV_OK;
}

}  // namespace sv

// ---------------------------------------------------------------- loss of Eq. 9-11
namespace sv {
namespace {

constexpr int kLossBlocks = 256;  // fixed grid: the summation order does not depend on timing

struct LossPair {
  const float* Y;
  const float* gt;
  const uint8_t* noc;
  const float* mu;
  const float* sg;
  float* gY;
  float* gmu;
  float* gsg;
  size_t P, nl;
};

__device__ double block_sum(double v, double* sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sm[i];
  __syncthreads();
  return t;
}

// Per block: partial sums of the weighted L1 term and of the KL term over all pairs, with the
// gradients written on the way (inv_p = 1 / total pixels, kl_scale = 256 / total latent).
__global__ void loss_paper_partial(const LossPair* __restrict__ lp, int n, double inv_p, double kl_scale,
                                   double* __restrict__ slots) {
  __shared__ double sm[32];
  double a = 0.0, b = 0.0;
  for (int i = 0; i < n; ++i) {
    const LossPair& q = lp[i];
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < q.P; p += (size_t)gridDim.x * blockDim.x) {
      const float e = q.gt[p] - q.Y[p];
      const float wgt = q.noc[p] ? 2.f : 1.f;
      a += (double)wgt * fabs((double)e);
      if (q.gY) q.gY[p] = (float)(e > 0.f ? -wgt * inv_p : e < 0.f ? wgt * inv_p : 0.0);
    }
    for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < q.nl; p += (size_t)gridDim.x * blockDim.x) {
      const double m = (double)q.mu[p] - 1.0, s = (double)q.sg[p] - 1.0;
      b += 0.5 * (m * m + exp(2.0 * s) - 1.0 - 2.0 * s);
      if (q.gmu) q.gmu[p] = (float)(kl_scale * m);
      if (q.gsg) q.gsg[p] = (float)(kl_scale * (exp(2.0 * s) - 1.0));
    }
  }
  a = block_sum(a, sm);
  b = block_sum(b, sm);
  if (threadIdx.x == 0) {
    slots[2 * blockIdx.x] = a;
    slots[2 * blockIdx.x + 1] = b;
  }
}

__global__ void loss_paper_finish(const double* __restrict__ slots, double inv_p256, double inv_nl, double* out) {
  if (threadIdx.x != 0) return;
  double a = 0.0, b = 0.0;
  for (int i = 0; i < kLossBlocks; ++i) {
    a += slots[2 * i];
    b += slots[2 * i + 1];
  }
  const double l1 = a * inv_p256, l2 = b * inv_nl;  // Loss_1 in normalised units (|gt - Y| / 256)
  out[0] = 256.0 * (l1 + l2);
  out[1] = l1;
  out[2] = l2;
}

}  // namespace

sv_status Ctx::loss_paper(const sv_pair* pairs, int n, const float* const* Y, const float* const* gt,
                          const uint8_t* const* noc, const float* const* mu, const float* const* sigma, double* out,
                          float* const* gY, float* const* gmu, float* const* gsigma, cudaStream_t st) {
  size_t P = 0, nl = 0;
  std::vector<LossPair> lp(n);
  for (int i = 0; i < n; ++i) {
    const Levels lv(pairs[i].height, pairs[i].width);
    lp[i] = LossPair{Y[i], gt[i], noc[i], mu[i], sigma[i], gY ? gY[i] : nullptr, gmu ? gmu[i] : nullptr,
                     gsigma ? gsigma[i] : nullptr, (size_t)pairs[i].width * pairs[i].height,
                     (size_t)lv.H[3] * lv.W[3]};
    P += lp[i].P;
    nl += lp[i].nl;
  }
  sv_status s;
  if ((s = cuda(loss_slots.ensure(sizeof(double) * 2 * kLossBlocks + sizeof(LossPair) * n), "alloc loss slots")))
    return s;
  double* slots = (double*)loss_slots.p;
  LossPair* d_lp = (LossPair*)(slots + 2 * kLossBlocks);
  if ((s = cuda(cudaMemcpyAsync(d_lp, lp.data(), sizeof(LossPair) * n, cudaMemcpyHostToDevice, st), "upload loss table")))
    return s;
  // d total / d Y_px = -w sign(gt - Y) / P (the 256 of Eq. 9 cancels the normalisation)
  {
    LaunchScope ls(*this, "loss_paper", st);
    loss_paper_partial<<<kLossBlocks, 256, 0, st>>>(d_lp, n, 1.0 / (double)P, 256.0 / (double)nl, slots);
    if ((s = cuda(cudaGetLastError(), "loss partial sums"))) return s;
  }
  LaunchScope ls(*this, "loss_paper", st);
  loss_paper_finish<<<1, 32, 0, st>>>(slots, 1.0 / (256.0 * (double)P), 1.0 / (double)nl, out);
  return cuda(cudaGetLastError(), "loss total");
}

}  // namespace sv

extern "C" sv_status sv_loss_paper(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const float* const* Y,
                                   const float* const* gt, const uint8_t* const* noc, const float* const* mu,
                                   const float* const* sigma, double* loss_out, float* const* grad_Y,
                                   float* const* grad_mu, float* const* grad_sigma, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  sv::Ctx* c = reinterpret_cast<sv::Ctx*>(ctx);
  c->err.clear();
  if (n_pairs <= 0 || !pairs || !Y || !gt || !noc || !mu || !sigma || !loss_out)
    return c->fail(SV_ERR_INVALID_ARG, "NULL argument or empty batch");
  for (int i = 0; i < n_pairs; ++i) {
    if (!Y[i] || !gt[i] || !noc[i] || !mu[i] || !sigma[i]) return c->fail(SV_ERR_INVALID_ARG, "pair %d: NULL buffer", i);
    if (pairs[i].width < 1 || pairs[i].height < 1 || pairs[i].width > sv::kMaxSide || pairs[i].height > sv::kMaxSide)
      return c->fail(SV_ERR_INVALID_ARG, "pair %d: size %dx%d", i, pairs[i].width, pairs[i].height);
  }
  sv::DeviceGuardInt g(c->device);
  return c->loss_paper(pairs, n_pairs, Y, gt, noc, mu, sigma, loss_out, grad_Y, grad_mu, grad_sigma,
                       (cudaStream_t)stream);
}
