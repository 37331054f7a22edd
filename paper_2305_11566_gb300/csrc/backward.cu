// backward.cu -- gradient kernels of the refinement network (FP32 and FP64), the
// transpose of the bilinear x4 upsampling, the loss and Adam.
//
//   dgrad_kernel    input gradient of a 3x3 / 1x1 conv read through a view (stride 1,
//                   stride 2, nearest x2 + crop): a gather over the taps and output pixels
//                   that read each input element, times the ReLU mask of the input.
//   wgrad_kernel    weight and bias gradient: each CTA reduces a chunk of output pixels for
//                   every weight it owns and adds the partial sum atomically.
//   latent_bwd      gradient through z = mu + eps exp(lv / 2) plus the loss's own mu / lv terms.
//   up4_bwd         transpose of the bilinear x4 upsampling (gather form, deterministic).
//   loss_*          smooth-L1 + KL per-block partial sums (summed in a fixed order) and the
//                   elementwise gradients.
//   adam_kernel     Adam on FP32 master weights.
#include "sv_internal.cuh"

namespace sv {

namespace {

__device__ __forceinline__ float atomic_add(float* a, float v) { return atomicAdd(a, v); }
__device__ __forceinline__ double atomic_add(double* a, double v) { return atomicAdd(a, v); }

// Input view V(vy, vx, ci) of the forward conv (zero outside), mode as in conv_direct.
template <typename T>
__device__ __forceinline__ T view_at(const T* in, int Hi, int Wi, int Ci, int Hv, int Wv, int mode, int vy, int vx,
                                     int ci) {
  if (vy < 0 || vx < 0 || vy >= Hv || vx >= Wv) return (T)0;
  const int iy = mode == CM_UP2 ? vy >> 1 : vy, ix = mode == CM_UP2 ? vx >> 1 : vx;
  return in[((size_t)iy * Wi + ix) * Ci + ci];
}

// One thread per (input pixel, ci).
template <typename T>
__global__ void dgrad_kernel(const T* __restrict__ gout, int Ho, int Wo, int Co, const T* __restrict__ w, int ks,
                             int mode, const T* __restrict__ mask_act, int Hi, int Wi, int Ci, int accumulate,
                             T* __restrict__ gin) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)Hi * Wi * Ci) return;
  const int ci = (int)(idx % Ci);
  const size_t pix = idx / Ci;
  const int iy = (int)(pix / Wi), ix = (int)(pix % Wi);
  const int pad = ks / 2, stride = mode == CM_S2 ? 2 : 1;
  T acc = 0;
  // virtual positions of the forward input that map to this element
  const int nvy = mode == CM_UP2 ? 2 : 1, nvx = nvy;
  for (int a = 0; a < nvy; ++a) {
    const int vy = mode == CM_UP2 ? 2 * iy + a : iy;
    if (mode == CM_UP2 && vy >= Ho) continue;  // cropped away
    for (int b = 0; b < nvx; ++b) {
      const int vx = mode == CM_UP2 ? 2 * ix + b : ix;
      if (mode == CM_UP2 && vx >= Wo) continue;
      for (int ky = 0; ky < ks; ++ky) {
        const int ny = vy - ky + pad;  // = oy * stride
        if (ny < 0 || ny % stride) continue;
        const int oy = ny / stride;
        if (oy >= Ho) continue;
        for (int kx = 0; kx < ks; ++kx) {
          const int nx = vx - kx + pad;
          if (nx < 0 || nx % stride) continue;
          const int ox = nx / stride;
          if (ox >= Wo) continue;
          const T* g = gout + ((size_t)oy * Wo + ox) * Co;
          const T* wp = w + ((size_t)ky * ks + kx) * Ci + ci;
          const size_t wstride = (size_t)ks * ks * Ci;
          for (int co = 0; co < Co; ++co) acc = fma(wp[co * wstride], g[co], acc);
        }
      }
    }
  }
  if (mask_act && !(mask_act[idx] > (T)0)) acc = 0;
  gin[idx] = accumulate ? gin[idx] + acc : acc;
}

// Weight + bias gradient.  Block = 256 threads over the weight elements (bias entries
// last); blockIdx.x = chunk of `chunk` output pixels.
template <typename T>
__global__ void wgrad_kernel(const T* __restrict__ gout, int Ho, int Wo, int Co, const T* __restrict__ in, int Hi,
                             int Wi, int Ci, int ks, int mode, int chunk, T* __restrict__ gw, T* __restrict__ gb) {
  const int nW = Co * ks * ks * Ci;
  const size_t P = (size_t)Ho * Wo;
  const size_t p0 = (size_t)blockIdx.x * chunk;
  const size_t p1 = p0 + chunk < P ? p0 + chunk : P;
  const int pad = ks / 2, stride = mode == CM_S2 ? 2 : 1;
  const int Hv = mode == CM_UP2 ? Ho : Hi, Wv = mode == CM_UP2 ? Wo : Wi;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < nW + Co; e += gridDim.y * blockDim.x) {
    T acc = 0;
    if (e < nW) {
      const int ci = e % Ci, t = e / Ci;
      const int kx = t % ks, ky = (t / ks) % ks, co = t / (ks * ks);
      for (size_t p = p0; p < p1; ++p) {
        const int oy = (int)(p / Wo), ox = (int)(p % Wo);
        const T g = gout[p * Co + co];
        if (g == (T)0) continue;
        acc = fma(g, view_at(in, Hi, Wi, Ci, Hv, Wv, mode, oy * stride + ky - pad, ox * stride + kx - pad, ci), acc);
      }
      atomic_add(gw + e, acc);
    } else {
      const int co = e - nW;
      for (size_t p = p0; p < p1; ++p) acc += gout[p * Co + co];
      atomic_add(gb + co, acc);
    }
  }
}

template <typename T>
__global__ void latent_bwd(const T* __restrict__ gz, const T* __restrict__ eps, const T* __restrict__ lv,
                           const T* __restrict__ gmu_ext, const T* __restrict__ glv_ext, size_t n, T* __restrict__ gmu,
                           T* __restrict__ glv) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  gmu[i] = gz[i] + (gmu_ext ? gmu_ext[i] : (T)0);
  glv[i] = (eps ? gz[i] * eps[i] * (T)0.5 * exp((T)0.5 * lv[i]) : (T)0) + (glv_ext ? glv_ext[i] : (T)0);
}

// Transpose of U = 4 * bilinear(coarse): each coarse pixel gathers the full-resolution
// gradients whose bilinear support includes it.  g = gU (+ gx0_ch1 / 256).
template <typename T>
__device__ __forceinline__ void up4_coeff(int X, int w, int& x0, int& x1, T& f) {
  T s = (T)X * (T)0.25 - (T)0.375;
  s = s < (T)0 ? (T)0 : (s > (T)(w - 1) ? (T)(w - 1) : s);
  x0 = (int)s;
  x1 = x0 + 1 < w ? x0 + 1 : w - 1;
  f = s - (T)x0;
}

template <typename T>
__global__ void up4_bwd(const T* __restrict__ gU, const T* __restrict__ gx0, int W, int H, int w, int h,
                        T* __restrict__ gc) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= w * h) return;
  const int x = idx % w, y = idx / w;
  // full-resolution columns / rows whose interpolation touches coarse column x / row y
  const int X0 = max(0, 4 * x - 4), X1 = min(W - 1, 4 * x + 5);
  const int Y0 = max(0, 4 * y - 4), Y1 = min(H - 1, 4 * y + 5);
  const int Xe = x == w - 1 ? W - 1 : X1, Ye = y == h - 1 ? H - 1 : Y1;
  const int Xs = x == 0 ? 0 : X0, Ys = y == 0 ? 0 : Y0;
  T acc = 0;
  for (int Y = Ys; Y <= Ye; ++Y) {
    int y0, y1;
    T fy;
    up4_coeff<T>(Y, h, y0, y1, fy);
    T wy = (y0 == y ? (T)1 - fy : (T)0) + (y1 == y ? fy : (T)0);
    if (wy == (T)0) continue;
    for (int X = Xs; X <= Xe; ++X) {
      int x0, x1;
      T fx;
      up4_coeff<T>(X, w, x0, x1, fx);
      T wx = (x0 == x ? (T)1 - fx : (T)0) + (x1 == x ? fx : (T)0);
      if (wx == (T)0) continue;
      const size_t p = (size_t)Y * W + X;
      T g = gU[p] + (gx0 ? gx0[p * 2 + 1] * (T)(1.0 / 256.0) : (T)0);
      acc += (T)4 * wy * wx * g;
    }
  }
  gc[idx] = acc;
}

template <typename T>
__global__ void add_inplace(T* a, const T* b, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] += b[i];
}

// x0 = (L / 256, U / 256) materialised for the enc1 weight gradient.
template <typename T>
__global__ void build_x0(const uint8_t* L, int pitch, int W, int H, const T* coarse, int w, int h, T* x0) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (size_t)W * H) return;
  const int X = (int)(p % W), Y = (int)(p / W);
  int x0i, x1i, y0i, y1i;
  T fx, fy;
  up4_coeff<T>(X, w, x0i, x1i, fx);
  up4_coeff<T>(Y, h, y0i, y1i, fy);
  const T top = ((T)1 - fx) * coarse[(size_t)y0i * w + x0i] + fx * coarse[(size_t)y0i * w + x1i];
  const T bot = ((T)1 - fx) * coarse[(size_t)y1i * w + x0i] + fx * coarse[(size_t)y1i * w + x1i];
  x0[2 * p] = (T)L[(size_t)Y * pitch + X] * (T)(1.0 / 256.0);
  x0[2 * p + 1] = (T)4 * (((T)1 - fy) * top + fy * bot) * (T)(1.0 / 256.0);
}

// Loss: every block writes its partial sum to its own slot (no atomics), loss_finish adds
// the slots in a fixed order, so the loss is bitwise reproducible.  Slot layout: for pair
// i, kLossBlocks smooth-L1 partials then kLossBlocks KL partials.
constexpr int kLossBlocks = 128;

template <typename T>
__global__ void loss_rec(const T* __restrict__ Y, const float* __restrict__ gt, size_t P, double inv_npix,
                         T* __restrict__ gY, double* __restrict__ slots) {
  __shared__ double red[256];
  double s = 0;
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
    const T e = Y[p] - (T)gt[p];
    const T a = e < (T)0 ? -e : e;
    s += a < (T)1 ? (double)((T)0.5 * e * e) : (double)(a - (T)0.5);
    if (gY) gY[p] = (a < (T)1 ? e : (e > (T)0 ? (T)1 : (T)-1)) * (T)inv_npix;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) slots[blockIdx.x] = red[0];
}

template <typename T>
__global__ void loss_kl(const T* __restrict__ mu, const T* __restrict__ lv, size_t n, double kl_scale,
                        T* __restrict__ gmu, T* __restrict__ glv, double* __restrict__ slots) {
  __shared__ double red[256];
  double s = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T m = mu[i], l = lv[i];
    const T el = exp(l);
    s += (double)((T)0.5 * (m * m + el - (T)1 - l));
    if (gmu) gmu[i] = (T)kl_scale * m;
    if (glv) glv[i] = (T)kl_scale * (T)0.5 * (el - (T)1);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) slots[kLossBlocks + blockIdx.x] = red[0];
}

template <typename T>
__global__ void loss_finish(const double* slots, int n_pairs, double inv_npix, double inv_nlat, double kl_w, T* out) {
  double rec = 0, kl = 0;
  for (int i = 0; i < n_pairs; ++i)
    for (int b = 0; b < kLossBlocks; ++b) {
      rec += slots[(size_t)i * 2 * kLossBlocks + b];
      kl += slots[(size_t)i * 2 * kLossBlocks + kLossBlocks + b];
    }
  rec *= inv_npix;
  kl *= inv_nlat;
  out[0] = (T)(rec + kl_w * kl);
  out[1] = (T)rec;
  out[2] = (T)kl;
}

template <typename T>
__global__ void adam_kernel(float* __restrict__ p, T* __restrict__ m, T* __restrict__ v, const T* __restrict__ g,
                            size_t n, T lr, T b1, T b2, T eps, T c1, T c2) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T gi = g[i];
  const T mi = b1 * m[i] + ((T)1 - b1) * gi;
  const T vi = b2 * v[i] + ((T)1 - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] = (float)((T)p[i] - lr * (mi / c1) / (sqrt(vi / c2) + eps));
}

inline unsigned blocks(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <typename T>
cudaError_t launch_dgrad(const T* gout, int Ho, int Wo, int Co, const T* w, int ks, int mode, const T* mask_act,
                         int Hi, int Wi, int Ci, int accumulate, T* gin, cudaStream_t st) {
  const size_t n = (size_t)Hi * Wi * Ci;
  dgrad_kernel<T><<<blocks(n), 256, 0, st>>>(gout, Ho, Wo, Co, w, ks, mode, mask_act, Hi, Wi, Ci, accumulate, gin);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_wgrad(const T* gout, int Ho, int Wo, int Co, const T* in, int Hi, int Wi, int Ci, int ks, int mode,
                         T* gw, T* gb, cudaStream_t st) {
  const int chunk = 256;
  const size_t P = (size_t)Ho * Wo;
  const int nW = Co * ks * ks * Ci + Co;
  dim3 grid((unsigned)((P + chunk - 1) / chunk), (unsigned)std::min(4, (nW + 255) / 256));
  wgrad_kernel<T><<<grid, 256, 0, st>>>(gout, Ho, Wo, Co, in, Hi, Wi, Ci, ks, mode, chunk, gw, gb);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_latent_bwd(const T* gz, const T* eps, const T* lv, const T* gmu_ext, const T* glv_ext, size_t n,
                              T* gmu, T* glv, cudaStream_t st) {
  latent_bwd<T><<<blocks(n), 256, 0, st>>>(gz, eps, lv, gmu_ext, glv_ext, n, gmu, glv);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_up4_bwd(const T* gU, const T* gx0, int W, int H, int w, int h, T* gc, cudaStream_t st) {
  up4_bwd<T><<<blocks((size_t)w * h), 256, 0, st>>>(gU, gx0, W, H, w, h, gc);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_build_x0(const uint8_t* L, int pitch, int W, int H, const T* coarse, int w, int h, T* x0,
                            cudaStream_t st) {
  build_x0<T><<<blocks((size_t)W * H), 256, 0, st>>>(L, pitch, W, H, coarse, w, h, x0);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add(T* a, const T* b, size_t n, cudaStream_t st) {
  add_inplace<T><<<blocks(n), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

size_t loss_slots_per_pair() { return 2 * kLossBlocks; }

template <typename T>
cudaError_t launch_loss_rec(const T* Y, const float* gt, size_t P, double inv_npix, T* gY, double* slots,
                            cudaStream_t st) {
  loss_rec<T><<<kLossBlocks, 256, 0, st>>>(Y, gt, P, inv_npix, gY, slots);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_loss_kl(const T* mu, const T* lv, size_t n, double kl_scale, T* gmu, T* glv, double* slots,
                           cudaStream_t st) {
  loss_kl<T><<<kLossBlocks, 256, 0, st>>>(mu, lv, n, kl_scale, gmu, glv, slots);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_loss_finish(const double* slots, int n_pairs, double inv_npix, double inv_nlat, double kl_w, T* out,
                               cudaStream_t st) {
  loss_finish<T><<<1, 1, 0, st>>>(slots, n_pairs, inv_npix, inv_nlat, kl_w, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_adam(float* p, T* m, T* v, const T* g, size_t n, double lr, double b1, double b2, double eps,
                        int t, cudaStream_t st) {
  const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  adam_kernel<T><<<blocks(n), 256, 0, st>>>(p, m, v, g, n, (T)lr, (T)b1, (T)b2, (T)eps, (T)c1, (T)c2);
  return cudaGetLastError();
}

#define SV_BWD_INST(T)                                                                                              \
  template cudaError_t launch_dgrad<T>(const T*, int, int, int, const T*, int, int, const T*, int, int, int, int, T*, \
                                       cudaStream_t);                                                                \
  template cudaError_t launch_wgrad<T>(const T*, int, int, int, const T*, int, int, int, int, int, T*, T*,           \
                                       cudaStream_t);                                                                \
  template cudaError_t launch_latent_bwd<T>(const T*, const T*, const T*, const T*, const T*, size_t, T*, T*,       \
                                            cudaStream_t);                                                           \
  template cudaError_t launch_up4_bwd<T>(const T*, const T*, int, int, int, int, T*, cudaStream_t);                 \
  template cudaError_t launch_build_x0<T>(const uint8_t*, int, int, int, const T*, int, int, T*, cudaStream_t);     \
  template cudaError_t launch_add<T>(T*, const T*, size_t, cudaStream_t);                                           \
  template cudaError_t launch_loss_rec<T>(const T*, const float*, size_t, double, T*, double*, cudaStream_t);        \
  template cudaError_t launch_loss_kl<T>(const T*, const T*, size_t, double, T*, T*, double*, cudaStream_t);        \
  template cudaError_t launch_loss_finish<T>(const double*, int, double, double, double, T*, cudaStream_t);         \
  template cudaError_t launch_adam<T>(float*, T*, T*, const T*, size_t, double, double, double, double, int,        \
                                      cudaStream_t);
SV_BWD_INST(float)
SV_BWD_INST(double)

}  // namespace sv
