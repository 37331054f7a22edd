// sv_api.cu -- the C ABI declared in include/stereovae.h: context, argument
// validation, workspaces and the order of launches of each entry point.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "sv_internal.cuh"
#include "sv_ctx.cuh"

namespace sv {

int NetDims::cout(int l) const {
  switch (l) {
    case L_ENC1: case L_ENC2: case L_ENC3: return enc[l - L_ENC1];
    case L_MU: case L_LV: return lat;
    case L_DEC1: case L_DEC2: case L_DEC3: return dec[l - L_DEC1];
    default: return 1;
  }
}
int NetDims::cin(int l) const {
  switch (l) {
    case L_ENC1: return 2;
    case L_ENC2: return enc[0];
    case L_ENC3: return enc[1];
    case L_MU: case L_LV: return enc[2];
    case L_DEC1: return lat;
    case L_DEC2: return dec[0];
    case L_DEC3: return dec[1];
    default: return dec[2];
  }
}
int NetDims::ks(int l) const { return (l == L_MU || l == L_LV) ? 1 : 3; }
size_t NetDims::w_off(int l) const {
  size_t o = 0;
  for (int i = 0; i < l; ++i) o += (size_t)cout(i) * ks(i) * ks(i) * cin(i) + cout(i);
  return o;
}
size_t NetDims::b_off(int l) const { return w_off(l) + (size_t)cout(l) * ks(l) * ks(l) * cin(l); }
size_t NetDims::count() const { return w_off(L_COUNT); }

cudaError_t DevBuf::ensure(size_t bytes) {
  if (n >= bytes) return cudaSuccess;
  if (p) cudaFree(p);
  p = nullptr;
  n = 0;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e == cudaSuccess) n = bytes;
  return e;
}
void DevBuf::release() {
  if (p) cudaFree(p);
  p = nullptr;
  n = 0;
}

namespace {

__global__ void f32_to_f64(const float* a, double* b, size_t n) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

}  // namespace

sv_status Ctx::fail(sv_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  err = buf;
  return s;
}

sv_status Ctx::cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return SV_OK;
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return fail(SV_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  }
  return fail(SV_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

sv_status Ctx::check_pairs(const sv_pair* pairs, int n_pairs) {
  if (n_pairs < 0) return fail(SV_ERR_INVALID_ARG, "n_pairs < 0");
  if (n_pairs > 0 && !pairs) return fail(SV_ERR_INVALID_ARG, "pairs is NULL");
  const int k = cfg.window;
  for (int i = 0; i < n_pairs; ++i) {
    const sv_pair& p = pairs[i];
    if (!p.left || !p.right) return fail(SV_ERR_INVALID_ARG, "pair %d: NULL image", i);
    if (((uintptr_t)p.left & 15) || ((uintptr_t)p.right & 15))
      return fail(SV_ERR_INVALID_ARG, "pair %d: image not 16-byte aligned", i);
    if (p.pitch % 16 || p.pitch < p.width) return fail(SV_ERR_INVALID_ARG, "pair %d: pitch %d invalid", i, p.pitch);
    if (p.width < 4 * k || p.height < 4 * k)
      return fail(SV_ERR_INVALID_ARG, "pair %d: %dx%d smaller than 4 * window", i, p.width, p.height);
    if (p.width > kMaxSide || p.height > kMaxSide)
      return fail(SV_ERR_UNSUPPORTED, "pair %d: side above %d", i, kMaxSide);
    if (p.max_disp < 1 || p.max_disp > kMaxDisp || p.max_disp > p.width / 4)
      return fail(SV_ERR_INVALID_ARG, "pair %d: max_disp %d outside [1, min(%d, W/4)]", i, p.max_disp, kMaxDisp);
  }
  return SV_OK;
}

// ---------------------------------------------------------------- coarse matching
void Ctx::coarse_prepare(const sv_pair* pairs, int n, int16_t* const* disp, float* const* best, float* const* second,
                         ZRun& z) {
  z.pairs.assign(n, ZPair{});
  z.jobs.clear();
  z.maxD = 1;
  for (int i = 0; i < n; ++i) z.maxD = std::max(z.maxD, pairs[i].max_disp);
  const int gx = kZnccWarps * zncc_tx(zncc_kd(z.maxD));
  for (int i = 0; i < n; ++i) {
    const sv_pair& p = pairs[i];
    ZPair& q = z.pairs[i];
    q.L = p.left; q.R = p.right; q.W = p.width; q.H = p.height; q.pitch = p.pitch; q.D = p.max_disp;
    q.w = p.width / 4; q.h = p.height / 4;
    q.disp = disp[i];
    q.best = best ? best[i] : nullptr;
    q.second = second ? second[i] : nullptr;
    for (int y0 = 0; y0 < q.h; y0 += kZnccTY)
      for (int x0 = 0; x0 < q.w; x0 += gx) z.jobs.push_back({i, y0, x0, 0});
  }
}

sv_status Ctx::coarse_launch(const ZRun& z, const ZPair* d_pairs, const ZJob* d_jobs, cudaStream_t st) {
  if (z.jobs.empty()) return SV_OK;
  LaunchScope ls(*this, "zncc_wta", st);
  bool scores = false;
  for (const ZPair& q : z.pairs) scores |= q.best != nullptr || q.second != nullptr;
  return cuda(launch_zncc_wta(d_pairs, d_jobs, (int)z.jobs.size(), cfg.window / 2, z.maxD, st, scores ? 1 : 0),
              "zncc_wta launch");
}

sv_status Ctx::coarse(const sv_pair* pairs, int n, int16_t* const* disp, float* const* best, float* const* second,
                      cudaStream_t st) {
  ZRun z;
  coarse_prepare(pairs, n, disp, best, second, z);
  if (z.jobs.empty()) return SV_OK;
  sv_status s;
  if ((s = cuda(zpairs.ensure(sizeof(ZPair) * n), "alloc pair table"))) return s;
  if ((s = cuda(zjobs.ensure(sizeof(ZJob) * z.jobs.size()), "alloc job table"))) return s;
  if ((s = cuda(cudaMemcpyAsync(zpairs.p, z.pairs.data(), sizeof(ZPair) * n, cudaMemcpyHostToDevice, st),
                "upload pairs")))
    return s;
  if ((s = cuda(cudaMemcpyAsync(zjobs.p, z.jobs.data(), sizeof(ZJob) * z.jobs.size(), cudaMemcpyHostToDevice, st),
                "upload jobs")))
    return s;
  return coarse_launch(z, (const ZPair*)zpairs.p, (const ZJob*)zjobs.p, st);
}

// ---------------------------------------------------------------- plain refinement
template <typename T>
sv_status Ctx::refine_direct(const sv_pair& p, const void* coarse_map, bool coarse_int16, const T* eps, T* Y, T* mu_out,
                             T* lv_out, T* const* saved, cudaStream_t st) {
  const Levels lv(p.height, p.width);
  const int w = p.width / 4, h = p.height / 4;
  const T* Wt = weights<T>();
  auto Wl = [&](int l) { return Wt + net.w_off(l); };
  auto Bl = [&](int l) { return Wt + net.b_off(l); };
  sv_status s;
  // workspaces: e1 e2 e3 z d1 d2 d3 (or the caller's saved buffers)
  const size_t P0 = (size_t)lv.H[0] * lv.W[0], P1 = (size_t)lv.H[1] * lv.W[1], P2 = (size_t)lv.H[2] * lv.W[2],
               P3 = (size_t)lv.H[3] * lv.W[3];
  const size_t need[7] = {P1 * net.enc[0], P2 * net.enc[1], P3 * net.enc[2], P3 * net.lat,
                          P2 * net.dec[0], P1 * net.dec[1], P0 * net.dec[2]};
  T* buf[7];
  for (int i = 0; i < 7; ++i) {
    if (saved && saved[i]) {
      buf[i] = saved[i];
      continue;
    }
    if ((s = cuda(act[i].ensure(need[i] * sizeof(T)), "alloc activations"))) return s;
    buf[i] = (T*)act[i].p;
  }
  T *e1 = buf[0], *e2 = buf[1], *e3 = buf[2], *z = buf[3], *d1 = buf[4], *d2 = buf[5], *d3 = buf[6];
  cudaError_t e;
#define SV_SCOPE(n) LaunchScope _ls_##n(*this, #n, st)
  {
  SV_SCOPE(enc1);
  if (coarse_int16)
    e = launch_enc1<T, int16_t>(p.left, p.pitch, p.width, p.height, (const int16_t*)coarse_map, w, h, Wl(L_ENC1),
                                Bl(L_ENC1), net.enc[0], e1, st);
  else
    e = launch_enc1<T, T>(p.left, p.pitch, p.width, p.height, (const T*)coarse_map, w, h, Wl(L_ENC1), Bl(L_ENC1),
                          net.enc[0], e1, st);
  }
  if ((s = cuda(e, "enc1"))) return s;
  DirectConvArgs<T> a{e1, lv.H[1], lv.W[1], net.enc[0], Wl(L_ENC2), Bl(L_ENC2), net.enc[1], lv.H[2], lv.W[2], 1, e2};
  { SV_SCOPE(enc2); s = cuda(launch_conv_direct<T>(a, CM_S2, 3, st), "enc2"); }
  if (s) return s;
  a = {e2, lv.H[2], lv.W[2], net.enc[1], Wl(L_ENC3), Bl(L_ENC3), net.enc[2], lv.H[3], lv.W[3], 1, e3};
  { SV_SCOPE(enc3); s = cuda(launch_conv_direct<T>(a, CM_S2, 3, st), "enc3"); }
  if (s) return s;
  const bool train = eps != nullptr || lv_out != nullptr;
  { SV_SCOPE(latent); s = cuda(launch_latent<T>(e3, lv.H[3], lv.W[3], net.enc[2], Wl(L_MU), Bl(L_MU), Wl(L_LV), Bl(L_LV), net.lat, eps, mu_out,
                                 train ? lv_out : nullptr, z, st),
                "latent"); }
  if (s) return s;
  a = {z, lv.H[3], lv.W[3], net.lat, Wl(L_DEC1), Bl(L_DEC1), net.dec[0], lv.H[2], lv.W[2], 1, d1};
  { SV_SCOPE(dec1); s = cuda(launch_conv_direct<T>(a, CM_UP2, 3, st), "dec1"); }
  if (s) return s;
  a = {d1, lv.H[2], lv.W[2], net.dec[0], Wl(L_DEC2), Bl(L_DEC2), net.dec[1], lv.H[1], lv.W[1], 1, d2};
  { SV_SCOPE(dec2); s = cuda(launch_conv_direct<T>(a, CM_UP2, 3, st), "dec2"); }
  if (s) return s;
  a = {d2, lv.H[1], lv.W[1], net.dec[1], Wl(L_DEC3), Bl(L_DEC3), net.dec[2], lv.H[0], lv.W[0], 1, d3};
  { SV_SCOPE(dec3); s = cuda(launch_conv_direct<T>(a, CM_UP2, 3, st), "dec3"); }
  if (s) return s;
  SV_SCOPE(final);
  if (coarse_int16)
    e = launch_final<T, int16_t, T>(d3, p.width, p.height, net.dec[2], Wl(L_FINAL), Bl(L_FINAL),
                                    (const int16_t*)coarse_map, w, h, Y, st);
  else
    e = launch_final<T, T, T>(d3, p.width, p.height, net.dec[2], Wl(L_FINAL), Bl(L_FINAL), (const T*)coarse_map, w, h,
                              Y, st);
  return cuda(e, "final");
#undef SV_SCOPE
}

template <> const float* Ctx::weights<float>() const { return (const float*)w32.p; }
template <> const double* Ctx::weights<double>() const { return (const double*)w64.p; }

template sv_status Ctx::refine_direct<float>(const sv_pair&, const void*, bool, const float*, float*, float*, float*,
                                             float* const*, cudaStream_t);
template sv_status Ctx::refine_direct<double>(const sv_pair&, const void*, bool, const double*, double*, double*,
                                              double*, double* const*, cudaStream_t);

sv_status Ctx::refresh_weight_copies_async(cudaStream_t st) {
  if (t1) return SV_OK;  // the Table I network runs on the FP32 master copy
  sv_status s;
  const size_t n = net.count();
  if ((s = cuda(w64.ensure(n * sizeof(double)), "alloc fp64 weights"))) return s;
  {
    LaunchScope ls(*this, "weights_f64", st);
    f32_to_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float*)w32.p, (double*)w64.p, n);
    if ((s = cuda(cudaGetLastError(), "weights to fp64"))) return s;
  }
  // (the FP8 form also runs its last decoder layer from the BF16 packs)
  if (cfg.precision == SV_BF16 || cfg.precision == SV_FP8)
    if ((s = pack_bf16_weights(st))) return s;
  if (cfg.precision == SV_FP8)
    if ((s = pack_fp8_weights(st))) return s;
  return SV_OK;
}

sv_status Ctx::refresh_weight_copies() {
  sv_status s = refresh_weight_copies_async(0);
  if (s) return s;
  return cuda(cudaDeviceSynchronize(), "weight refresh");
}

}  // namespace sv

using sv::Ctx;

using DeviceGuard = sv::DeviceGuardInt;

extern "C" {

const char* sv_status_string(sv_status s) {
  switch (s) {
    case SV_OK: return "SV_OK";
    case SV_ERR_INVALID_ARG: return "SV_ERR_INVALID_ARG";
    case SV_ERR_CUDA: return "SV_ERR_CUDA";
    case SV_ERR_OOM: return "SV_ERR_OOM";
    case SV_ERR_UNSUPPORTED: return "SV_ERR_UNSUPPORTED";
    case SV_ERR_TIMEOUT: return "SV_ERR_TIMEOUT";
    case SV_ERR_STATE: return "SV_ERR_STATE";
  }
  return "SV_ERR_UNKNOWN";
}

const char* sv_last_error(const sv_ctx* ctx) {
  if (!ctx) return "NULL context";
  return reinterpret_cast<const Ctx*>(ctx)->err.c_str();
}

static bool config_ok(const sv_config* c) {
  if (!c) return false;
  if (c->window < 3 || c->window > 15 || c->window % 2 == 0) return false;
  if (c->flags == SV_NET_TABLE1) return c->precision == SV_FP32;  // widths fixed by Table I
  for (int i = 0; i < 3; ++i)
    if (!sv::valid_width_pub(c->enc_ch[i]) || !sv::valid_width_pub(c->dec_ch[i])) return false;
  if (!sv::valid_width_pub(c->latent_ch)) return false;
  if (c->precision < SV_FP32 || c->precision > SV_FP8) return false;
  if (c->precision == SV_FP8) {
    // E4M3 operands: a quantised layer's input width is a whole number of 32-element K steps
    const int in_w[5] = {c->enc_ch[0], c->enc_ch[1], c->enc_ch[2], c->latent_ch, c->dec_ch[0]};
    for (int w : in_w)
      if (w % 32) return false;
  }
  if (c->flags != 0) return false;
  return true;
}

size_t sv_param_count(const sv_config* c) {
  if (!config_ok(c)) return 0;
  if (c->flags == SV_NET_TABLE1) return sv::t1_param_count();
  sv::NetDims n{{c->enc_ch[0], c->enc_ch[1], c->enc_ch[2]}, c->latent_ch, {c->dec_ch[0], c->dec_ch[1], c->dec_ch[2]}};
  return n.count();
}

sv_status sv_create(const sv_config* cfg, int device, sv_ctx** out) {
  if (!out) return SV_ERR_INVALID_ARG;
  *out = nullptr;
  if (!config_ok(cfg)) return SV_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return SV_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return SV_ERR_INVALID_ARG;
  DeviceGuard g(device);
  Ctx* c = new Ctx();
  c->cfg = *cfg;
  c->device = device;
  c->t1 = cfg->flags == SV_NET_TABLE1;
  if (!c->t1)
    c->net = sv::NetDims{{cfg->enc_ch[0], cfg->enc_ch[1], cfg->enc_ch[2]}, cfg->latent_ch,
                         {cfg->dec_ch[0], cfg->dec_ch[1], cfg->dec_ch[2]}};
  const size_t n = c->n_params();
  sv_status s = c->cuda(c->err_flag.ensure(sizeof(int)), "alloc error flag");
  if (!s) s = c->cuda(cudaMemset(c->err_flag.p, 0, sizeof(int)), "zero error flag");
  if (!s) s = c->cuda(c->w32.ensure(n * sizeof(float)), "alloc weights");
  if (!s) s = c->cuda(cudaMemset(c->w32.p, 0, n * sizeof(float)), "zero weights");
  if (!s) s = c->refresh_weight_copies();
  if (s) {
    delete c;
    return s;
  }
  *out = reinterpret_cast<sv_ctx*>(c);
  return SV_OK;
}

sv_status sv_destroy(sv_ctx* ctx) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  {
    DeviceGuard g(c->device);
    cudaDeviceSynchronize();
    c->release_all();
  }
  delete c;
  return SV_OK;
}

sv_status sv_set_weights(sv_ctx* ctx, const float* params, size_t n) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!params) return c->fail(SV_ERR_INVALID_ARG, "params is NULL");
  if (n != c->n_params()) return c->fail(SV_ERR_INVALID_ARG, "expected %zu parameters, got %zu", c->n_params(), n);
  DeviceGuard g(c->device);
  sv_status s = c->cuda(cudaMemcpy(c->w32.p, params, n * sizeof(float), cudaMemcpyDefault), "copy weights");
  if (s) return s;
  c->adam_t = 0;
  return c->refresh_weight_copies();
}

sv_status sv_get_weights(sv_ctx* ctx, float* params, size_t n) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!params) return c->fail(SV_ERR_INVALID_ARG, "params is NULL");
  if (n != c->n_params()) return c->fail(SV_ERR_INVALID_ARG, "expected %zu parameters, got %zu", c->n_params(), n);
  DeviceGuard g(c->device);
  return c->cuda(cudaMemcpy(params, c->w32.p, n * sizeof(float), cudaMemcpyDefault), "copy weights out");
}

sv_status sv_coarse_match(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, int16_t* const* disp_out,
                          float* const* best, float* const* second, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  c->err.clear();
  sv_status s = c->check_pairs(pairs, n_pairs);
  if (s) return s;
  if (n_pairs == 0) return SV_OK;
  if (!disp_out) return c->fail(SV_ERR_INVALID_ARG, "disp_out is NULL");
  for (int i = 0; i < n_pairs; ++i)
    if (!disp_out[i]) return c->fail(SV_ERR_INVALID_ARG, "disp_out[%d] is NULL", i);
  DeviceGuard g(c->device);
  return c->coarse(pairs, n_pairs, disp_out, best, second, (cudaStream_t)stream);
}

sv_status sv_refine(sv_ctx* ctx, const sv_pair* pairs, const int16_t* const* coarse, int n_pairs,
                    float* const* disp_out, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  c->err.clear();
  sv_status s = c->check_pairs(pairs, n_pairs);
  if (s) return s;
  if (n_pairs == 0) return SV_OK;
  if (!coarse || !disp_out) return c->fail(SV_ERR_INVALID_ARG, "coarse / disp_out is NULL");
  for (int i = 0; i < n_pairs; ++i)
    if (!coarse[i] || !disp_out[i]) return c->fail(SV_ERR_INVALID_ARG, "coarse[%d] / disp_out[%d] is NULL", i, i);
  DeviceGuard g(c->device);
  return c->refine_infer(pairs, coarse, n_pairs, disp_out, (cudaStream_t)stream);
}

sv_status sv_pipeline(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, float* const* disp_out, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  c->err.clear();
  sv_status s = c->check_pairs(pairs, n_pairs);
  if (s) return s;
  if (n_pairs == 0) return SV_OK;
  if (!disp_out) return c->fail(SV_ERR_INVALID_ARG, "disp_out is NULL");
  for (int i = 0; i < n_pairs; ++i)
    if (!disp_out[i]) return c->fail(SV_ERR_INVALID_ARG, "disp_out[%d] is NULL", i);
  DeviceGuard g(c->device);
  return c->pipeline(pairs, n_pairs, disp_out, (cudaStream_t)stream);
}

sv_status sv_pipeline_host(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, float* const* disp_out,
                           sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  c->err.clear();
  if (n_pairs < 0 || (n_pairs > 0 && (!pairs || !disp_out))) return c->fail(SV_ERR_INVALID_ARG, "bad arguments");
  if (n_pairs == 0) return SV_OK;
  std::vector<sv_pair> dev(n_pairs);
  std::vector<size_t> img_off(n_pairs + 1, 0), out_off(n_pairs + 1, 0);
  for (int i = 0; i < n_pairs; ++i) {
    const sv_pair& p = pairs[i];
    if (!p.left || !p.right || !disp_out[i] || p.pitch < p.width || p.width <= 0 || p.height <= 0)
      return c->fail(SV_ERR_INVALID_ARG, "pair %d: bad host buffers", i);
    const int dpitch = (p.width + 15) / 16 * 16;
    img_off[i + 1] = img_off[i] + 2 * (size_t)dpitch * p.height;
    out_off[i + 1] = out_off[i] + (size_t)p.width * p.height;
  }
  DeviceGuard g(c->device);
  cudaStream_t st = (cudaStream_t)stream;
  sv_status s = c->cuda(c->host_img.ensure(img_off[n_pairs]), "alloc image staging");
  if (!s) s = c->cuda(c->host_out.ensure(out_off[n_pairs] * sizeof(float)), "alloc output staging");
  if (s) return s;
  // Device-accessible views of the host buffers (pinned or mapped host memory, reached
  // through the unified address space): with all of them, one kernel gathers every image
  // and one scatters every result; otherwise (pageable memory) one copy call per buffer.
  auto dev_view = [](const void* ptr) -> void* {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
  };
  bool direct = c->host_copy > 0;
  const bool scatter = c->host_copy > 1;
  std::vector<sv::HostRowCopy> jobs(3 * (size_t)n_pairs);
  std::vector<float*> dout(n_pairs);
  int max_rows = 0;
  for (int i = 0; i < n_pairs; ++i) {
    const sv_pair& p = pairs[i];
    const int dpitch = (p.width + 15) / 16 * 16;
    uint8_t* L = (uint8_t*)c->host_img.p + img_off[i];
    uint8_t* R = L + (size_t)dpitch * p.height;
    dev[i] = p;
    dev[i].left = L;
    dev[i].right = R;
    dev[i].pitch = dpitch;
    dout[i] = (float*)c->host_out.p + out_off[i];
    max_rows = std::max(max_rows, p.height);
    if (direct) {
      void* lv = dev_view(p.left);
      void* rv = dev_view(p.right);
      void* ov = scatter ? dev_view(disp_out[i]) : (void*)1;
      if (!lv || !rv || !ov) {
        direct = false;
      } else {
        jobs[2 * i] = {(const unsigned char*)lv, L, p.pitch, dpitch, p.width, p.height};
        jobs[2 * i + 1] = {(const unsigned char*)rv, R, p.pitch, dpitch, p.width, p.height};
        const int ob = (int)sizeof(float) * p.width;
        jobs[2 * (size_t)n_pairs + i] = {(const unsigned char*)dout[i], (unsigned char*)ov, ob, ob, ob, p.height};
      }
    }
  }
  if ((s = c->check_pairs(dev.data(), n_pairs))) return s;
  if (direct && !scatter) {
    // the batch in parts of at least 8 pairs: each part's images are gathered on the input
    // stream ahead of its compute (the next part's arrive while the current one computes),
    // and its results go back on the copy stream while the next part computes
    const size_t jb = sizeof(sv::HostRowCopy) * jobs.size();
    if ((s = c->cuda(c->host_jobs.ensure(jb), "alloc copy jobs"))) return s;
    const int nch = std::max(1, std::min(c->host_chunks, n_pairs / 8));
    if (!c->copy_stream && (s = c->cuda(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking), "stream")))
      return s;
    if (!c->in_stream && (s = c->cuda(cudaStreamCreateWithFlags(&c->in_stream, cudaStreamNonBlocking), "stream")))
      return s;
    for (auto* e : {&c->chunk_done[0], &c->chunk_done[1], &c->chunk_done[2], &c->chunk_done[3], &c->gather_done[0],
                    &c->gather_done[1], &c->gather_done[2], &c->gather_done[3], &c->call_start})
      if (!*e && (s = c->cuda(cudaEventCreateWithFlags(e, cudaEventDisableTiming), "event"))) return s;
    // the input stream starts after the work already queued on the caller's stream
    if ((s = c->cuda(cudaEventRecord(c->call_start, st), "record"))) return s;
    if ((s = c->cuda(cudaStreamWaitEvent(c->in_stream, c->call_start, 0), "wait"))) return s;
    if ((s = c->cuda(cudaMemcpyAsync(c->host_jobs.p, jobs.data(), jb, cudaMemcpyHostToDevice, c->in_stream),
                     "copy jobs")))
      return s;
    const sv::HostRowCopy* dj = (const sv::HostRowCopy*)c->host_jobs.p;
    // part sizes in the ratio 1 : 2 : ... : 2 : 1 (two parts: 1 : 1): the first part's gather
    // and the last part's copy-back are the only transfers nothing overlaps, so those parts
    // are the small ones
    std::vector<int> first(nch + 1, 0);
    const int units = nch <= 2 ? nch : 2 * nch - 2;
    for (int ch = 0, u = 0; ch < nch; ++ch) {
      u += nch <= 2 || ch == 0 || ch == nch - 1 ? 1 : 2;
      first[ch + 1] = ch + 1 == nch ? n_pairs : (int)((long long)n_pairs * u / units);
    }
    for (int ch = 0; ch < nch && !s; ++ch) {
      int rows = 0;
      for (int i = first[ch]; i < first[ch + 1]; ++i) rows = std::max(rows, pairs[i].height);
      s = c->cuda(sv::launch_copy_rows(dj + 2 * first[ch], 2 * (first[ch + 1] - first[ch]), rows, 1, c->in_stream),
                  "gather images");
      if (!s) s = c->cuda(cudaEventRecord(c->gather_done[ch], c->in_stream), "record");
    }
    for (int ch = 0; ch < nch && !s; ++ch) {
      const int start = first[ch], cnt = first[ch + 1] - first[ch];
      if ((s = c->cuda(cudaStreamWaitEvent(st, c->gather_done[ch], 0), "wait"))) break;
      if ((s = c->pipeline(dev.data() + start, cnt, dout.data() + start, st))) break;
      if ((s = c->cuda(cudaEventRecord(c->chunk_done[ch], st), "record"))) break;
      if ((s = c->cuda(cudaStreamWaitEvent(c->copy_stream, c->chunk_done[ch], 0), "wait"))) break;
      for (int i = start; i < start + cnt && !s; ++i)
        s = c->cuda(cudaMemcpyAsync(disp_out[i], dout[i], sizeof(float) * pairs[i].width * pairs[i].height,
                                    cudaMemcpyDeviceToHost, c->copy_stream), "D2H");
    }
    const sv_status s0 = c->cuda(cudaStreamSynchronize(c->in_stream), "synchronise gathers");
    const sv_status s1 = c->cuda(cudaStreamSynchronize(st), "synchronise");
    const sv_status s2 = c->cuda(cudaStreamSynchronize(c->copy_stream), "synchronise copies");
    return s ? s : s0 ? s0 : s1 ? s1 : s2;
  }
  if (direct) {  // gather and scatter kernels around one whole-batch pipeline
    const size_t jb = sizeof(sv::HostRowCopy) * jobs.size();
    if ((s = c->cuda(c->host_jobs.ensure(jb), "alloc copy jobs"))) return s;
    if ((s = c->cuda(cudaMemcpyAsync(c->host_jobs.p, jobs.data(), jb, cudaMemcpyHostToDevice, st), "copy jobs")))
      return s;
    const sv::HostRowCopy* dj = (const sv::HostRowCopy*)c->host_jobs.p;
    if ((s = c->cuda(sv::launch_copy_rows(dj, 2 * n_pairs, max_rows, 1, st), "gather images"))) return s;
    if ((s = c->pipeline(dev.data(), n_pairs, dout.data(), st))) return s;
    if ((s = c->cuda(sv::launch_copy_rows(dj + 2 * n_pairs, n_pairs, max_rows, 1, st), "scatter results"))) return s;
    return c->cuda(cudaStreamSynchronize(st), "synchronise");
  }
  for (int i = 0; i < n_pairs; ++i) {
    const sv_pair& p = pairs[i];
    s = c->cuda(cudaMemcpy2DAsync((void*)dev[i].left, dev[i].pitch, p.left, p.pitch, p.width, p.height,
                                  cudaMemcpyHostToDevice, st), "H2D");
    if (!s) s = c->cuda(cudaMemcpy2DAsync((void*)dev[i].right, dev[i].pitch, p.right, p.pitch, p.width, p.height,
                                          cudaMemcpyHostToDevice, st), "H2D");
    if (s) return s;
  }
  if ((s = c->pipeline(dev.data(), n_pairs, dout.data(), st))) return s;
  for (int i = 0; i < n_pairs; ++i)
    if ((s = c->cuda(cudaMemcpyAsync(disp_out[i], dout[i], sizeof(float) * pairs[i].width * pairs[i].height,
                                     cudaMemcpyDeviceToHost, st), "D2H")))
      return s;
  return c->cuda(cudaStreamSynchronize(st), "synchronise");
}

sv_status sv_profile_enable(sv_ctx* ctx, int enable) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  reinterpret_cast<Ctx*>(ctx)->prof_on = enable != 0;
  return SV_OK;
}

sv_status sv_profile_read(sv_ctx* ctx, sv_profile_entry* out, int max_entries, int* n_out, int reset) {
  if (!ctx || max_entries < 0 || (max_entries > 0 && !out)) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  DeviceGuard g(c->device);
  c->prof_flush();
  int i = 0;
  for (auto& kv : c->prof_tot) {
    if (i < max_entries) {
      memset(out[i].name, 0, sizeof(out[i].name));
      strncpy(out[i].name, kv.first.c_str(), sizeof(out[i].name) - 1);
      out[i].launches = kv.second.first;
      out[i].total_ms = kv.second.second;
    }
    ++i;
  }
  if (n_out) *n_out = (int)c->prof_tot.size();
  if (reset) c->prof_tot.clear();
  return SV_OK;
}

sv_status sv_synchronize(sv_ctx* ctx, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  DeviceGuard g(c->device);
  sv_status s = c->cuda(cudaStreamSynchronize((cudaStream_t)stream), "synchronise");
  if (s) return s;
  int code = 0;
  if ((s = c->cuda(cudaMemcpy(&code, c->err_flag.p, sizeof(int), cudaMemcpyDeviceToHost), "read error flag")))
    return s;
  if (code) {
    cudaMemset(c->err_flag.p, 0, sizeof(int));
    static const char* where[] = {"",           "producer",           "MMA issuer", "MMA drain",
                                  "epilogue",   "copy drain",         "final-conv staging", "enc1 MMA"};
    return c->fail(SV_ERR_TIMEOUT, "a device-side wait ran out (%s, code %d)", code >= 1 && code <= 7 ? where[code] : "?",
                   code);
  }
  return SV_OK;
}

sv_status sv_set_option(sv_ctx* ctx, const char* key, long long value) {
  if (!ctx || !key) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (!strcmp(key, "spin_limit")) {
    if (value < 1) return c->fail(SV_ERR_INVALID_ARG, "spin_limit must be >= 1");
    c->spin_limit = value;
    return SV_OK;
  }
  if (!strcmp(key, "graphs")) {
    if (value != 0 && value != 1) return c->fail(SV_ERR_INVALID_ARG, "graphs must be 0 or 1");
    c->use_graphs = value != 0;
    if (!c->use_graphs) c->drop_graphs();
    return SV_OK;
  }
  if (!strcmp(key, "host_chunks")) {
    if (value < 1 || value > 4) return c->fail(SV_ERR_INVALID_ARG, "host_chunks must be 1..4");
    c->host_chunks = (int)value;
    return SV_OK;
  }
  if (!strcmp(key, "host_copy")) {
    if (value < 0 || value > 2) return c->fail(SV_ERR_INVALID_ARG, "host_copy must be 0, 1 or 2");
    c->host_copy = (int)value;
    return SV_OK;
  }
  if (!strcmp(key, "fused_final")) {
    if (value != 0 && value != 1) return c->fail(SV_ERR_INVALID_ARG, "fused_final must be 0 or 1");
    c->fused_final = (int)value;
    c->drop_graphs();
    return SV_OK;
  }
  if (!strcmp(key, "split_rows")) {
    if (value != 0 && value != 1) return c->fail(SV_ERR_INVALID_ARG, "split_rows must be 0 or 1");
    c->split_rows = (int)value;
    c->drop_graphs();
    return SV_OK;
  }
  if (!strcmp(key, "enc1_tensor")) {
    if (value != 0 && value != 1) return c->fail(SV_ERR_INVALID_ARG, "enc1_tensor must be 0 or 1");
    c->enc1_tensor = (int)value;
    c->drop_graphs();
    return SV_OK;
  }
  if (!strcmp(key, "fused_prefetch")) {
    if (value < 0 || value > 16) return c->fail(SV_ERR_INVALID_ARG, "fused_prefetch must be 0..16");
    c->fused_prefetch = (int)value;
    c->drop_graphs();
    return SV_OK;
  }
  if (!strcmp(key, "fused_ring")) {
    if (value != 0 && (value < 4 || value > 16)) return c->fail(SV_ERR_INVALID_ARG, "fused_ring must be 0 or 4..16");
    c->fused_ring = (int)value;
    c->drop_graphs();
    return SV_OK;
  }
  if (!strcmp(key, "debug_plans")) {
    if (value != 0 && value != 1) return c->fail(SV_ERR_INVALID_ARG, "debug_plans must be 0 or 1");
    c->debug_plans = (int)value;
    return SV_OK;
  }
  if (!strcmp(key, "tc_ctas_per_sm")) {
    if (value < 0 || value > 4) return c->fail(SV_ERR_INVALID_ARG, "tc_ctas_per_sm must be 0..4");
    c->tc_ctas_per_sm = (int)value;
    c->drop_graphs();
    return SV_OK;
  }
  if (!strcmp(key, "tc_strip_rows")) {
    if (value < 0 || value > 4096) return c->fail(SV_ERR_INVALID_ARG, "tc_strip_rows out of range");
    c->tc_strip_rows = (int)value;
    return SV_OK;
  }
  return c->fail(SV_ERR_INVALID_ARG, "unknown option '%s'", key);
}

sv_status sv_debug_activation(sv_ctx* ctx, int which, int pair, void* dst, size_t bytes) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  if (c->t1) return c->fail(SV_ERR_UNSUPPORTED, "not available for the Table I network");
  if (which < 0 || which > 6 || pair < 0 || pair >= (int)c->tc_off.size() || !dst)
    return c->fail(SV_ERR_INVALID_ARG, "no such activation");
  // FP8 contexts keep e1 .. d1 as E4M3 codes (one byte per element; e1's codes in tc_act[7])
  const bool f8 = c->cfg.precision == SV_FP8 && which <= 4;
  const size_t es = f8 ? 1 : sizeof(__nv_bfloat16);
  const int buf = f8 && which == 0 ? 7 : which;
  if (bytes != c->tc_len[pair][which] * es)
    return c->fail(SV_ERR_INVALID_ARG, "activation has %zu bytes", c->tc_len[pair][which] * es);
  if (which == 6 && c->last_fused)
    return c->fail(SV_ERR_STATE, "d3 stayed on chip (fused final conv); set option fused_final 0 to keep it");
  DeviceGuard g(c->device);
  return c->cuda(cudaMemcpy(dst, (const unsigned char*)c->tc_act[buf].p + c->tc_off[pair][which] * es, bytes,
                            cudaMemcpyDeviceToHost), "copy activation");
}

long long sv_launch_count(const sv_ctx* ctx) {
  if (!ctx) return -1;
  return reinterpret_cast<const Ctx*>(ctx)->launches;
}

}  // extern "C"
