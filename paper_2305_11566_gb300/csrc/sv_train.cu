// sv_train.cu -- differentiation form: training forward (saves the decoder activations
// and the latent), backward through every refinement layer and the fused bilinear
// upsampling (the encoder is recomputed, not stored), loss and Adam.  FP32 for SV_FP32 /
// SV_BF16 contexts, FP64 for SV_FP64_CHECK contexts.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "sv_ctx.cuh"

namespace sv {

template <typename T>
cudaError_t launch_dgrad(const T* gout, int Ho, int Wo, int Co, const T* w, int ks, int mode, const T* mask_act,
                         int Hi, int Wi, int Ci, int accumulate, T* gin, cudaStream_t st);
template <typename T>
cudaError_t launch_wgrad(const T* gout, int Ho, int Wo, int Co, const T* in, int Hi, int Wi, int Ci, int ks, int mode,
                         T* gw, T* gb, cudaStream_t st);
template <typename T>
cudaError_t launch_latent_bwd(const T* gz, const T* eps, const T* lv, const T* gmu_ext, const T* glv_ext, size_t n,
                              T* gmu, T* glv, cudaStream_t st);
template <typename T>
cudaError_t launch_up4_bwd(const T* gU, const T* gx0, int W, int H, int w, int h, T* gc, cudaStream_t st);
template <typename T>
cudaError_t launch_build_x0(const uint8_t* L, int pitch, int W, int H, const T* coarse, int w, int h, T* x0,
                            cudaStream_t st);
template <typename T>
cudaError_t launch_loss_rec(const T* Y, const float* gt, size_t P, double inv_npix, T* gY, double* acc,
                            cudaStream_t st);
template <typename T>
cudaError_t launch_loss_kl(const T* mu, const T* lv, size_t n, double kl_scale, T* gmu, T* glv, double* acc,
                           cudaStream_t st);
template <typename T>
cudaError_t launch_loss_finish(const double* slots, int n_pairs, double inv_npix, double inv_nlat, double kl_w, T* out,
                               cudaStream_t st);
size_t loss_slots_per_pair();
template <typename T>
cudaError_t launch_adam(float* p, T* m, T* v, const T* g, size_t n, double lr, double b1, double b2, double eps,
                        int t, cudaStream_t st);

namespace {

// saved per pair: z, d1, d2, d3, lv, eps  (element type T)
enum { S_Z = 0, S_D1, S_D2, S_D3, S_LV, S_EPS, S_COUNT };

template <typename T>
size_t saved_sizes(const NetDims& net, const Levels& lv, size_t out[S_COUNT]) {
  const size_t P0 = (size_t)lv.H[0] * lv.W[0], P1 = (size_t)lv.H[1] * lv.W[1], P2 = (size_t)lv.H[2] * lv.W[2],
               P3 = (size_t)lv.H[3] * lv.W[3];
  out[S_Z] = P3 * net.lat;
  out[S_D1] = P2 * net.dec[0];
  out[S_D2] = P1 * net.dec[1];
  out[S_D3] = P0 * net.dec[2];
  out[S_LV] = P3 * net.lat;
  out[S_EPS] = P3 * net.lat;
  size_t t = 0;
  for (int i = 0; i < S_COUNT; ++i) t += (out[i] + 1) / 2 * 2;
  return t;
}

}  // namespace

template <typename T>
sv_status Ctx::train_forward(const sv_pair* pairs, const void* const* coarse, const void* const* eps, int n,
                             void* const* Y, void* const* mu, void* const* lv, cudaStream_t st) {
  sv_status s;
  std::vector<size_t> off(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    size_t sz[S_COUNT];
    off[i + 1] = off[i] + saved_sizes<T>(net, Levels(pairs[i].height, pairs[i].width), sz);
  }
  if ((s = cuda(train_saved.ensure(std::max<size_t>(off[n], 2) * sizeof(T)), "alloc saved activations"))) return s;
  train_pairs.assign(pairs, pairs + n);
  train_coarse.assign(coarse, coarse + n);
  train_off = off;
  train_elem = sizeof(T);
  for (int i = 0; i < n; ++i) {
    const Levels lv_(pairs[i].height, pairs[i].width);
    size_t sz[S_COUNT];
    saved_sizes<T>(net, lv_, sz);
    T* base = (T*)train_saved.p + off[i];
    T* sv[S_COUNT];
    for (int k = 0; k < S_COUNT; ++k) {
      sv[k] = base;
      base += (sz[k] + 1) / 2 * 2;
    }
    T* saved[7] = {nullptr, nullptr, nullptr, sv[S_Z], sv[S_D1], sv[S_D2], sv[S_D3]};
    if ((s = refine_direct<T>(pairs[i], coarse[i], false, (const T*)eps[i], (T*)Y[i], mu ? (T*)mu[i] : nullptr, sv[S_LV],
                              saved, st)))
      return s;
    if (lv && lv[i] && (s = cuda(cudaMemcpyAsync(lv[i], sv[S_LV], sz[S_LV] * sizeof(T), cudaMemcpyDeviceToDevice, st),
                                 "copy logvar")))
      return s;
    if ((s = cuda(cudaMemcpyAsync(sv[S_EPS], eps[i], sz[S_EPS] * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy eps")))
      return s;
  }
  train_ready = true;
  return SV_OK;
}

// Training forward of the BF16 form: the tensor-core encoder and decoder (BF16 operands,
// FP32 accumulation), the training latent in FP32 on CUDA cores, the final conv in FP32.
// The decoder activations and the latent are saved as FP32 for the FP32 backward.
sv_status Ctx::train_forward_bf16(const sv_pair* pairs, const void* const* coarse, const void* const* eps, int n,
                                  void* const* Y, void* const* mu, void* const* lv, cudaStream_t st) {
  using T = float;
  sv_status s;
  std::vector<size_t> off(n + 1, 0);
  size_t lat_total = 0;
  for (int i = 0; i < n; ++i) {
    size_t sz[S_COUNT];
    off[i + 1] = off[i] + saved_sizes<T>(net, Levels(pairs[i].height, pairs[i].width), sz);
    lat_total += (sz[S_LV] + 1) / 2 * 2;
  }
  if ((s = cuda(train_saved.ensure(std::max<size_t>(off[n], 2) * sizeof(T)), "alloc saved activations"))) return s;
  if ((s = cuda(train_mu.ensure(std::max<size_t>(lat_total, 2) * sizeof(T)), "alloc latent scratch"))) return s;
  train_pairs.assign(pairs, pairs + n);
  train_coarse.assign(coarse, coarse + n);
  train_off = off;
  train_elem = sizeof(T);
  std::vector<float*> outs(n);
  for (int i = 0; i < n; ++i) outs[i] = (float*)Y[i];
  TcRun r;
  if ((s = tc_prepare(pairs, nullptr, n, outs.data(), r, (const float* const*)coarse))) return s;
  if ((s = cuda(tc_tables.ensure(r.host.size()), "alloc tables"))) return s;
  if ((s = cuda(cudaMemcpyAsync(tc_tables.p, r.host.data(), r.host.size(), cudaMemcpyHostToDevice, st),
                "upload tables")))
    return s;
  TcTrainLatent tl;
  std::vector<T*> svb(n * S_COUNT);
  size_t mo = 0;
  for (int i = 0; i < n; ++i) {
    const Levels lv_(pairs[i].height, pairs[i].width);
    size_t sz[S_COUNT];
    saved_sizes<T>(net, lv_, sz);
    T* base = (T*)train_saved.p + off[i];
    for (int k = 0; k < S_COUNT; ++k) {
      svb[i * S_COUNT + k] = base;
      base += (sz[k] + 1) / 2 * 2;
    }
    tl.e3.push_back((const __nv_bfloat16*)tc_act[2].p + tc_off[i][2]);
    tl.P3.push_back(lv_.H[3] * lv_.W[3]);
    tl.eps.push_back((const float*)eps[i]);
    float* m = mu && mu[i] ? (float*)mu[i] : (float*)train_mu.p + mo;
    mo += (sz[S_LV] + 1) / 2 * 2;
    tl.mu.push_back(m);
    tl.lv.push_back(svb[i * S_COUNT + S_LV]);
    tl.z.push_back((__nv_bfloat16*)tc_act[3].p + tc_off[i][3]);
  }
  if ((s = tc_launch(r, (const unsigned char*)tc_tables.p, st, &tl))) return s;
  for (int i = 0; i < n; ++i) {
    const int acts[4] = {3, 4, 5, 6};
    const int slots[4] = {S_Z, S_D1, S_D2, S_D3};
    for (int k = 0; k < 4; ++k) {
      LaunchScope _ls(*this, "save_bf16_to_f32", st);
      if ((s = cuda(launch_bf16_to_f32((const __nv_bfloat16*)tc_act[acts[k]].p + tc_off[i][acts[k]],
                                       svb[i * S_COUNT + slots[k]], tc_len[i][acts[k]], st),
                    "save activations")))
        return s;
    }
    size_t sz[S_COUNT];
    saved_sizes<T>(net, Levels(pairs[i].height, pairs[i].width), sz);
    if (lv && lv[i] &&
        (s = cuda(cudaMemcpyAsync(lv[i], svb[i * S_COUNT + S_LV], sz[S_LV] * sizeof(T), cudaMemcpyDeviceToDevice, st),
                  "copy logvar")))
      return s;
    if ((s = cuda(cudaMemcpyAsync(svb[i * S_COUNT + S_EPS], eps[i], sz[S_EPS] * sizeof(T), cudaMemcpyDeviceToDevice, st),
                  "copy eps")))
      return s;
  }
  train_ready = true;
  return SV_OK;
}

template <typename T>
sv_status Ctx::train_backward(const void* const* gY, const void* const* gmu_ext, const void* const* glv_ext, T* gparams,
                              void* const* gcoarse, cudaStream_t st) {
  sv_status s;
  const int n = (int)train_pairs.size();
  const T* Wt = weights<T>();
  auto Wl = [&](int l) { return Wt + net.w_off(l); };
  auto Bl = [&](int l) { return Wt + net.b_off(l); };
  auto GW = [&](int l) { return gparams + net.w_off(l); };
  auto GB = [&](int l) { return gparams + net.b_off(l); };
  if ((s = cuda(cudaMemsetAsync(gparams, 0, net.count() * sizeof(T), st), "zero grads"))) return s;
  // scratch for one pair at a time: gd3 gd2 gd1 gz gmu glv ge3 ge2 ge1 gx0 x0
  size_t need = 0;
  for (int i = 0; i < n; ++i) {
    const Levels lv(train_pairs[i].height, train_pairs[i].width);
    const size_t P0 = (size_t)lv.H[0] * lv.W[0], P1 = (size_t)lv.H[1] * lv.W[1], P2 = (size_t)lv.H[2] * lv.W[2],
                 P3 = (size_t)lv.H[3] * lv.W[3];
    size_t t = P0 * net.dec[2] + P1 * net.dec[1] + P2 * net.dec[0] + 3 * P3 * net.lat + P3 * net.enc[2] +
               P2 * net.enc[1] + P1 * net.enc[0] + 4 * P0 + 64;
    need = std::max(need, t);
  }
  if ((s = cuda(train_scratch.ensure(need * sizeof(T)), "alloc backward scratch"))) return s;
  // FP32: the tiled gradient kernels (per-CTA weight-gradient slots, reduced in a fixed
  // order); FP64 (the check form): the plain gather kernels
  if constexpr (std::is_same<T, float>::value) {
    size_t maxw = 0;
    for (int l = 0; l < L_COUNT; ++l)
      maxw = std::max(maxw, (size_t)net.cout(l) * net.ks(l) * net.ks(l) * net.cin(l) + net.cout(l));
    if ((s = cuda(wgrad_slots.ensure(4 * 152 * maxw * sizeof(float)), "alloc weight-gradient slots"))) return s;
  }
  auto DG = [&](const T* go, int Ho, int Wo, int Co, const T* wt, int ks, int mode, const T* mask, int Hi, int Wi, int Ci,
                int accum, T* gi) -> cudaError_t {
    if constexpr (std::is_same<T, float>::value)
      return launch_dgrad_tiled(go, Ho, Wo, Co, wt, ks, mode, mask, Hi, Wi, Ci, accum, gi, st);
    else
      return launch_dgrad<T>(go, Ho, Wo, Co, wt, ks, mode, mask, Hi, Wi, Ci, accum, gi, st);
  };
  auto WG = [&](const T* go, int Ho, int Wo, int Co, const T* in, int Hi, int Wi, int Ci, int ks, int mode, T* gw,
                T* gb) -> cudaError_t {
    if constexpr (std::is_same<T, float>::value)
      return launch_wgrad_tiled(go, Ho, Wo, Co, in, Hi, Wi, Ci, ks, mode, gw, gb, (float*)wgrad_slots.p,
                                wgrad_slots.n / sizeof(float), st);
    else
      return launch_wgrad<T>(go, Ho, Wo, Co, in, Hi, Wi, Ci, ks, mode, gw, gb, st);
  };
  for (int i = 0; i < n; ++i) {
    const sv_pair& p = train_pairs[i];
    const Levels lv(p.height, p.width);
    const int H = lv.H[0], W = lv.W[0], w = p.width / 4, h = p.height / 4;
    const size_t P0 = (size_t)H * W, P1 = (size_t)lv.H[1] * lv.W[1], P2 = (size_t)lv.H[2] * lv.W[2],
                 P3 = (size_t)lv.H[3] * lv.W[3];
    size_t sz[S_COUNT];
    saved_sizes<T>(net, lv, sz);
    const T* base = (const T*)train_saved.p + train_off[i];
    const T* sv[S_COUNT];
    for (int k = 0; k < S_COUNT; ++k) {
      sv[k] = base;
      base += (sz[k] + 1) / 2 * 2;
    }
    T* q = (T*)train_scratch.p;
    auto take = [&](size_t cnt) { T* r = q; q += (cnt + 1) / 2 * 2; return r; };
    T *gd3 = take(P0 * net.dec[2]), *gd2 = take(P1 * net.dec[1]), *gd1 = take(P2 * net.dec[0]);
    T *gz = take(P3 * net.lat), *gmu = take(P3 * net.lat), *glv = take(P3 * net.lat);
    T *ge3 = take(P3 * net.enc[2]), *ge2 = take(P2 * net.enc[1]), *ge1 = take(P1 * net.enc[0]);
    T *gx0 = take(2 * P0), *x0 = take(2 * P0);
    const T* gYi = (const T*)gY[i];
    const T* coarse = (const T*)train_coarse[i];
    cudaError_t e;
#define SV_BW(name, expr)                      \
  {                                            \
    LaunchScope _ls(*this, name, st);          \
    if ((s = cuda((expr), name))) return s;    \
  }
    // final: Y = U + conv(d3) + b
    SV_BW("bwd_final_dgrad", DG(gYi, H, W, 1, Wl(L_FINAL), 3, CM_S1, sv[S_D3], H, W, net.dec[2], 0, gd3));
    SV_BW("bwd_final_wgrad", WG(gYi, H, W, 1, sv[S_D3], H, W, net.dec[2], 3, CM_S1, GW(L_FINAL), GB(L_FINAL)));
    // decoder (nearest x2 + crop + 3x3 conv + ReLU)
    SV_BW("bwd_dec3_dgrad", DG(gd3, H, W, net.dec[2], Wl(L_DEC3), 3, CM_UP2, sv[S_D2], lv.H[1], lv.W[1],
                                            net.dec[1], 0, gd2));
    SV_BW("bwd_dec3_wgrad", WG(gd3, H, W, net.dec[2], sv[S_D2], lv.H[1], lv.W[1], net.dec[1], 3, CM_UP2,
                                            GW(L_DEC3), GB(L_DEC3)));
    SV_BW("bwd_dec2_dgrad", DG(gd2, lv.H[1], lv.W[1], net.dec[1], Wl(L_DEC2), 3, CM_UP2, sv[S_D1], lv.H[2],
                                            lv.W[2], net.dec[0], 0, gd1));
    SV_BW("bwd_dec2_wgrad", WG(gd2, lv.H[1], lv.W[1], net.dec[1], sv[S_D1], lv.H[2], lv.W[2], net.dec[0], 3,
                                            CM_UP2, GW(L_DEC2), GB(L_DEC2)));
    SV_BW("bwd_dec1_dgrad", DG(gd1, lv.H[2], lv.W[2], net.dec[0], Wl(L_DEC1), 3, CM_UP2, nullptr, lv.H[3],
                                            lv.W[3], net.lat, 0, gz));
    SV_BW("bwd_dec1_wgrad", WG(gd1, lv.H[2], lv.W[2], net.dec[0], sv[S_Z], lv.H[3], lv.W[3], net.lat, 3,
                                            CM_UP2, GW(L_DEC1), GB(L_DEC1)));
    // latent: z = mu + eps exp(lv / 2), plus the loss's own terms
    SV_BW("bwd_latent", launch_latent_bwd<T>(gz, sv[S_EPS], sv[S_LV], gmu_ext && gmu_ext[i] ? (const T*)gmu_ext[i] : nullptr,
                                             glv_ext && glv_ext[i] ? (const T*)glv_ext[i] : nullptr, P3 * net.lat, gmu, glv, st));
    // recompute the encoder (not stored by the forward)
    T* rec[7] = {(T*)act[0].p, (T*)act[1].p, (T*)act[2].p, nullptr, nullptr, nullptr, nullptr};
    {
      const size_t needE[3] = {P1 * net.enc[0], P2 * net.enc[1], P3 * net.enc[2]};
      for (int k = 0; k < 3; ++k) {
        if ((s = cuda(act[k].ensure(needE[k] * sizeof(T)), "alloc encoder recompute"))) return s;
        rec[k] = (T*)act[k].p;
      }
      {
        LaunchScope _ls(*this, "recompute_enc1", st);
        e = launch_enc1<T, T>(p.left, p.pitch, p.width, p.height, coarse, w, h, Wl(L_ENC1), Bl(L_ENC1), net.enc[0],
                              rec[0], st);
        if ((s = cuda(e, "recompute enc1"))) return s;
      }
      DirectConvArgs<T> a{rec[0], lv.H[1], lv.W[1], net.enc[0], Wl(L_ENC2), Bl(L_ENC2), net.enc[1], lv.H[2], lv.W[2], 1,
                          rec[1]};
      SV_BW("recompute_enc2", launch_conv_direct<T>(a, CM_S2, 3, st));
      a = {rec[1], lv.H[2], lv.W[2], net.enc[1], Wl(L_ENC3), Bl(L_ENC3), net.enc[2], lv.H[3], lv.W[3], 1, rec[2]};
      SV_BW("recompute_enc3", launch_conv_direct<T>(a, CM_S2, 3, st));
    }
    const T *e1 = rec[0], *e2 = rec[1], *e3 = rec[2];
    // latent heads (1x1): e3 -> mu, e3 -> logvar
    SV_BW("bwd_mu_dgrad", DG(gmu, lv.H[3], lv.W[3], net.lat, Wl(L_MU), 1, CM_S1, e3, lv.H[3], lv.W[3],
                                          net.enc[2], 0, ge3));
    SV_BW("bwd_lv_dgrad", DG(glv, lv.H[3], lv.W[3], net.lat, Wl(L_LV), 1, CM_S1, e3, lv.H[3], lv.W[3],
                                          net.enc[2], 1, ge3));
    SV_BW("bwd_mu_wgrad", WG(gmu, lv.H[3], lv.W[3], net.lat, e3, lv.H[3], lv.W[3], net.enc[2], 1, CM_S1,
                                          GW(L_MU), GB(L_MU)));
    SV_BW("bwd_lv_wgrad", WG(glv, lv.H[3], lv.W[3], net.lat, e3, lv.H[3], lv.W[3], net.enc[2], 1, CM_S1,
                                          GW(L_LV), GB(L_LV)));
    // encoder (3x3 stride 2 + ReLU)
    SV_BW("bwd_enc3_dgrad", DG(ge3, lv.H[3], lv.W[3], net.enc[2], Wl(L_ENC3), 3, CM_S2, e2, lv.H[2], lv.W[2],
                                            net.enc[1], 0, ge2));
    SV_BW("bwd_enc3_wgrad", WG(ge3, lv.H[3], lv.W[3], net.enc[2], e2, lv.H[2], lv.W[2], net.enc[1], 3, CM_S2,
                                            GW(L_ENC3), GB(L_ENC3)));
    SV_BW("bwd_enc2_dgrad", DG(ge2, lv.H[2], lv.W[2], net.enc[1], Wl(L_ENC2), 3, CM_S2, e1, lv.H[1], lv.W[1],
                                            net.enc[0], 0, ge1));
    SV_BW("bwd_enc2_wgrad", WG(ge2, lv.H[2], lv.W[2], net.enc[1], e1, lv.H[1], lv.W[1], net.enc[0], 3, CM_S2,
                                            GW(L_ENC2), GB(L_ENC2)));
    SV_BW("bwd_build_x0", launch_build_x0<T>(p.left, p.pitch, W, H, coarse, w, h, x0, st));
    SV_BW("bwd_enc1_wgrad", WG(ge1, lv.H[1], lv.W[1], net.enc[0], x0, H, W, 2, 3, CM_S2, GW(L_ENC1),
                                            GB(L_ENC1)));
    if (gcoarse && gcoarse[i]) {
      // through the network input (channel U / 256) and the residual Y = U + ...
      SV_BW("bwd_enc1_dgrad", DG(ge1, lv.H[1], lv.W[1], net.enc[0], Wl(L_ENC1), 3, CM_S2, nullptr, H, W, 2, 0,
                                              gx0));
      SV_BW("bwd_upsample4", launch_up4_bwd<T>(gYi, gx0, W, H, w, h, (T*)gcoarse[i], st));
    }
#undef SV_BW
  }
  return SV_OK;
}

template <typename T>
sv_status Ctx::loss(const sv_pair* pairs, int n, const void* const* Y, const float* const* gt, const void* const* mu,
                    const void* const* lv, double kl_w, void* out, void* const* gY, void* const* gmu, void* const* glv,
                    cudaStream_t st) {
  sv_status s;
  const size_t per = loss_slots_per_pair();
  if ((s = cuda(loss_acc.ensure(per * n * sizeof(double)), "alloc loss partials"))) return s;
  double npix = 0, nlat = 0;
  for (int i = 0; i < n; ++i) {
    const Levels lv_(pairs[i].height, pairs[i].width);
    npix += (double)pairs[i].width * pairs[i].height;
    nlat += (double)lv_.H[3] * lv_.W[3] * net.lat;
  }
  for (int i = 0; i < n; ++i) {
    double* acc = (double*)loss_acc.p + per * i;
    const Levels lv_(pairs[i].height, pairs[i].width);
    const size_t P = (size_t)pairs[i].width * pairs[i].height, nl = (size_t)lv_.H[3] * lv_.W[3] * net.lat;
    {
      LaunchScope _ls(*this, "loss_rec", st);
      if ((s = cuda(launch_loss_rec<T>((const T*)Y[i], gt[i], P, 1.0 / npix, gY && gY[i] ? (T*)gY[i] : nullptr, acc, st),
                    "loss rec")))
        return s;
    }
    LaunchScope _ls(*this, "loss_kl", st);
    if ((s = cuda(launch_loss_kl<T>((const T*)mu[i], (const T*)lv[i], nl, kl_w / nlat, gmu && gmu[i] ? (T*)gmu[i] : nullptr,
                                    glv && glv[i] ? (T*)glv[i] : nullptr, acc, st),
                  "loss kl")))
      return s;
  }
  LaunchScope _ls(*this, "loss_finish", st);
  return cuda(launch_loss_finish<T>((const double*)loss_acc.p, n, 1.0 / npix, 1.0 / nlat, kl_w, (T*)out, st),
              "loss finish");
}

template <typename T>
sv_status Ctx::adam(const T* g, int step, double lr, double b1, double b2, double eps, cudaStream_t st) {
  sv_status s;
  const size_t n = net.count();
  if (adam_elem != (int)sizeof(T) || !adam_m.p) {
    if ((s = cuda(adam_m.ensure(n * sizeof(T)), "alloc adam m"))) return s;
    if ((s = cuda(adam_v.ensure(n * sizeof(T)), "alloc adam v"))) return s;
    if ((s = cuda(cudaMemsetAsync(adam_m.p, 0, n * sizeof(T), st), "zero adam"))) return s;
    if ((s = cuda(cudaMemsetAsync(adam_v.p, 0, n * sizeof(T), st), "zero adam"))) return s;
    adam_elem = (int)sizeof(T);
  }
  {
    LaunchScope _ls(*this, "adam", st);
    if ((s = cuda(launch_adam<T>((float*)w32.p, (T*)adam_m.p, (T*)adam_v.p, g, n, lr, b1, b2, eps, step, st), "adam")))
      return s;
  }
  return refresh_weight_copies_async(st);
}

template sv_status Ctx::train_forward<float>(const sv_pair*, const void* const*, const void* const*, int, void* const*,
                                             void* const*, void* const*, cudaStream_t);
template sv_status Ctx::train_forward<double>(const sv_pair*, const void* const*, const void* const*, int, void* const*,
                                              void* const*, void* const*, cudaStream_t);
template sv_status Ctx::train_backward<float>(const void* const*, const void* const*, const void* const*, float*,
                                              void* const*, cudaStream_t);
template sv_status Ctx::train_backward<double>(const void* const*, const void* const*, const void* const*, double*,
                                               void* const*, cudaStream_t);

}  // namespace sv

using sv::Ctx;

extern "C" {

sv_status sv_refine_train(sv_ctx* ctx, const sv_pair* pairs, const void* const* coarse, const void* const* eps,
                          int n_pairs, void* const* disp_out, void* const* mu_out, void* const* logvar_out,
                          sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  c->err.clear();
  sv_status s = c->check_pairs(pairs, n_pairs);
  if (s) return s;
  if (n_pairs == 0) return SV_OK;
  if (!coarse || !eps || !disp_out) return c->fail(SV_ERR_INVALID_ARG, "coarse / eps / disp_out is NULL");
  for (int i = 0; i < n_pairs; ++i)
    if (!coarse[i] || !eps[i] || !disp_out[i]) return c->fail(SV_ERR_INVALID_ARG, "pair %d: NULL buffer", i);
  sv::DeviceGuardInt g(c->device);
  c->train_ready = false;
  if (c->t1)  // forward with the reparameterisation of Eq. 8; logvar_out receives sigma
    return c->t1_forward(pairs, n_pairs, nullptr, (const float* const*)coarse, (const float* const*)eps,
                         (float* const*)disp_out, (float* const*)mu_out, (float* const*)logvar_out,
                         (cudaStream_t)stream);
  if (c->cfg.precision == SV_FP8) return c->fail(SV_ERR_UNSUPPORTED, "the FP8 form is inference only");
  if (c->cfg.precision == SV_FP64_CHECK)
    return c->train_forward<double>(pairs, coarse, eps, n_pairs, disp_out, mu_out, logvar_out, (cudaStream_t)stream);
  if (c->cfg.precision == SV_BF16)
    return c->train_forward_bf16(pairs, coarse, eps, n_pairs, disp_out, mu_out, logvar_out, (cudaStream_t)stream);
  return c->train_forward<float>(pairs, coarse, eps, n_pairs, disp_out, mu_out, logvar_out, (cudaStream_t)stream);
}

sv_status sv_refine_backward(sv_ctx* ctx, const void* const* grad_disp, const void* const* grad_mu,
                             const void* const* grad_logvar, void* grad_params, void* const* grad_coarse,
                             sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  c->err.clear();
  if (c->t1) return c->fail(SV_ERR_UNSUPPORTED, "no backward for the Table I network");
  if (!c->train_ready) return c->fail(SV_ERR_STATE, "sv_refine_backward needs a preceding sv_refine_train");
  if (!grad_disp || !grad_params) return c->fail(SV_ERR_INVALID_ARG, "grad_disp / grad_params is NULL");
  for (size_t i = 0; i < c->train_pairs.size(); ++i)
    if (!grad_disp[i]) return c->fail(SV_ERR_INVALID_ARG, "grad_disp[%zu] is NULL", i);
  sv::DeviceGuardInt g(c->device);
  if (c->train_elem == (int)sizeof(double))
    return c->train_backward<double>(grad_disp, grad_mu, grad_logvar, (double*)grad_params, grad_coarse,
                                     (cudaStream_t)stream);
  return c->train_backward<float>(grad_disp, grad_mu, grad_logvar, (float*)grad_params, grad_coarse,
                                  (cudaStream_t)stream);
}

sv_status sv_loss(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const void* const* disp, const float* const* gt,
                  const void* const* mu, const void* const* logvar, double kl_weight, void* loss_out,
                  void* const* grad_disp, void* const* grad_mu, void* const* grad_logvar, sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  c->err.clear();
  if (c->t1) return c->fail(SV_ERR_UNSUPPORTED, "the Table I network's loss is sv_loss_paper");
  sv_status s = c->check_pairs(pairs, n_pairs);
  if (s) return s;
  if (n_pairs == 0 || !disp || !gt || !mu || !logvar || !loss_out) return c->fail(SV_ERR_INVALID_ARG, "NULL argument");
  for (int i = 0; i < n_pairs; ++i)
    if (!disp[i] || !gt[i] || !mu[i] || !logvar[i]) return c->fail(SV_ERR_INVALID_ARG, "pair %d: NULL buffer", i);
  sv::DeviceGuardInt g(c->device);
  if (c->cfg.precision == SV_FP64_CHECK)
    return c->loss<double>(pairs, n_pairs, disp, gt, mu, logvar, kl_weight, loss_out, grad_disp, grad_mu, grad_logvar,
                           (cudaStream_t)stream);
  return c->loss<float>(pairs, n_pairs, disp, gt, mu, logvar, kl_weight, loss_out, grad_disp, grad_mu, grad_logvar,
                        (cudaStream_t)stream);
}

sv_status sv_adam_step(sv_ctx* ctx, const void* grad, int step, double lr, double beta1, double beta2, double eps,
                       sv_stream stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  c->err.clear();
  if (c->t1) return c->fail(SV_ERR_UNSUPPORTED, "no training step for the Table I network");
  if (!grad || step < 1) return c->fail(SV_ERR_INVALID_ARG, "grad is NULL or step < 1");
  sv::DeviceGuardInt g(c->device);
  if (c->cfg.precision == SV_FP64_CHECK)
    return c->adam<double>((const double*)grad, step, lr, beta1, beta2, eps, (cudaStream_t)stream);
  return c->adam<float>((const float*)grad, step, lr, beta1, beta2, eps, (cudaStream_t)stream);
}

}  // extern "C"
