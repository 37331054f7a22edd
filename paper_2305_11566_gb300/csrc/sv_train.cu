// sv_train.cu -- differentiation form: training forward, loss, backward, Adam.
#include "sv_ctx.cuh"

extern "C" {

sv_status sv_refine_train(sv_ctx* ctx, const sv_pair*, const void* const*, const void* const*, int, void* const*,
                          void* const*, void* const*, sv_stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  return reinterpret_cast<sv::Ctx*>(ctx)->fail(SV_ERR_UNSUPPORTED, "training form not built yet");
}
sv_status sv_refine_backward(sv_ctx* ctx, const void* const*, const void* const*, const void* const*, void*,
                             void* const*, sv_stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  return reinterpret_cast<sv::Ctx*>(ctx)->fail(SV_ERR_UNSUPPORTED, "training form not built yet");
}
sv_status sv_loss(sv_ctx* ctx, const sv_pair*, int, const void* const*, const float* const*, const void* const*,
                  const void* const*, double, void*, void* const*, void* const*, void* const*, sv_stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  return reinterpret_cast<sv::Ctx*>(ctx)->fail(SV_ERR_UNSUPPORTED, "training form not built yet");
}
sv_status sv_adam_step(sv_ctx* ctx, const void*, int, double, double, double, double, sv_stream) {
  if (!ctx) return SV_ERR_INVALID_ARG;
  return reinterpret_cast<sv::Ctx*>(ctx)->fail(SV_ERR_UNSUPPORTED, "training form not built yet");
}

}  // extern "C"
