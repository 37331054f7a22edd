// sv_forms.cu -- inference entry points of the context: plain refinement (per-pair
// launches on CUDA cores, FP32 or FP64), the tensor-core form, and the pipeline.
#include <algorithm>
#include <vector>

#include "sv_ctx.cuh"

namespace sv {

sv_status Ctx::refine_infer(const sv_pair* pairs, const int16_t* const* coarse, int n, float* const* out,
                            cudaStream_t st) {
  if (cfg.precision == SV_BF16) return refine_tc(pairs, coarse, n, out, st);
  if (cfg.precision == SV_FP64_CHECK)
    return fail(SV_ERR_UNSUPPORTED, "inference entry points produce FP32; use sv_refine_train on FP64_CHECK contexts");
  for (int i = 0; i < n; ++i) {
    sv_status s = refine_direct<float>(pairs[i], coarse[i], true, nullptr, out[i], nullptr, nullptr, nullptr, st);
    if (s) return s;
  }
  return SV_OK;
}

sv_status Ctx::pipeline(const sv_pair* pairs, int n, float* const* out, cudaStream_t st) {
  std::vector<size_t> off(n + 1, 0);
  for (int i = 0; i < n; ++i) off[i + 1] = off[i] + (size_t)(pairs[i].width / 4) * (pairs[i].height / 4);
  sv_status s = cuda(coarse_maps.ensure(off[n] * sizeof(int16_t)), "alloc coarse maps");
  if (s) return s;
  std::vector<int16_t*> maps(n);
  for (int i = 0; i < n; ++i) maps[i] = (int16_t*)coarse_maps.p + off[i];
  if ((s = coarse(pairs, n, maps.data(), nullptr, nullptr, st))) return s;
  std::vector<const int16_t*> cm(maps.begin(), maps.end());
  return refine_infer(pairs, cm.data(), n, out, st);
}

}  // namespace sv
