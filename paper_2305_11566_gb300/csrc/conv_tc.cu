// conv_tc.cu -- implicit-GEMM convolutions on the tcgen05 tensor cores (BF16 operands,
// FP32 accumulation in tensor memory).
#include "sv_ctx.cuh"

namespace sv {

sv_status Ctx::pack_bf16_weights() { return SV_OK; }

sv_status Ctx::refine_tc(const sv_pair*, const int16_t* const*, int, float* const*, cudaStream_t) {
  return fail(SV_ERR_UNSUPPORTED, "BF16 tensor-core refinement not built yet");
}

}  // namespace sv
