// zncc_static.cu -- a coarse-matching entry point that allocates no device memory.
//
// Some callers cannot call cudaMalloc when they need a disparity map: a real-time loop
// that must not block on the allocator (cudaMalloc may synchronise the device and has no
// latency bound), or a plugin whose host owns every byte of device memory and hands the
// library only its inputs and outputs.  sv_coarse_match keeps its per-call work tables in
// memory its context allocated; this variant keeps them in a fixed array that is part of
// the library image instead, so a call needs nothing but the caller's inputs and outputs.
// The tables are uploaded from host memory that lives only for the duration of the call.
#include <mutex>
#include <vector>

#include "sv_ctx.cuh"

namespace {

constexpr int kStaticMaxPairs = 256;
constexpr int kStaticMaxJobs = 32768;
constexpr size_t kPairBytes = sizeof(sv::ZPair) * kStaticMaxPairs;
constexpr size_t kJobOffset = (kPairBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kJobOffset + sizeof(sv::ZJob) * kStaticMaxJobs;

// The work tables of one call (pair descriptors, then job list).  Every GPU that loads the
// library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_zncc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_zncc_scratch on the current device, looked up once per device
// ordinal and cached.  In host code the symbol's name is only a host-side handle, never a
// device pointer.  The cache assumes the device's primary context lives as long as the
// process: after cudaDeviceReset the cached address is stale, so a process that resets a
// device must not call this entry point on it again.
cudaError_t scratch_address(void** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_zncc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

// The validation of sv_coarse_match, with the same status codes.
sv_status pair_check(const sv_pair& p, int k) {
  if (!p.left || !p.right) return SV_ERR_INVALID_ARG;
  if (((uintptr_t)p.left & 15) || ((uintptr_t)p.right & 15)) return SV_ERR_INVALID_ARG;
  if (p.pitch % 16 || p.pitch < p.width) return SV_ERR_INVALID_ARG;
  if (p.width < 4 * k || p.height < 4 * k) return SV_ERR_INVALID_ARG;
  if (p.width > sv::kMaxSide || p.height > sv::kMaxSide) return SV_ERR_UNSUPPORTED;
  if (p.max_disp < 1 || p.max_disp > sv::kMaxDisp || p.max_disp > p.width / 4) return SV_ERR_INVALID_ARG;
  return SV_OK;
}

}  // namespace

extern "C" sv_status sv_coarse_match_static(const sv_pair* pairs, int n_pairs, int window, int16_t* const* disp_out,
                                            float* const* best, float* const* second, sv_stream stream) {
  if (window < 3 || window > 15 || window % 2 == 0) return SV_ERR_INVALID_ARG;
  if (n_pairs < 0 || (n_pairs > 0 && (!pairs || !disp_out))) return SV_ERR_INVALID_ARG;
  if (n_pairs == 0) return SV_OK;
  if (n_pairs > kStaticMaxPairs) return SV_ERR_UNSUPPORTED;
  int maxD = 1;
  for (int i = 0; i < n_pairs; ++i) {
    const sv_status ps = pair_check(pairs[i], window);
    if (ps != SV_OK) return ps;
    if (!disp_out[i]) return SV_ERR_INVALID_ARG;
    if (pairs[i].max_disp > maxD) maxD = pairs[i].max_disp;
  }
  const int gx = sv::kZnccWarps * sv::zncc_tx(sv::zncc_kd(maxD));
  std::vector<sv::ZPair> zp(n_pairs);
  std::vector<sv::ZJob> jobs;
  for (int i = 0; i < n_pairs; ++i) {
    const sv_pair& p = pairs[i];
    sv::ZPair& z = zp[i];
    z.L = p.left; z.R = p.right; z.W = p.width; z.H = p.height; z.pitch = p.pitch; z.D = p.max_disp;
    z.w = p.width / 4; z.h = p.height / 4;
    z.disp = disp_out[i];
    z.best = best ? best[i] : nullptr;
    z.second = second ? second[i] : nullptr;
    for (int y0 = 0; y0 < z.h; y0 += sv::kZnccTY)
      for (int x0 = 0; x0 < z.w; x0 += gx) jobs.push_back({i, y0, x0, 0});
  }
  if ((int)jobs.size() > kStaticMaxJobs) return SV_ERR_UNSUPPORTED;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return SV_ERR_CUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaStream_t st = (cudaStream_t)stream;
  // both tables are rewritten in full by every call: nothing has to start at zero
  if (cudaMemcpyAsync(b, zp.data(), sizeof(sv::ZPair) * n_pairs, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SV_ERR_CUDA;
  if (cudaMemcpyAsync(b + kJobOffset, jobs.data(), sizeof(sv::ZJob) * jobs.size(), cudaMemcpyHostToDevice, st) !=
      cudaSuccess)
    return SV_ERR_CUDA;
  bool scores = false;
  for (const sv::ZPair& q : zp) scores |= q.best != nullptr || q.second != nullptr;
  if (sv::launch_zncc_wta(reinterpret_cast<const sv::ZPair*>(b), reinterpret_cast<const sv::ZJob*>(b + kJobOffset),
                          (int)jobs.size(), window / 2, maxD, st, scores ? 1 : 0) != cudaSuccess)
    return SV_ERR_CUDA;
  return SV_OK;
}
