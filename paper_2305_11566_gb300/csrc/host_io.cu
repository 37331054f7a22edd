// host_io.cu -- one-launch staging for sv_pipeline_host: when every host buffer of a call is
// device-accessible (pinned / mapped host memory, reached through the unified address
// space over the CPU-GPU link), one kernel gathers all images into the device workspace
// and one kernel scatters all disparity maps back, instead of one copy call per image.
#include "sv_internal.cuh"

namespace sv {

namespace {

// One row-copy job per image: rows of `width` bytes (or floats) from src (pitch spitch) to
// dst (pitch dpitch).  A warp copies one row; 16-byte accesses when both sides allow them.
__global__ void copy_rows_kernel(const HostRowCopy* __restrict__ jobs, int njobs, int elem_bytes) {
  const HostRowCopy J = jobs[blockIdx.y];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nw = blockDim.x >> 5;
  const size_t row_bytes = (size_t)J.width * elem_bytes;
  const bool vec = ((reinterpret_cast<uintptr_t>(J.src) | reinterpret_cast<uintptr_t>(J.dst) | (uintptr_t)J.spitch |
                     (uintptr_t)J.dpitch | row_bytes) & 15) == 0;
  for (int y = blockIdx.x * nw + warp; y < J.height; y += gridDim.x * nw) {
    const unsigned char* s = J.src + (size_t)y * J.spitch;
    unsigned char* d = J.dst + (size_t)y * J.dpitch;
    if (vec) {
      for (size_t o = (size_t)lane * 16; o < row_bytes; o += 32 * 16)
        *reinterpret_cast<uint4*>(d + o) = *reinterpret_cast<const uint4*>(s + o);
    } else {
      for (size_t o = lane; o < row_bytes; o += 32) d[o] = s[o];
    }
  }
  (void)njobs;
}

}  // namespace

cudaError_t launch_copy_rows(const HostRowCopy* jobs, int njobs, int max_rows, int elem_bytes, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  const int warps = 8;
  dim3 grid((unsigned)std::max(1, std::min(64, (max_rows + warps - 1) / warps)), (unsigned)njobs);
  copy_rows_kernel<<<grid, warps * 32, 0, st>>>(jobs, njobs, elem_bytes);
  return cudaGetLastError();
}

}  // namespace sv
