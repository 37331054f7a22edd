// conv_tc.cu -- refinement convolutions as implicit GEMMs on the tcgen05 tensor cores:
// BF16 operands in shared memory, FP32 accumulators in tensor memory (TMEM).
//
// GEMM view of one tile: M = 128 consecutive output units of one row, N = NT output
// channels, K = taps x Cin.  Instead of an im2col copy per tap, the input rows a tile
// needs are staged ONCE in shared memory as K-major swizzled pixel rows: channel block kb
// (RB / 2 channels, RB = 128, 64 or 32 bytes per pixel) of every staged pixel, pixel
// after pixel, in the 128/64/32-byte swizzle that one TMA box per block writes.  The A
// operand of every tap is the same staged rows seen from a start address shifted by
// whole pixels (matrix descriptor: swizzled K-major, SBO = 8 pixels); the K steps of 16
// channels inside a pixel row advance the start by 32 bytes.  Consecutive tiles of a CTA
// walk down the rows of a column strip and reuse staged rows (ring of row slots, or of
// one-channel-block slots where the weights leave no room for a spare row).
//
// Modes:
//   TM_S2  3x3 stride-2 conv (encoder): staged rows 2i-1, 2i, 2i+1 with odd and even
//          pixels de-interleaved into two pixel sets, so each tap is a unit-stride view.
//   TM_UP2 nearest-x2 upsample + 3x3 conv (decoder), computed as four output phases
//          (py, px) of 2x2 convs on the low-resolution input with the 3x3 weights summed
//          per phase (rows/cols {0} and {1,2} for phase 0, {0,1} and {2} for phase 1):
//          4 taps per output instead of 9.  The last row / column of an odd-sized
//          (cropped) output is recomputed exactly by edge_up2fix (tc_edges.cu) afterwards.
//   TM_P1  1x1 conv (latent mean head).
//
// Warp roles (192 threads): warps 0-3 epilogue (TMEM lanes 0-127: tcgen05.ld, bias,
// ReLU, BF16 store), warp 4 TMEM allocation + MMA issue (the whole warp runs the loop with
// warp-uniform descriptors advanced by constant increments; one elect.sync lane issues each
// tcgen05.mma / tcgen05.commit), warp 5 one thread
// loading every staged row with TMA (cp.async.bulk.tensor, one box of RB / 2 channels x
// the staged pixels per channel block and pixel set; the hardware fills the halo outside
// the image with zeros) and signalling the row's mbarrier by transaction count.  Every wait is bounded; on
// timeout the kernel records an error code and returns.
#include <algorithm>
#include <cstdio>
#include <vector>

#include <cuda.h>
#include <cuda_fp8.h>
#include <type_traits>
#include <cudaTypedefs.h>

#include "sv_ctx.cuh"

namespace sv {

namespace tc {

using bf16 = __nv_bfloat16;

enum Mode { TM_S2 = 0, TM_UP2 = 1, TM_P1 = 2 };

struct alignas(128) LayerPair {
  const bf16* in;
  bf16* out;
  int Hi, Wi;  // input size
  int Ho, Wo;  // output size
  int Hu, Wu;  // unit grid covered by tiles (S2 / P1: output; UP2: low-resolution input)
  int pad[6];
  CUtensorMap tm[2];  // TMA view of the input: S2 [0] odd pixels, [1] even pixels; others [0]
};

struct Strip {
  int pair, j0, i0, cnt;
};

struct Params {
  const LayerPair* lp;
  const Strip* strips;
  int n_strips;
  const bf16* wpack;  // [G][T][NT * cin] in the core-matrix layout
  const float* bias;  // [cout]
  int cin, cout, G, relu, ring;  // ring: staged units (rows, or channel blocks of rows if split)
  int split;                      // 1: a ring unit is one channel block of a row
  int* err;
  long long spin;
  // FP8 form (E4M3 operands): cin counts pairs of FP8 channels (the operand bytes / 2, so
  // that every byte-level layout is the BF16 one); scale [cout] dequantises the
  // accumulator (per-output-channel weight scale); out_f8: the output is stored as E4M3
  // codes (else BF16)
  const float* scale;
  int out_f8;
};

// RA staged rows per tile, STEP new rows per next tile, T taps, NSET pixel sets per row
// (stride 2: odd and even pixels), NPX pixels per set.
template <int MODE> struct Geo;
template <> struct Geo<TM_S2> { static constexpr int RA = 3, STEP = 2, T = 9, NSET = 2, NPX = 129; };
template <> struct Geo<TM_UP2> { static constexpr int RA = 2, STEP = 1, T = 4, NSET = 1, NPX = 129; };
template <> struct Geo<TM_P1> { static constexpr int RA = 1, STEP = 1, T = 1, NSET = 1, NPX = 128; };

constexpr int kThreads = 192;
constexpr int kBarBytes = 8;

__host__ __device__ inline int nset(int mode) { return mode == TM_S2 ? 2 : 1; }
__host__ __device__ inline int npx(int mode) { return mode == TM_P1 ? 128 : 129; }
// bytes per staged pixel and channel block: the widest swizzle span whose channel count
// divides cin (128 B = 64 channels, 64 B = 32, 32 B = 16)
__host__ __device__ inline int rb_of(int cin) { return cin % 64 == 0 ? 128 : cin % 32 == 0 ? 64 : 32; }
// one channel block of every staged pixel of one set, 1024-byte aligned (swizzle atom)
__host__ __device__ inline uint32_t kb_stride(int mode, int rb) { return (uint32_t)((npx(mode) * rb + 1023) / 1024 * 1024); }
__host__ __device__ inline size_t row_bytes(int mode, int cin) {
  const int rb = rb_of(cin);
  return (size_t)nset(mode) * (cin * 2 / rb) * kb_stride(mode, rb);
}
__host__ __device__ inline int taps(int mode) { return mode == TM_S2 ? 9 : mode == TM_UP2 ? 4 : 1; }
__host__ __device__ inline size_t b_bytes(int mode, int NT, int cin) { return (size_t)taps(mode) * NT * cin * 2; }
// ring: staged units, whole rows or (split) one channel block of a row each
// f8: the FP8 form also keeps a per-channel scale beside the bias
// epilogue staging: per epilogue warp 32 pixels x 32 BF16 channels (the stores leave shared
// memory as whole 64-byte pixel segments instead of one 16-byte piece per pixel and lane)
constexpr uint32_t kStageBytes = 4 * 32 * 64;
__host__ __device__ inline size_t smem_bytes(int mode, int NT, int cin, int ring, bool split = false, bool f8 = false) {
  const size_t unit = split ? row_bytes(mode, cin) / (cin * 2 / rb_of(cin)) : row_bytes(mode, cin);
  return 1024 + (b_bytes(mode, NT, cin) + (size_t)NT * (f8 ? 8 : 4) + kStageBytes + 1023) / 1024 * 1024 +
         (size_t)ring * unit + (size_t)(2 * ring + 4) * kBarBytes + 16;
}

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// Wait for the phase with the given parity to complete; false after `spin` cycles.  The
// common case (already complete) costs one try_wait.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long spin) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (clock64() - t0 > spin) return false;
  }
}
// Every lane of the warp waits (one shared-memory access per try for the warp); the result
// is made warp-uniform.
__device__ __forceinline__ bool mbar_wait_warp(uint32_t bar, uint32_t parity, long long spin) {
  return __all_sync(0xffffffffu, mbar_wait(bar, parity, spin));
}
// position in the ring of staged rows, advanced without division
struct RingPos {
  uint32_t slot = 0, pass = 0;  // pass = number of completed trips round the ring
  __device__ __forceinline__ void next(uint32_t ring) {
    if (++slot == ring) {
      slot = 0;
      ++pass;
    }
  }
};
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(bar), "r"(bytes)
               : "memory");
}
// 3-D TMA tile load (box: RB / 2 channels x staged pixels x 1 row) completing on `bar`.
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* tm, int c, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// L2 prefetch of a 3-D TMA box (no shared memory, no completion): a later load of the same
// box then finds it in L2.
__device__ __forceinline__ void tma_prefetch3(const CUtensorMap* tm, int c, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(c), "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void tensormap_acquire(const CUtensorMap* tm) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(reinterpret_cast<uint64_t>(tm)) : "memory");
}

// tcgen05 shared-memory matrix descriptors as two 32-bit words.  Low word: start address
// >> 4 (bits 0-13), leading byte offset >> 4 (bits 16-29).  High word: stride byte offset
// >> 4 (bits 0-13), version 1 (bit 14), base offset 0, layout (bits 29-31: 0 none,
// 2 128-byte swizzle, 4 64-byte, 6 32-byte).  The start field stays below 2^14 for any
// shared address (< 256 KB), so adding to the low word never carries into the LBO field.
__host__ __device__ constexpr uint32_t desc_lo(uint32_t addr, uint32_t lbo) { return (addr >> 4) | ((lbo >> 4) << 16); }
__host__ __device__ constexpr uint32_t desc_hi(uint32_t sbo, uint32_t layout) {
  return ((sbo >> 4) & 0x3FFFu) | (1u << 14) | (layout << 29);
}
__host__ __device__ constexpr uint32_t swz_layout(int rb) { return rb == 128 ? 2u : rb == 64 ? 4u : 6u; }

// MMA issue and commit, warp-wide: the whole warp runs the issue loop (its descriptors are
// warp-uniform values) and one lane, chosen by elect.sync, issues each instruction.
__device__ __forceinline__ void mma_bf16_elect(uint32_t tmem_d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                               uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .b64 da, db;\n .reg .pred p, e;\n .reg .b32 r;\n elect.sync r|e, 0xffffffff;\n"
      " mov.b64 da, {%1, %2};\n mov.b64 db, {%3, %4};\n setp.ne.b32 p, %6, 0;\n"
      " @e tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %5, p;\n}\n" ::"r"(tmem_d),
      "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc));
}
// The same with E4M3 A and B (kind::f8f6f4: K = 32 elements, the same 32 bytes per K step).
__device__ __forceinline__ void mma_f8_elect(uint32_t tmem_d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                             uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .b64 da, db;\n .reg .pred p, e;\n .reg .b32 r;\n elect.sync r|e, 0xffffffff;\n"
      " mov.b64 da, {%1, %2};\n mov.b64 db, {%3, %4};\n setp.ne.b32 p, %6, 0;\n"
      " @e tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], da, db, %5, p;\n}\n" ::"r"(tmem_d),
      "r"(alo), "r"(ahi), "r"(blo), "r"(bhi), "r"(idesc), "r"(acc));
}
template <bool F8>
__device__ __forceinline__ void mma_elect(uint32_t tmem_d, uint32_t alo, uint32_t ahi, uint32_t blo, uint32_t bhi,
                                          uint32_t idesc, uint32_t acc) {
  if constexpr (F8)
    mma_f8_elect(tmem_d, alo, ahi, blo, bhi, idesc, acc);
  else
    mma_bf16_elect(tmem_d, alo, ahi, blo, bhi, idesc, acc);
}
__device__ __forceinline__ void mma_commit_elect(uint32_t bar) {
  asm volatile(
      "{\n .reg .pred e;\n .reg .b32 r;\n elect.sync r|e, 0xffffffff;\n"
      " @e tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n}\n" ::"r"(bar)
      : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
      "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// tcgen05.ld of 32 columns without the wait: several loads in flight, then tmem_wait_ld()
__device__ __forceinline__ void tmem_ld32_nowait(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%"
      "20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// ------------------------------------------------------------------ geometry
// first input row staged for unit row i (phase row py for UP2)
template <int MODE>
__device__ __forceinline__ int first_row(int i, int py) {
  return MODE == TM_S2 ? 2 * i - 1 : MODE == TM_UP2 ? i + py - 1 : i;
}
// TMA x coordinate of the first staged pixel of set s (in that set's tensor map)
template <int MODE>
__device__ __forceinline__ int set_x0(int s, int j0, int px) {
  if (MODE == TM_S2) return s == 0 ? j0 - 1 : j0;  // odd pixels 2(j0+t)-1, even pixels 2(j0+t)
  if (MODE == TM_UP2) return j0 + px - 1;
  return j0;
}
// (staged row offset, pixel set, pixel start) of tap t
template <int MODE>
__device__ __forceinline__ void tap_geo(int t, int& row, int& set, int& col) {
  if (MODE == TM_S2) {
    row = t / 3;
    const int dx = t % 3;
    set = dx == 1 ? 1 : 0;
    col = dx == 2 ? 1 : 0;
  } else if (MODE == TM_UP2) {
    row = t >> 1;
    set = 0;
    col = t & 1;
  } else {
    row = 0;
    set = 0;
    col = 0;
  }
}

template <int MODE, int NT, int RB, bool SPLIT = false, bool F8 = false>
__global__ void __launch_bounds__(kThreads, 1) conv_tc_kernel(const __grid_constant__ Params p) {
  using G_ = Geo<MODE>;
  constexpr int RA = G_::RA, STEP = G_::STEP, T = G_::T, NSET = G_::NSET, NPX = G_::NPX;
  constexpr int KPR = RB / 32;                                 // 16-channel K steps per pixel row
  constexpr uint32_t KBS = (NPX * RB + 1023) / 1024 * 1024;    // channel-block stride
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const int cin = p.cin;
  const uint32_t ring = (uint32_t)p.ring;
  const int KB = cin * 2 / RB;  // channel blocks
  // ring units: whole rows, or (split) one channel block of a row, so that a row's first
  // blocks can be reloaded while its last ones are still read
  const int UPR = SPLIT ? KB : 1, KPU = KB / UPR;  // units per row, channel blocks per unit (KB or 1)
  const uint32_t unitb = NSET * KPU * KBS;
  const uint32_t sB = base;
  const uint32_t sBias = sB + (uint32_t)T * NT * cin * 2;
  const uint32_t sStage = sBias + NT * (F8 ? 8 : 4);  // 16-byte aligned (NT >= 16)
  const uint32_t sA = (sStage + kStageBytes + 1023u) & ~1023u;
  const uint32_t bars = sA + ring * unitb;
  const uint32_t full0 = bars, empty0 = bars + ring * 8, accf0 = bars + 2 * ring * 8, acce0 = accf0 + 16;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(gbase + (acce0 + 16 - base));
  const float* bias_s = reinterpret_cast<const float*>(gbase + (sBias - base));

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = blockIdx.x % p.G, crank = blockIdx.x / p.G, cpg = gridDim.x / p.G;
  const int phase = MODE == TM_UP2 ? (g & 3) : 0;
  const int nslice = MODE == TM_UP2 ? (g >> 2) : g;
  const int py = phase >> 1, px = phase & 1;
  const int n0 = nslice * NT;

  // ---- weights and bias of this CTA's set, resident for the kernel's lifetime
  {
    const uint4* src = reinterpret_cast<const uint4*>(p.wpack + (size_t)g * T * NT * cin);
    uint4* dst = reinterpret_cast<uint4*>(gbase);
    const int n16 = T * NT * cin / 8;
    for (int e = tid; e < n16; e += kThreads) dst[e] = src[e];
    float* bs = reinterpret_cast<float*>(gbase + (sBias - base));
    for (int e = tid; e < NT; e += kThreads) bs[e] = p.bias[n0 + e];
    if constexpr (F8)
      for (int e = tid; e < NT; e += kThreads) bs[NT + e] = p.scale[n0 + e];
  }
  if (tid == 0) {
    for (uint32_t r = 0; r < ring; ++r) {
      mbar_init(full0 + 8 * r, 1);
      mbar_init(empty0 + 8 * r, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, 4);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  constexpr uint32_t kCols = NT * 2 <= 32 ? 32 : NT * 2 <= 64 ? 64 : NT * 2 <= 128 ? 128 : NT * 2 <= 256 ? 256 : 512;
  if (warp == 4) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool ok = true;

  if (warp == 5) {
    // ------------------------------------------------------------ TMA producer (one thread)
    if (lane == 0) {
      const uint32_t unit_tx = (uint32_t)(NSET * KPU * NPX * RB);
      RingPos w;  // slot of the next unit to load; unit q goes to slot q % ring on pass q / ring
      uint32_t q = 0;
      int last_pair = -1;
      Strip nxt = crank < p.n_strips ? p.strips[crank] : Strip{};
      for (int s = crank; s < p.n_strips && ok; s += cpg) {
        const Strip st = nxt;
        if (s + cpg < p.n_strips) nxt = p.strips[s + cpg];  // in flight while this strip loads
        const LayerPair* L = p.lp + st.pair;
        if (st.pair != last_pair) {
          for (int k = 0; k < NSET; ++k) tensormap_acquire(&L->tm[k]);
          last_pair = st.pair;
        }
        const int nrows = STEP * (st.cnt - 1) + RA;
        const int y0 = first_row<MODE>(st.i0, py);
        for (int r = 0; r < nrows && ok; ++r)
          for (int u = 0; u < UPR; ++u, ++q, w.next(ring)) {
            // the slot's previous unit must have been consumed (pass > 0: released once)
            if (w.pass > 0 && !mbar_wait(empty0 + 8 * w.slot, (w.pass - 1) & 1, p.spin)) {
              atomicCAS(p.err, 0, 1);
              ok = false;
              break;
            }
            const uint32_t fb = full0 + 8 * w.slot;
            mbar_expect_tx(fb, unit_tx);
            const uint32_t dst0 = sA + w.slot * unitb;
            for (int k = 0; k < NSET; ++k) {
              const int x0 = set_x0<MODE>(k, st.j0, px);
              for (int kk = 0; kk < KPU; ++kk)
                tma_load3(dst0 + (k * KPU + kk) * KBS, &L->tm[k], (u * KPU + kk) * (RB / 2), x0, y0 + r, fb);
            }
          }
      }
      // no copy may still be writing shared memory when the CTA ends (also after a
      // timeout): wait for the most recent load of every slot
      const long long drain = p.spin > 2000000000LL ? p.spin : 2000000000LL;
      for (uint32_t k = 0; k < ring && k < q; ++k) {
        const uint32_t row = q - 1 - k;
        if (!mbar_wait(full0 + 8 * (row % ring), (row / ring) & 1, drain)) atomicCAS(p.err, 0, 5);
      }
    }
    __syncwarp();
  } else if (warp == 4) {
    // ------------------------------------------------------------ MMA issuer (the whole warp
    // runs the loop with warp-uniform descriptors; one elected lane issues each instruction)
    {
      // FP32 accumulator; A, B BF16 (format 1) or E4M3 (format 0); K-major; N; M = 128
      const uint32_t idesc = (1u << 4) | (F8 ? 0u : (1u << 7) | (1u << 10)) | ((uint32_t)(NT >> 3) << 17) |
                             ((128u >> 4) << 24);
      const uint32_t bsz = NT * cin * 2;
      // A: swizzled K-major pixel rows, SBO = 8 pixels (LBO unused: one swizzle span per
      // row); B: no-swizzle K-major core matrices, LBO = 128 B (next 8 channels), SBO =
      // 8 output channels x cin
      constexpr uint32_t a_hi = desc_hi(8 * RB, swz_layout(RB));
      const uint32_t b_hi = desc_hi((uint32_t)cin * 16, 0);
      // B descriptors (K step 0) of every tap: fixed for the CTA's lifetime
      uint32_t b0[T];
#pragma unroll
      for (int t = 0; t < T; ++t) b0[t] = desc_lo(sB + t * bsz, 128);
      uint32_t tseq = 0;
      RingPos wt;  // next unit to wait for (units are waited for in load order)
      RingPos tb;  // slot of the first unit of the current tile
      Strip nxt = crank < p.n_strips ? p.strips[crank] : Strip{};
      for (int s = crank; s < p.n_strips && ok; s += cpg) {
        const Strip st = nxt;
        if (s + cpg < p.n_strips) nxt = p.strips[s + cpg];
        int waited = 0;  // units of this strip waited for
        for (int ii = 0; ii < st.cnt && ok; ++ii) {
          const uint32_t buf = tseq & 1, use = tseq >> 1;
          const uint32_t dcol = tmem + buf * NT;
          const int nrel = ii + 1 < st.cnt ? STEP : RA;  // rows the strip's next tile no longer reads
          if (!SPLIT) {
            // whole-row units: the tile's rows, then one descriptor set for all channel blocks
            for (; waited < STEP * ii + RA; ++waited, wt.next(ring))
              if (!mbar_wait_warp(full0 + 8 * wt.slot, wt.pass & 1, p.spin)) {
                ok = false;
                break;
              }
            if (ok && use > 0 && !mbar_wait_warp(acce0 + 8 * buf, (use - 1) & 1, p.spin)) ok = false;
            if (ok) {
              tc_fence_after();
              // A descriptors (K step 0) of every tap for this tile's staged rows; all MMAs
              // of a channel block then issue back to back from independent additions
              uint32_t a0[T];
#pragma unroll
              for (int t = 0; t < T; ++t) {
                int ro, se, co;
                tap_geo<MODE>(t, ro, se, co);
                const uint32_t sl = tb.slot + (uint32_t)ro;
                a0[t] = desc_lo(sA + (sl >= ring ? sl - ring : sl) * unitb + (uint32_t)(se * KB) * KBS + (uint32_t)co * RB,
                                16);
              }
              // taps run in row order (T / RA taps per staged row); in the last channel block a
              // row the strip's next tile no longer reads goes back to the producer as soon as
              // the MMAs issued up to its last tap complete (a commit on its empty barrier), so
              // that its reload overlaps the rest of the tile's MMAs
              constexpr int TPR = T / RA;
              for (int kb = 0; kb < KB; ++kb) {
                const uint32_t ak = (uint32_t)kb * (KBS >> 4), bk = (uint32_t)kb * (16 * KPR);
#pragma unroll
                for (int t = 0; t < T; ++t) {
#pragma unroll
                  for (int k4 = 0; k4 < KPR; ++k4)
                    // next 16 channels: +32 B inside the swizzled pixel row, +256 B in B
                    mma_elect<F8>(dcol, a0[t] + ak + 2 * k4, a_hi, b0[t] + bk + 16 * k4, b_hi, idesc,
                                  (kb | t | k4) != 0 ? 1u : 0u);
                  if (kb == KB - 1 && (t + 1) % TPR == 0 && (t + 1) / TPR <= nrel) {
                    const uint32_t sl = tb.slot + (uint32_t)((t + 1) / TPR - 1);
                    mma_commit_elect(empty0 + 8 * (sl >= ring ? sl - ring : sl));
                  }
                }
              }
              mma_commit_elect(accf0 + 8 * buf);
            }
          }
          if (SPLIT && use > 0 && !mbar_wait_warp(acce0 + 8 * buf, (use - 1) & 1, p.spin)) ok = false;
          for (int kb = 0; SPLIT && kb < KB && ok; ++kb) {
            // channel-block units (KPU = 1): wait, issue and release block by block
            for (const int upto = (STEP * ii + RA - 1) * UPR + kb; waited <= upto; ++waited, wt.next(ring))
              if (!mbar_wait_warp(full0 + 8 * wt.slot, wt.pass & 1, p.spin)) {
                ok = false;
                break;
              }
            if (!ok) break;
            tc_fence_after();
            uint32_t a0[T];
#pragma unroll
            for (int t = 0; t < T; ++t) {
              int ro, se, co;
              tap_geo<MODE>(t, ro, se, co);
              const uint32_t sl = tb.slot + (uint32_t)(ro * UPR + kb);
              a0[t] = desc_lo(sA + (sl >= ring ? sl - ring : sl) * unitb + (uint32_t)se * KBS + (uint32_t)co * RB, 16);
            }
            const uint32_t bk = (uint32_t)kb * (16 * KPR);
#pragma unroll
            for (int t = 0; t < T; ++t)
#pragma unroll
              for (int k4 = 0; k4 < KPR; ++k4)
                mma_elect<F8>(dcol, a0[t] + 2 * k4, a_hi, b0[t] + bk + 16 * k4, b_hi, idesc, (kb | t | k4) != 0 ? 1u : 0u);
            // block kb of the rows the next tile no longer reads goes back to the producer
            for (int r = 0; r < nrel; ++r) {
              const uint32_t sl = tb.slot + (uint32_t)(r * UPR + kb);
              mma_commit_elect(empty0 + 8 * (sl >= ring ? sl - ring : sl));
            }
          }
          if (!ok) {
            if (lane == 0) atomicCAS(p.err, 0, 2);
            break;
          }
          if (SPLIT) mma_commit_elect(accf0 + 8 * buf);
          tb.slot += (uint32_t)(nrel * UPR);  // first unit of the next tile
          while (tb.slot >= ring) tb.slot -= ring;
          ++tseq;
        }
      }
      // drain, also after a timeout: the last commit arrives when every MMA issued by this
      // CTA has completed, so tensor memory is released only once nothing writes to it
      if (tseq > 0) {
        const uint32_t last = tseq - 1;
        const long long drain = p.spin > 2000000000LL ? p.spin : 2000000000LL;
        if (!mbar_wait_warp(accf0 + 8 * (last & 1), (last >> 1) & 1, drain) && lane == 0) atomicCAS(p.err, 0, 3);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (warps 0-3)
    const int m = warp * 32 + lane;
    uint32_t tseq = 0;
    for (int s = crank; s < p.n_strips && ok; s += cpg) {
      const Strip st = p.strips[s];
      const LayerPair* L = p.lp + st.pair;
      const int Hu = L->Hu, Wu = L->Wu, Ho = L->Ho, Wo = L->Wo;
      bf16* const out = L->out;
      for (int ii = 0; ii < st.cnt; ++ii, ++tseq) {
        const uint32_t buf = tseq & 1;
        // lane 0 waits for the accumulator and tells the warp (a warp-uniform decision)
        bool got = true;
        if (lane == 0) got = mbar_wait(accf0 + 8 * buf, (tseq >> 1) & 1, p.spin);
        got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
        if (!got) {
          if (lane == 0) atomicCAS(p.err, 0, 4);
          ok = false;
          break;
        }
        __syncwarp();  // orders the other lanes after lane 0's acquire of the barrier
        tc_fence_after();
        const int i = st.i0 + ii, j = st.j0 + m;
        const int oy = MODE == TM_UP2 ? 2 * i + py : i;
        const int ox = MODE == TM_UP2 ? 2 * j + px : j;
        const bool valid = i < Hu && j < Wu && oy < Ho && ox < Wo;
        bf16* op = out + ((size_t)oy * Wo + ox) * p.cout + n0;
        const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16) + buf * NT;
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += 32) {
          uint32_t r[32];
          if (NT >= 32) tmem_ld32(trow + c0, r);
          else tmem_ld16(trow + c0, r);
          constexpr int CW = NT >= 32 ? 32 : NT;
          const bool f8out = F8 && p.out_f8;  // warp-uniform
          if (f8out && CW == 32) {
            // E4M3 codes: relu(scale * acc + bias), 4 per word, through the warp's stage: lane =
            // pixel writes its two 16-byte pieces (piece q at slot q ^ ((pixel >> 2) & 1):
            // conflict-free), then two lanes per pixel store its 32 bytes, sixteen pixels per
            // instruction
            uint32_t packed[8];
#pragma unroll
            for (int e = 0; e < 32; e += 4) {
              float v[4];
#pragma unroll
              for (int q = 0; q < 4; ++q) {
                v[q] = fmaf(__uint_as_float(r[e + q]), bias_s[NT + c0 + e + q], bias_s[c0 + e + q]);
                if (p.relu) v[q] = fmaxf(v[q], 0.f);
              }
              const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[0], v[1]), __NV_SATFINITE, __NV_E4M3);
              const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[2], v[3]), __NV_SATFINITE, __NV_E4M3);
              packed[e / 4] = lo | (hi << 16);
            }
            uint4* sw = reinterpret_cast<uint4*>(gbase + (sStage - base)) + warp * 128;
#pragma unroll
            for (int q = 0; q < 2; ++q)
              sw[lane * 2 + (q ^ ((lane >> 2) & 1))] =
                  make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
            __syncwarp();
#pragma unroll
            for (int s16 = 0; s16 < 2; ++s16) {
              const int pp = 16 * s16 + (lane >> 1), q = lane & 1;
              const uint4 v = sw[pp * 2 + (q ^ ((pp >> 2) & 1))];
              const int jp = st.j0 + warp * 32 + pp;
              const int oxp = MODE == TM_UP2 ? 2 * jp + px : jp;
              if (i < Hu && jp < Wu && oy < Ho && oxp < Wo)
                *reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(out) + ((size_t)oy * Wo + oxp) * p.cout + n0 + c0 +
                                          16 * q) = v;
            }
            __syncwarp();
          } else if (f8out) {
            if (valid) {
              // E4M3 codes: relu(scale * acc + bias), 4 per word, 16 per 16-byte store
              uint32_t packed[CW / 4];
#pragma unroll
              for (int e = 0; e < CW; e += 4) {
                float v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                  v[q] = fmaf(__uint_as_float(r[e + q]), bias_s[NT + c0 + e + q], bias_s[c0 + e + q]);
                  if (p.relu) v[q] = fmaxf(v[q], 0.f);
                }
                const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(v[0], v[1]), __NV_SATFINITE, __NV_E4M3);
                const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(v[2], v[3]), __NV_SATFINITE, __NV_E4M3);
                packed[e / 4] = lo | (hi << 16);
              }
              uint8_t* ob = reinterpret_cast<uint8_t*>(out) + ((size_t)oy * Wo + ox) * p.cout + n0 + c0;
              if constexpr (CW >= 16) {
                uint4* dst = reinterpret_cast<uint4*>(ob);
#pragma unroll
                for (int v = 0; v < CW / 16; ++v)
                  dst[v] = make_uint4(packed[4 * v], packed[4 * v + 1], packed[4 * v + 2], packed[4 * v + 3]);
              }
            }
          } else {
            uint32_t packed[CW / 2];
#pragma unroll
            for (int e = 0; e < CW; e += 2) {
              float a = __uint_as_float(r[e]), b = __uint_as_float(r[e + 1]);
              if constexpr (F8) {
                a = fmaf(a, bias_s[NT + c0 + e], bias_s[c0 + e]);
                b = fmaf(b, bias_s[NT + c0 + e + 1], bias_s[c0 + e + 1]);
              } else {
                a += bias_s[c0 + e];
                b += bias_s[c0 + e + 1];
              }
              if (p.relu) {
                a = fmaxf(a, 0.f);
                b = fmaxf(b, 0.f);
              }
              __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
              packed[e / 2] = *reinterpret_cast<uint32_t*>(&h);
            }
            if constexpr (CW == 32) {
              // through the warp's stage: lane = pixel writes its four 16-byte pieces (piece
              // q at slot q ^ ((pixel >> 1) & 3): conflict-free), then four lanes per pixel
              // store its 64 bytes, eight pixels per instruction
              uint4* sw = reinterpret_cast<uint4*>(gbase + (sStage - base)) + warp * 128;
#pragma unroll
              for (int q = 0; q < 4; ++q)
                sw[lane * 4 + (q ^ ((lane >> 1) & 3))] =
                    make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
              __syncwarp();
#pragma unroll
              for (int s8 = 0; s8 < 4; ++s8) {
                const int pp = 8 * s8 + (lane >> 2), q = lane & 3;
                const uint4 v = sw[pp * 4 + (q ^ ((pp >> 1) & 3))];
                const int jp = st.j0 + warp * 32 + pp;
                const int oxp = MODE == TM_UP2 ? 2 * jp + px : jp;
                if (i < Hu && jp < Wu && oy < Ho && oxp < Wo)
                  *reinterpret_cast<uint4*>(out + ((size_t)oy * Wo + oxp) * p.cout + n0 + c0 + 8 * q) = v;
              }
              __syncwarp();
            } else if (valid) {
              uint4* dst = reinterpret_cast<uint4*>(op + c0);
#pragma unroll
              for (int v = 0; v < CW / 8; ++v)
                dst[v] = make_uint4(packed[4 * v], packed[4 * v + 1], packed[4 * v + 2], packed[4 * v + 3]);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce0 + 8 * buf);  // the warp's TMEM reads are complete
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 4) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// ------------------------------------------------------------------ fused dec3 + final
// The last decoder layer (nearest x2 + crop + 3x3 conv + ReLU), the final 3x3 conv to one
// channel and the residual onto U in one kernel, so that d3 never leaves the SM.  A CTA
// computes all four output phases of 128 input pixels of one row per tile (one MMA per
// staged view and K step, the phases reading the view stacked along N: 10 MMAs per K step
// into four TMEM accumulators, see fused_view) and writes the two resulting d3 rows (BF16,
// 256 columns) into shared memory, in the swizzled K-major layout of an MMA operand.  The
// final conv runs on the tensor cores as well: with a d3 row as A (M = 128 columns, K = the
// d3 channels) and one B holding all nine taps' weights (N = 32: each weight split into a
// BF16 high part and a BF16 low part, hi + lo = w to about 2^-16 relative), one MMA pass
// per row and column half gives every pixel's nine tap products P_r(x, ky, kx).  The
// epilogue adds them: out(y, x) = sum over (ky, kx) of P_{y+ky-1}(x+kx-1, ky, kx), the kx
// shifts by warp shuffles, the ky rows through two partial sums per column carried from
// tile to tile, so that tile i (d3 rows 2i, 2i + 1) completes output rows 2i - 1 and 2i.
// Column strips step by 127 input pixels (tile = input pixels j0 .. j0 + 127 with
// j0 = 127 s - 1), so each strip's 254 final columns 2 j0 + 1 .. 2 j0 + 254 have both
// neighbours in the tile; a strip starts with one halo tile above its first row (none at
// row 0, where the carried sums start at zero: the padding above).  d3 outside the output
// is stored as zero (the final conv's padding), and the rows below an even-height output
// are zero, so the carried sum of the last row is complete after the last tile.  An odd
// output height crops half of the last up-sampled row: the last tile's phase-0 rows then
// subtract the kernel row that falls on the cropped half (4 extra MMA groups with B
// negated, reusing phase-1 blocks), which gives the cropped conv.  Odd output widths are not
// handled here.
struct alignas(128) FusedPair {
  float* Y;                    // refined disparity [Ho][Wo]
  const int16_t* coarse;       // coarse map [h4][w4]
  int Hu, Wu, Ho, Wo, w4, h4;  // input (d2) rows / cols, output size, coarse-map size
  int pad[4];
  CUtensorMap tm;              // TMA view of d2 (box: cin channels x 130 pixels x 1 row)
};

struct FusedParams {
  const FusedPair* fp;
  const Strip* strips;
  int n_strips;
  const bf16* wpack;  // [16][NT x cin] decoder blocks, then the final conv's [32 x NT] block
  const float* bias;  // [NT] decoder bias
  const float* bf;    // final bias
  int ring;
  int pf;             // rows the producer prefetches into L2 ahead of the row it loads
  int* err;
  long long spin;
};

constexpr int kFusedNpx = 130;
constexpr int kFinalN = 32;  // final conv MMA width: 9 high parts, 9 low parts, 14 zero rows
__host__ __device__ inline uint32_t fused_kbs(int rb) { return (uint32_t)((kFusedNpx * rb + 1023) / 1024 * 1024); }
__host__ __device__ inline size_t fused_wpack_elems(int NT, int cin) {
  return (size_t)16 * NT * cin + (size_t)kFinalN * NT;
}
// decoder bias [NT], final bias (+ 3 pad), tap-sum exchange [2 parities][8 warps][2 sides][8]
__host__ __device__ inline size_t fused_param_bytes(int NT) { return (size_t)(NT + 4 + 256) * 4; }
__host__ __device__ inline size_t fused_smem_bytes(int NT, int cin, int ring) {
  const size_t head = (fused_wpack_elems(NT, cin) * 2 + fused_param_bytes(NT) + 1023) / 1024 * 1024;
  return 1024 + head + (size_t)ring * fused_kbs(cin * 2) + (size_t)4 * 256 * NT * 2 + (size_t)(2 * ring + 8) * 8 + 16;
}

// 320 threads: warps 0-7 epilogue, warp 8 TMEM allocation + MMA issue, warp 9 TMA.
constexpr int kFusedThreads = 320, kFusedEpi = 256;
// Named barrier 1 over the 256 epilogue threads (warps 0-7) only; the producer and MMA warps
// never take part.
__device__ __forceinline__ void named_sync_epi() { asm volatile("bar.sync 1, 256;" ::: "memory"); }
// Same barrier with an OR over the 256 threads' predicates.
__device__ __forceinline__ bool epi_any(bool v) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)v)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void tmem_ld2_nowait(uint32_t taddr, uint32_t& a, uint32_t& b) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(a), "=r"(b) : "r"(taddr));
}

// Instruction descriptor: BF16 A and B, FP32 accumulator, K-major, M = 128, width N.
__host__ __device__ constexpr uint32_t idesc_n(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
}
// The 16 (phase, tap) products of a tile read 9 distinct views of the staged rows: phase
// (py, px) with tap (ro, co) reads staged row py + ro at pixel shift px + co.  Each view is
// one MMA whose N stacks the phases reading it, so the accumulators of those phases must be
// adjacent in TMEM: blocks (units of NT columns) 0: (0, 0), 1: (0, 1), 2: (1, 1), 3: (1, 0).
// The four phases form the cycle (0,0)-(0,1)-(1,1)-(1,0)-(0,0) under "share a view"; the
// view (1, 0), shared by (1, 0) and (0, 0), closes it and is issued as two MMAs: 10 MMAs
// per K step.  A view's weights are `nb` consecutive packed blocks starting at `blk`
// (pack_fused_kernel writes them in this order); `col` is its first accumulator block.
// (The issue loops are unrolled, so every call below folds to constants.)
struct FusedView {
  int r, s, blk, nb, col;
};
constexpr int kFusedViewMMAs = 10;
__host__ __device__ constexpr FusedView fused_view(int v) {
  switch (v) {
    case 0: return {1, 1, 0, 4, 0};   // (0,0) t(1,1), (0,1) t(1,0), (1,1) t(0,0), (1,0) t(0,1)
    case 1: return {0, 1, 4, 2, 0};   // (0,0) t(0,1), (0,1) t(0,0)
    case 2: return {2, 1, 6, 2, 2};   // (1,1) t(1,0), (1,0) t(1,1)
    case 3: return {1, 2, 8, 2, 1};   // (0,1) t(1,1), (1,1) t(0,1)
    case 4: return {1, 0, 10, 1, 3};  // (1,0) t(0,0)
    case 5: return {1, 0, 11, 1, 0};  // (0,0) t(1,0)
    case 6: return {0, 0, 12, 1, 0};  // (0,0) t(0,0)
    case 7: return {0, 2, 13, 1, 1};  // (0,1) t(0,1)
    case 8: return {2, 0, 14, 1, 3};  // (1,0) t(1,0)
    default: return {2, 2, 15, 1, 2};  // (1,1) t(1,1)
  }
}
// Odd output height, last tile: the taps (ro = 1) of phases (0, px) hold kernel rows 1 + 2;
// row 2 falls on the cropped-away up-sampled row.  It is subtracted with the block of phase
// (1, px), tap (1, co), which holds kernel row 2 alone with the same column folding.
__host__ __device__ constexpr FusedView fused_crop_view(int v) {
  switch (v) {
    case 0: return {1, 0, 14, 1, 0};  // (0,0) t(1,0) - row 2 of (1,0) t(1,0)
    case 1: return {1, 1, 7, 1, 0};   // (0,0) t(1,1) - row 2 of (1,0) t(1,1)
    case 2: return {1, 1, 6, 1, 1};   // (0,1) t(1,0) - row 2 of (1,1) t(1,0)
    default: return {1, 2, 15, 1, 1};  // (0,1) t(1,1) - row 2 of (1,1) t(1,1)
  }
}
// packed block -> phase 2 py + px (high digit) and tap 2 ro + co (low digit), in the
// order of fused_view
__host__ __device__ constexpr int fused_block_pt(int blk) {
  constexpr int pt[16] = {3, 12, 30, 21, 1, 10, 32, 23, 13, 31, 20, 2, 0, 11, 22, 33};
  return pt[blk];
}

template <int NT, int RB>
__global__ void __launch_bounds__(kFusedThreads, 1) dec3f_kernel(const __grid_constant__ FusedParams p) {
  constexpr int RA = 3, KPR = RB / 32, CIN = RB / 2;
  constexpr uint32_t KBS = (kFusedNpx * RB + 1023) / 1024 * 1024;
  constexpr int NCH = NT / 8;                                  // 16-byte chunks per d3 pixel
  constexpr int SWS = NCH == 4 ? 1 : 2;                        // d3 chunk swizzle: col >> SWS
  constexpr uint32_t PXB = NT * 2;                             // bytes per d3 pixel
  constexpr uint32_t BBLK = NT * CIN * 2;                      // one (phase, tap) weight block
  constexpr int FKS = NT / 16;                                 // K steps of the final conv
  constexpr uint32_t kCols = 512;                              // 2 x 4 x NT accumulators + 2 x 128 partials
  constexpr uint32_t FCOL = 8 * NT;                            // first TMEM column of the final partials
  static_assert(NT == 16 || NT == 32, "fused decoder widths");
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  unsigned char* gbase = smem_raw + (base - raw);
  const uint32_t ring = (uint32_t)p.ring;
  const uint32_t sB = base;
  const uint32_t sF = sB + 16 * BBLK;                          // final conv B [32 x NT]
  const uint32_t sPar = sF + kFinalN * NT * 2;
  const uint32_t sA = (sPar + (uint32_t)fused_param_bytes(NT) + 1023u) & ~1023u;
  const uint32_t sD = sA + ring * KBS;                         // d3 rows [4][256][NCH] x 16 B
  const uint32_t bars = sD + 4 * 256 * PXB;
  const uint32_t full0 = bars, empty0 = bars + ring * 8, accf0 = bars + 2 * ring * 8, acce0 = accf0 + 16;
  const uint32_t finf0 = acce0 + 16, fine0 = finf0 + 16;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(gbase + (fine0 + 16 - base));
  float* bias_s = reinterpret_cast<float*>(gbase + (sPar - base));
  float* bf_s = bias_s + NT;
  float* edge_s = bias_s + NT + 4;
  uint4* d3r = reinterpret_cast<uint4*>(gbase + (sD - base));
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int crank = blockIdx.x, cpg = gridDim.x;

  {
    const uint4* src = reinterpret_cast<const uint4*>(p.wpack);
    uint4* dst = reinterpret_cast<uint4*>(gbase);
    for (int e = tid; e < (int)((16 * BBLK + kFinalN * NT * 2) / 16); e += kFusedThreads) dst[e] = src[e];
    for (int e = tid; e < NT; e += kFusedThreads) bias_s[e] = p.bias[e];
    if (tid == 0) bf_s[0] = p.bf[0];
  }
  if (tid == 0) {
    for (uint32_t r = 0; r < ring; ++r) {
      mbar_init(full0 + 8 * r, 1);
      mbar_init(empty0 + 8 * r, 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(accf0 + 8 * b, 1);
      mbar_init(acce0 + 8 * b, kFusedEpi / 32);  // one arrival per epilogue warp
      mbar_init(finf0 + 8 * b, 1);
      mbar_init(fine0 + 8 * b, kFusedEpi / 32);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  bool ok = true;

  if (warp == 9) {
    // ------------------------------------------------------------ TMA producer (one thread)
    if (lane == 0) {
      const uint32_t row_tx = (uint32_t)(kFusedNpx * RB);
      RingPos w;
      uint32_t q = 0;
      int last_pair = -1;
      for (int s = crank; s < p.n_strips && ok; s += cpg) {
        const Strip st = p.strips[s];
        const FusedPair* F = p.fp + st.pair;
        if (st.pair != last_pair) {
          tensormap_acquire(&F->tm);
          last_pair = st.pair;
        }
        const int first = st.i0 > 0 ? st.i0 - 1 : st.i0;
        const int nrows = (st.i0 + st.cnt - first) - 1 + RA;
        const int Hu = F->Hu;
        for (int r = 0; r < nrows; ++r, ++q, w.next(ring)) {
          if (w.pass > 0 && !mbar_wait(empty0 + 8 * w.slot, (w.pass - 1) & 1, p.spin)) {
            atomicCAS(p.err, 0, 1);
            ok = false;
            break;
          }
          const uint32_t fb = full0 + 8 * w.slot;
          mbar_expect_tx(fb, row_tx);
          tma_load3(sA + w.slot * KBS, &F->tm, 0, st.j0 - 1, first - 1 + r, fb);
          const int yp = first - 1 + r + p.pf;  // L2 prefetch (inside the image, x clamped at 0)
          if (p.pf > 0 && r + p.pf < nrows && yp >= 0 && yp < Hu) tma_prefetch3(&F->tm, 0, st.j0 > 1 ? st.j0 - 1 : 0, yp);
        }
      }
      const long long drain = p.spin > 2000000000LL ? p.spin : 2000000000LL;
      for (uint32_t k = 0; k < ring && k < q; ++k) {
        const uint32_t row = q - 1 - k;
        if (!mbar_wait(full0 + 8 * (row % ring), (row / ring) & 1, drain)) atomicCAS(p.err, 0, 5);
      }
    }
    __syncwarp();
  } else if (warp == 8) {
    // ------------------------------------------------------------ MMA issuer (the whole warp
    // runs the loop with warp-uniform descriptors; one elected lane issues each instruction)
    {
      const uint32_t fdesc = idesc_n(kFinalN);
      constexpr uint32_t a_hi = desc_hi(8 * RB, swz_layout(RB));
      constexpr uint32_t b_hi = desc_hi((uint32_t)CIN * 16, 0);
      constexpr uint32_t fa_hi = desc_hi(8 * PXB, swz_layout(PXB));  // d3 rows: swizzled K-major
      constexpr uint32_t fb_hi = desc_hi((uint32_t)NT * 16, 0);
      const uint32_t fb0 = desc_lo(sF, 128);
      uint32_t tseq = 0, fseq = 0;
      RingPos wt, tb;
      // Final conv MMAs of the tile with sequence number fseq and image row i (d3 rows 2i and
      // 2i + 1): waits until the epilogue has written those rows (the same arrival that frees
      // the tile's accumulators) and has read out the partial-sum buffer's previous use.
      auto issue_final = [&](int i) -> bool {
        const uint32_t b = fseq & 1, use = fseq >> 1;
        if (!mbar_wait_warp(acce0 + 8 * b, use & 1, p.spin)) return false;
        if (use > 0 && !mbar_wait_warp(fine0 + 8 * b, (use - 1) & 1, p.spin)) return false;
        tc_fence_after();
#pragma unroll
        for (int rho = 0; rho < 2; ++rho)
#pragma unroll
          for (int mu = 0; mu < 2; ++mu) {
            const uint32_t a0 = desc_lo(sD + ((uint32_t)((2 * i + rho) & 3) * 256u + 128u * mu) * PXB, 16);
            const uint32_t d = tmem + FCOL + b * 128 + 32 * (2 * rho + mu);
#pragma unroll
            for (int ks = 0; ks < FKS; ++ks)
              mma_bf16_elect(d, a0 + 2 * ks, fa_hi, fb0 + 16 * ks, fb_hi, fdesc, ks != 0 ? 1u : 0u);
          }
        mma_commit_elect(finf0 + 8 * b);
        ++fseq;
        return true;
      };
      for (int s = crank; s < p.n_strips && ok; s += cpg) {
        const Strip st = p.strips[s];
        const FusedPair* F = p.fp + st.pair;
        const int Hu = F->Hu, Ho = F->Ho;
        const int first = st.i0 > 0 ? st.i0 - 1 : st.i0;
        const int ntiles = st.i0 + st.cnt - first;
        for (int k = 0; k < ntiles && ok; ++k) {
          const int rlo = k == 0 ? 0 : k - 1 + RA;
          for (int r = rlo; r < k + RA; ++r, wt.next(ring)) {
            if (!mbar_wait_warp(full0 + 8 * wt.slot, wt.pass & 1, p.spin)) {
              ok = false;
              break;
            }
          }
          const uint32_t buf = tseq & 1, use = tseq >> 1;
          if (ok && use > 0 && !mbar_wait_warp(acce0 + 8 * buf, (use - 1) & 1, p.spin)) ok = false;
          if (!ok) {
            if (lane == 0) atomicCAS(p.err, 0, 2);
            break;
          }
          tc_fence_after();
          uint32_t slot_of_row[RA];
#pragma unroll
          for (int r = 0; r < RA; ++r) {
            const uint32_t sl = tb.slot + r;
            slot_of_row[r] = sA + (sl >= ring ? sl - ring : sl) * KBS;
          }
          const bool crop_row = (first + k == Hu - 1) && (Ho & 1);  // odd height: last row's py = 0
          // One MMA per staged view (row r, pixel shift s) and K step, N = the phases that
          // read that view stacked (fused_view); the first view (all four phases)
          // initialises the accumulators.  The crop case then subtracts the kernel row that
          // falls on the cropped-away half (B negated through the instruction descriptor).
          const uint32_t dbase = tmem + buf * (4 * NT);
#pragma unroll
          for (int v = 0; v < kFusedViewMMAs; ++v) {
            const FusedView fv = fused_view(v);
            const uint32_t a0 = desc_lo(slot_of_row[fv.r] + (uint32_t)fv.s * RB, 16);
            const uint32_t b0 = desc_lo(sB + (uint32_t)fv.blk * BBLK, 128);
            const uint32_t vdesc = idesc_n(NT * fv.nb);
#pragma unroll
            for (int k4 = 0; k4 < KPR; ++k4)
              mma_bf16_elect(dbase + fv.col * NT, a0 + 2 * k4, a_hi, b0 + 16 * k4, b_hi, vdesc, (v != 0 || k4 != 0) ? 1u : 0u);
          }
          if (crop_row) {
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const FusedView fv = fused_crop_view(v);
              const uint32_t a0 = desc_lo(slot_of_row[fv.r] + (uint32_t)fv.s * RB, 16);
              const uint32_t b0 = desc_lo(sB + (uint32_t)fv.blk * BBLK, 128);
#pragma unroll
              for (int k4 = 0; k4 < KPR; ++k4)
                mma_bf16_elect(dbase + fv.col * NT, a0 + 2 * k4, a_hi, b0 + 16 * k4, b_hi, idesc_n(NT) | (1u << 14), 1u);
            }
          }
          mma_commit_elect(accf0 + 8 * buf);
          // rows no later tile of the strip reads go back to the producer when these MMAs
          // complete (one commit per row on its empty barrier)
          {
            const int nrel = k + 1 < ntiles ? 1 : RA;
            for (int r = 0; r < nrel; ++r) {
              const uint32_t sl = tb.slot + r;
              mma_commit_elect(empty0 + 8 * (sl >= ring ? sl - ring : sl));
            }
          }
          tb.slot += 1;
          if (k + 1 == ntiles) tb.slot += RA - 1;
          while (tb.slot >= ring) tb.slot -= ring;
          ++tseq;
          // the previous tile's final conv runs while this tile's decoder MMAs are queued
          if (k > 0 && !issue_final(first + k - 1)) {
            if (lane == 0) atomicCAS(p.err, 0, 2);
            ok = false;
          }
        }
        if (ok && ntiles > 0 && !issue_final(first + ntiles - 1)) {
          if (lane == 0) atomicCAS(p.err, 0, 2);
          ok = false;
        }
      }
      const long long drain = p.spin > 2000000000LL ? p.spin : 2000000000LL;
      if (tseq > 0) {
        const uint32_t last = tseq - 1;
        if (!mbar_wait_warp(accf0 + 8 * (last & 1), (last >> 1) & 1, drain) && lane == 0) atomicCAS(p.err, 0, 3);
      }
      if (fseq > 0) {
        const uint32_t last = fseq - 1;
        if (!mbar_wait_warp(finf0 + 8 * (last & 1), (last >> 1) & 1, drain) && lane == 0) atomicCAS(p.err, 0, 3);
      }
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue (warps 0-7)
    // Decoder part: warps 0-3 convert phases (0, 0), (0, 1) (d3 row 2i), warps 4-7 phases
    // (1, 0), (1, 1) (row 2i + 1); TMEM lane quarter = warp % 4.  Final part: thread tid owns
    // local d3 column tid (TMEM lane tid % 128 of column half tid / 128), so warp w holds
    // columns 32 w .. 32 w + 31.
    const int m = tid & 127;  // input pixel j0 + m of the tile / TMEM lane
    const int grp = tid >> 7;
    uint32_t tseq = 0, fseq = 0;
    auto ring_at = [&](int y, int col, int q) -> uint4* {  // row y (any integer), local column col
      return d3r + (((uint32_t)y & 3u) * 256u + (uint32_t)col) * NCH + (uint32_t)(q ^ ((col >> SWS) & (NCH - 1)));
    };
    // residual U at output row Yr, column X: the four raw coarse values around it and the
    // bilinear fractions (loads only; interpolated at the store)
    auto coarse4 = [](const int16_t* cmap, int w4, int h4, int X, int Yr, int16_t (&cv)[4], float& fx, float& fy) {
      float sx = (float)X * 0.25f - 0.375f;
      sx = fminf(fmaxf(sx, 0.f), (float)(w4 - 1));
      const int x0 = (int)sx, x1 = min(x0 + 1, w4 - 1);
      float sy = (float)Yr * 0.25f - 0.375f;
      sy = fminf(fmaxf(sy, 0.f), (float)(h4 - 1));
      const int y0 = (int)sy, y1 = min(y0 + 1, h4 - 1);
      const int16_t* c0p = cmap + (size_t)y0 * w4;
      const int16_t* c1p = cmap + (size_t)y1 * w4;
      cv[0] = __ldg(c0p + x0);
      cv[1] = __ldg(c0p + x1);
      cv[2] = __ldg(c1p + x0);
      cv[3] = __ldg(c1p + x1);
      fx = sx - (float)x0;
      fy = sy - (float)y0;
    };
    auto residual = [](const int16_t (&cv)[4], float fx, float fy) {
      const float top = (1.f - fx) * (float)cv[0] + fx * (float)cv[1];
      const float bot = (1.f - fx) * (float)cv[2] + fx * (float)cv[3];
      return 4.f * ((1.f - fy) * top + fy * bot);
    };
    for (int s = crank; s < p.n_strips && ok; s += cpg) {
      const Strip st = p.strips[s];
      const FusedPair* F = p.fp + st.pair;
      const int Hu = F->Hu, Wu = F->Wu, Ho = F->Ho, Wo = F->Wo;
      const int j0 = st.j0;
      const int first = st.i0 > 0 ? st.i0 - 1 : st.i0;
      const int ntiles = st.i0 + st.cnt - first;
      const bool below = st.i0 + st.cnt == Hu && Ho == 2 * Hu;  // zero rows under the last row
      const int16_t* cmap = F->coarse;
      float* Yout = F->Y;
      const int w4 = F->w4, h4 = F->h4;
      const int X = 2 * j0 + tid;                                // this thread's output column
      const bool col_out = tid >= 1 && tid <= 254 && X >= 0 && X < Wo;
      float c1 = 0.f, c2 = 0.f;  // carried partial sums of output rows 2i + 1 and 2i + 2
      // raw coarse values of the residual U for the rows finished in the next iteration,
      // loaded one iteration ahead so that their latency is hidden
      int16_t cv[2][4] = {}, cvn[2][4] = {};
      float fxy[2][2] = {}, fxyn[2][2] = {};
      for (int k = 0; k <= ntiles; ++k) {
        const int i = first + k;
        if (k < ntiles && col_out) {
          // iteration k + 1 finishes rows 2 (i + 1) - 3 and 2 (i + 1) - 2
#pragma unroll
          for (int r = 0; r < 2; ++r)
            coarse4(cmap, w4, h4, X, min(max(2 * i - 1 + r, 0), Ho - 1), cvn[r], fxyn[r][0], fxyn[r][1]);
        }
        if (k < ntiles) {
          const uint32_t buf = tseq & 1;
          // lane 0 of each warp waits; the OR below makes the decision uniform
          const bool got = lane != 0 || mbar_wait(accf0 + 8 * buf, (tseq >> 1) & 1, p.spin);
          // all epilogue threads take the same decision, so none is left waiting at a
          // named barrier
          if (epi_any(!got)) {
            if (tid == 0) atomicCAS(p.err, 0, 4);
            ok = false;
            break;
          }
          tc_fence_after();
          // accumulator blocks (units of NT columns): phase (0, 0) = 0, (0, 1) = 1, (1, 1) = 2,
          // (1, 0) = 3; this group's phases (grp, 0), (grp, 1)
          const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + buf * (4 * NT);
          const uint32_t c0 = grp == 0 ? 0u : 3u * NT, c1 = grp == 0 ? (uint32_t)NT : 2u * NT;
          uint32_t rr[2][32];
          if (NT == 32) {
            tmem_ld32_nowait(trow + c0, rr[0]);
            tmem_ld32_nowait(trow + c1, rr[1]);
          } else {
            tmem_ld16_nowait(trow + c0, rr[0]);
            tmem_ld16_nowait(trow + c1, rr[1]);
          }
          tmem_wait_ld();
          const int oy = 2 * i + grp;
          // lanes m and m ^ 4 store the two columns of a pixel pair in opposite order, so that
          // each group of eight lanes fills both halves of a 128-byte bank row (with the
          // chunk swizzle q ^ (m & 3): eight distinct 16-byte slots, no bank conflict)
          const int sw = (m >> 2) & 1;
#pragma unroll
          for (int q = 0; q < NCH; ++q) {
            const float4 bl = *reinterpret_cast<const float4*>(bias_s + q * 8);
            const float4 bh = *reinterpret_cast<const float4*>(bias_s + q * 8 + 4);
            const float2 bv[4] = {make_float2(bl.x, bl.y), make_float2(bl.z, bl.w), make_float2(bh.x, bh.y),
                                  make_float2(bh.z, bh.w)};
            uint4 pk[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int ox = 2 * (j0 + m) + h;
              // outside the output: the final conv's zero padding
              const bool valid = oy < Ho && ox >= 0 && ox < Wo && j0 + m < Wu;
              uint32_t w4[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const int c0 = q * 8 + 2 * e;
                // bias (packed add), BF16 rounding, then ReLU on the pair: rounding to
                // nearest commutes with max(., 0)
                const float2 v = __fadd2_rn(make_float2(__uint_as_float(rr[h][c0]), __uint_as_float(rr[h][c0 + 1])), bv[e]);
                const __nv_bfloat162 hh = __hmax2(__floats2bfloat162_rn(v.x, v.y), __float2bfloat162_rn(0.f));
                w4[e] = valid ? *reinterpret_cast<const uint32_t*>(&hh) : 0u;
              }
              pk[h] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
            }
#pragma unroll
            for (int b = 0; b < 2; ++b) {
              const int px = sw ^ b;
              *ring_at(oy, 2 * m + px, q) = px ? pk[1] : pk[0];
            }
          }
          // the d3 rows are read by the tensor cores next: generic-proxy writes made visible
          // to the async proxy before the warp's arrival
          fence_proxy_async();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acce0 + 8 * buf);  // TMEM read out, d3 rows written
          ++tseq;
        }
        if (k > 0) {
          // final conv of the previous tile (image row ip, d3 rows 2 ip and 2 ip + 1)
          const int ip = i - 1;
          const uint32_t fb = fseq & 1;
          const bool got = lane != 0 || mbar_wait(finf0 + 8 * fb, (fseq >> 1) & 1, p.spin);
          if (epi_any(!got)) {
            if (tid == 0) atomicCAS(p.err, 0, 4);
            ok = false;
            break;
          }
          tc_fence_after();
          uint32_t q0[32], q1[32];
          const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + FCOL + fb * 128 + 32 * grp;
          tmem_ld16_nowait(taddr, q0);
          tmem_ld2_nowait(taddr + 16, q0[16], q0[17]);
          tmem_ld16_nowait(taddr + 64, q1);
          tmem_ld2_nowait(taddr + 64 + 16, q1[16], q1[17]);
          tmem_wait_ld();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(fine0 + 8 * fb);  // partial-sum buffer read out
          // d3 row r adds S_0 to output row r + 1, S_1 to row r, S_2 to row r - 1, with
          // S_ky(x) = P_r(x - 1, ky, 0) + P_r(x, ky, 1) + P_r(x + 1, ky, 2).  The four sums
          // this tile contributes to (rows 2 ip - 1 .. 2 ip + 2, from d3 rows 2 ip and 2 ip + 1)
          // are formed per kx first, so that only 4 values cross to each neighbour.
          // tap products: high part + low part of the weights
          const auto p0 = [&](int t) { return __uint_as_float(q0[t]) + __uint_as_float(q0[t + 9]); };
          const auto p1 = [&](int t) { return __uint_as_float(q1[t]) + __uint_as_float(q1[t + 9]); };
          float part[3][4];  // [kx][row 2 ip - 1 + i]
#pragma unroll
          for (int kx = 0; kx < 3; ++kx) {
            part[kx][0] = p0(6 + kx);
            part[kx][1] = p0(3 + kx) + p1(6 + kx);
            part[kx][2] = p0(kx) + p1(3 + kx);
            part[kx][3] = p1(kx);
          }
          // kx = 0 parts go to the right neighbour, kx = 2 parts to the left one; lanes 0
          // and 31 exchange with the neighbouring warps through shared memory
          float* eb = edge_s + (fseq & 1) * 128;
          if (lane == 31) *reinterpret_cast<float4*>(eb + (warp * 2 + 0) * 8) = make_float4(part[0][0], part[0][1], part[0][2], part[0][3]);
          if (lane == 0) *reinterpret_cast<float4*>(eb + (warp * 2 + 1) * 8) = make_float4(part[2][0], part[2][1], part[2][2], part[2][3]);
          named_sync_epi();
          float4 le = make_float4(0.f, 0.f, 0.f, 0.f), re = make_float4(0.f, 0.f, 0.f, 0.f);
          if (lane == 0 && warp > 0) le = *reinterpret_cast<const float4*>(eb + ((warp - 1) * 2 + 0) * 8);
          if (lane == 31 && warp < 7) re = *reinterpret_cast<const float4*>(eb + ((warp + 1) * 2 + 1) * 8);
          const float lev[4] = {le.x, le.y, le.z, le.w}, rev[4] = {re.x, re.y, re.z, re.w};
          float Tsum[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            float l = __shfl_up_sync(0xffffffffu, part[0][i], 1);
            float r = __shfl_down_sync(0xffffffffu, part[2][i], 1);
            if (lane == 0) l = lev[i];
            if (lane == 31) r = rev[i];
            Tsum[i] = l + part[1][i] + r;
          }
          const float outA = c1 + Tsum[0];  // row 2 ip - 1: complete
          const float outB = c2 + Tsum[1];  // row 2 ip: complete
          c1 = Tsum[2];                     // row 2 ip + 1
          c2 = Tsum[3];                     // row 2 ip + 2
          ++fseq;
          if (ip >= st.i0 && col_out) {
            const float b = bf_s[0];
            const int yA = 2 * ip - 1, yB = 2 * ip;
            if (yA >= 0 && yA < Ho) Yout[(size_t)yA * Wo + X] = residual(cv[0], fxy[0][0], fxy[0][1]) + (b + outA);
            if (yB < Ho) Yout[(size_t)yB * Wo + X] = residual(cv[1], fxy[1][0], fxy[1][1]) + (b + outB);
          }
        }
#pragma unroll
        for (int r = 0; r < 2; ++r) {
#pragma unroll
          for (int e = 0; e < 4; ++e) cv[r][e] = cvn[r][e];
          fxy[r][0] = fxyn[r][0];
          fxy[r][1] = fxyn[r][1];
        }
      }
      if (ok && below && col_out) {
        // last output row 2 Hu - 1: its rows below (2 Hu, 2 Hu + 1) are zero
        int16_t cc[4];
        float fx, fy;
        const int yC = 2 * Hu - 1;
        coarse4(cmap, w4, h4, X, yC, cc, fx, fy);
        Yout[(size_t)yC * Wo + X] = residual(cc, fx, fy) + (bf_s[0] + c1);
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 8) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

// ------------------------------------------------------------------ weight packing
// Value the tensor-core form multiplies for output channel co, input channel k and tap t
// (phase ph of an up-sampling layer): the weight itself (stride-2, 1 x 1), or the sum of the
// 3 x 3 weights the phase folds onto the tap (rows / columns {0} and {1, 2} for phase 0,
// {0, 1} and {2} for phase 1), summed in FP32 in row-major tap order.
__device__ __forceinline__ float tc_weight(const float* __restrict__ W, int mode, int ph, int t, int co, int k, int cin) {
  if (mode == TM_P1) return W[(size_t)co * cin + k];
  if (mode == TM_S2) return W[((size_t)co * 9 + t) * cin + k];
  const int py = ph >> 1, px = ph & 1, a = t >> 1, b = t & 1;
  const int ky0 = py == 0 ? (a == 0 ? 0 : 1) : (a == 0 ? 0 : 2);
  const int ky1 = py == 0 ? (a == 0 ? 0 : 2) : (a == 0 ? 1 : 2);
  const int kx0 = px == 0 ? (b == 0 ? 0 : 1) : (b == 0 ? 0 : 2);
  const int kx1 = px == 0 ? (b == 0 ? 0 : 2) : (b == 0 ? 1 : 2);
  float v = 0.f;
  for (int ky = ky0; ky <= ky1; ++ky)
    for (int kx = kx0; kx <= kx1; ++kx) v += W[((size_t)co * 9 + ky * 3 + kx) * cin + k];
  return v;
}

// FP8 form: per-output-channel scale max |v| / 448 over every value the layer multiplies for
// that channel (all phases and taps; 1 if all are zero).  unfolded: the 3 x 3 weights as they
// are (the border recompute of up-sampling layers).
__global__ void fp8_scale_kernel(const float* __restrict__ W, int mode, int cin, int cout, int unfolded,
                                 float* __restrict__ scale) {
  const int co = blockIdx.x * blockDim.x + threadIdx.x;
  if (co >= cout) return;
  float m = 0.f;
  if (unfolded) {
    for (int i = 0; i < 9 * cin; ++i) m = fmaxf(m, fabsf(W[(size_t)co * 9 * cin + i]));
  } else {
    const int T = taps(mode), NPH = mode == TM_UP2 ? 4 : 1;
    for (int ph = 0; ph < NPH; ++ph)
      for (int t = 0; t < T; ++t)
        for (int k = 0; k < cin; ++k) m = fmaxf(m, fabsf(tc_weight(W, mode, ph, t, co, k, cin)));
  }
  scale[co] = m > 0.f ? m / 448.0f : 1.0f;
}

// Packed B of the FP8 form: the E4M3 codes of v / scale[co] in the byte layout of the BF16
// pack with cin / 2 channels (two FP8 channels per BF16 slot, the even one first).
__global__ void pack_fp8_kernel(const float* __restrict__ W, int mode, int NT, int G, int cin, int cout,
                                const float* __restrict__ scale, uint8_t* __restrict__ out) {
  const int T = taps(mode);
  const size_t total = (size_t)G * T * NT * cin;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int k = (int)(idx % cin);
  size_t r = idx / cin;
  const int n = (int)(r % NT);
  r /= NT;
  const int t = (int)(r % T);
  const int g = (int)(r / T);
  const int nsl = mode == TM_UP2 ? g / 4 : g;
  const int co = nsl * NT + n;
  uint8_t q = 0;
  if (co < cout)
    q = (uint8_t)__nv_cvt_float_to_fp8(tc_weight(W, mode, g % 4, t, co, k, cin) / scale[co], __NV_SATFINITE, __NV_E4M3);
  const int cb = cin / 2, kb = k >> 1;
  const size_t slot = (size_t)(n % 8) * 8 + (size_t)(n / 8) * cb * 8 + (kb % 8) + (size_t)(kb / 8) * 64;
  out[((size_t)g * T + t) * NT * cin + 2 * slot + (k & 1)] = q;
}

// E4M3 codes of the unfolded 3 x 3 weights [co][3][3][ci] (the border recompute).
__global__ void quant_unfolded_kernel(const float* __restrict__ W, int cout, int cin, const float* __restrict__ scale,
                                      uint8_t* __restrict__ out) {
  const size_t n = (size_t)cout * 9 * cin;
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = (uint8_t)__nv_cvt_float_to_fp8(W[i] / scale[i / (9 * (size_t)cin)], __NV_SATFINITE, __NV_E4M3);
}

// Packed B of one layer: [G][T][NT rows (output channels) x cin] in the no-swizzle
// K-major core-matrix layout: element (n, k) at (n%8)*8 + (n/8)*cin*8 + (k%8) + (k/8)*64.
__global__ void pack_kernel(const float* __restrict__ W, int mode, int NT, int G, int cin, int cout,
                            bf16* __restrict__ out) {
  const int T = taps(mode);
  const size_t total = (size_t)G * T * NT * cin;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int k = (int)(idx % cin);
  size_t r = idx / cin;
  const int n = (int)(r % NT);
  r /= NT;
  const int t = (int)(r % T);
  const int g = (int)(r / T);
  const int nsl = mode == TM_UP2 ? g / 4 : g;
  const int co = nsl * NT + n;
  const float v = co < cout ? tc_weight(W, mode, g % 4, t, co, k, cin) : 0.f;
  const size_t dst = ((size_t)g * T + t) * NT * cin + (size_t)(n % 8) * 8 + (size_t)(n / 8) * cin * 8 + (k % 8) +
                     (size_t)(k / 8) * 64;
  out[dst] = __float2bfloat16_rn(v);
}


// Packed B of the fused dec3 kernel: 16 blocks of [NT output channels x cin] in the same
// core-matrix layout, one per (phase (py, px), tap (ro, co)) of the 4-phase form (3x3 weights
// summed per phase as in pack_kernel), in the stacking order of fused_view.
__global__ void pack_fused_kernel(const float* __restrict__ W, int NT, int cin, bf16* __restrict__ out) {
  const size_t total = (size_t)16 * NT * cin;
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int k = (int)(idx % cin);
  const int n = (int)((idx / cin) % NT);
  const int blk = (int)(idx / ((size_t)cin * NT));
  const int ph = fused_block_pt(blk) / 10, t = fused_block_pt(blk) % 10;
  const int py = ph >> 1, px = ph & 1, a = t >> 1, b = t & 1;
  const int ky0 = py == 0 ? (a == 0 ? 0 : 1) : (a == 0 ? 0 : 2);
  const int ky1 = py == 0 ? (a == 0 ? 0 : 2) : (a == 0 ? 1 : 2);
  const int kx0 = px == 0 ? (b == 0 ? 0 : 1) : (b == 0 ? 0 : 2);
  const int kx1 = px == 0 ? (b == 0 ? 0 : 2) : (b == 0 ? 1 : 2);
  float v = 0.f;
  for (int ky = ky0; ky <= ky1; ++ky)
    for (int kx = kx0; kx <= kx1; ++kx) v += W[((size_t)n * 9 + ky * 3 + kx) * cin + k];
  const size_t dst = (size_t)blk * NT * cin + (size_t)(n % 8) * 8 + (size_t)(n / 8) * cin * 8 + (k % 8) + (size_t)(k / 8) * 64;
  out[dst] = __float2bfloat16_rn(v);
}

// Packed B of the fused kernel's final conv: [32 rows x NT channels] in the same core-matrix
// layout.  Rows 0-8: the BF16 high parts hi = bf16(w) of the nine taps' weights (row
// 3 ky + kx), rows 9-17: the low parts bf16(w - hi), rows 18-31: zero.  hi + lo equals the
// FP32 weight to about 2^-16 relative, so the tensor-core final conv keeps FP32-weight
// accuracy.
__global__ void pack_final_kernel(const float* __restrict__ wf, int NT, bf16* __restrict__ out) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= kFinalN * NT) return;
  const int k = idx % NT, n = idx / NT;
  float v = 0.f;
  if (n < 18) {
    const float w = wf[(n % 9) * NT + k];
    const float hi = __bfloat162float(__float2bfloat16_rn(w));
    v = n < 9 ? hi : w - hi;
  }
  out[(size_t)(n % 8) * 8 + (size_t)(n / 8) * NT * 8 + (k % 8) + (size_t)(k / 8) * 64] = __float2bfloat16_rn(v);
}

template <int NT, int RB>
cudaError_t launch_fused_nt(const FusedParams& p, int grid, size_t smem, cudaStream_t st) {
  auto k = dec3f_kernel<NT, RB>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<grid, kFusedThreads, smem, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_fused(const FusedParams& p, int NT, int cin, int grid, size_t smem, cudaStream_t st) {
  if (NT == 32 && cin == 64) return launch_fused_nt<32, 128>(p, grid, smem, st);
  if (NT == 16 && cin == 64) return launch_fused_nt<16, 128>(p, grid, smem, st);
  if (NT == 32 && cin == 32) return launch_fused_nt<32, 64>(p, grid, smem, st);
  if (NT == 16 && cin == 32) return launch_fused_nt<16, 64>(p, grid, smem, st);
  return cudaErrorInvalidValue;
}

// The fused dec3 + final kernel applies to decoder widths (cout, cin) in {16, 32} x {32, 64}
// when its shared memory fits.
bool fused_supported(int cout, int cin) {
  return (cout == 16 || cout == 32) && (cin == 32 || cin == 64) && fused_smem_bytes(cout, cin, 4) <= 232448;
}

template <int MODE, int NT, int RB, bool F8>
cudaError_t launch_mode_nt(const Params& p, int grid, size_t smem, cudaStream_t st) {
  // channel-block rings are planned only for up-sampling layers with 128-byte channel blocks
  auto k = conv_tc_kernel<MODE, NT, RB, false, F8>;
  if constexpr (MODE == TM_UP2 && RB == 128) {
    if (p.split) k = conv_tc_kernel<MODE, NT, RB, true, F8>;
  } else {
    if (p.split) return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // all of the SM's unified L1 / shared storage as shared memory: co-resident CTAs
  e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  k<<<grid, kThreads, smem, st>>>(p);
  return cudaGetLastError();
}

template <int MODE, int RB, bool F8>
cudaError_t launch_mode_rb(const Params& p, int NT, int grid, size_t smem, cudaStream_t st) {
  switch (NT) {
    case 16: return launch_mode_nt<MODE, 16, RB, F8>(p, grid, smem, st);
    case 32: return launch_mode_nt<MODE, 32, RB, F8>(p, grid, smem, st);
    case 64: return launch_mode_nt<MODE, 64, RB, F8>(p, grid, smem, st);
    case 128: return launch_mode_nt<MODE, 128, RB, F8>(p, grid, smem, st);
    case 256:
      if constexpr (!F8) return launch_mode_nt<MODE, 256, RB, F8>(p, grid, smem, st);  // FP8 plans cap N at 128
      break;
  }
  return cudaErrorInvalidValue;
}

template <int MODE, bool F8>
cudaError_t launch_mode(const Params& p, int NT, int grid, size_t smem, cudaStream_t st) {
  switch (rb_of(p.cin)) {
    case 128: return launch_mode_rb<MODE, 128, F8>(p, NT, grid, smem, st);
    case 64: return launch_mode_rb<MODE, 64, F8>(p, NT, grid, smem, st);
    case 32: return launch_mode_rb<MODE, 32, F8>(p, NT, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_conv(int mode, const Params& p, int NT, int grid, size_t smem, cudaStream_t st, bool f8 = false) {
  switch (mode) {
    case TM_S2: return f8 ? launch_mode<TM_S2, true>(p, NT, grid, smem, st) : launch_mode<TM_S2, false>(p, NT, grid, smem, st);
    case TM_UP2:
      return f8 ? launch_mode<TM_UP2, true>(p, NT, grid, smem, st) : launch_mode<TM_UP2, false>(p, NT, grid, smem, st);
    case TM_P1: return f8 ? launch_mode<TM_P1, true>(p, NT, grid, smem, st) : launch_mode<TM_P1, false>(p, NT, grid, smem, st);
  }
  return cudaErrorInvalidValue;
}

// CTAs of one layer that fit an SM.  Computed from the kernel's resources: the occupancy
// API answers 1 for any kernel that allocates tensor memory, although the hardware runs
// several such CTAs per SM when their columns fit the SM's 512.
template <int MODE, int NT, int RB>
static int regs_of() {
  cudaFuncAttributes fa{};
  if (cudaFuncGetAttributes(&fa, conv_tc_kernel<MODE, NT, RB>) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return fa.numRegs;
}
template <int MODE, int RB>
static int regs_rb(int NT) {
  switch (NT) {
    case 16: return regs_of<MODE, 16, RB>();
    case 32: return regs_of<MODE, 32, RB>();
    case 64: return regs_of<MODE, 64, RB>();
    case 128: return regs_of<MODE, 128, RB>();
    case 256: return regs_of<MODE, 256, RB>();
  }
  return -1;
}
template <int MODE>
static int regs_mode(int NT, int cin) {
  switch (rb_of(cin)) {
    case 128: return regs_rb<MODE, 128>(NT);
    case 64: return regs_rb<MODE, 64>(NT);
    case 32: return regs_rb<MODE, 32>(NT);
  }
  return -1;
}

int blocks_per_sm(int mode, int NT, int cin, size_t smem, int device) {
  const int regs = mode == TM_S2 ? regs_mode<TM_S2>(NT, cin) : mode == TM_UP2 ? regs_mode<TM_UP2>(NT, cin)
                                                                               : regs_mode<TM_P1>(NT, cin);
  int per_sm = 0, reserved = 0, regfile = 0, max_threads = 0;
  if (regs <= 0 || cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&regfile, cudaDevAttrMaxRegistersPerMultiprocessor, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&max_threads, cudaDevAttrMaxThreadsPerMultiProcessor, device) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const int by_smem = (int)((size_t)per_sm / (smem + (size_t)reserved));
  const int warp_regs = (regs * 32 + 255) / 256 * 256;  // allocated per warp in units of 256
  const int by_regs = regfile / (warp_regs * (kThreads / 32));
  const int by_threads = max_threads / kThreads;
  // tensor memory: co-resident CTAs must fit 512 columns
  const int cols = NT * 2 <= 32 ? 32 : NT * 2 <= 64 ? 64 : NT * 2 <= 128 ? 128 : NT * 2 <= 256 ? 256 : 512;
  return std::max(0, std::min(std::min(by_smem, by_regs), std::min(by_threads, 512 / cols)));
}

}  // namespace tc

// ------------------------------------------------------------------ host side
namespace {
constexpr size_t kSmemLimit = 232448;  // 227 KB opt-in per block
constexpr int kPrefetchSteps = 8;      // row steps staged ahead of the tile being computed
}  // namespace

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to libcuda).
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }
  return fn;
}

// TMA view of a BF16 NHWC activation: dims (channels, pixels of the set, rows), box of
// one channel block (RB / 2 channels) x `box_px` pixels x 1 row in the RB-byte swizzle,
// zero fill outside.  `px_step` = 2 for the odd / even pixel sets of a stride-2 layer.
static bool make_tmap(CUtensorMap* m, const __nv_bfloat16* base, int C, int npix, int H, int W, int px_step,
                      int box_px) {
  auto fn = encode_fn();
  if (!fn || npix < 1) return false;
  const int rb = tc::rb_of(C);
  cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)npix, (cuuint64_t)H};
  cuuint64_t strides[2] = {(cuuint64_t)px_step * C * 2, (cuuint64_t)W * C * 2};
  cuuint32_t box[3] = {(cuuint32_t)(rb / 2), (cuuint32_t)box_px, 1};
  cuuint32_t es[3] = {1, 1, 1};
  const CUtensorMapSwizzle sw = rb == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                : rb == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                           : CU_TENSOR_MAP_SWIZZLE_32B;
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA view of a BF16 NHWC map [H][W][C] for a whole-pixel tile: box C x box_w x box_h, no
// swizzle (pixels contiguous in shared memory), zero fill outside.
static bool make_tmap_tile(CUtensorMap* m, const __nv_bfloat16* base, int C, int W, int H, int box_w, int box_h) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H};
  cuuint64_t strides[2] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2};
  cuuint32_t box[3] = {(cuuint32_t)C, (cuuint32_t)box_w, (cuuint32_t)box_h};
  cuuint32_t es[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
         CUDA_SUCCESS;
}

// BF16 copies of the decoder weights in their canonical [co][3][3][ci] order (border fix),
// stored after the packed GEMM operands; returns their offsets.
static size_t unfolded_offsets(const NetDims& net, size_t packed_total, size_t ofs[3]) {
  size_t o = (packed_total + 7) / 8 * 8;
  const int layers[3] = {L_DEC1, L_DEC2, L_DEC3};
  for (int k = 0; k < 3; ++k) {
    ofs[k] = o;
    o += ((size_t)net.cout(layers[k]) * 9 * net.cin(layers[k]) + 7) / 8 * 8;
  }
  return o;
}

__global__ void to_bf16_kernel(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = __float2bfloat16_rn(a[i]);
}

// f8: the FP8 form, whose operands are E4M3 bytes: a layer of cin channels is planned as cin / 2
// BF16-sized channels (the same bytes), N at most 128, bias and scale beside the weights.
static void plan_layers(const NetDims& net, std::vector<TcLayerPlan>& plans, size_t& total, bool f8 = false) {
  plans.clear();
  total = 0;
  const int layers[6] = {L_ENC2, L_ENC3, L_MU, L_DEC1, L_DEC2, L_DEC3};
  for (int l : layers) {
    TcLayerPlan pl{};
    pl.layer = l;
    pl.mode = (l == L_ENC2 || l == L_ENC3) ? tc::TM_S2 : l == L_MU ? tc::TM_P1 : tc::TM_UP2;
    pl.f8 = f8 ? 1 : 0;
    pl.cin = f8 ? net.cin(l) / 2 : net.cin(l);
    pl.cout = net.cout(l);
    pl.relu = l != L_MU;
    const int RA = pl.mode == tc::TM_S2 ? 3 : pl.mode == tc::TM_UP2 ? 2 : 1;
    const int STEP = pl.mode == tc::TM_S2 ? 2 : 1;
    int NT = std::min(f8 ? 128 : 256, pl.cout & -pl.cout);  // a power of two dividing cout (widths are multiples of 16)
    int ring = RA + STEP;
    while (true) {
      size_t sm = tc::smem_bytes(pl.mode, NT, pl.cin, ring, false, f8);
      if (sm <= kSmemLimit) break;
      if (ring > RA) { --ring; continue; }
      NT /= 2;
      ring = RA + STEP;
    }
    // spend leftover shared memory on deeper row prefetch: a staged row is needed by one
    // tile of MMAs only, so many rows in flight hide the load latency
    while (ring < RA + kPrefetchSteps * STEP && tc::smem_bytes(pl.mode, NT, pl.cin, ring + 1, false, f8) <= kSmemLimit)
      ++ring;
    pl.NT = NT;
    pl.ring = ring;
    const int nsl = (pl.cout + NT - 1) / NT;
    pl.G = pl.mode == tc::TM_UP2 ? 4 * nsl : nsl;
    pl.smem = tc::smem_bytes(pl.mode, NT, pl.cin, ring, false, f8);
    pl.wofs = total;
    pl.fix_wofs = 0;
    total += (size_t)pl.G * tc::taps(pl.mode) * NT * pl.cin;
    plans.push_back(pl);
  }
  size_t unf[3];
  unfolded_offsets(net, total, unf);
  for (auto& pl : plans)
    if (pl.mode == tc::TM_UP2) pl.fix_wofs = unf[pl.layer == L_DEC1 ? 0 : pl.layer == L_DEC2 ? 1 : 2];
}

sv_status Ctx::pack_bf16_weights(cudaStream_t st) {
  std::vector<TcLayerPlan> plans;
  size_t total;
  plan_layers(net, plans, total);
  size_t unf[3];
  const size_t all = unfolded_offsets(net, total, unf);
  sv_status s = cuda(wbf.ensure(all * sizeof(__nv_bfloat16)), "alloc packed weights");
  if (s) return s;
  const int dl[3] = {L_DEC1, L_DEC2, L_DEC3};
  for (int k = 0; k < 3; ++k) {
    const size_t n = (size_t)net.cout(dl[k]) * 9 * net.cin(dl[k]);
    LaunchScope ls(*this, "pack_bf16", st);
    to_bf16_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float*)w32.p + net.w_off(dl[k]),
                                                                (__nv_bfloat16*)wbf.p + unf[k], n);
    if ((s = cuda(cudaGetLastError(), "unfolded weights"))) return s;
  }
  if (tc::fused_supported(net.dec[2], net.dec[1])) {
    const size_t n = (size_t)16 * net.dec[2] * net.dec[1];
    if ((s = cuda(wfuse.ensure(tc::fused_wpack_elems(net.dec[2], net.dec[1]) * sizeof(__nv_bfloat16)),
                  "alloc fused weights")))
      return s;
    LaunchScope ls(*this, "pack_bf16", st);
    tc::pack_fused_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float*)w32.p + net.w_off(L_DEC3), net.dec[2],
                                                                  net.dec[1], (__nv_bfloat16*)wfuse.p);
    if ((s = cuda(cudaGetLastError(), "fused weights"))) return s;
    const int nf = tc::kFinalN * net.dec[2];
    tc::pack_final_kernel<<<(unsigned)((nf + 255) / 256), 256, 0, st>>>((const float*)w32.p + net.w_off(L_FINAL),
                                                                    net.dec[2], (__nv_bfloat16*)wfuse.p + n);
    if ((s = cuda(cudaGetLastError(), "fused final weights"))) return s;
  }
  for (auto& pl : plans) {
    const size_t n = (size_t)pl.G * tc::taps(pl.mode) * pl.NT * pl.cin;
    LaunchScope ls(*this, "pack_bf16", st);
    tc::pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float*)w32.p + net.w_off(pl.layer), pl.mode, pl.NT,
                                                           pl.G, pl.cin, pl.cout, (__nv_bfloat16*)wbf.p + pl.wofs);
    if ((s = cuda(cudaGetLastError(), "pack weights"))) return s;
  }
  return SV_OK;
}

// FP8 form: per quantised layer (enc2 .. dec2) the E4M3 codes of the packed operand (in the
// BF16 pack's byte layout) and its per-output-channel scales; for dec1, dec2 also the codes of
// the unfolded 3 x 3 weights and their scales (the border recompute).  Offsets: the plan's wofs (BF16
// units of wf8), scale offsets f8_scale_ofs[6] and f8_unf_ofs / f8_unf_scale_ofs[3].
sv_status Ctx::pack_fp8_weights(cudaStream_t st) {
  std::vector<TcLayerPlan> plans;
  size_t total;
  plan_layers(net, plans, total, true);
  const int dl[3] = {L_DEC1, L_DEC2, L_DEC3};
  size_t unf_bytes = 0, nscale = 0;
  for (int k = 0; k < 3; ++k) {
    f8_unf_ofs[k] = unf_bytes;
    unf_bytes += ((size_t)net.cout(dl[k]) * 9 * net.cin(dl[k]) + 15) / 16 * 16;
  }
  for (size_t li = 0; li < plans.size(); ++li) {
    f8_scale_ofs[li] = nscale;
    nscale += (size_t)(plans[li].cout + 3) / 4 * 4;
  }
  for (int k = 0; k < 3; ++k) {
    f8_unf_scale_ofs[k] = nscale;
    nscale += (size_t)(net.cout(dl[k]) + 3) / 4 * 4;
  }
  sv_status s;
  if ((s = cuda(wf8.ensure(total * 2), "alloc FP8 weights"))) return s;
  if ((s = cuda(wf8u.ensure(std::max<size_t>(unf_bytes, 16)), "alloc FP8 unfolded weights"))) return s;
  if ((s = cuda(wf8s.ensure(nscale * sizeof(float)), "alloc FP8 scales"))) return s;
  float* sc = (float*)wf8s.p;
  const float* W = (const float*)w32.p;
  for (size_t li = 0; li < plans.size(); ++li) {
    const TcLayerPlan& pl = plans[li];
    if (pl.layer == L_DEC3) continue;  // the last decoder layer runs from the BF16 packs
    const int cin = net.cin(pl.layer);
    LaunchScope ls(*this, "pack_fp8", st);
    tc::fp8_scale_kernel<<<(pl.cout + 127) / 128, 128, 0, st>>>(W + net.w_off(pl.layer), pl.mode, cin, pl.cout, 0,
                                                               sc + f8_scale_ofs[li]);
    if ((s = cuda(cudaGetLastError(), "FP8 scales"))) return s;
    const size_t n = (size_t)pl.G * tc::taps(pl.mode) * pl.NT * cin;
    tc::pack_fp8_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W + net.w_off(pl.layer), pl.mode, pl.NT, pl.G, cin,
                                                                     pl.cout, sc + f8_scale_ofs[li],
                                                                     (uint8_t*)((__nv_bfloat16*)wf8.p + pl.wofs));
    if ((s = cuda(cudaGetLastError(), "pack FP8 weights"))) return s;
  }
  for (int k = 0; k < 2; ++k) {  // dec1, dec2 (dec3's border fix uses the BF16 weights)
    const int cout = net.cout(dl[k]), cin = net.cin(dl[k]);
    LaunchScope ls(*this, "pack_fp8", st);
    tc::fp8_scale_kernel<<<(cout + 127) / 128, 128, 0, st>>>(W + net.w_off(dl[k]), tc::TM_S2, cin, cout, 1,
                                                            sc + f8_unf_scale_ofs[k]);
    if ((s = cuda(cudaGetLastError(), "FP8 unfolded scales"))) return s;
    const size_t n = (size_t)cout * 9 * cin;
    tc::quant_unfolded_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(W + net.w_off(dl[k]), cout, cin,
                                                                           sc + f8_unf_scale_ofs[k],
                                                                           (uint8_t*)wf8u.p + f8_unf_ofs[k]);
    if ((s = cuda(cudaGetLastError(), "FP8 unfolded weights"))) return s;
  }
  return SV_OK;
}

// Host side of one tensor-core refinement call: activation workspaces (allocated here),
// per-layer descriptor and strip tables (built here, uploaded by the caller) and launch
// geometry.  Nothing is enqueued on a stream.
sv_status Ctx::tc_prepare(const sv_pair* pairs, const int16_t* const* coarse, int n, float* const* out, TcRun& r,
                          const float* const* coarse_f) {
  using tc::LayerPair;
  using tc::Strip;
  size_t wtotal;
  const bool f8 = cfg.precision == SV_FP8;
  plan_layers(net, r.plans, wtotal, f8);
  if (f8) {  // the FP8 form's last decoder layer runs as in the BF16 form (BF16 pack, BF16 d2)
    std::vector<TcLayerPlan> bfp;
    size_t bft;
    plan_layers(net, bfp, bft, false);
    for (size_t li = 0; li < r.plans.size(); ++li)
      if (r.plans[li].layer == L_DEC3) r.plans[li] = bfp[li];
  }
  for (size_t li = 0; li < r.plans.size(); ++li) {
    // autotuned narrower N slice (more weight sets, more CTAs per pair): only for one-tap
    // layers, whose packed weights are the same bytes for any slice width (a multi-tap layer's
    // pack interleaves the taps per slice of the planned width)
    if (tc_nt_override[li] > 0 && tc_nt_override[li] <= r.plans[li].NT && r.plans[li].mode == tc::TM_P1) {
      TcLayerPlan& pl = r.plans[li];
      const int NT = tc_nt_override[li];
      pl.NT = NT;
      const int nsl = (pl.cout + NT - 1) / NT;
      pl.G = pl.mode == tc::TM_UP2 ? 4 * nsl : nsl;
      const int RA = pl.mode == tc::TM_S2 ? 3 : pl.mode == tc::TM_UP2 ? 2 : 1;
      const int STEP = pl.mode == tc::TM_S2 ? 2 : 1;
      while (pl.ring < RA + kPrefetchSteps * STEP &&
             tc::smem_bytes(pl.mode, NT, pl.cin, pl.ring + 1, false, pl.f8 != 0) <= kSmemLimit)
        ++pl.ring;
      pl.smem = tc::smem_bytes(pl.mode, NT, pl.cin, pl.ring, false, pl.f8 != 0);
    }
  }
  {
    // shallower rings so that k CTAs share an SM (k per layer from the autotuner, else the
    // context option); one CTA's control overhead between its MMA batches is then
    // covered by the other CTAs' MMAs
    int per_sm = 0, reserved = 0;
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
    cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
    for (size_t li = 0; li < r.plans.size(); ++li) {
      const int k = tc_ctas_override[li] > 0 ? tc_ctas_override[li] : tc_ctas_per_sm;
      if (k <= 1) continue;
      TcLayerPlan& pl = r.plans[li];
      const size_t budget = (size_t)per_sm / k - (size_t)reserved;
      const int RA = pl.mode == tc::TM_S2 ? 3 : pl.mode == tc::TM_UP2 ? 2 : 1;
      const int STEP = pl.mode == tc::TM_S2 ? 2 : 1;
      while (pl.ring > RA + STEP && tc::smem_bytes(pl.mode, pl.NT, pl.cin, pl.ring, false, pl.f8 != 0) > budget) --pl.ring;
      pl.smem = tc::smem_bytes(pl.mode, pl.NT, pl.cin, pl.ring, false, pl.f8 != 0);
    }
  }
  // a layer whose ring holds no row beyond the tile's own (the weights fill shared memory)
  // stages channel blocks instead of whole rows: a row's first blocks are reloaded while the
  // tile still reads its last ones, so the next tile's input arrives ahead of it
  for (size_t li = 0; li < r.plans.size(); ++li) {
    TcLayerPlan& pl = r.plans[li];
    pl.split = 0;
    const int RA = pl.mode == tc::TM_S2 ? 3 : pl.mode == tc::TM_UP2 ? 2 : 1;
    const int KB = pl.cin * 2 / tc::rb_of(pl.cin);
    if (!split_rows || pl.mode != tc::TM_UP2 || tc::rb_of(pl.cin) != 128 || pl.ring > RA || KB < 2) continue;
    const int k = tc_ctas_override[li] > 0 ? tc_ctas_override[li] : tc_ctas_per_sm;
    size_t budget = kSmemLimit;
    if (k > 1) {
      int per_sm = 0, reserved = 0;
      cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, device);
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, device);
      const size_t share = (size_t)per_sm / k - (size_t)reserved;
      if (pl.smem <= share) budget = share;  // else k CTAs do not fit anyway: one per SM
    }
    int units = RA * KB;
    while (units < 3 * RA * KB && tc::smem_bytes(pl.mode, pl.NT, pl.cin, units + 1, true, pl.f8 != 0) <= budget) ++units;
    if (units <= RA * KB) continue;  // no unit of look-ahead fits
    pl.split = 1;
    pl.ring = units;
    pl.smem = tc::smem_bytes(pl.mode, pl.NT, pl.cin, units, true, pl.f8 != 0);
  }
  sv_status s;
  int nsm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device);
  std::vector<Levels> lv(n);
  size_t cnt[7] = {0};
  std::vector<std::array<size_t, 7>> off(n), lens;
  for (int i = 0; i < n; ++i) {
    lv[i] = Levels(pairs[i].height, pairs[i].width);
    const size_t P[4] = {(size_t)lv[i].H[0] * lv[i].W[0], (size_t)lv[i].H[1] * lv[i].W[1],
                         (size_t)lv[i].H[2] * lv[i].W[2], (size_t)lv[i].H[3] * lv[i].W[3]};
    const size_t need[7] = {P[1] * net.enc[0], P[2] * net.enc[1], P[3] * net.enc[2], P[3] * net.lat,
                            P[2] * net.dec[0], P[1] * net.dec[1], P[0] * net.dec[2]};
    for (int k = 0; k < 7; ++k) {
      off[i][k] = cnt[k];
      cnt[k] += (need[k] + 15) / 16 * 16;  // 16-byte aligned per pair (BF16 and E4M3)
    }
    lens.push_back({need[0], need[1], need[2], need[3], need[4], need[5], need[6]});
  }
  // BF16 activations; the FP8 form keeps e2 .. d1 (the inputs of its quantised layers) as E4M3
  // codes (one byte per channel) and the E4M3 codes of e1 in tc_act[7]
  auto esize = [&](int k) { return f8 && k >= 1 && k <= 4 ? (size_t)1 : sizeof(__nv_bfloat16); };
  for (int k = 0; k < 7; ++k)
    if ((s = cuda(tc_act[k].ensure(std::max<size_t>(cnt[k], 16) * esize(k)), "alloc activations"))) return s;
  if (f8 && (s = cuda(tc_act[7].ensure(std::max<size_t>(cnt[0], 16)), "alloc FP8 e1"))) return s;
  // (an FP8 tensor is addressed as BF16 of half the channels: offsets are element counts / 2)
  auto act = [&](int k, int i) {
    return esize(k) == 1 ? (__nv_bfloat16*)((uint8_t*)tc_act[k].p + off[i][k]) : (__nv_bfloat16*)tc_act[k].p + off[i][k];
  };
  auto act_in = [&](int k, int i) {  // a tensor-core layer's input: e1 as E4M3 codes in the FP8 form
    return f8 && k == 0 ? (__nv_bfloat16*)((uint8_t*)tc_act[7].p + off[i][0]) : act(k, i);
  };
  tc_off = off;
  tc_len = lens;
  r.host.clear();
  auto put = [&](const void* src, size_t bytes) {
    size_t o = (r.host.size() + 127) / 128 * 128;  // the structs holding tensor maps are 128-byte aligned
    r.host.resize(o + bytes);
    memcpy(r.host.data() + o, src, bytes);
    return o;
  };
  r.tabs.assign(r.plans.size(), {});
  for (size_t li = 0; li < r.plans.size(); ++li) {
    const TcLayerPlan& pl = r.plans[li];
    std::vector<LayerPair> lps(n);
    const int in_act = pl.layer == L_ENC2 ? 0 : pl.layer == L_ENC3 ? 1 : pl.layer == L_MU ? 2 : pl.layer == L_DEC1 ? 3
                       : pl.layer == L_DEC2 ? 4 : 5;
    const int out_act = in_act + 1;
    const int lin = pl.layer == L_ENC2 ? 1 : pl.layer == L_ENC3 ? 2 : pl.layer == L_MU ? 3 : pl.layer == L_DEC1 ? 3
                    : pl.layer == L_DEC2 ? 2 : 1;
    const int lout = pl.layer == L_ENC2 ? 2 : pl.layer == L_ENC3 ? 3 : pl.layer == L_MU ? 3 : pl.layer == L_DEC1 ? 2
                     : pl.layer == L_DEC2 ? 1 : 0;
    long long units = 0;
    std::vector<UpFixPair> fix(n);
    for (int i = 0; i < n; ++i) {
      LayerPair& L = lps[i];
      memset(&L, 0, sizeof(L));
      L.in = act_in(in_act, i);
      L.out = act(out_act, i);
      L.Hi = lv[i].H[lin]; L.Wi = lv[i].W[lin];
      L.Ho = lv[i].H[lout]; L.Wo = lv[i].W[lout];
      if (pl.mode == tc::TM_UP2) { L.Hu = L.Hi; L.Wu = L.Wi; }
      else { L.Hu = L.Ho; L.Wu = L.Wo; }
      units += (long long)L.Hu * ((L.Wu + 127) / 128);
      bool okm;
      if (pl.mode == tc::TM_S2)
        okm = make_tmap(&L.tm[0], L.in + pl.cin, pl.cin, L.Wi / 2, L.Hi, L.Wi, 2, 129) &&
              make_tmap(&L.tm[1], L.in, pl.cin, (L.Wi + 1) / 2, L.Hi, L.Wi, 2, 129);
      else
        okm = make_tmap(&L.tm[0], L.in, pl.cin, L.Wi, L.Hi, L.Wi, 1, tc::npx(pl.mode));
      if (!okm) return fail(SV_ERR_CUDA, "layer %d: cuTensorMapEncodeTiled failed", pl.layer);
      fix[i] = {L.in, L.out, L.Hi, L.Wi, L.Ho, L.Wo, L.Hu, L.Wu};
    }
    int bps = tc::blocks_per_sm(pl.mode, pl.NT, pl.cin, pl.smem, device);
    if (bps <= 0) return fail(SV_ERR_UNSUPPORTED, "layer %d: tensor-core kernel does not fit an SM", pl.layer);
    int grid = std::max(pl.G, (nsm * bps) / pl.G * pl.G);
    const int cpg = grid / pl.G;
    // strip height: about four strips per CTA of a weight set, at least 2 rows, unless tuned
    const long long want = std::max<long long>(1, (long long)cpg * 4);
    int hs = (int)std::max<long long>(2, (units + want - 1) / want);
    if (tc_strip_rows > 0) hs = tc_strip_rows;
    if (tc_rows_override[li] > 0) hs = tc_rows_override[li];
    std::vector<Strip> strips;
    for (int i = 0; i < n; ++i)
      for (int j0 = 0; j0 < lps[i].Wu; j0 += 128)
        for (int i0 = 0; i0 < lps[i].Hu; i0 += hs) strips.push_back({i, j0, i0, std::min(hs, lps[i].Hu - i0)});
    grid = (int)std::min<long long>(grid, (long long)pl.G * (long long)strips.size());
    r.tabs[li].lp_ofs = put(lps.data(), sizeof(LayerPair) * n);
    r.tabs[li].fix_ofs = put(fix.data(), sizeof(UpFixPair) * n);
    r.tabs[li].strip_ofs = put(strips.data(), sizeof(Strip) * strips.size());
    r.tabs[li].n_strips = (int)strips.size();
    r.tabs[li].grid = grid;
    r.tabs[li].hs = hs;
    if (debug_plans)
      fprintf(stderr,
              "[sv] tc layer %d: mode %d cin %d cout %d NT %d ring %d%s smem %zu blocks/SM %d grid %d strips %zu rows %d\n",
              pl.layer, pl.mode, pl.cin, pl.cout, pl.NT, pl.ring, pl.split ? " (channel blocks)" : "", pl.smem, bps, grid,
              strips.size(), hs);
    int mb = 0;
    for (int i = 0; i < n; ++i) mb = std::max(mb, upfix_segments(lps[i].Ho, lps[i].Wo));
    r.tabs[li].fix_segments = mb;
  }
  std::vector<EdgePair> eps_(n);
  r.maxW = r.maxH = r.maxW1 = r.maxH1 = 0;
  for (int i = 0; i < n; ++i) {
    const sv_pair& p = pairs[i];
    eps_[i] = {p.left, p.pitch, p.width, p.height, p.width / 4, p.height / 4, coarse ? coarse[i] : nullptr,
               coarse_f ? coarse_f[i] : nullptr, act(0, i), act(6, i), out[i],
               f8 && enc1_on_tc() ? (uint8_t*)act_in(0, i) : nullptr, CUtensorMap{}};
    if (final_staged_by_tma(net.dec[2]) &&
        !make_tmap_tile(&eps_[i].d3_map, act(6, i), net.dec[2], p.width, p.height, 34, final_tile_rows(net.dec[2]) + 2))
      return fail(SV_ERR_CUDA, "pair %d: cuTensorMapEncodeTiled failed (final conv)", i);
    r.maxW = std::max(r.maxW, p.width);
    r.maxH = std::max(r.maxH, p.height);
    r.maxW1 = std::max(r.maxW1, lv[i].W[1]);
    r.maxH1 = std::max(r.maxH1, lv[i].H[1]);
  }
  r.edge_ofs = put(eps_.data(), sizeof(EdgePair) * n);
  r.n = n;
  r.e1_count = cnt[0];

  // fused last decoder layer + final conv: inference only (training keeps d3 for backward)
  r.fused = false;
  bool even = true;
  for (int i = 0; i < n; ++i) even = even && (pairs[i].width % 2 == 0);
  if (!coarse_f && fused_final && even && tc::fused_supported(net.dec[2], net.dec[1]) && wfuse.p) {
    const int NT = net.dec[2], cin = net.dec[1];
    int ring = 4;  // 3 rows per tile + 1 ahead; more where shared memory allows
    while (ring < 3 + kPrefetchSteps && tc::fused_smem_bytes(NT, cin, ring + 1) <= kSmemLimit) ++ring;
    if (fused_ring > 0) ring = std::min(ring, fused_ring);
    std::vector<tc::FusedPair> fps(n);
    long long units = 0;
    for (int i = 0; i < n; ++i) {
      tc::FusedPair& F = fps[i];
      memset(&F, 0, sizeof(F));
      F.Y = out[i];
      F.coarse = coarse ? coarse[i] : nullptr;
      F.Hu = lv[i].H[1];
      F.Wu = lv[i].W[1];
      F.Ho = lv[i].H[0];
      F.Wo = lv[i].W[0];
      F.w4 = pairs[i].width / 4;
      F.h4 = pairs[i].height / 4;
      if (!make_tmap(&F.tm, act(5, i), cin, F.Wu, F.Hu, F.Wu, 1, tc::kFusedNpx))
        return fail(SV_ERR_CUDA, "pair %d: cuTensorMapEncodeTiled failed (fused decoder)", i);
      units += (long long)F.Hu * ((F.Wo + 1 + 253) / 254);
    }
    const int grid0 = nsm;  // one CTA per SM (about 214 KB of shared memory each)
    int hs = (int)std::max<long long>(2, (units + grid0 * 4LL - 1) / (grid0 * 4LL));
    if (tc_strip_rows > 0) hs = tc_strip_rows;
    if (tc_rows_override[5] > 0) hs = tc_rows_override[5];
    std::vector<tc::Strip> strips;
    for (int i = 0; i < n; ++i)
      for (int sx = 0; 254 * sx - 1 < fps[i].Wo; ++sx)
        for (int i0 = 0; i0 < fps[i].Hu; i0 += hs) strips.push_back({i, 127 * sx - 1, i0, std::min(hs, fps[i].Hu - i0)});
    r.fused_fp_ofs = put(fps.data(), sizeof(tc::FusedPair) * n);
    r.fused_strip_ofs = put(strips.data(), sizeof(tc::Strip) * strips.size());
    r.fused_n_strips = (int)strips.size();
    r.fused_grid = (int)std::min<long long>(grid0, (long long)strips.size());
    r.fused_ring = ring;
    r.fused_hs = hs;
    r.fused_smem = tc::fused_smem_bytes(NT, cin, ring);
    r.fused = true;
    if (debug_plans)
      fprintf(stderr, "[sv] fused dec3+final: NT %d cin %d ring %d smem %zu grid %d strips %zu rows %d\n", NT, cin, ring,
              r.fused_smem, r.fused_grid, strips.size(), hs);
  }
  return SV_OK;
}

// Kernel launches of a prepared call; `tables` holds r.host on the device.  Only kernel
// launches: safe inside a stream capture.
sv_status Ctx::tc_launch(const TcRun& r, const unsigned char* tables, cudaStream_t st, const TcTrainLatent* tl) {
  using tc::LayerPair;
  using tc::Strip;
  sv_status s;
  const float* W = (const float*)w32.p;
  const EdgePair* d_edges = (const EdgePair*)(tables + r.edge_ofs);
  {
    LaunchScope ls(*this, "edge_enc1", st);
    if ((s = cuda(launch_edge_enc1(d_edges, r.n, r.maxW1, r.maxH1, W + net.w_off(L_ENC1), W + net.b_off(L_ENC1),
                                   net.enc[0], (int*)err_flag.p, spin_limit, enc1_tensor != 0, st),
                  "enc1")))
      return s;
  }
  const bool f8 = cfg.precision == SV_FP8;
  if (f8 && !enc1_on_tc()) {  // (the tensor-core enc1 writes the codes itself)
    LaunchScope ls(*this, "e1_to_e4m3", st);
    if ((s = cuda(launch_bf16_to_e4m3((const __nv_bfloat16*)tc_act[0].p, (uint8_t*)tc_act[7].p, r.e1_count, st),
                  "e1 to E4M3")))
      return s;
  }
  static const char* names[6] = {"tc_enc2", "tc_enc3", "tc_latent", "tc_dec1", "tc_dec2", "tc_dec3"};
  for (size_t li = 0; li < r.plans.size(); ++li) {
    const TcLayerPlan& pl = r.plans[li];
    tc::Params prm{};
    prm.lp = (const LayerPair*)(tables + r.tabs[li].lp_ofs);
    prm.strips = (const Strip*)(tables + r.tabs[li].strip_ofs);
    prm.n_strips = r.tabs[li].n_strips;
    const bool lf8 = pl.f8 != 0;
    prm.wpack = (const __nv_bfloat16*)(lf8 ? wf8.p : wbf.p) + pl.wofs;
    prm.bias = W + net.b_off(pl.layer);
    prm.scale = lf8 ? (const float*)wf8s.p + f8_scale_ofs[li] : nullptr;
    prm.out_f8 = lf8 && pl.layer != L_DEC2;  // dec2 writes the BF16 d2 of the last decoder layer
    prm.cin = pl.cin;
    prm.cout = pl.cout;
    prm.G = pl.G;
    prm.relu = pl.relu;
    prm.ring = pl.ring;
    prm.split = pl.split;
    prm.err = (int*)err_flag.p;
    prm.spin = spin_limit;
    if (tl && pl.layer == L_MU) {
      // training: mu, logvar and the reparameterised z instead of z = mu
      for (int i = 0; i < r.n; ++i) {
        LaunchScope ls(*this, "train_latent", st);
        if ((s = cuda(launch_train_latent_bf16(tl->e3[i], tl->P3[i], net.enc[2], W + net.w_off(L_MU), W + net.b_off(L_MU),
                                               W + net.w_off(L_LV), W + net.b_off(L_LV), net.lat, tl->eps[i], tl->mu[i],
                                               tl->lv[i], tl->z[i], st),
                      "train latent")))
          return s;
      }
      continue;
    }
    if (r.fused && pl.layer == L_DEC3) {
      tc::FusedParams fp{};
      fp.fp = (const tc::FusedPair*)(tables + r.fused_fp_ofs);
      fp.strips = (const Strip*)(tables + r.fused_strip_ofs);
      fp.n_strips = r.fused_n_strips;
      fp.wpack = (const __nv_bfloat16*)wfuse.p;
      fp.bias = prm.bias;
      fp.bf = W + net.b_off(L_FINAL);
      fp.ring = r.fused_ring;
      fp.pf = fused_prefetch;
      fp.err = (int*)err_flag.p;
      fp.spin = spin_limit;
      LaunchScope ls(*this, "tc_dec3_final", st);
      if ((s = cuda(tc::launch_fused(fp, net.dec[2], net.dec[1], r.fused_grid, r.fused_smem, st), "fused dec3 + final")))
        return s;
      continue;  // no border fix: the crop is exact inside the fused kernel
    }
    {
      LaunchScope ls(*this, names[li], st);
      if ((s = cuda(tc::launch_conv(pl.mode, prm, pl.NT, r.tabs[li].grid, pl.smem, st, lf8), names[li]))) return s;
    }
    if (lf8 && pl.mode == tc::TM_UP2 && r.tabs[li].fix_segments > 0) {
      const int k = pl.layer == L_DEC1 ? 0 : pl.layer == L_DEC2 ? 1 : 2;
      LaunchScope ls(*this, "edge_up2fix", st);
      if ((s = cuda(launch_edge_up2fix_f8((const UpFixPair*)(tables + r.tabs[li].fix_ofs), r.n, r.tabs[li].fix_segments,
                                          (const uint8_t*)wf8u.p + f8_unf_ofs[k],
                                          (const float*)wf8s.p + f8_unf_scale_ofs[k], prm.bias, net.cin(pl.layer),
                                          pl.cout, 1, prm.out_f8, st),
                    "border fix")))
        return s;
    } else if (pl.mode == tc::TM_UP2 && r.tabs[li].fix_segments > 0) {
      LaunchScope ls(*this, "edge_up2fix", st);
      if ((s = cuda(launch_edge_up2fix((const UpFixPair*)(tables + r.tabs[li].fix_ofs), r.n, r.tabs[li].fix_segments,
                                       (const __nv_bfloat16*)wbf.p + pl.fix_wofs, prm.bias, pl.cin, pl.cout, 1, st),
                    "border fix")))
        return s;
    }
  }
  last_fused = r.fused;
  if (r.fused) return SV_OK;  // the final conv ran inside the fused decoder kernel
  {
    LaunchScope ls(*this, "edge_final", st);
    if ((s = cuda(launch_edge_final(d_edges, r.n, r.maxW, r.maxH, W + net.w_off(L_FINAL), W + net.b_off(L_FINAL),
                                    net.dec[2], (int*)err_flag.p, spin_limit, st),
                  "final")))
      return s;
  }
  return SV_OK;
}

sv_status Ctx::refine_tc(const sv_pair* pairs, const int16_t* const* coarse, int n, float* const* out,
                         cudaStream_t st) {
  TcRun r;
  sv_status s = tc_prepare(pairs, coarse, n, out, r);
  if (s) return s;
  if ((s = cuda(tc_tables.ensure(r.host.size()), "alloc tables"))) return s;
  if ((s = cuda(cudaMemcpyAsync(tc_tables.p, r.host.data(), r.host.size(), cudaMemcpyHostToDevice, st),
                "upload tables")))
    return s;
  return tc_launch(r, (const unsigned char*)tc_tables.p, st);
}

}  // namespace sv
