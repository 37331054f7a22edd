// sv_ctx.cuh -- the library context behind the opaque sv_ctx handle.
#pragma once

#include <map>
#include <string>
#include <vector>

#include "sv_internal.cuh"

namespace sv {

constexpr int kMaxSide = 16384;  // largest accepted image width / height
constexpr int kMaxDisp = 128;    // largest accepted D (4 disparities per lane of a warp)

inline bool valid_width_pub(int c) { return c >= 16 && c <= 256 && c % 16 == 0; }

// Device allocation that only grows.
struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
  cudaError_t ensure(size_t bytes);
  void release();
};

// Launch plan of one tensor-core layer.
struct TcLayerPlan {
  int layer, mode, NT, G, ring, cin, cout, relu;
  int split;  // 1: ring units are channel blocks of rows (ring counts units)
  size_t wofs, smem;
  size_t fix_wofs;  // decoder layers: BF16 [co][3][3][ci] weights of the border fix
  int f8;           // E4M3 operands (the FP8 form's quantised layers; cin counts channel pairs)
};

// Prepared tensor-core refinement call: plans, table bytes and launch geometry.
struct TcRun {
  std::vector<TcLayerPlan> plans;
  struct Tab {
    size_t lp_ofs, strip_ofs, fix_ofs;
    int n_strips, grid, fix_segments, hs;  // fix_segments: border-fix blocks per pair (max)
  };
  std::vector<Tab> tabs;
  std::vector<unsigned char> host;
  size_t edge_ofs = 0;
  int n = 0, maxW = 0, maxH = 0, maxW1 = 0, maxH1 = 0;
  size_t e1_count = 0;  // elements of the e1 workspace (all pairs)
  // fused last decoder layer + final conv (inference, even output widths)
  bool fused = false;
  size_t fused_fp_ofs = 0, fused_strip_ofs = 0, fused_smem = 0;
  int fused_n_strips = 0, fused_grid = 0, fused_ring = 0, fused_hs = 0;
};

// Prepared coarse-matching call.
struct ZRun {
  std::vector<ZPair> pairs;
  std::vector<ZJob> jobs;
  int maxD = 1;
};

// Per-pair buffers of the training latent of the tensor-core form.
struct TcTrainLatent {
  std::vector<const __nv_bfloat16*> e3;
  std::vector<int> P3;
  std::vector<const float*> eps;
  std::vector<float*> mu, lv;
  std::vector<__nv_bfloat16*> z;
};

// One captured batched step (coarse match + tensor-core refinement) and what it needs.
struct GraphEntry {
  std::vector<uint64_t> key;
  std::vector<uint64_t> pkey;  // the call signature that led to it (before any preparation)
  std::vector<std::array<size_t, 7>> off, len;  // per-pair activation offsets of the call
  bool fused = false;
  cudaGraphExec_t exec = nullptr;
  void* tables = nullptr;  // device copy of the step's tables (owned)
  struct Rec { std::string name; cudaEvent_t a, b; };
  std::vector<Rec> prof;   // event pairs captured around each kernel (profiling on)
  long long kernels = 0;
  long long last_use = 0;
};

size_t t1_param_count();  // the paper's Table I network (t1net.cu)

struct Ctx {
  sv_config cfg{};
  NetDims net{};
  bool t1 = false;               // the paper's Table I network (sv_config.flags SV_NET_TABLE1)
  size_t n_params() const { return t1 ? t1_param_count() : net.count(); }
  int device = 0;
  std::string err;

  DevBuf w32, w64, wbf;          // FP32 master, FP64 copy, packed BF16 GEMM operands
  DevBuf wfuse;                  // packed BF16 operands of the fused last decoder layer
  DevBuf wf8, wf8u, wf8s;        // FP8 form: packed E4M3 operands, unfolded decoder E4M3 weights, scales
  size_t f8_scale_ofs[6] = {0}, f8_unf_ofs[3] = {0}, f8_unf_scale_ofs[3] = {0};
  DevBuf zpairs, zjobs;          // coarse-matcher tables
  DevBuf coarse_maps;            // int16 coarse maps of sv_pipeline
  DevBuf act[7];                 // activations e1 e2 e3 z d1 d2 d3 (direct path)
  DevBuf tc_act[8];              // BF16 activations of the tensor-core path
  DevBuf tc_tables;              // tensor-core job tables
  int adam_t = 0;
  int adam_elem = 0;
  DevBuf adam_m, adam_v;
  // differentiation form: state saved by the last training forward
  DevBuf train_saved, train_scratch, loss_acc, train_mu;
  DevBuf wgrad_slots;            // per-CTA partial weight gradients of the FP32 backward
  std::vector<sv_pair> train_pairs;
  std::vector<const void*> train_coarse;
  std::vector<size_t> train_off;
  int train_elem = 0;
  bool train_ready = false;
  DevBuf host_img, host_out;     // device staging of sv_pipeline_host
  DevBuf host_jobs;              // row-copy job tables of sv_pipeline_host (gather + scatter)
  DevBuf sgm_s, sgm_c, sgm_a, sgm_tab;  // coarse-stage variants: box sums, cost, aggregated cost, pairs
  DevBuf x_codes, x_maps;               // census codes; winner-take-all and intermediate maps
  DevBuf t1_act, t1_tab;                // Table I network: activations, per-call tables
  DevBuf loss_slots;                    // per-block partial sums of sv_loss_paper
  cudaStream_t copy_stream = nullptr;    // sv_pipeline_host: results go back here while the
  cudaEvent_t chunk_done[4] = {nullptr, nullptr, nullptr, nullptr};  // next part computes
  cudaStream_t in_stream = nullptr;      // sv_pipeline_host: parts' images gathered ahead of their compute
  cudaEvent_t gather_done[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t call_start = nullptr;
  int host_chunks = 3;                  // parts of an sv_pipeline_host batch (>= 8 pairs each)
  std::vector<unsigned char> tc_host_tables;
  long long spin_limit = 4000000000LL;  // clock64 cycles a device-side wait may spin
  int tc_strip_rows = 0;                // 0: automatic
  int debug_plans = 0;                  // 1: print each tensor-core layer's launch plan to stderr
  int fused_final = 1;                  // 1: last decoder layer + final conv in one kernel when possible
  int fused_ring = 0;                   // fused kernel's staged-row ring: 0 as deep as shared memory allows
  int fused_prefetch = 4;               // fused kernel: rows prefetched into L2 ahead of the loaded row
  int enc1_tensor = 1;                  // 1: enc1 on the tensor cores where its width allows
  bool enc1_on_tc() const { return enc1_tensor && (net.enc[0] == 16 || net.enc[0] == 32 || net.enc[0] == 64); }
  int split_rows = 1;                   // 1: layers without a spare staged row stage channel blocks
  int host_copy = 1;                    // sv_pipeline_host: 0 copy calls, 1 gather kernel in, 2 kernels both ways
  bool last_fused = false;              // the last tensor-core call did not materialise d3
  int tc_ctas_per_sm = 0;               // 0: deepest row ring (one CTA per SM); k: ring sized for k
  int tc_rows_override[6] = {0, 0, 0, 0, 0, 0};  // per tensor-core layer, set by the autotuner
  int tc_nt_override[6] = {0, 0, 0, 0, 0, 0};
  int tc_ctas_override[6] = {0, 0, 0, 0, 0, 0};  // CTAs per SM the ring is sized for (0: tc_ctas_per_sm)
  bool use_graphs = true;
  bool tune_loaded = false;
  double tune_us[6] = {0, 0, 0, 0, 0, 0};
  DevBuf tune_out;
  std::vector<GraphEntry> graphs;
  long long graph_clock = 0;
  std::vector<std::array<size_t, 7>> tc_off;   // per pair offsets of the last tensor-core call
  std::vector<std::array<size_t, 7>> tc_len;
  DevBuf err_flag;                      // device int: first failure code of a kernel

  // launch accounting and optional per-kernel event timing
  long long launches = 0;
  bool prof_on = false;
  struct ProfRec { std::string name; cudaEvent_t a, b; bool pooled = true; };  // pooled: events return to ev_free
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> ev_free;
  std::map<std::string, std::pair<long long, double>> prof_tot;
  cudaEvent_t take_event() {
    cudaEvent_t e = nullptr;
    if (!ev_free.empty()) { e = ev_free.back(); ev_free.pop_back(); }
    else cudaEventCreate(&e);
    return e;
  }

  sv_status fail(sv_status s, const char* fmt, ...);
  sv_status cuda(cudaError_t e, const char* what);
  sv_status check_pairs(const sv_pair* pairs, int n_pairs);

  sv_status coarse(const sv_pair* pairs, int n, int16_t* const* disp, float* const* best, float* const* second,
                   cudaStream_t st);
  sv_status coarse_ext(const sv_pair* pairs, int n, const sv_coarse_opts& o, int16_t* const* disp,
                       float* const* cost_out, cudaStream_t st);
  sv_status post_launch(const void* table, int n, int maxw, int maxh, int post, cudaStream_t st);
  sv_status postprocess(const sv_pair* pairs, int n, const int16_t* const* in, int post, int16_t* const* out,
                        cudaStream_t st);
  sv_status pipeline_ex(const sv_pair* pairs, int n, const sv_coarse_opts& o, float* const* out, cudaStream_t st);
  sv_status t1_forward(const sv_pair* pairs, int n, const int16_t* const* coarse_i, const float* const* coarse_f,
                       const float* const* eps, float* const* Y, float* const* mu, float* const* sigma,
                       cudaStream_t st);
  sv_status loss_paper(const sv_pair* pairs, int n, const float* const* Y, const float* const* gt,
                       const uint8_t* const* noc, const float* const* mu, const float* const* sigma, double* out,
                       float* const* gY, float* const* gmu, float* const* gsigma, cudaStream_t st);
  template <typename T> const T* weights() const;
  template <typename T>
  sv_status refine_direct(const sv_pair& p, const void* coarse_map, bool coarse_int16, const T* eps, T* Y, T* mu_out,
                          T* lv_out, T* const* saved, cudaStream_t st);
  sv_status refine_infer(const sv_pair* pairs, const int16_t* const* coarse, int n, float* const* out,
                         cudaStream_t st);
  sv_status pipeline(const sv_pair* pairs, int n, float* const* out, cudaStream_t st);
  sv_status refresh_weight_copies();
  sv_status refresh_weight_copies_async(cudaStream_t st);
  sv_status pack_bf16_weights(cudaStream_t st = 0);
  sv_status pack_fp8_weights(cudaStream_t st = 0);
  template <typename T>
  sv_status train_forward(const sv_pair* pairs, const void* const* coarse, const void* const* eps, int n,
                          void* const* Y, void* const* mu, void* const* lv, cudaStream_t st);
  template <typename T>
  sv_status train_backward(const void* const* gY, const void* const* gmu_ext, const void* const* glv_ext, T* gparams,
                           void* const* gcoarse, cudaStream_t st);
  template <typename T>
  sv_status loss(const sv_pair* pairs, int n, const void* const* Y, const float* const* gt, const void* const* mu,
                 const void* const* lv, double kl_w, void* out, void* const* gY, void* const* gmu, void* const* glv,
                 cudaStream_t st);
  template <typename T>
  sv_status adam(const T* g, int step, double lr, double b1, double b2, double eps, cudaStream_t st);
  sv_status refine_tc(const sv_pair* pairs, const int16_t* const* coarse, int n, float* const* out, cudaStream_t st);
  sv_status tc_prepare(const sv_pair* pairs, const int16_t* const* coarse, int n, float* const* out, TcRun& r,
                       const float* const* coarse_f = nullptr);
  sv_status tc_launch(const TcRun& r, const unsigned char* tables, cudaStream_t st, const TcTrainLatent* tl = nullptr);
  sv_status train_forward_bf16(const sv_pair* pairs, const void* const* coarse, const void* const* eps, int n,
                               void* const* Y, void* const* mu, void* const* lv, cudaStream_t st);
  void coarse_prepare(const sv_pair* pairs, int n, int16_t* const* disp, float* const* best, float* const* second,
                      ZRun& z);
  sv_status coarse_launch(const ZRun& z, const ZPair* d_pairs, const ZJob* d_jobs, cudaStream_t st);
  sv_status pipeline_graph(const sv_pair* pairs, int n, float* const* out, cudaStream_t st);
  sv_status autotune(const sv_pair* pairs, int n, const char* cache_path, cudaStream_t st);
  void drop_graphs() {
    prof_flush();  // pending records may point at graph-owned events
    for (auto& g : graphs) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      if (g.tables) cudaFree(g.tables);
      for (auto& r : g.prof) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
    }
    graphs.clear();
  }

  void prof_flush() {
    for (auto& r : prof_pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
        auto& t = prof_tot[r.name];
        t.first += 1;
        t.second += ms;
      }
      if (r.pooled) {
        ev_free.push_back(r.a);
        ev_free.push_back(r.b);
      }
    }
    prof_pending.clear();
  }

  void release_all() {
    prof_flush();
    drop_graphs();
    if (copy_stream) cudaStreamSynchronize(copy_stream);
    if (in_stream) cudaStreamSynchronize(in_stream);
    for (auto& e : chunk_done)
      if (e) {
        cudaEventDestroy(e);
        e = nullptr;
      }
    for (auto& e : gather_done)
      if (e) {
        cudaEventDestroy(e);
        e = nullptr;
      }
    if (call_start) cudaEventDestroy(call_start);
    call_start = nullptr;
    if (copy_stream) cudaStreamDestroy(copy_stream);
    copy_stream = nullptr;
    if (in_stream) cudaStreamDestroy(in_stream);
    in_stream = nullptr;
    for (auto e : ev_free) cudaEventDestroy(e);
    ev_free.clear();
    host_img.release(); host_out.release(); host_jobs.release(); err_flag.release(); tune_out.release();
    sgm_s.release(); sgm_c.release(); sgm_a.release(); sgm_tab.release(); x_codes.release(); x_maps.release();
    t1_act.release(); t1_tab.release(); loss_slots.release();
    w32.release(); w64.release(); wbf.release(); wfuse.release(); wf8.release(); wf8u.release(); wf8s.release(); zpairs.release(); zjobs.release();
    coarse_maps.release();
    for (auto& b : act) b.release();
    for (auto& b : tc_act) b.release();
    tc_tables.release(); adam_m.release(); adam_v.release();
    train_saved.release(); train_scratch.release(); loss_acc.release(); train_mu.release(); wgrad_slots.release();
  }
};

}  // namespace sv

namespace sv {
// Makes a device current for the scope of an ABI call and restores the caller's.
struct DeviceGuardInt {
  int prev = -1;
  explicit DeviceGuardInt(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuardInt() {
    int cur;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// Counts one kernel launch and, when profiling is on, brackets it with events.
struct LaunchScope {
  Ctx& c;
  const char* name;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  unsigned flags = cudaEventRecordDefault;
  LaunchScope(Ctx& ctx, const char* n, cudaStream_t s) : c(ctx), name(n), st(s) {
    ++c.launches;
    if (c.prof_on) {
      // inside a stream capture only an "external" record becomes an event-record node
      cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
      if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        flags = cudaEventRecordExternal;
      a = c.take_event();
      cudaEventRecordWithFlags(a, st, flags);
    }
  }
  ~LaunchScope() {
    if (c.prof_on && a) {
      cudaEvent_t b = c.take_event();
      cudaEventRecordWithFlags(b, st, flags);
      c.prof_pending.push_back({name, a, b});
    }
  }
};
}  // namespace sv
