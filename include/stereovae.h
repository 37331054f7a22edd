/*
 * stereovae.h -- C ABI of the GB300 StereoVAE hot path (arXiv 2305.11566).
 *
 * The library computes, for rectified grayscale stereo pairs:
 *   1. a quarter-size coarse disparity map: 4x4 box downsampling (Sec. I, IV-A
 *      "quarter size"), ZNCC matching scores (Eq. 1-3) over d = 0..D-1 and
 *      winner-take-all (Eq. 6);
 *   2. its refinement to full resolution by a small VAE-style network
 *      (Sec. III-B): bilinear x4 upsampling of the coarse map ("linear scaling",
 *      Sec. IV-C), a stride-2 conv encoder, latent mean / log-variance heads
 *      (Table I "mu & sigma"), a nearest-x2 upsampling conv decoder and a final
 *      conv whose output is added to the upsampled coarse map.
 *
 * Conventions for every entry point:
 *   - All image, map and tensor pointers are DEVICE pointers owned by the caller,
 *     except where a comment says "host".  The context owns its weights and
 *     workspaces.
 *   - Work is enqueued asynchronously on the given stream (0 = legacy default
 *     stream); the call returns once it is enqueued.  Outputs are valid after the
 *     stream is synchronised.
 *   - Arguments are validated on the host before anything is launched; an invalid
 *     call returns SV_ERR_INVALID_ARG (or SV_ERR_UNSUPPORTED) and launches nothing.
 *     No call aborts, throws or traps.  A CUDA failure returns SV_ERR_CUDA; a
 *     device-side bounded wait that ran out returns SV_ERR_TIMEOUT.  The text of the
 *     last error of a context is available from sv_last_error().
 *   - A context is not thread safe: one host thread at a time.
 *   - Images are uint8, row-major with a row pitch in bytes; pitch % 16 == 0 and
 *     base pointers 16-byte aligned (rows are read with 16-byte vector loads).
 *   - Coarse maps are (height / 4) x (width / 4) (floor), row-major, dense.
 *   - Full-resolution outputs are height x width FP32, row-major, dense.
 */
#ifndef STEREOVAE_H
#define STEREOVAE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SV_API __attribute__((visibility("default")))
#else
#define SV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* sv_stream; /* == cudaStream_t */

typedef enum {
  SV_OK = 0,
  SV_ERR_INVALID_ARG = 1,
  SV_ERR_CUDA = 2,
  SV_ERR_OOM = 3,
  SV_ERR_UNSUPPORTED = 4,
  SV_ERR_TIMEOUT = 5,
  SV_ERR_STATE = 6
} sv_status;

/* Arithmetic of the refinement convolutions.
 * SV_FP32: FP32 CUDA-core direct convolutions (the plain method).
 * SV_BF16: implicit-GEMM convolutions on the tcgen05 tensor cores, BF16 operands,
 *          FP32 accumulation; the last conv and the residual stay FP32.
 * SV_FP64_CHECK: FP64 CUDA-core convolutions, for gradient checks on small crops.
 * SV_FP8: the quantised refinement the paper names as future work (Sec. V), inference
 *          only: the quantised layers enc2, enc3, latent, dec1 and dec2 take E4M3 operands
 *          (tcgen05 kind::f8f6f4, FP32 accumulation).  Weights: per layer and output channel
 *          co the scale s_co = max |w| / 448 over the channel's GEMM operand (for dec1 and dec2
 *          the FP32 sums of the nearest-x2 phase folding; the border pixels of an odd crop use
 *          the unfolded 3 x 3 weights with their own scales), codes E4M3(w / s_co) (round to
 *          nearest even, saturating at 448).  Activations carry scale 1: e1 (BF16 from the
 *          first layer) and the outputs of enc2 .. dec1 are stored as E4M3 codes of
 *          relu(s_co * acc + bias); dec2 writes BF16.  The first layer, the last decoder layer
 *          (fused with the final conv where the widths allow), the upsampling and the residual
 *          are as SV_BF16.  enc, latent and dec1 widths are multiples of 32.  sv_refine_train
 *          returns SV_ERR_UNSUPPORTED;
 *          sv_debug_activation returns e1 .. d1 as E4M3 bytes. */
typedef enum { SV_FP32 = 0, SV_BF16 = 1, SV_FP64_CHECK = 2, SV_FP8 = 3 } sv_precision;

/* sv_config.flags: selects the refinement network.
 * 0: the small VAE-style net described above (widths from enc_ch / latent_ch / dec_ch).
 * SV_NET_TABLE1: the paper's own network (Sec. III-B1, Table I), FP32 only (precision
 *   SV_FP32; the width fields are ignored).  At half resolution (ceil(H/2) x ceil(W/2)) the
 *   inputs are X_0 = 4 x bilinear x2 of the coarse map / 256 (the disparity in
 *   full-resolution pixels, normalised) and X_1 = 2 x 2 box mean of the left image / 256;
 *   FE_1 = conv5(X_0) and FE_2 = conv5(X_1) (32 channels each); encoder EN_1 = conv5 s2
 *   (FE_1 & FE_2) -> 16, EN_1_R = conv5(EN_1) -> 8, EN_2 = conv5 s2 (EN_1 & EN_1_R) -> 32,
 *   EN_2_R = conv5(EN_2) -> 16, heads = conv1(EN_2 & EN_2_R) -> mu, sigma; decoder input
 *   (mu - 1) + eps exp(sigma - 1) (Eq. 8; eps = 0 at inference), D_1 = conv1 -> 32, D_1_R =
 *   conv5(D_1 & EN_2 & EN_2_R) -> 16, D_2 = deconv5 s2 (D_1 & EN_2 & EN_2_R & D_1_R) -> 16,
 *   D_2_R = conv5(D_2 & EN_1 & EN_1_R) -> 8, D = deconv5 s2 (D_2 & EN_1 & EN_1_R & D_2_R) -> 16;
 *   output Y = deconv5 s2 (D & X_0 & FE_1 & FE_2) -> 1 at H x W; "&" concatenates channels
 *   in that order; leaky ReLU 0.1 after every layer but the heads and Y; every conv and
 *   deconv has a bias and padding 2 (5 x 5); a stride-2 conv gives ceil(n/2) and a stride-2
 *   deconv 2n cropped to the size of the level it returns to.  The refined disparity is 256 Y
 *   (pixels).  Parameters: per layer in the order above W[co][ky][kx][ci] then b[co]
 *   (162,380).  sv_refine / sv_pipeline / sv_pipeline_ex / sv_pipeline_host run it;
 *   sv_refine_train runs its training forward (eps and mu / sigma of [H8][W8][1], sigma in the
 *   logvar_out slot); sv_loss_paper is its loss; sv_refine_backward, sv_loss, sv_adam_step,
 *   sv_autotune and sv_debug_activation return SV_ERR_UNSUPPORTED on such a context. */
enum { SV_NET_TABLE1 = 1 };

/* Network and matcher configuration (copied by sv_create). */
typedef struct {
  int window;     /* ZNCC window side k: odd, 3 <= k <= 15 (Eq. 1-3 window W) */
  int enc_ch[3];  /* encoder widths, each a multiple of 16, <= 256 */
  int latent_ch;  /* latent (mean / logvar) width, multiple of 16, <= 256 */
  int dec_ch[3];  /* decoder widths, each a multiple of 16, <= 256 */
  int precision;  /* sv_precision */
  int flags;      /* 0 or SV_NET_TABLE1 */
} sv_config;

/* One stereo pair.  left / right: device, [height][pitch] uint8. */
typedef struct {
  const uint8_t* left;
  const uint8_t* right;
  int width;    /* W >= 4 * window; W / 4 coarse columns */
  int height;   /* H >= 4 * window; H / 4 coarse rows */
  int pitch;    /* bytes per row, >= width, multiple of 16 */
  int max_disp; /* D: candidates d = 0..D-1 coarse pixels; 1 <= D <= 128 and D <= W / 4 */
} sv_pair;

typedef struct sv_ctx sv_ctx;

/* Status code name (static string). */
SV_API const char* sv_status_string(sv_status s);

/* Text of the last error on this context ("" if none); valid until the next call. */
SV_API const char* sv_last_error(const sv_ctx* ctx);

/* Number of FP32 parameters of a configuration.  Flat layout, per layer in the
 * order enc1, enc2, enc3, mu, logvar, dec1, dec2, dec3, final: W[cout][kh][kw][cin]
 * then b[cout].  enc1 has cin = 2 (left / 256, upsampled disparity / 256), the
 * latent heads are 1x1, final has cout = 1; all other kernels are 3x3.
 * Returns 0 for an invalid configuration. */
SV_API size_t sv_param_count(const sv_config* cfg);

/* Create a context on CUDA device `device` (made current for the call).
 * Weights start at zero; set them with sv_set_weights. */
SV_API sv_status sv_create(const sv_config* cfg, int device, sv_ctx** out);

/* Release a context and everything it owns (synchronises its device). */
SV_API sv_status sv_destroy(sv_ctx* ctx);

/* Copy n = sv_param_count() FP32 parameters (host or device pointer) into the
 * context's FP32 master copy and refresh the BF16 / FP64 copies. Synchronous. */
SV_API sv_status sv_set_weights(sv_ctx* ctx, const float* params, size_t n);

/* Copy the FP32 master parameters out (host or device pointer). Synchronous. */
SV_API sv_status sv_get_weights(sv_ctx* ctx, float* params, size_t n);

/* Coarse matching of n_pairs pairs (Eq. 1-3, Eq. 6).
 * For pair i, disp_out[i] receives the (H/4) x (W/4) int16 WTA disparity
 * d* = argmax_d rho(x, y, d) over valid candidates (x - d >= 0, d < D), lowest d
 * on ties; rho is the ZNCC of the k x k windows of 4x4 box sums centred at (x, y)
 * in the left and (x - d, y) in the right image, window pixels clamped to the
 * image, rho = 0 for a window of zero variance.  best[i] / second[i] (the arrays,
 * or any of their entries, may be NULL) receive FP32 rho(d*) and the largest rho of
 * the other valid candidates (-2 when there is none).
 * All pairs are processed by one launch. */
SV_API sv_status sv_coarse_match(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, int16_t* const* disp_out,
                          float* const* best, float* const* second, sv_stream stream);

/* Inference refinement (z = mu) of n_pairs pairs given their coarse maps
 * (coarse[i]: (H/4) x (W/4) int16, e.g. from sv_coarse_match; values are used as
 * disparities in coarse pixels).  disp_out[i]: H x W FP32 refined disparity in
 * full-resolution pixels: Y = U + net(L / 256, U / 256) where U is the bilinear x4
 * upsampled coarse map times 4. */
SV_API sv_status sv_refine(sv_ctx* ctx, const sv_pair* pairs, const int16_t* const* coarse, int n_pairs,
                    float* const* disp_out, sv_stream stream);

/* Semi-global matching variant of the coarse stage (Sec. III-A, Eq. 1 and 4-6).  For every
 * pair: the ZNCC cost volume C = 1 - rho of Eq. 1-3 on the quarter-size images (window side =
 * the context's window, clamp-to-edge windows; candidates with x - d < 0 cost 2, the largest
 * value of Eq. 1), aggregated by Eq. 4 along `npaths` directions taken in the order
 * left-to-right, right-to-left, top-to-bottom, bottom-to-top (1..4) and summed (Eq. 5), then
 * winner-take-all (Eq. 6, lowest d on ties) into disp_out[i] ((H/4) x (W/4) int16, device).
 * P1 (change of one disparity) and P2 (larger changes) are the penalties of Eq. 4, both >= 0;
 * the paper does not give their values.  cost_out (nullable array; entries nullable)
 * receives the aggregated volume [H/4][W/4][max_disp] FP32 (device).  Returns
 * SV_ERR_INVALID_ARG for a negative penalty, npaths outside 1..4 or a NULL disp_out entry.
 * Equivalent to sv_coarse_match_ex with SV_COST_ZNCC, SV_AGG_SGM and no post-processing.
 * Asynchronous on `stream`; the context's work buffers are reused by the next call. */
SV_API sv_status sv_coarse_match_sgm(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, float P1, float P2, int npaths,
                                     int16_t* const* disp_out, float* const* cost_out, sv_stream stream);

/* Matching cost of the coarse stage: ZNCC (Eq. 1-3) or the census cost the paper's
 * robustness study pairs with it (Sec. IV-C, settings S1 and S2). */
typedef enum { SV_COST_ZNCC = 0, SV_COST_CENSUS = 1 } sv_cost_kind;

/* Cost aggregation: none (plain winner-take-all, Eq. 6), semi-global matching (Eq. 4-5) or
 * the domain-transform aggregation of the robustness study (Sec. IV-C, settings S1, S3). */
typedef enum { SV_AGG_NONE = 0, SV_AGG_SGM = 1, SV_AGG_DT = 2 } sv_aggregation;

/* Post-processing of the winner-take-all map (Sec. III-A, Eq. 7 and the text after it),
 * applied in this order when both are set. */
enum { SV_POST_SMP = 1, SV_POST_MEDIAN = 2 };

/* Options of sv_coarse_match_ex / sv_pipeline_ex.
 *  census_window: SV_COST_CENSUS: odd side kc of the census window, 3, 5 or 7 (bit = 1 where a
 *                 window pixel of the quarter-size image is below the centre, clamped window;
 *                 cost = Hamming distance of the codes of (x, y) and (x - d, y), kc^2 - 1 where
 *                 x - d < 0).
 *  P1, P2, npaths: SV_AGG_SGM: penalties (>= 0, units of the cost) and directions (1..4), as
 *                 for sv_coarse_match_sgm.
 *  dt_sigma_s, dt_sigma_r, dt_iters: SV_AGG_DT: spatial scale (coarse pixels, > 0), range
 *                 scale (intensity levels 0..255 of the quarter-size left image, > 0) and
 *                 iterations (1..8) of the recursive domain-transform filter applied to every
 *                 disparity slice, rows (both ways) then columns (both ways) per iteration,
 *                 iteration i of N at scale dt_sigma_s sqrt(3) 2^(N-i) / sqrt(4^N - 1).
 *  post:          SV_POST_* flags. */
typedef struct {
  int cost;
  int census_window;
  int aggregation;
  float P1, P2;
  int npaths;
  float dt_sigma_s, dt_sigma_r;
  int dt_iters;
  int post;
} sv_coarse_opts;

/* Coarse stage with a chosen cost, aggregation and post-processing.  For every pair: the cost
 * volume of `opts->cost` on the quarter-size images (ZNCC: C = 1 - rho with the context's
 * window, 2 where x - d < 0), aggregated by `opts->aggregation`, winner-take-all (argmin over
 * d, lowest d on ties; with SV_COST_ZNCC and SV_AGG_NONE the exact argmax of rho of
 * sv_coarse_match), then the single-matching-phase check (SV_POST_SMP: of two pixels of a row
 * matched to the same target column x - d within D, the left one keeps its disparity; every
 * other pixel takes the disparity of the nearest kept pixel of its row, the left one at equal
 * distance) and a 3 x 3 median filter with clamped edges (SV_POST_MEDIAN).  disp_out[i]:
 * (H/4) x (W/4) int16 (device).  cost_out (nullable array; entries nullable): the aggregated
 * volume [H/4][W/4][max_disp] FP32 (the raw cost with SV_AGG_NONE).  SV_ERR_INVALID_ARG for a
 * NULL or out-of-range option.  Asynchronous on `stream`. */
SV_API sv_status sv_coarse_match_ex(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const sv_coarse_opts* opts,
                                    int16_t* const* disp_out, float* const* cost_out, sv_stream stream);

/* The post-processing of sv_coarse_match_ex alone, on given coarse maps: disp_in[i] and
 * disp_out[i] are (H/4) x (W/4) int16 device maps of pair i (sizes and max_disp are taken
 * from pairs[i]; the image pointers are not read and may be NULL); post = SV_POST_* flags
 * (0 copies).  disp_out[i] must not overlap disp_in[i].  Asynchronous on `stream`. */
SV_API sv_status sv_postprocess(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const int16_t* const* disp_in,
                                int post, int16_t* const* disp_out, sv_stream stream);

/* sv_pipeline with the coarse stage of sv_coarse_match_ex: coarse maps by `opts`, then the
 * refinement of sv_refine (the context's form), into disp_out[i] (H x W FP32, device). */
SV_API sv_status sv_pipeline_ex(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const sv_coarse_opts* opts,
                                float* const* disp_out, sv_stream stream);

/* Coarse matching followed by refinement (sv_coarse_match + sv_refine) with the
 * coarse maps kept in the context's workspace. */
SV_API sv_status sv_pipeline(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, float* const* disp_out, sv_stream stream);

/* Training forward of n_pairs pairs: z = mu + eps * exp(logvar / 2) (the
 * reparameterisation of Eq. 8 in its standard form).  Saves in the context what
 * sv_refine_backward needs (decoder activations and the latent; the encoder is
 * recomputed there).  On SV_BF16 contexts the encoder and decoder convolutions run on
 * the tensor cores (BF16 operands, FP32 accumulation, FP32 master weights) and the
 * backward runs in FP32; SV_FP32 runs FP32 throughout, SV_FP64_CHECK FP64.  Element type of coarse, eps, disp_out, mu_out and logvar_out
 * is float for SV_FP32 / SV_BF16 contexts and double for SV_FP64_CHECK contexts.
 * coarse[i]: (H/4) x (W/4) real-valued coarse map; eps[i], mu_out[i], logvar_out[i]:
 * latent tensors [H3][W3][latent_ch] with H3 = ceil(ceil(ceil(H/2)/2)/2) (same for W3);
 * disp_out[i]: H x W. */
SV_API sv_status sv_refine_train(sv_ctx* ctx, const sv_pair* pairs, const void* const* coarse, const void* const* eps,
                          int n_pairs, void* const* disp_out, void* const* mu_out, void* const* logvar_out,
                          sv_stream stream);

/* Backward of the last sv_refine_train on this context.  grad_disp[i],
 * grad_mu[i], grad_logvar[i]: gradients of the loss w.r.t. that call's outputs
 * (grad_mu / grad_logvar arrays or entries may be NULL = zero).  grad_params
 * (device, sv_param_count elements, same element type rule) is OVERWRITTEN with the
 * gradient summed over the pairs.  grad_coarse (array or entries may be NULL)
 * receives d loss / d coarse[i] (through the residual and the network input).
 * Returns SV_ERR_STATE if no training forward preceded it. */
SV_API sv_status sv_refine_backward(sv_ctx* ctx, const void* const* grad_disp, const void* const* grad_mu,
                             const void* const* grad_logvar, void* grad_params, void* const* grad_coarse,
                             sv_stream stream);

/* Loss of Sec. III-B2 as used here: smooth-L1 (beta = 1 px) of disp - gt summed over
 * all pixels of all pairs and divided by their number, plus kl_weight times the KL
 * divergence of N(mu, exp(logvar)) from N(0, 1) summed over all latent elements and
 * divided by their number.  loss_out (device, 3 values of the context's element
 * type): total, reconstruction, KL.  grad_* (arrays or entries nullable) receive
 * the gradients of the total w.r.t. disp, mu and logvar.  Element types as for
 * sv_refine_train; gt[i] is always float. */
SV_API sv_status sv_loss(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const void* const* disp, const float* const* gt,
                  const void* const* mu, const void* const* logvar, double kl_weight, void* loss_out,
                  void* const* grad_disp, void* const* grad_mu, void* const* grad_logvar, sv_stream stream);

/* Loss of the paper's Table I network (Sec. III-B2, Eq. 9-11), as read here:
 * Loss_1 = (sum over non-occluded pixels of |gt - Y| / 256 + sum over all pixels of
 * |gt - Y| / 256) / (number of pixels), i.e. non-occluded pixels weigh twice the occluded
 * ones; Loss_2 = mean over the latent elements of the KL divergence of N(mu - 1,
 * exp(sigma - 1)^2) (the distribution Eq. 8 samples) from N(0, 1),
 * 0.5 ((mu - 1)^2 + exp(2 (sigma - 1)) - 1 - 2 (sigma - 1)); total = 256 (Loss_1 + Loss_2).
 * Sums run over all pairs of the call.  Y[i], gt[i]: H x W FP32 disparities in pixels (device);
 * noc[i]: H x W uint8, non-zero where the pixel is not occluded; mu[i], sigma[i]: [H8][W8] FP32
 * (H8 = ceil(ceil(ceil(H/2)/2)/2)).  loss_out: device, 3 doubles (total, Loss_1, Loss_2).
 * grad_* (arrays or entries nullable): FP32 gradients of the total w.r.t. Y, mu and sigma
 * (the subgradient 0 where Y = gt).  The reduction order is fixed: repeated calls give
 * identical sums.  Available on every context. */
SV_API sv_status sv_loss_paper(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const float* const* Y,
                               const float* const* gt, const uint8_t* const* noc, const float* const* mu,
                               const float* const* sigma, double* loss_out, float* const* grad_Y,
                               float* const* grad_mu, float* const* grad_sigma, sv_stream stream);

/* One Adam step (Sec. IV-A) on the context's master weights with gradient grad
 * (device, sv_param_count elements, context element type): t = step (1-based),
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, p -= lr mhat / (sqrt(vhat) + eps).
 * Refreshes the BF16 copies. */
SV_API sv_status sv_adam_step(sv_ctx* ctx, const void* grad, int step, double lr, double beta1, double beta2, double eps,
                       sv_stream stream);

/* sv_pipeline with HOST buffers: pairs[i].left / right are host pointers (pinned or
 * pageable; any pitch >= width, no alignment rule) and disp_out[i] host H x W FP32.
 * The images are copied into the context's device workspace on `stream`, the
 * pipeline runs there and the results are copied back; returns after the stream has
 * been synchronised.  With option "host_copy" and device-accessible host memory (pinned /
 * mapped) one kernel gathers all images (and optionally one writes all results back),
 * reading and writing host memory directly; otherwise one copy call per buffer. */
SV_API sv_status sv_pipeline_host(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, float* const* disp_out,
                                  sv_stream stream);

/* Per-kernel timing.  While enabled, every kernel the context launches is bracketed by
 * two CUDA events recorded on the launching stream. */
typedef struct {
  char name[32];   /* kernel / layer name */
  long long launches;
  double total_ms;
} sv_profile_entry;

SV_API sv_status sv_profile_enable(sv_ctx* ctx, int enable);

/* Synchronises the pending events, adds them to the per-name totals, copies up to
 * max_entries totals into out (sorted by name) and sets *n_out to the number of names.
 * reset != 0 clears the totals afterwards. */
SV_API sv_status sv_profile_read(sv_ctx* ctx, sv_profile_entry* out, int max_entries, int* n_out, int reset);

/* Autotuner of the tensor-core forms (SV_BF16, SV_FP8): for each tensor-core layer picks
 * the strip height (rows of 128-unit tiles one work item walks down), the output-channel
 * slice per CTA and
 * the number of CTAs sharing an SM (1-3; the row prefetch ring shrinks to fit) that run
 * fastest on this batch, timing every candidate with CUDA events on `stream`.
 * The choice stays in the context and applies to later calls.  cache_path (nullable): a
 * JSON-lines file; an entry for this (GPU, SM count, network, window, precision,
 * batch-shape bucket) is loaded instead of tuning, a new result is appended.  Synchronous.
 * Returns SV_ERR_UNSUPPORTED on other precisions. */
SV_API sv_status sv_autotune(sv_ctx* ctx, const sv_pair* pairs, int n_pairs, const char* cache_path,
                             sv_stream stream);

/* The tuned launch shape (6 layers: enc2, enc3, latent, dec1, dec2, dec3): strip rows
 * (0 = automatic), N slice (0 = full width), CTAs per SM (0 = the "tc_ctas_per_sm"
 * option) and the measured microseconds per launch (-1 when loaded from a cache).  Any
 * pointer may be NULL. */
SV_API sv_status sv_tuning(const sv_ctx* ctx, int* rows6, int* nt6, int* ctas6, double* us6);

/* Waits for `stream` and reports device-side failures recorded since the previous
 * call: SV_ERR_TIMEOUT if a kernel's bounded wait ran out (the kernel then returned
 * early and its outputs are undefined), SV_ERR_CUDA for a CUDA error.  Clears the
 * recorded state. */
SV_API sv_status sv_synchronize(sv_ctx* ctx, sv_stream stream);

/* Tuning / test options (0 = default where noted):
 *   "spin_limit"     clock cycles one device-side wait may spin before it gives up
 *                    (default 4e9, about 2 s)
 *   "tc_strip_rows"  rows per work item of the tensor-core convolutions (0 = automatic)
 *   "tc_ctas_per_sm" 0 (default): each tensor-core convolution stages as many input rows
 *                    ahead as shared memory holds; k = 1..4: fewer, so that k CTAs share
 *                    an SM
 *   "fused_final"    1 (default): an SV_BF16 inference call computes the last decoder
 *                    layer, the final conv and the residual in one kernel (d3 stays in
 *                    shared memory) when the decoder widths allow it and every output
 *                    width is even; 0: separate kernels (d3 materialised in HBM)
 *   "fused_ring"     0 (default): the fused kernel stages as many input rows ahead as
 *                    shared memory holds; 4..16: at most this many rows in its ring
 *   "split_rows"     1 (default): a tensor-core layer whose shared memory holds no staged
 *                    row beyond its tile's own stages channel blocks of rows, so that the
 *                    next tile's input loads while the current tile still computes; 0: rows
 *   "enc1_tensor"    1 (default): the first encoder layer of an SV_BF16 context runs on the
 *                    tensor cores (im2col tile in shared memory; widths 16, 32, 64); 0: CUDA
 *                    cores (FP32 FMA)
 *   "fused_prefetch" 0..16 (default 4): the fused kernel's producer prefetches the input row
 *                    this many rows ahead into L2 (0: no prefetch)
 *   "host_copy"      sv_pipeline_host with device-accessible (pinned) host buffers: 0 one
 *                    copy call per buffer, 1 (default) one kernel gathers the images and
 *                    the results go back by copy calls, 2 kernels both ways (GPU writes
 *                    to host memory were the slowest of the three on GB300)
 *   "host_chunks"    1..4 (default 3): sv_pipeline_host computes a batch in up to this many
 *                    parts (at least 8 pairs each) and copies a part's results back while
 *                    the next part computes
 *   "debug_plans"    1: print each tensor-core layer's launch plan (ring depth, shared
 *                    memory, CTAs per SM, grid, strips) to stderr when a call is prepared
 *   "graphs"         1 (default): sv_pipeline on an SV_BF16 or SV_FP8 context captures each batch
 *                    signature in a CUDA graph and replays it (not on the legacy or
 *                    per-thread default stream); 0: launch eagerly
 * Returns SV_ERR_INVALID_ARG for an unknown key or a value out of range. */
SV_API sv_status sv_set_option(sv_ctx* ctx, const char* key, long long value);

/* Test hook: copies activation `which` (0 e1, 1 e2, 2 e3, 3 z, 4 d1, 5 d2, 6 d3; NHWC
 * BF16) of pair `pair` of the last SV_BF16 refinement call into host memory `dst`
 * (`bytes` must equal the activation's size).  Synchronous.  d3 is SV_ERR_STATE after a
 * call that fused the final conv (option "fused_final"). */
SV_API sv_status sv_debug_activation(sv_ctx* ctx, int which, int pair, void* dst, size_t bytes);

/* sv_coarse_match without any device allocation, and without a context.
 *
 * For callers that cannot allocate device memory at the moment they need a coarse map:
 * real-time loops that must not block on the allocator (cudaMalloc can synchronise the
 * device), and plugins whose host owns the whole device memory budget and hands the
 * library only its inputs and outputs.  The paper has no counterpart: this is a
 * deployment entry point.
 *
 * Same inputs, outputs, results and status codes as sv_coarse_match; `window` is the ZNCC
 * window side (odd, 3..15).  The call's work tables are kept in a fixed array compiled
 * into the library (540,672 bytes, held on every GPU that loads the library until the
 * process exits): at most 256 pairs and 32768 jobs per call, where a pair of W x H needs
 * ceil((H/4) / 8) * ceil((W/4) / (8 * TX)) jobs (TX = 32, 20, 16, 12 for D up to 32, 64,
 * 96, 128).  Larger calls return SV_ERR_UNSUPPORTED and launch nothing; other invalid
 * arguments return SV_ERR_INVALID_ARG.  The tables are uploaded on `stream` from host
 * memory that lives only for the duration of the call.  The first call on a device looks
 * up the array's device address with that device current and caches it for the life of
 * the process: do not call this entry point on a device after cudaDeviceReset.  All calls
 * share the one array and each overwrites it: calls whose work can overlap on the GPU
 * (other streams, no ordering between them) race and must be ordered by the caller.  It
 * calls no cudaMalloc, cudaFree or allocating library routine. */
SV_API sv_status sv_coarse_match_static(const sv_pair* pairs, int n_pairs, int window, int16_t* const* disp_out,
                                        float* const* best, float* const* second, sv_stream stream);

/* Number of kernels the context has launched since it was created. */
SV_API long long sv_launch_count(const sv_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* STEREOVAE_H */
