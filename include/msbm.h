/*
 * msbm.h -- C ABI of libmsbm: multi-scale hierarchical ZNCC block matching on one GPU.
 *
 * Method: Kaushik & Lall, "Fast Hierarchical depth map computation from stereo" (arXiv
 * 1901.09593).  A K-level Gaussian pyramid of a rectified stereo pair (Sec. III, Fig. 1);
 * a full-range zero-mean normalised cross-correlation (ZNCC, Eq. 1-2) winner-take-all
 * search at the coarsest level (Sec. III-A, Eq. 3-4); at every finer level a ZNCC search
 * restricted to a radius around the 2x nearest-neighbour upsample of the coarser disparity
 * (Sec. III-C, Eq. 8-9, first branch).
 *
 * Conventions shared by every entry point:
 *   - Images are 8-bit grayscale, row-major, (y, x) = (row, column).  The LEFT image is
 *     the reference: candidate disparity z compares left column x with right column x - z.
 *   - Candidates at level 0 are 0..D-1; at level k there are D_k = ceil(D / 2^k); a
 *     candidate is admissible only if z <= x.  Level k is ceil(W_{k-1}/2) x ceil(H_{k-1}/2).
 *   - Windows are (2n+1) x (2n+1), read clamp-to-edge.  A window with zero variance on
 *     either side scores 0.  Ties go to the smallest z.
 *   - Pyramid step: 5-tap binomial [1 4 6 4 1]/16 per axis, clamp-to-edge, 2x decimation,
 *     integer result rounded to nearest.
 *   - Device pointers are owned by the caller and must stay valid until the enqueued work
 *     has finished; the context owns only its internal buffers.  Output maps are dense
 *     (row pitch = width).  Disparities are int16, costs float32 (the winning ZNCC value,
 *     within about 1e-6 of its exact value).
 *   - Work is asynchronous on the stream given at creation.  Argument errors are returned
 *     synchronously before anything is enqueued.  CUDA launch errors are returned as
 *     MSBM_ERR_CUDA.  Device-side failures (a bounded wait that gave up) are recorded in the
 *     context and returned by msbm_sync.  No entry point aborts, throws or traps.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef MSBM_H
#define MSBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum msbm_status {
    MSBM_OK = 0,
    MSBM_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of range */
    MSBM_ERR_ALIGNMENT = 2,     /* a buffer misses its required alignment (the soft-argmax
                                   backward's workspace, 256 bytes) */
    MSBM_ERR_OOM = 3,           /* device or host allocation failed */
    MSBM_ERR_CUDA = 4,          /* a CUDA runtime call or launch failed */
    MSBM_ERR_TIMEOUT = 5,       /* a bounded device wait gave up (see MSBM_FLAG_TEST_TIMEOUT) */
    MSBM_ERR_UNSUPPORTED = 6    /* no usable sm_103a device, or a size beyond a kernel limit */
} msbm_status;

/* msbm_disparity enqueues its kernels directly instead of replaying a CUDA graph. */
#define MSBM_FLAG_NO_GRAPH 1u
/* Test hook: every bounded device wait gives up at once.  The kernel records
 * MSBM_ERR_TIMEOUT, drains its own copies in flight and returns without writing outputs. */
#define MSBM_FLAG_TEST_TIMEOUT 2u
/* The gated steps of the full method (Sec. III), each optional; none of them is the plain
 * method's hot path:
 *   ALPHA_REFINE     Eq. 5-7: at the coarsest level, pixels whose cost is not above alpha
 *                    take the argmax of the ZNCC averaged over their 3 x 3 neighbourhood;
 *   BETA_FALLBACK    Eq. 8-9, second branch: at finer levels, pixels whose bicubic cost
 *                    prior BI(C^{k+1}) (fine pixel (y, x) at coarse (y/2, x/2)) is not above
 *                    beta take the full search instead of the restricted one;
 *   SELECTIVE_MEDIAN Eq. 10: after each finer level, pixels whose cost is not above alpha
 *                    take the lower median of the 5 x 5 neighbours whose cost is above it. */
#define MSBM_FLAG_ALPHA_REFINE 4u
#define MSBM_FLAG_BETA_FALLBACK 8u
#define MSBM_FLAG_SELECTIVE_MEDIAN 16u
#define MSBM_FLAGS_FULL_METHOD (MSBM_FLAG_ALPHA_REFINE | MSBM_FLAG_BETA_FALLBACK | MSBM_FLAG_SELECTIVE_MEDIAN)
/* Per-level block size (Sec. III: the matching block size halves at every pyramid level):
 * `window` is level 0's; level k matches with half-width n_k = max(1, n_0 >> k), i.e.
 * windows 2 n_k + 1 (11, 5, 3, 3, ... for the paper's 11 x 11). */
#define MSBM_FLAG_WINDOW_HALVING 32u
/* Batch execution mode (msbm_batch_create, taken from pairs[0].flags): instead of one
 * persistent launch over the (pair, stage, tile) queue, one launch per group of stages that
 * share a tile function (pyramid groups, coarsest searches, statistics planes, then each
 * restricted level from the coarsest down), all pairs' tiles of a group in one grid,
 * captured in one CUDA graph.  Same results. */
#define MSBM_FLAG_BATCH_GROUPED 64u

/* Problem statement (Sec. III; window and pyramid depth as in Sec. IV). */
typedef struct msbm_params {
    int32_t width, height; /* level-0 size, 1..16384 each                                  */
    int32_t max_disp;      /* D, 1..4096: level-0 candidates 0..D-1                        */
    int32_t levels;        /* K, 1..12; K = 1 is flat full-range block matching             */
    int32_t window;        /* odd window side 2n+1, 3..13 (int32-exact sums up to 13x13);
                              level 0's with MSBM_FLAG_WINDOW_HALVING                      */
    int32_t radius;        /* r, 0..16: refinement candidates dhat-r .. dhat+r              */
    uint32_t flags;        /* MSBM_FLAG_*                                                   */
    float alpha;           /* threshold of ALPHA_REFINE and SELECTIVE_MEDIAN (paper: 0.9);
                              inside (-2, 2) when either flag is set (NaN is rejected)     */
    float beta;            /* threshold of BETA_FALLBACK (paper: 0.9); inside (-2, 2) when
                              that flag is set                                             */
} msbm_params;

typedef struct msbm_ctx msbm_ctx;

/* Library version (major*10000 + minor*100 + patch). */
int msbm_version(void);
/* Static text for a status code. */
const char *msbm_status_string(msbm_status s);

/* Validate params, allocate the pyramid and per-level output buffers on the current
 * device, and bind the context to `cuda_stream` (a cudaStream_t; NULL = legacy default).
 * *out is NULL on failure. */
msbm_status msbm_create(const msbm_params *params, void *cuda_stream, msbm_ctx **out);
/* Synchronise the stream and free everything the context owns.  NULL is accepted. */
msbm_status msbm_destroy(msbm_ctx *ctx);
/* Rebind the context to another stream (later work is enqueued there). */
msbm_status msbm_set_stream(msbm_ctx *ctx, void *cuda_stream);

/* Size and candidate count D_k of level `level` (0 = full resolution). */
msbm_status msbm_level_shape(const msbm_ctx *ctx, int32_t level, int32_t *w, int32_t *h,
                             int32_t *d_k);

/* Sec. III, Fig. 1: build all K levels of both images into the context.  `d_left`,
 * `d_right`: device images of the context's width x height, row pitch `pitch_bytes`
 * (>= width; any value). */
msbm_status msbm_pyramid(msbm_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right,
                         size_t pitch_bytes);

/* Copy level `level` of the left (which = 0) or right (which = 1) pyramid into the dense
 * device buffer `d_out` (W_k x H_k bytes).  For tests and inspection. */
msbm_status msbm_level_image(msbm_ctx *ctx, int32_t level, int32_t which, uint8_t *d_out);

/* One level of winner-take-all on the pyramid built by msbm_pyramid.
 *   d_prior == NULL: full search over 0..min(D_k-1, x)              (Sec. III-A, Eq. 3-4)
 *   d_prior != NULL: dense int16 map of level+1 (W_{k+1} x H_{k+1}); candidates
 *                    dhat-r .. dhat+r with dhat = 2*prior(y/2, x/2), clipped to
 *                    0..min(D_k-1, x) (dhat itself is first clamped into that range)
 *                                                                  (Sec. III-C, Eq. 8-9)
 * Writes d_out (int16, W_k x H_k) and cost_out (float, W_k x H_k, may be NULL). */
msbm_status msbm_match_level(msbm_ctx *ctx, int32_t level, const int16_t *d_prior,
                             int16_t *d_out, float *cost_out);

/* Gated steps on caller buffers of level `level` (dense W_k x H_k), for step-by-step use and
 * tests; msbm_disparity chains them itself when the flags ask for them.
 *   msbm_alpha_refine      : Eq. 5-7 in place on (d, cost), using the pyramid built by
 *                            msbm_pyramid; pixels with cost > alpha are untouched.
 *   msbm_selective_median  : Eq. 10, d_out from (d_in, cost); d_out must not alias d_in.
 *   msbm_match_level_beta  : Eq. 8-9 with both branches: prior and cost_prior are the
 *                            coarser level's maps (W_{k+1} x H_{k+1}); fallback_out (may
 *                            be NULL) receives 1 where the full search was taken. */
msbm_status msbm_alpha_refine(msbm_ctx *ctx, int32_t level, int16_t *d, float *cost);
msbm_status msbm_selective_median(msbm_ctx *ctx, int32_t level, const int16_t *d_in,
                                  const float *cost, int16_t *d_out);
msbm_status msbm_match_level_beta(msbm_ctx *ctx, int32_t level, const int16_t *d_prior,
                                  const float *cost_prior, int16_t *d_out, float *cost_out,
                                  uint8_t *fallback_out);

/* The whole hierarchical pass on device images: pyramid, coarsest full search, then the
 * restricted search at every finer level, with the gated steps the context's flags select.
 * Writes the level-0 maps (with SELECTIVE_MEDIAN, d_out holds the filtered map and cost_out
 * the matching cost it was filtered with).  Replays a CUDA graph
 * (re-captured when a pointer changes) unless MSBM_FLAG_NO_GRAPH. */
msbm_status msbm_disparity(msbm_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right,
                           size_t pitch_bytes, int16_t *d_out, float *cost_out);

/* Same pass on HOST buffers, waiting for the result: the images are copied into device
 * staging buffers (owned by the context, allocated on the first call), the pass runs on them
 * and the maps are copied back.  h_cost may be NULL (the disparity map alone comes back).
 * Page-locked buffers (cudaHostAlloc / cudaHostRegister, e.g. torch pin_memory) make the
 * copies asynchronous DMA transfers; pageable ones work too, at the driver's pageable-copy
 * speed.  The same as msbm_disparity_host_frames with one frame. */
msbm_status msbm_disparity_host(msbm_ctx *ctx, const uint8_t *h_left, const uint8_t *h_right,
                                size_t pitch_bytes, int16_t *h_d, float *h_cost);

/* A sequence of n_frames stereo pairs in HOST memory (a video stream), pipelined, waiting
 * for the last result.  Frame i (arrays of n_frames host pointers; images width x height at
 * pitch_bytes; maps dense) is uploaded on an upload stream into one of P device staging sets
 * (P = min(n_frames, 6)), matched, and its maps downloaded on a download stream, so that the
 * uploads of the next frames and the downloads of the previous ones overlap the pass of
 * frame i (they need page-locked buffers to overlap).  Frame i is matched on pass pipeline
 * i mod P: pipeline 0 is the context's stream, the others are contexts of the same
 * parameters with their own level buffers and streams, created on the first call that needs
 * them and freed with the context.  So consecutive frames' passes (chains of small,
 * latency-bound grids) run side by side.  The other pipelines' evaluations are not added to
 * msbm_eval_count.  h_costs may be NULL or hold NULLs (no cost map for that frame).  Results
 * equal msbm_disparity_host frame by frame.  Returns the first CUDA error, or the device
 * error word of any pipeline as msbm_sync does. */
msbm_status msbm_disparity_host_frames(msbm_ctx *ctx, int32_t n_frames, const uint8_t *const *h_lefts,
                                       const uint8_t *const *h_rights, size_t pitch_bytes,
                                       int16_t *const *h_ds, float *const *h_costs);

/* Copy the maps of an intermediate level (1..K-1) left by the last msbm_disparity into
 * the caller's dense device buffers (W_k x H_k; cost_out may be NULL).  Level 0 is written
 * to the caller's buffers by msbm_disparity itself. */
msbm_status msbm_level_result(msbm_ctx *ctx, int32_t level, int16_t *d_out, float *cost_out);

/* Timing aid: run the whole pass once with direct launches, recording a CUDA event
 * before the first kernel and after each stage on the context's stream, wait, and write
 * each stage's milliseconds to stage_ms in launch order:
 *   [0]          the pyramid (level-0 copy and reduces to levels 1 .. K-1, fused launches),
 *   [1]          the right-window statistics planes of levels 0 .. K-2 (one launch here;
 *                the pass itself runs them on side streams, beside the coarsest level's
 *                search and the coarser restricted levels; 0 when K = 1),
 *   [2]          full search at level K-1 (+ alpha refinement when enabled),
 *   [3 .. K+1]   levels K-2 .. 0: restricted search (+ beta gate and the fallback pixels' full search,
 *                + selective median, when enabled).
 * n_stages must be K + 2.  Results equal msbm_disparity's. */
msbm_status msbm_profile_disparity(msbm_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right,
                                   size_t pitch_bytes, int16_t *d_out, float *cost_out,
                                   float *stage_ms, int32_t n_stages);

/* Wait for the context's stream; return the first device-side error recorded since the
 * last msbm_sync (and clear it), else MSBM_OK. */
msbm_status msbm_sync(msbm_ctx *ctx);

/* Number of (pixel, candidate) ZNCC evaluations performed since the last call with
 * reset != 0 (synchronises the stream). */
msbm_status msbm_eval_count(msbm_ctx *ctx, int64_t *count, int32_t reset);

/* Kernel launches in one msbm_disparity call: the kernel nodes of the pass graph captured
 * by the last msbm_disparity (0 before the first call or with MSBM_FLAG_NO_GRAPH). */
msbm_status msbm_pass_kernel_count(const msbm_ctx *ctx, int32_t *count);

/* Tuning of the full-range search at `level` (used at the coarsest level and by K = 1):
 * tiles of 32*sx columns x 8 rows (sx in {1, 2, 4}) and z-blocks of `zblock` candidates
 * staged per pass (a multiple of 32; 0 = the largest the tile allows).  Results do not
 * depend on it.  The next msbm_disparity re-captures its graph. */
msbm_status msbm_set_level_tuning(msbm_ctx *ctx, int32_t level, int32_t sx, int32_t zblock);

/* ---------------------------------------------------------------------------------------
 * Batching: many pairs of different sizes, disparity ranges, depths, windows and radii
 * through the whole hierarchical pass (pyramid, coarsest full search, restricted levels)
 * in ONE persistent kernel launch over a (pair, stage, tile) work queue, replayed from a
 * CUDA graph.  The paper processes one pair at a time; this is a throughput addition with
 * the same per-pair results as msbm_disparity.
 *   pairs[i]         : per-pair parameters as for msbm_create (window 3..9 here; the flag
 *                      MSBM_FLAG_TEST_TIMEOUT on pairs[0] makes the queue withhold its first
 *                      stage so that every dependent wait gives up after ~1 ms: test hook).
 *   full_sx[i]       : NULL or the coarsest-level tile width 32*sx, sx in {1, 2}.
 *   full_zblock[i]   : NULL or the coarsest-level z-block (multiple of 32, 0 = maximum).
 * The batch owns each pair's pyramid and intermediate maps. */
typedef struct msbm_batch msbm_batch;
msbm_status msbm_batch_create(const msbm_params *pairs, int32_t n_pairs, const int32_t *full_sx,
                              const int32_t *full_zblock, void *cuda_stream, msbm_batch **out);
/* Enqueue one pass over all pairs.  Arrays of n_pairs device pointers (images width x
 * height at pitches[i]; level-0 maps dense; cost_outs may be NULL or hold NULLs).  When a
 * pointer differs from the previous call, the device pointer table is re-uploaded (this
 * waits for the stream).  Asynchronous otherwise. */
msbm_status msbm_batch_run(msbm_batch *b, const uint8_t *const *d_lefts,
                           const uint8_t *const *d_rights, const size_t *pitches,
                           int16_t *const *d_outs, float *const *cost_outs);
/* Wait for the stream; return (and clear) a recorded device error (MSBM_ERR_TIMEOUT). */
msbm_status msbm_batch_sync(msbm_batch *b);
msbm_status msbm_batch_eval_count(msbm_batch *b, int64_t *count, int32_t reset);
/* Copy pair `pair`'s map of level `level` (1 <= level < levels) from the last completed
 * run into caller device buffers (dense W_k x H_k; cost_out may be NULL), on the batch's
 * stream.  These are the priors the pair's finer levels searched around (Sec. III-C), so
 * each level of a batched pair can be checked on its own. */
msbm_status msbm_batch_level_result(msbm_batch *b, int32_t pair, int32_t level, int16_t *d_out,
                                    float *cost_out);
/* Queue length, persistent grid size (CTAs) and number of (pair, stage) segments. */
msbm_status msbm_batch_info(const msbm_batch *b, int64_t *n_items, int32_t *grid,
                            int32_t *n_segments);
msbm_status msbm_batch_destroy(msbm_batch *b);

/* ---------------------------------------------------------------------------------------
 * Differentiable level: soft-argmax readout of a ZNCC cost volume (Eq. 2 on float images).
 * For each pixel of each image of a batch (B x H x W, float32, dense, row-major):
 *   rho_z = sum ac*bc / sqrt((sum ac^2 + eps)(sum bc^2 + eps)) over the (2n+1)^2 window
 *           (ac, bc centred on their window means, clamp-to-edge reads), for the admissible
 *           candidates 0 <= z <= min(ndisp - 1, x);
 *   p_z    = softmax_z(rho_z / temperature);   d_soft = sum_z z p_z.
 * The cost volume is never stored.  window: odd 3..9; ndisp 1..256; batch 1..65535;
 * temperature > 0;
 * eps >= 0 (1e-6 * window^2 is the default used by the Python binding).
 * Forward writes d_soft, and the softmax statistics m_out (max of rho_z * log2(e) / T) and
 * l_out (sum of 2^(rho_z log2(e)/T - m)) that the backward reuses. */
msbm_status msbm_zncc_softargmax_fwd(const float *d_left, const float *d_right, int32_t batch,
                                     int32_t height, int32_t width, int32_t window, int32_t ndisp,
                                     float temperature, float eps, float *d_soft, float *m_out,
                                     float *l_out, void *cuda_stream);

/* Bytes of device workspace msbm_zncc_softargmax_bwd needs (0 for invalid sizes): the
 * per-(pixel, z) coefficient volume, six per-pixel arrays and four floats per position of
 * the window-extended image ((height + 2n) x (width + 2n), n = window / 2). */
size_t msbm_zncc_softargmax_workspace_bytes(int32_t batch, int32_t height, int32_t width,
                                            int32_t window, int32_t ndisp);

/* Backward of msbm_zncc_softargmax_fwd: given g_d = dLoss/dd_soft, writes g_left and
 * g_right (dLoss/dLeft, dLoss/dRight, same layout as the images; overwritten).  The window
 * statistics and rho are recomputed, not read from the forward.  workspace: caller-owned
 * device memory of at least msbm_zncc_softargmax_workspace_bytes, 256-byte aligned
 * (MSBM_ERR_ALIGNMENT otherwise).  Asynchronous on cuda_stream. */
msbm_status msbm_zncc_softargmax_bwd(const float *d_left, const float *d_right, int32_t batch,
                                     int32_t height, int32_t width, int32_t window, int32_t ndisp,
                                     float temperature, float eps, const float *d_soft,
                                     const float *m_in, const float *l_in, const float *g_d,
                                     float *g_left, float *g_right, void *workspace,
                                     size_t workspace_bytes, void *cuda_stream);

/* Bytes of caller-owned device memory msbm_zncc_softargmax_fwd_saved keeps for the backward
 * (0 for invalid sizes): rho for every (image, z, pixel), float [batch][ndisp][height][width],
 * then the left and right window statistics {mean, rsqrt(sum c^2 + eps)}, float2
 * [batch][height][width] each; every part 256-byte aligned. */
size_t msbm_zncc_softargmax_saved_bytes(int32_t batch, int32_t height, int32_t width, int32_t window,
                                        int32_t ndisp);

/* msbm_zncc_softargmax_fwd that also keeps, in `saved` (at least
 * msbm_zncc_softargmax_saved_bytes, 256-byte aligned: MSBM_ERR_ALIGNMENT otherwise), the
 * costs rho of Eq. 2 it evaluated (admissible z only) and the window statistics, for
 * msbm_zncc_softargmax_bwd_saved.  The same d_soft, m, l as msbm_zncc_softargmax_fwd. */
msbm_status msbm_zncc_softargmax_fwd_saved(const float *d_left, const float *d_right, int32_t batch,
                                           int32_t height, int32_t width, int32_t window, int32_t ndisp,
                                           float temperature, float eps, float *d_soft, float *m_out,
                                           float *l_out, void *saved, size_t saved_bytes, void *cuda_stream);

/* msbm_zncc_softargmax_bwd reading rho and the window statistics from `saved` (written by
 * msbm_zncc_softargmax_fwd_saved for the same images and arguments, unchanged since) instead
 * of recomputing them; the same gradients (the saved values are the recomputed ones).
 * workspace as for msbm_zncc_softargmax_bwd.  Asynchronous on cuda_stream. */
msbm_status msbm_zncc_softargmax_bwd_saved(const float *d_left, const float *d_right, int32_t batch,
                                           int32_t height, int32_t width, int32_t window, int32_t ndisp,
                                           float temperature, float eps, const float *d_soft,
                                           const float *m_in, const float *l_in, const float *g_d,
                                           const void *saved, size_t saved_bytes, float *g_left,
                                           float *g_right, void *workspace, size_t workspace_bytes,
                                           void *cuda_stream);

/* ---------------------------------------------------------------------------------------
 * Measurement support (the paper has no counterpart): issue-rate probe of one instruction
 * class, the denominator of the matching kernels' rooflines.
 *   kind   : 0 = 4-way byte dot product (dp4a), 1 = 32-bit funnel shift, 2 = FP32 FMA,
 *            3 = 32-bit integer add / logic, 4 = 32-bit shared-memory load.
 *   blocks : CTAs of 256 threads (1 .. 65536); iters: loop iterations (1 .. 2^24), each
 *            8 independent chains x 16 operations per thread.
 * Runs one launch on cuda_stream and waits for it; *ms = its CUDA-event time, *lane_ops =
 * the operations executed (blocks * 256 * iters * 128).  Allocates and frees a small
 * result buffer; changes no clock or device setting. */
msbm_status msbm_pipe_probe(int32_t kind, int32_t blocks, int32_t iters, void *cuda_stream, float *ms,
                            double *lane_ops);

/* ---------------------------------------------------------------------------------------
 * Allocation-free flat matching.  The paper has no counterpart: this is a deployment aid.
 *
 * Some callers cannot call cudaMalloc: cudaMalloc and cudaFree may synchronise the whole
 * device, which a real-time loop sharing the GPU with other streams cannot afford while a
 * frame is in flight, and some host frameworks own all device memory through their own
 * pool and forbid allocations made outside it.  For them this entry point runs flat
 * full-range block matching (the K = 1 case of msbm_disparity: every admissible candidate
 * 0 <= z <= min(max_disp - 1, x), winner-take-all, ties to the smallest z) without
 * allocating: it calls no cudaMalloc, cudaFree or other allocating routine.  Its scratch
 * (two replicated-apron image buffers and a status word) is a fixed device array of
 * MSBM_NOALLOC_SCRATCH_BYTES compiled into the library; every GPU that loads this part of
 * the library keeps that array until the process exits.
 *   d_left, d_right : device images, width x height, row pitch pitch_bytes (>= width).
 *   d_out           : device int16 map, width x height, dense.          (written)
 *   cost_out        : device float map, width x height, dense, or NULL. (written)
 *   d_status        : device int32, or NULL.  Set to 0 on the stream before the kernels
 *                     run; a device wait that gave up leaves MSBM_ERR_TIMEOUT there.
 *   cuda_stream     : cudaStream_t the work is enqueued on (asynchronous).
 * Sizes: width, height 1..16384, max_disp 1..4096, window odd 3..13.  A size whose two
 * apron buffers, (round_up(width + 32, 128) * (height + 16) bytes each, rounded up to 256)
 * plus 256 bytes, exceed MSBM_NOALLOC_SCRATCH_BYTES returns MSBM_ERR_UNSUPPORTED before
 * any work is enqueued (2880 x 1984 fits; 4096 x 2160 does not).
 * Every call resolves the array's device address in the current context with
 * cudaGetSymbolAddress and sets the kernel's shared-memory attribute (host calls that
 * allocate nothing), so a context re-created after cudaDeviceReset is served correctly.
 * The first call on a device may load the library's device code (CUDA's lazy module
 * loading); make that first call outside any stream capture.  All calls share the one array and it keeps the
 * last call's contents: calls whose work overlaps on the GPU (on different streams, or
 * from different host threads without ordering) race on it and must be serialised by the
 * caller. */
#define MSBM_NOALLOC_SCRATCH_BYTES (16 << 20)
msbm_status msbm_flat_disparity_noalloc(const uint8_t *d_left, const uint8_t *d_right,
                                        size_t pitch_bytes, int32_t width, int32_t height,
                                        int32_t max_disp, int32_t window, int16_t *d_out,
                                        float *cost_out, int32_t *d_status, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MSBM_H */
