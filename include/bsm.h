/*
 * bsm.h - C ABI of the GB300-native Binary Stereo Matching library (libbsm.so).
 *
 * Method: K. Zhang, J. Li, Y. Li, W. Hu, L. Sun, S. Yang, "Binary Stereo Matching", Sec. 3.
 *   describe              Eq. 2-3 (BRIEF descriptor B(x)) and Eq. 5-7 (binary mask Phi(x))
 *   cost_aggregate_wta    Eq. 8 (masked Hamming cost), a square-window box sum of that cost,
 *                         and Eq. 1 (winner-take-all), for the left and for the right view
 *   refine                the left/right check and the voting refinement of Eq. 9-10
 *
 * Conventions for every entry point:
 *   - Image, descriptor, disparity and cost buffers are DEVICE pointers owned by the caller; the
 *     library never frees them and keeps no reference after the call returns.
 *   - RGB images are 8-bit, 3 bytes per pixel (R, G, B), rows of pitch_bytes >= 3 * width.
 *   - Descriptor planes B and Phi are uint32 [height][width][n_bits / 32]; pair i (0-based) of the
 *     sampling table is bit (i % 32) of word (i / 32), i.e. the weight 2^(i-1) of the paper's
 *     1-based sum in Eq. 2 and Eq. 7.
 *   - Disparity maps are int32 [height][width]; the cost volume is uint16 [height][width][dmax]
 *     (d fastest).
 *   - `stream` is a cudaStream_t (NULL selects the legacy default stream). Work is enqueued
 *     asynchronously on it; argument errors are returned synchronously before anything is
 *     enqueued. Errors detected inside a kernel (a bounded wait that gave up) are latched in a
 *     device status word read by bsm_last_error().
 *   - A context is not thread-safe: use one context per host thread. Its calls share the
 *     context's scratch memory, so calls on one context must not overlap on the GPU: issue them on
 *     one stream, or order the streams with events.
 *   - Calls allocate nothing except where stated: bsm_describe and bsm_refine grow the context's
 *     scratch the first time they see an image larger than any before (bsm_reserve sizes it up
 *     front, which is required before capturing calls into a CUDA graph).
 *   - No C++ exception crosses this ABI.
 */
#ifndef BSM_H
#define BSM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bsm_ctx bsm_ctx;

typedef enum {
  BSM_OK = 0,
  BSM_ERR_INVALID_ARG = 1,   /* a size, pointer or parameter is out of its documented range */
  BSM_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation of the context failed */
  BSM_ERR_CUDA = 3,          /* a CUDA runtime call or a kernel launch failed */
  BSM_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up (see bsm_last_error) */
  BSM_ERR_UNSUPPORTED = 5    /* valid per the paper, not built in this library version */
} bsm_status;

/* Parameters of the method, fixed at bsm_create. */
typedef struct {
  int32_t n_bits;        /* descriptor length n (Eq. 2): a multiple of 32; this version builds the
                            powers of two 32 ... 4096 (the paper uses 4096, Sec. 4.1). Batching and
                            serving take n_bits <= 256. */
  int32_t window_S;      /* sampling window S (Sec. 3): every offset satisfies |off| <= S / 2;
                            3..63 */
  const int8_t *pairs;   /* HOST pointer to n_bits entries of 4 int8 (px, py, qx, qy): the offsets of
                            p_i and q_i from the centre pixel (Eq. 2). Copied at create; the caller
                            keeps ownership. */
  int32_t agg_window;    /* odd side of the square box window that sums Eq. 8's cost before Eq. 1;
                            1 is the paper's method exactly. n_bits * agg_window^2 <= 65535;
                            this version builds 1, 3, 5 and 7. */
  int32_t mask_rank;     /* k: T of Eq. 6 is the k-th smallest weight (1-based), 1..n_bits;
                            0 selects n_bits / 4 (the paper's "quarter smallest value") */
  int32_t dmax;          /* largest disparity range any call will use: d in [0, dmax-1]
                            (Eq. 1); 1..256 */
  int32_t lr_tol;        /* left/right check tolerance in pixels (>= 0; default 1) */
  int32_t vote_radius;   /* R: the refinement votes over a (2R+1)^2 window (0..31; default 15) */
  int32_t lambda_c;      /* lambda_c of Eq. 10 (paper: 9), > 0 */
  int32_t lambda_e;      /* lambda_e of Eq. 10 (paper: 16), > 0 */
  int32_t mask_mode;     /* which mask weights Eq. 8's Hamming distance (BSM_MASK_*):
                            BSM_MASK_REFERENCE (0): the reference pixel's Phi, the paper's method;
                            BSM_MASK_NONE (1): no mask, the plain descriptor distance of Eq. 4
                            (Phi is written as all ones; mask_rank must be 0 or n_bits);
                            BSM_MASK_BOTH (2): Phi of the reference pixel AND Phi of its match, an
                            ablation of the paper's choice (n_bits >= 256; per-pair calls only) */
} bsm_params;

#define BSM_MASK_REFERENCE 0
#define BSM_MASK_NONE 1
#define BSM_MASK_BOTH 2

/*
 * Create a context on the current CUDA device: validates the parameters, uploads the sampling
 * pairs, builds the 2^24-entry colour table (packed CIELAB + intensity, see bsm_copy_color_table)
 * and the integer vote tables of Eq. 10 on that device. Synchronous.
 * Returns BSM_ERR_INVALID_ARG / BSM_ERR_UNSUPPORTED for bad parameters (before touching the GPU),
 * BSM_ERR_OUT_OF_MEMORY or BSM_ERR_CUDA on device failure. *out is set only on BSM_OK.
 */
bsm_status bsm_create(const bsm_params *params, bsm_ctx **out);

/* Release the context and everything it owns. Synchronises the device first. NULL is allowed. */
void bsm_destroy(bsm_ctx *ctx);

/*
 * Size the context's scratch for images of up to max_w x max_h pixels (synchronises the device if
 * the scratch grows). Afterwards no call on images within that size allocates.
 */
bsm_status bsm_reserve(bsm_ctx *ctx, int32_t max_w, int32_t max_h);

/*
 * Eq. 2-3 and Eq. 5-7 for every pixel of one view.
 *   rgb_dev      device RGB image, h rows of pitch_bytes
 *   B_dev        device uint32 [h][w][n_bits/32] output: B(x), bit i = [I(p_i) > I(q_i)]
 *   Phi_dev      device uint32 [h][w][n_bits/32] output: Phi(x), bit i = [w_i <= T] with
 *                w_i = max(SAD(x, p_i), SAD(x, q_i)) in integer CIELAB and T the mask_rank-th
 *                smallest w_i
 * Intensity is I = (77 R + 150 G + 29 B + 128) >> 8. Sampling positions outside the image are
 * clamped to the border. Sizes: 1 <= w, h <= 16384, pitch_bytes >= 3 w. B and Phi must be
 * 16-byte aligned. Uses the context's scratch (a w * h colour plane), grown here if too small.
 */
bsm_status bsm_describe(bsm_ctx *ctx, const uint8_t *rgb_dev, int32_t w, int32_t h, int32_t pitch_bytes,
                        uint32_t *B_dev, uint32_t *Phi_dev, void *stream);

/*
 * Eq. 8 + box aggregation + Eq. 1, once with the left view as reference (match x - d) and once with
 * the right view as reference (match x + d).
 *   C(x, d) = popcount((B_ref(x) XOR B_other(x_d)) AND Phi_ref(x)); a match outside the image
 *   costs n_bits. A(x, d) = sum of C over the in-image pixels of the agg_window^2 box around x.
 *   disp(x) = the smallest d in [0, dmax-1] with the minimum A(x, d).
 *   dispL, dispR  device int32 [h][w] outputs (left and right reference)
 *   costL_or_null optional device uint16 [h][w][dmax] output: A(x, d) for the left reference
 * dmax <= the context's dmax. Descriptor planes must be 16-byte aligned.
 */
bsm_status bsm_cost_aggregate_wta(bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                                  const uint32_t *PhiR, int32_t w, int32_t h, int32_t dmax, int32_t *dispL,
                                  int32_t *dispR, uint16_t *costL_or_null, void *stream);

/*
 * bsm_cost_aggregate_wta writing both aggregated cost volumes: costL[y][x][d] = A(x, d) with the left
 * view as reference (match x - d) and costR[y][x][d] with the right view as reference (match x + d),
 * device uint16 [h][w][dmax] each (both required). Same kernels, same WTA outputs, same errors.
 */
bsm_status bsm_cost_volumes(bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                            const uint32_t *PhiR, int32_t w, int32_t h, int32_t dmax, int32_t *dispL, int32_t *dispR,
                            uint16_t *costL, uint16_t *costR, void *stream);

/*
 * Global optimisation of a cost volume, the extension the paper names as future work (Sec. 5):
 * semi-global aggregation of the (box-aggregated) Eq. 8 cost along `paths` image directions, then
 * Eq. 1 on the result. Directions: 4 = left-to-right, right-to-left, top-down, bottom-up; 8 adds the
 * four diagonals. Per direction r, with m = min_k L_r(p - r, k):
 *   L_r(p, d) = C(p, d) + min(L_r(p-r, d), L_r(p-r, d-1) + P1, L_r(p-r, d+1) + P1, m + P2) - m,
 * and L_r(p, d) = C(p, d) where p - r leaves the image.
 *   cost  device uint16 [h][w][dmax], e.g. bsm_cost_volumes' costL or costR (read only)
 *   S     device uint32 [h][w][dmax] output: S(p, d) = sum over the directions of L_r(p, d)
 *   disp  device int32 [h][w] output: the smallest d with the minimum S(p, d)
 * 0 <= P1 <= P2 <= 65535; paths 4 or 8; dmax <= the context's dmax. Asynchronous on `stream`.
 * Where the volume's largest cost + P2 < 65536 (decided on the device) every direction runs at once
 * on the context's own streams (forked from and joined back into `stream` with events), writing
 * 16-bit path costs into the context's SGM scratch (paths * w * h * dmax * 2 bytes, grown here if too
 * small, synchronously); otherwise the directions run one after another on `stream`, accumulating
 * into S. Errors: BSM_ERR_INVALID_ARG for a NULL or misaligned pointer or a value out of range.
 */
bsm_status bsm_sgm(bsm_ctx *ctx, const uint16_t *cost, int32_t w, int32_t h, int32_t dmax, int32_t P1, int32_t P2,
                   int32_t paths, uint32_t *S, int32_t *disp, void *stream);

/* One stereo pair of a batch: every pointer is a DEVICE pointer owned by the caller. */
typedef struct {
  const uint8_t *rgbL, *rgbR;  /* RGB views, h rows of pitch_bytes each */
  int32_t w, h, pitch_bytes;   /* 1 <= w, h <= 16384, pitch_bytes >= 3 w */
  int32_t dmax;                /* 1 <= dmax <= the context's dmax */
  uint32_t *BL, *PhiL, *BR, *PhiR; /* [h][w][n_bits/32] descriptor and mask outputs, 16-byte aligned */
  int32_t *dispL, *dispR;      /* [h][w] WTA outputs (left and right reference) */
  int32_t *out;                /* [h][w] refined left map */
} bsm_pair_desc;

/* Largest number of pairs in one bsm_batch_run call. */
#define BSM_MAX_BATCH 1024

/*
 * The whole method (describe both views, cost_aggregate_wta, refine) for `count` pairs of any sizes
 * and dmax in four persistent launches; the first three are replayed from one CUDA graph the context
 * captures on its first batch. Pairs of at least 1280 x 720 x 128 pixel-disparities instead take the
 * tensor-core cost kernel (one launch each, after the graph) where n_bits is 256 and the tuning's
 * cost_variant is 0 or 3. Every pair's outputs are bit-identical to the per-pair calls. `pairs` is a HOST array
 * read before the call returns. Work is asynchronous on `stream`. The context's batch scratch (the
 * colour planes of all 2 * count views) grows here if too small (bsm_reserve_batch sizes it up
 * front); the call waits until the previous batch's ticket table has been copied to the device.
 * Errors: BSM_ERR_INVALID_ARG for a bad descriptor or count outside 1..BSM_MAX_BATCH;
 * BSM_ERR_UNSUPPORTED when the context's n_bits exceeds 256 (long descriptors run per pair) or its
 * mask_mode is BSM_MASK_BOTH.
 */
bsm_status bsm_batch_run(bsm_ctx *ctx, const bsm_pair_desc *pairs, int32_t count, void *stream);

/* Size the batch scratch for batches of up to `total_pixels` pixels per view summed over the pairs. */
bsm_status bsm_reserve_batch(bsm_ctx *ctx, int64_t total_pixels);

/*
 * Serving engine: continuous batching of requests on the current device.
 *
 * A scheduler thread owns `lanes` lanes (each a context with the engine's parameters and its own
 * stream). Whenever a lane is free it admits queued requests in arrival order while the engine's
 * device-memory budget allows, and runs them with the copies of their views in and their refined maps
 * out: the small requests as one bsm_batch_run, the large ones (w h dmax >= 1280 x 720 x 128) through
 * the per-pair calls with the tensor-core cost kernel where the parameters allow it. Batches of
 * different lanes overlap on the device and requests that arrive while others run are admitted as soon
 * as a lane and memory free up. Request buffers are allocated from the engine's own stream-ordered
 * pool; each lane's context also keeps batch and per-pair scratch (grown to the largest seen) outside
 * the budget. Results are bit-identical to the per-pair calls.
 */
typedef struct bsm_server bsm_server;

typedef struct {
  int32_t lanes;          /* batches in flight at once, 1..8 */
  int32_t max_batch;      /* requests per batch, 1..BSM_MAX_BATCH */
  int64_t device_budget;  /* bytes of device memory the engine may hold for request buffers and its lanes'
                             colour-plane scratch (4 bytes per pixel of a lane's largest batch and of its
                             largest per-pair request, kept once reserved); 0 selects half the free memory */
  int64_t max_batch_work; /* cap on a batch's sum of w * h * dmax (a larger request still runs alone);
                             0 = no cap. Keeps large requests from holding small ones in one batch. */
} bsm_server_config;

typedef struct {
  uint64_t id;                 /* caller's identifier, returned with the completion */
  const uint8_t *rgbL, *rgbR;  /* HOST views, h rows of pitch_bytes; pinned memory lets copies overlap */
  int32_t w, h, pitch_bytes, dmax;
  int32_t *out;                /* HOST int32 [h][w]: the refined left map (pinned memory recommended) */
} bsm_request;                 /* the buffers must stay valid until the request completes */

typedef struct {
  uint64_t id;
  bsm_status status;           /* BSM_OK, or why the request failed */
  double latency_us;           /* from bsm_server_submit to the scheduler seeing the result */
} bsm_completion;

typedef struct {
  int64_t submitted, completed, failed, batches, max_batch_seen, queued, bytes_in_use, budget;
  int64_t scratch_bytes;  /* lane scratch reserved so far, charged to the budget beside bytes_in_use */
} bsm_server_stats;

/* Start an engine (creates `lanes` contexts: synchronous, allocates). BSM_ERR_UNSUPPORTED for
 * n_bits > 256 or mask_mode BSM_MASK_BOTH, which the batched kernels do not serve. */
bsm_status bsm_server_create(const bsm_params *params, const bsm_server_config *cfg, bsm_server **out);

/* Queue a request (any thread, non-blocking). A malformed request, or one whose buffers and lane
 * scratch exceed the whole budget, completes at once with BSM_ERR_INVALID_ARG, also returned here. */
bsm_status bsm_server_submit(bsm_server *s, const bsm_request *req);

/* Up to max_out completions; waits up to timeout_us for the first (0: none, < 0: forever).
 * Returns how many were written (-1 on a bad argument). */
int32_t bsm_server_poll(bsm_server *s, bsm_completion *out, int32_t max_out, int32_t timeout_us);

/* Wait until every submitted request has completed (timeout_ms < 0: forever); BSM_ERR_TIMEOUT if not. */
bsm_status bsm_server_drain(bsm_server *s, int32_t timeout_ms);

bsm_status bsm_server_get_stats(bsm_server *s, bsm_server_stats *out);

/* Finish every queued request, then stop the scheduler and release everything. */
void bsm_server_destroy(bsm_server *s);

/* Largest image, in pixels (width * height), that bsm_describe_noalloc accepts: 2^22. */
#define BSM_NOALLOC_MAX_PIXELS 4194304

/*
 * bsm_describe for callers that cannot allocate device memory. The paper has no counterpart; this is
 * a deployment variant of the same computation. bsm_describe grows its scratch with cudaMalloc the
 * first time it sees a larger image; callers that capture streams into graphs, that run under a
 * device-memory budget fixed up front, or that cannot accept the device synchronisation of an
 * allocation use this call instead. It computes exactly what bsm_describe computes, with the same
 * arguments, requirements and outputs, and allocates nothing:
 *   - its scratch is one fixed array of BSM_NOALLOC_MAX_PIXELS colour words (16 MiB) in the
 *     library's device code, which every GPU that loads it holds until the process exits. The CUDA
 *     driver reserves those 16 MiB when it loads the module that holds the array: at library load
 *     with eager module loading, or, with CUDA's default lazy loading, at this call's first use on
 *     each device; make that first call during set-up, while memory is still free;
 *   - images with w * h > BSM_NOALLOC_MAX_PIXELS are rejected with BSM_ERR_INVALID_ARG;
 *   - the context must already exist (bsm_create allocates; create it during set-up);
 *   - the first call on a device looks up that device's address of the array with the device current
 *     and caches it (a host-side lookup; no cudaMalloc); make that first call before any stream
 *     capture. The cached address belongs to the current CUDA context of that device: after
 *     cudaDeviceReset do not call this function again in the same process;
 *   - errors map as bsm_describe's do (a failed lookup or launch returns BSM_ERR_CUDA, or
 *     BSM_ERR_OUT_OF_MEMORY when the driver could not load the module, with the CUDA error recorded
 *     for bsm_last_cuda_error);
 *   - every call on a device shares the one array, and each call overwrites every word it reads,
 *     so nothing needs clearing between calls; two calls that overlap on the GPU (different streams
 *     without ordering) race on the array and give undefined results.
 */
bsm_status bsm_describe_noalloc(bsm_ctx *ctx, const uint8_t *rgb_dev, int32_t w, int32_t h, int32_t pitch_bytes,
                                uint32_t *B_dev, uint32_t *Phi_dev, void *stream);

/*
 * Left/right check and the voting refinement of Eq. 9-10 on the left map.
 *   valid(x) = x - dL(x) >= 0 and |dL(x) - dR(x - dL(x))| <= lr_tol. Valid pixels keep dL(x).
 *   An invalid pixel x takes the smallest d maximising W(x, d) = sum over valid p with dL(p) = d in
 *   the (2R+1)^2 window of floor(Ec[c] * Es[e2] / 2^15), c = CIELAB SAD(x, p), e2 = |x - p|^2,
 *   Ec[c] = round(32768 exp(-c / lambda_c)), Es[e2] = round(32768 exp(-sqrt(e2) / lambda_e)).
 *   If no vote is positive: the smaller of the nearest valid dL to the left and to the right on
 *   the row, the one that exists, else 0.
 *   rgbL_dev  device left RGB image (h rows of pitch_bytes); out  device int32 [h][w]
 * Every dL value must lie in [0, dmax-1]. Uses the context's scratch (a w * h plane; it holds each
 * pixel's CIELAB colour, check result and disparity or row fallback as one word), grown here if too
 * small.
 */
bsm_status bsm_refine(bsm_ctx *ctx, const uint8_t *rgbL_dev, int32_t pitch_bytes, const int32_t *dispL,
                      const int32_t *dispR, int32_t w, int32_t h, int32_t dmax, int32_t *out, void *stream);

/*
 * The whole method for one pair with HOST buffers: copies both views to the device, runs
 * describe (both views), cost_aggregate_wta and refine, and copies the refined left map back.
 * Device buffers come from a workspace the context owns and grows on demand (this call may
 * allocate). Synchronous: returns after the result is in out_host.
 *   rgbL_host, rgbR_host  host RGB images, h rows of pitch_bytes (pinned memory is fastest)
 *   out_host              host int32 [h][w]
 */
bsm_status bsm_match_host(bsm_ctx *ctx, const uint8_t *rgbL_host, const uint8_t *rgbR_host, int32_t w, int32_t h,
                          int32_t pitch_bytes, int32_t dmax, int32_t *out_host, void *stream);

/*
 * Read and clear the device status word that kernels latch errors into (BSM_OK if none).
 * Synchronises the context's device.
 */
bsm_status bsm_last_error(bsm_ctx *ctx);

/*
 * Test hooks for failure detection (off by default; every hook only withholds work, it never faults).
 *   BSM_DEBUG_WITHHOLD_ARRIVALS (1): value 1 makes the cost kernels' staging thread skip its mbarrier
 *     arrivals, so every bounded wait of the next cost launch runs out (about a second per wave of
 *     CTAs); the kernel then latches BSM_ERR_TIMEOUT and returns, and the context stays usable. It
 *     reaches the one-column kernel (cost_variant 0, 1 or 2: the two-column kernel completes its copies
 *     by cp.async groups and has no wait to withhold) and, with cost_variant 3, the tensor-core kernel,
 *     whose producer then issues no copies, so its operand builders', MMA issuer's and epilogue's waits
 *     all run out; no disparity of the launch is written.
 */
#define BSM_DEBUG_WITHHOLD_ARRIVALS 1
bsm_status bsm_debug_set(bsm_ctx *ctx, int32_t key, int32_t value);

/* Name of the CUDA runtime error behind the context's most recent BSM_ERR_CUDA ("" if none). */
const char *bsm_last_cuda_error(bsm_ctx *ctx);

/* Static, human-readable name of a status code. */
const char *bsm_status_string(bsm_status s);

/*
 * Copy the context's colour table to dst_dev (device uint32 [2^24], index (R << 16) | (G << 8) | B):
 * byte 0 = L, byte 1 = a + 128, byte 2 = b + 128 (integer CIELAB, D65, each rounded half away from
 * zero), byte 3 = intensity I. Asynchronous on `stream`.
 */
bsm_status bsm_copy_color_table(bsm_ctx *ctx, uint32_t *dst_dev, void *stream);

/*
 * Host-side integer vote tables of Eq. 10 (no GPU needed): Ec[c] for c in [0, nc), Es[e2] for
 * e2 in [0, ne). Returns BSM_ERR_INVALID_ARG for non-positive lambdas or sizes.
 */
bsm_status bsm_vote_tables(int32_t lambda_c, int32_t lambda_e, int32_t nc, int32_t ne, uint32_t *Ec, uint32_t *Es);

/*
 * Launch shapes of a context's kernels. Results never depend on them (every shape computes the same
 * bits); only speed does. The autotuner of the Python package searches them per GPU and workload.
 * A zero field selects the library's heuristic.
 */
typedef struct {
  int32_t cost_rows;       /* rows per CTA band of the cost/aggregation/WTA kernel: 0 or 8..512
                              (n_bits > 256: the chunked long-descriptor kernel's band) */
  int32_t cost_popc_plain; /* popcount form of the cost kernel (n_bits = 256; results identical):
                              0 carry-save tree over 8 words, 1 plain POPC per word, 2 two 3-word
                              carry-save adders plus 2 plain words (two-column kernel only) */
  int32_t batch_rows;      /* rows per task of bsm_batch_run's cost stage: 0 (64) or 8..512 */
  int32_t cost_variant;    /* 0: automatic (tensor cores for pairs of >= 1280 x 720 x 128 pixel-
                              disparities where variant 3 is supported; else two columns per lane
                              for n_bits 128 and 256, one otherwise);
                              1: one column per lane; 2: two columns per lane (n_bits 128 or 256);
                              3: tensor cores (Eq. 8 as an exact E4M3 product on tcgen05, n_bits 256,
                              reference or no mask) */
  int32_t describe_variant; /* 0: automatic (warp per pixel from n_bits 256 on, thread per pixel below);
                               1: thread per pixel (n_bits <= 256); 2: warp per pixel (n_bits / 32 even;
                               always for n_bits > 256). Results identical. */
  int32_t describe_copies; /* copies of the colour-plane tile the warp-per-pixel describe kernel keeps in
                              shared memory, 0 (one) or 1..4: with more, each sample is read from the copy
                              that keeps its load's 32 addresses in distinct banks (bsm_describe_gather_plan);
                              fewer bank conflicts, more staging and shared memory. Results identical. */
  int32_t reserved[2];     /* must be zero */
} bsm_tuning;

/* Set / read the context's launch shapes. Synchronous, host only. */
bsm_status bsm_set_tuning(bsm_ctx *ctx, const bsm_tuning *tuning);
bsm_status bsm_get_tuning(bsm_ctx *ctx, bsm_tuning *tuning);

/* The cost / aggregation / WTA launch that bsm_cost_aggregate_wta and bsm_cost_volumes make for a
   w x h pair with this dmax under the context's current tuning (Eq. 8, box aggregation, Eq. 1): which
   kernel, and the output rows per CTA row band (band b covers rows [b rows_per_band, (b + 1)
   rows_per_band); every band reads rows_per_band + agg_window - 1 input rows). Host only, no GPU work;
   for tests that place checks on band boundaries and for profiling. BSM_ERR_INVALID_ARG on bad sizes. */
typedef struct {
  int32_t kernel;         /* 1 one column per lane, 2 two columns per lane, 3 tensor cores, 4 long descriptors */
  int32_t rows_per_band;  /* output rows per CTA band */
  int32_t launches;       /* kernel launches per call */
  int32_t reserved;
} bsm_cost_plan_info;
bsm_status bsm_cost_plan(bsm_ctx *ctx, int32_t w, int32_t h, int32_t dmax, bsm_cost_plan_info *out);

/* The shared-memory gather plan of the warp-per-pixel describe kernel for a pair table (Eq. 2-3 and 5 read
   the two samples of every sampling pair around the pixel; bit l of descriptor word j is pair 32 j + l's,
   so lane l of a warp reads pair 32 j + l's samples, one load per word and sample). The kernel keeps
   `copies` copies of its colour-plane tile (row pitch *pitch words) at bases in different banks and reads
   each sample from the copy the plan assigns, so that a load's 32 addresses share as few banks as
   possible. Host only, no GPU work; bsm_create plans the context's table with 4 copies (fewer for a large
   pair window). pairs: n_bits x (px, py, qx, qy) as in bsm_params; n_bits a multiple of 32 up to 256;
   copies 1..4. Outputs (caller-owned, any may be NULL): *pitch; *copies_used (copies, or fewer when the
   tile copies would exceed 64 KB); copy_base[copies_used] (word offsets of the copies, copy 0 at 0);
   offsets[n_bits][2] (each sample's word offset from the pixel in copy 0: its copy's base +
   dy * pitch + dx); wavefronts[2 n_bits / 32] (the bank-conflict degree of load 2 j + s, 1 = none).
   BSM_ERR_INVALID_ARG on a NULL pair table, a bad n_bits or copies, or an offset beyond 31. */
bsm_status bsm_describe_gather_plan(const int8_t *pairs, int32_t n_bits, int32_t copies, int32_t *pitch,
                                    int32_t *copies_used, int32_t *copy_base, int32_t *offsets, int32_t *wavefronts);

/* Validate parameters without touching the GPU: the checks bsm_create performs first. */
bsm_status bsm_validate_params(const bsm_params *params);

/* ABI version of this header (incremented on any incompatible change). */
int32_t bsm_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* BSM_H */
