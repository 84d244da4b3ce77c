// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/bsm.h"

namespace bsm {

constexpr int kMaxBits = 4096;     // longest descriptor (the paper's n, Sec. 4.1)
constexpr int kMaxShortBits = 256; // longest descriptor of the short-descriptor kernels
constexpr int kMaxDmax = 256;
constexpr int kMaxHalo = 31;       // largest |offset| of a sampling pair
constexpr int kMaxVoteRadius = 31;
constexpr int kMaxSad = 3 * 255;   // largest CIELAB SAD of Eq. 5 on 8-bit channels
constexpr int kVoteShift = 15;     // votes are floor(Ec * Es / 2^15)
// pixel-disparities of a pair from which the automatic cost variant takes the tensor-core kernel
constexpr long long kTcAutoWork = 1280LL * 720 * 128;

// Byte layout of a colour-table entry: L | (a + 128) << 8 | (b + 128) << 16 | I << 24.
constexpr uint32_t kLabMask = 0x00FFFFFFu;

// Pair offsets in the shared-memory tile of the describe kernels: element i is, for each of pair i's two
// samples, its offset from the centre pixel, dy * pitch + dx for the tile pitch chosen at launch, plus the
// base of the tile copy the sample is read from. The warp-per-pixel kernel keeps `copies` copies of its
// tile at bases that fall in different shared-memory banks and reads each sample from the copy that
// spreads its warp's 32 loads over the banks; the other kernels keep one copy at base 0.
constexpr int kMaxTileCopies = 4;
struct PairTable {
  int32_t off[kMaxShortBits][2];
  int32_t copy_base[kMaxTileCopies];
  int32_t copies;
};

// ---------------------------------------------------------------- batched execution

constexpr int kMaxBatch = 1024;   // pairs per bsm_batch_run call
constexpr int kRefineTX = 32, kRefineTY = 32;  // output block of one refinement CTA (per pair and batched)
constexpr int kMaxRefineTiles = (16384 / kRefineTX) * (16384 / kRefineTY);  // blocks of the largest image
constexpr int kBatchDisp = 64;    // disparities per CTA of the batched cost kernel (8 warps)

// One pair of a batch, as the batched kernels see it (built on the host, copied to the device).
struct BatchPair {
  const uint8_t *rgb[2];
  uint32_t *B[2], *Phi[2];
  int32_t *disp[2];
  int32_t *out;
  uint32_t *plane[2];  // colour planes in the batch scratch
  int w, h, pitch, dmax;
  int pre_base, desc_base, cost_base, ref_base;  // first ticket of this pair in each stage
  int desc_tx, desc_ty;                          // describe tiles per view
  int cost_cb, cost_bands, cost_dr;              // column blocks, row bands, disparity ranges
  int ref_tx, ref_ty;                            // refine tiles
};

struct BatchHeader {
  int count;
  int total[4];        // tickets per stage: pre-pass rows, describe tiles, cost tasks, refine tiles
  int band_rows;       // rows per cost task
  unsigned counters[4];  // next ticket per stage; the host writes zeros with every batch
  int pad[6];
};

}  // namespace bsm

struct bsm_ctx {
  int device = 0;
  bsm_params p{};
  int nw = 0;        // n_bits / 32
  int halo = 0;      // max |offset| over the pair table
  int mask_rank = 0; // resolved k
  int8_t pairs[bsm::kMaxBits * 4] = {};
  uint32_t *color_table = nullptr;  // device, 2^24 entries
  uint32_t *vote_ec = nullptr;      // device, kMaxSad + 1 entries
  uint32_t *vote_es = nullptr;      // device, 2 R^2 + 1 entries
  uint32_t *status = nullptr;       // device status word (bsm_status latched by kernels)
  int32_t *wide_offs = nullptr;     // device pair offsets of the long-descriptor describe kernel
  bsm::PairTable warp_pt{};         // gather plan of the warp-per-pixel describe kernel (tile copies)
  int32_t *refine_tiles = nullptr;  // device, 2 x kMaxRefineTiles: refinement blocks' invalid counts and their order
  // Launch shapes (bsm_set_tuning); 0 selects the library's heuristic.
  int cost_rows = 0;        // rows per CTA band of the cost kernel
  int cost_plain_popc = 0;  // 1: plain popcount in the cost kernel instead of the carry-save tree
  // Scratch: packed colour plane of the describe pre-pass (grown on demand, or by bsm_reserve).
  uint32_t *plane = nullptr;
  size_t plane_px = 0;
  int batch_rows = 0;       // rows per task of the batched cost kernel
  int cost_variant = 0;     // 0 automatic, 1 one column per lane, 2 two columns per lane, 3 tensor cores
  int describe_variant = 0; // 0 automatic, 1 thread per pixel, 2 warp per pixel
  int describe_copies = 0;  // tile copies of the warp-per-pixel describe kernel (0: the library's default)
  int withhold_arrivals = 0;  // test hook: cost kernels skip their mbarrier arrivals
  // Batched execution (bsm_batch_run).
  int sms = 0;
  uint8_t *batch_table_host = nullptr;  // pinned ticket table
  uint8_t *batch_table_dev = nullptr;
  cudaEvent_t batch_copied = nullptr;   // the graph's table copy has finished
  cudaStream_t batch_capture = nullptr; // stream the graph is captured on
  cudaStream_t copy_stream = nullptr;   // bsm_match_host: the right view's upload beside the left's describe
  cudaEvent_t copy_after = nullptr;     // ... ordered after the caller's earlier work and the left view's upload
  cudaEvent_t copy_done = nullptr;      // ... and awaited before the right view's describe
  uint16_t *sgm_ws = nullptr;           // bsm_sgm: 16-bit path-cost planes of every direction + the largest cost
  size_t sgm_ws_bytes = 0;
  cudaStream_t sgm_streams[8] = {};     // ... one per direction of the concurrent schedule
  cudaEvent_t sgm_fork = nullptr, sgm_join[8] = {};
  cudaGraphExec_t batch_graph = nullptr;
  int batch_graph_variant = -1;         // popcount form and describe variant the graph was captured with
  int batch_grid[4] = {0, 0, 0, 0};     // persistent grid sizes of the four batched kernels
  uint32_t *batch_plane = nullptr;      // colour planes of every view of a batch
  size_t batch_plane_words = 0;
  cudaError_t last_cuda = cudaSuccess;  // last CUDA error behind a BSM_ERR_CUDA of this context
  // Workspace of bsm_match_host (grown on demand).
  void *ws = nullptr;
  size_t ws_bytes = 0;
  // Scratch of the tensor-core cost kernel: E4M3 operand planes and popcount(Phi AND B) of both views.
};

namespace bsm {

// Launchers (each returns cudaGetLastError() after enqueueing).
cudaError_t build_color_table(uint32_t *table, const double *lin256, cudaStream_t s);
cudaError_t launch_color_plane(const bsm_ctx *ctx, const uint8_t *rgb, int w, int h, int pitch, uint32_t *plane,
                               cudaStream_t s);
cudaError_t launch_describe_plane(const bsm_ctx *ctx, const uint32_t *plane, int w, int h, uint32_t *B,
                                  uint32_t *Phi, cudaStream_t s);
cudaError_t launch_describe(const bsm_ctx *ctx, const uint8_t *rgb, int w, int h, int pitch, uint32_t *plane,
                            uint32_t *B, uint32_t *Phi, cudaStream_t s);
cudaError_t launch_cost_wta(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                            const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *costL, uint16_t *costR,
                            cudaStream_t s);
// Batched kernels: prepare_* sets kernel attributes and returns the persistent grid (outside any
// stream capture); launch_* only enqueues.
cudaError_t prepare_describe_batch(const bsm_ctx *ctx, int *grid);
cudaError_t prepare_cost_batch(const bsm_ctx *ctx, int *grid);
cudaError_t prepare_refine_batch(const bsm_ctx *ctx, int *grid);
void wide_offsets(const bsm_ctx *ctx, int32_t *out);
// Gather plan of the warp-per-pixel describe kernel for the context's pair table and tile copies (host
// only): the copies' bases and every sample's copy.
PairTable warp_pair_table(const bsm_ctx *ctx);
// The same plan for any pair table and number of copies; wavefronts[l] (2 n_bits / 32 entries, or nullptr)
// receives the shared-memory wavefronts of load l (word j's first samples at 2 j, its second at 2 j + 1).
// Returns the number of copies used (fewer than asked when the tile is large), or 0 on bad arguments.
int plan_tile_gathers(const int8_t *pairs, int n_bits, int copies, PairTable *pt, int *pitch, int *wavefronts);
cudaError_t launch_describe_wide(const bsm_ctx *ctx, const uint32_t *plane, int w, int h, uint32_t *B, uint32_t *Phi,
                                 cudaStream_t s);
cudaError_t launch_cost_long(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                             const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *costL, uint16_t *costR,
                             cudaStream_t s);
bool cost2_supported(const bsm_ctx *ctx);
bool cost_tc_supported(const bsm_ctx *ctx);
// Output rows per CTA band of each cost kernel for a w x h pair (the context's cost_rows, else the
// kernel's heuristic), and the plan launch_cost_wta follows.
int cost1_rows(const bsm_ctx *ctx, int w, int h, int dmax);
int cost2_rows(const bsm_ctx *ctx, int w, int h, int dmax);
int cost_tc_rows(const bsm_ctx *ctx, int w, int h, int dmax);
int cost_long_rows(const bsm_ctx *ctx, int w, int h, int dmax);
struct CostPlan {
  int kernel;  // 1 one column per lane, 2 two columns per lane, 3 tensor cores, 4 long descriptors
  int rows;
  int launches;
};
CostPlan cost_plan(const bsm_ctx *ctx, int w, int h, int dmax);
cudaError_t launch_cost_tc(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                           const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *costL,
                           uint16_t *costR, cudaStream_t s);
size_t sgm_scratch_bytes(int w, int h, int dmax, int paths);
cudaError_t launch_sgm(bsm_ctx *ctx, const uint16_t *C, int w, int h, int dmax, int P1, int P2, int paths,
                       uint32_t *S, int32_t *disp, cudaStream_t s);
cudaError_t launch_cost2(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                         const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *costL, uint16_t *costR,
                         cudaStream_t s);
cudaError_t launch_refine(const bsm_ctx *ctx, const uint8_t *rgb, int pitch, const int32_t *dL, const int32_t *dR,
                          int w, int h, int dmax, int32_t *out, uint32_t *near, cudaStream_t s);

}  // namespace bsm
