// Internal declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/bsm.h"

namespace bsm {

constexpr int kMaxBits = 256;      // descriptor length supported by the kernels of this version
constexpr int kMaxWords = kMaxBits / 32;
constexpr int kMaxDmax = 256;
constexpr int kMaxHalo = 31;       // largest |offset| of a sampling pair
constexpr int kMaxVoteRadius = 31;
constexpr int kMaxSad = 3 * 255;   // largest CIELAB SAD of Eq. 5 on 8-bit channels
constexpr int kVoteShift = 15;     // votes are floor(Ec * Es / 2^15)

// Byte layout of a colour-table entry: L | (a + 128) << 8 | (b + 128) << 16 | I << 24.
constexpr uint32_t kLabMask = 0x00FFFFFFu;

// Pair offsets in the shared-memory tile of the describe kernel: element i is
// (dy_p * pitch + dx_p, dy_q * pitch + dx_q) for the tile pitch chosen at launch.
struct PairTable {
  int32_t off[kMaxBits][2];
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
  // Launch shapes (bsm_set_tuning); 0 selects the library's heuristic.
  int cost_rows = 0;        // rows per CTA band of the cost kernel
  int cost_plain_popc = 0;  // 1: plain popcount in the cost kernel instead of the carry-save tree
  // Scratch: packed colour plane of the describe pre-pass (grown on demand, or by bsm_reserve).
  uint32_t *plane = nullptr;
  size_t plane_px = 0;
  // Workspace of bsm_match_host (grown on demand).
  void *ws = nullptr;
  size_t ws_bytes = 0;
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
                            const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *cost,
                            cudaStream_t s);
cudaError_t launch_refine(const bsm_ctx *ctx, const uint8_t *rgb, int pitch, const int32_t *dL, const int32_t *dR,
                          int w, int h, int dmax, int32_t *out, cudaStream_t s);

}  // namespace bsm
