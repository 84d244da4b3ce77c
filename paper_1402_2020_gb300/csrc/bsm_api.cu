// Host side of the C ABI declared in include/bsm.h: parameter validation, context set-up (sampling
// pairs, colour table, vote tables), argument checks and kernel launches.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "bsm_internal.cuh"

namespace {

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bsm_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return BSM_OK;
  if (e == cudaErrorMemoryAllocation) return BSM_ERR_OUT_OF_MEMORY;
  return BSM_ERR_CUDA;
}

bsm_status from_cuda(bsm_ctx *ctx, cudaError_t e) {
  if (e != cudaSuccess) ctx->last_cuda = e;
  return from_cuda(e);
}

bool size_ok(int32_t w, int32_t h) { return w >= 1 && h >= 1 && w <= 16384 && h <= 16384; }

// sRGB transfer curve (IEC 61966-2-1) for the 256 channel values; the colour-table kernel takes
// the rest of the CIELAB conversion from here.
void srgb_linear_table(double *lin) {
  for (int v = 0; v < 256; ++v) {
    const double c = v / 255.0;
    lin[v] = c <= 0.04045 ? c / 12.92 : std::pow((c + 0.055) / 1.055, 2.4);
  }
}

// Grow the context's colour-plane scratch to at least `pixels` words. Growing waits for all work on
// the device, because earlier calls may still read the old plane.

cudaError_t ensure_plane(bsm_ctx *ctx, size_t pixels) {
  if (ctx->plane_px >= pixels) return cudaSuccess;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return e;
  cudaFree(ctx->plane);
  ctx->plane = nullptr;
  ctx->plane_px = 0;
  e = cudaMalloc(&ctx->plane, pixels * sizeof(uint32_t));
  if (e == cudaSuccess) ctx->plane_px = pixels;
  return e;
}

}  // namespace

extern "C" {

int32_t bsm_abi_version(void) { return 3; }

const char *bsm_status_string(bsm_status s) {
  switch (s) {
    case BSM_OK: return "ok";
    case BSM_ERR_INVALID_ARG: return "invalid argument";
    case BSM_ERR_OUT_OF_MEMORY: return "out of memory";
    case BSM_ERR_CUDA: return "CUDA error";
    case BSM_ERR_TIMEOUT: return "device-side wait timed out";
    case BSM_ERR_UNSUPPORTED: return "unsupported by this version";
  }
  return "unknown status";
}

bsm_status bsm_validate_params(const bsm_params *p) {
  if (p == nullptr || p->pairs == nullptr) return BSM_ERR_INVALID_ARG;
  if (p->n_bits < 32 || p->n_bits % 32 != 0 || p->n_bits > 4096) return BSM_ERR_INVALID_ARG;
  if (p->window_S < 3 || p->window_S > 2 * bsm::kMaxHalo + 1) return BSM_ERR_INVALID_ARG;
  if (p->agg_window < 1 || p->agg_window % 2 == 0) return BSM_ERR_INVALID_ARG;
  if ((int64_t)p->n_bits * p->agg_window * p->agg_window > 65535) return BSM_ERR_INVALID_ARG;
  if (p->mask_rank < 0 || p->mask_rank > p->n_bits) return BSM_ERR_INVALID_ARG;
  if (p->dmax < 1 || p->dmax > 1024) return BSM_ERR_INVALID_ARG;
  if (p->lr_tol < 0) return BSM_ERR_INVALID_ARG;
  if (p->vote_radius < 0 || p->vote_radius > bsm::kMaxVoteRadius) return BSM_ERR_INVALID_ARG;
  if (p->lambda_c <= 0 || p->lambda_e <= 0) return BSM_ERR_INVALID_ARG;
  const int half = p->window_S / 2;
  for (int i = 0; i < 4 * p->n_bits; ++i)
    if (std::abs((int)p->pairs[i]) > half) return BSM_ERR_INVALID_ARG;
  if (p->mask_mode < BSM_MASK_REFERENCE || p->mask_mode > BSM_MASK_BOTH) return BSM_ERR_INVALID_ARG;
  if (p->mask_mode == BSM_MASK_NONE && p->mask_rank != 0 && p->mask_rank != p->n_bits) return BSM_ERR_INVALID_ARG;
  // Valid per the method, not built in this version.
  if (p->n_bits & (p->n_bits - 1)) return BSM_ERR_UNSUPPORTED;  // 32, 64, ..., 4096
  if (p->mask_mode == BSM_MASK_BOTH && p->n_bits < 256) return BSM_ERR_UNSUPPORTED;
  if (p->agg_window > 7) return BSM_ERR_UNSUPPORTED;
  if (p->dmax > bsm::kMaxDmax) return BSM_ERR_UNSUPPORTED;
  return BSM_OK;
}

bsm_status bsm_vote_tables(int32_t lambda_c, int32_t lambda_e, int32_t nc, int32_t ne, uint32_t *Ec, uint32_t *Es) {
  if (lambda_c <= 0 || lambda_e <= 0 || nc <= 0 || ne <= 0 || Ec == nullptr || Es == nullptr)
    return BSM_ERR_INVALID_ARG;
  // Eq. 10 with integer weights: Ec[c] = round(2^15 exp(-c / lambda_c)), Es[e2] = round(2^15 exp(-sqrt(e2) / lambda_e)).
  for (int32_t c = 0; c < nc; ++c) Ec[c] = (uint32_t)std::lround(32768.0 * std::exp(-(double)c / (double)lambda_c));
  for (int32_t e = 0; e < ne; ++e)
    Es[e] = (uint32_t)std::lround(32768.0 * std::exp(-std::sqrt((double)e) / (double)lambda_e));
  return BSM_OK;
}

void bsm_destroy(bsm_ctx *ctx) {
  if (ctx == nullptr) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  cudaFree(ctx->color_table);
  cudaFree(ctx->vote_ec);
  cudaFree(ctx->vote_es);
  cudaFree(ctx->status);
  cudaFree(ctx->wide_offs);
  cudaFree(ctx->refine_tiles);
  cudaFree(ctx->ws);
  cudaFree(ctx->plane);
  if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
  if (ctx->batch_copied) cudaEventDestroy(ctx->batch_copied);
  if (ctx->batch_capture) cudaStreamDestroy(ctx->batch_capture);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  if (ctx->copy_after) cudaEventDestroy(ctx->copy_after);
  if (ctx->copy_done) cudaEventDestroy(ctx->copy_done);
  cudaFree(ctx->sgm_ws);
  for (int r = 0; r < 8; ++r) {
    if (ctx->sgm_streams[r]) cudaStreamDestroy(ctx->sgm_streams[r]);
    if (ctx->sgm_join[r]) cudaEventDestroy(ctx->sgm_join[r]);
  }
  if (ctx->sgm_fork) cudaEventDestroy(ctx->sgm_fork);
  cudaFreeHost(ctx->batch_table_host);
  cudaFree(ctx->batch_table_dev);
  cudaFree(ctx->batch_plane);
  cudaSetDevice(prev);
  delete ctx;
}

bsm_status bsm_create(const bsm_params *p, bsm_ctx **out) {
  if (out == nullptr) return BSM_ERR_INVALID_ARG;
  const bsm_status v = bsm_validate_params(p);
  if (v != BSM_OK) return v;
  bsm_ctx *ctx = new (std::nothrow) bsm_ctx();
  if (ctx == nullptr) return BSM_ERR_OUT_OF_MEMORY;
  ctx->p = *p;
  ctx->p.pairs = nullptr;  // the copy below is the context's own
  ctx->nw = p->n_bits / 32;
  ctx->mask_rank = p->mask_rank == 0 ? p->n_bits / 4 : p->mask_rank;
  // No mask (Eq. 4): T of rank n is the largest weight, so every bit of Phi is set.
  if (p->mask_mode == BSM_MASK_NONE) ctx->mask_rank = p->n_bits;
  std::memcpy(ctx->pairs, p->pairs, (size_t)4 * p->n_bits);
  int halo = 0;
  for (int i = 0; i < 4 * p->n_bits; ++i) halo = std::max(halo, std::abs((int)p->pairs[i]));
  ctx->halo = halo;
  ctx->warp_pt = bsm::warp_pair_table(ctx);

  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
  const int ne = 2 * p->vote_radius * p->vote_radius + 1;
  double *lin_dev = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&ctx->color_table, sizeof(uint32_t) << 24);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->vote_ec, sizeof(uint32_t) * (bsm::kMaxSad + 1));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->vote_es, sizeof(uint32_t) * ne);
  if (e == cudaSuccess) e = cudaMalloc(&ctx->status, sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&lin_dev, sizeof(double) * 256);
  if (e == cudaSuccess) {
    double lin[256];
    srgb_linear_table(lin);
    uint32_t Ec[bsm::kMaxSad + 1];
    uint32_t *Es = new (std::nothrow) uint32_t[ne];
    if (Es == nullptr) {
      e = cudaErrorMemoryAllocation;
    } else {
      bsm_vote_tables(p->lambda_c, p->lambda_e, bsm::kMaxSad + 1, ne, Ec, Es);
      e = cudaMemcpy(lin_dev, lin, sizeof(lin), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(ctx->vote_ec, Ec, sizeof(Ec), cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaMemcpy(ctx->vote_es, Es, sizeof(uint32_t) * ne, cudaMemcpyHostToDevice);
      delete[] Es;
    }
  }
  if (e == cudaSuccess) {  // pair offsets of the warp-per-pixel describe kernel (every n)
    int32_t *offs = new (std::nothrow) int32_t[p->n_bits];
    if (offs == nullptr) {
      e = cudaErrorMemoryAllocation;
    } else {
      bsm::wide_offsets(ctx, offs);
      e = cudaMalloc(&ctx->wide_offs, sizeof(int32_t) * p->n_bits);
      if (e == cudaSuccess) e = cudaMemcpy(ctx->wide_offs, offs, sizeof(int32_t) * p->n_bits, cudaMemcpyHostToDevice);
      delete[] offs;
    }
  }
  if (e == cudaSuccess) e = cudaMalloc(&ctx->refine_tiles, sizeof(int32_t) * 2 * bsm::kMaxRefineTiles);
  if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(uint32_t));
  if (e == cudaSuccess) e = bsm::build_color_table(ctx->color_table, lin_dev, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaFree(lin_dev);
  if (e != cudaSuccess) {
    const bsm_status st = from_cuda(e);
    bsm_destroy(ctx);
    return st;
  }
  *out = ctx;
  return BSM_OK;
}

bsm_status bsm_describe(bsm_ctx *ctx, const uint8_t *rgb_dev, int32_t w, int32_t h, int32_t pitch_bytes,
                        uint32_t *B_dev, uint32_t *Phi_dev, void *stream) {
  if (ctx == nullptr || rgb_dev == nullptr || B_dev == nullptr || Phi_dev == nullptr) return BSM_ERR_INVALID_ARG;
  if (!size_ok(w, h) || pitch_bytes < 3 * w || !aligned16(B_dev) || !aligned16(Phi_dev)) return BSM_ERR_INVALID_ARG;
  cudaError_t e = ensure_plane(ctx, (size_t)w * h);
  if (e != cudaSuccess) return from_cuda(ctx, e);
  return from_cuda(ctx, bsm::launch_describe(ctx, rgb_dev, w, h, pitch_bytes, ctx->plane, B_dev, Phi_dev,
                                             (cudaStream_t)stream));
}

bsm_status bsm_cost_aggregate_wta(bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                                  const uint32_t *PhiR, int32_t w, int32_t h, int32_t dmax, int32_t *dispL,
                                  int32_t *dispR, uint16_t *costL_or_null, void *stream) {
  if (ctx == nullptr || BL == nullptr || PhiL == nullptr || BR == nullptr || PhiR == nullptr || dispL == nullptr ||
      dispR == nullptr)
    return BSM_ERR_INVALID_ARG;
  if (!size_ok(w, h) || dmax < 1 || dmax > ctx->p.dmax) return BSM_ERR_INVALID_ARG;
  if (!aligned16(BL) || !aligned16(PhiL) || !aligned16(BR) || !aligned16(PhiR)) return BSM_ERR_INVALID_ARG;
  return from_cuda(ctx, bsm::launch_cost_wta(ctx, BL, PhiL, BR, PhiR, w, h, dmax, dispL, dispR, costL_or_null,
                                             nullptr, (cudaStream_t)stream));
}

bsm_status bsm_cost_volumes(bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                            const uint32_t *PhiR, int32_t w, int32_t h, int32_t dmax, int32_t *dispL, int32_t *dispR,
                            uint16_t *costL, uint16_t *costR, void *stream) {
  if (ctx == nullptr || BL == nullptr || PhiL == nullptr || BR == nullptr || PhiR == nullptr || dispL == nullptr ||
      dispR == nullptr || costL == nullptr || costR == nullptr)
    return BSM_ERR_INVALID_ARG;
  if (!size_ok(w, h) || dmax < 1 || dmax > ctx->p.dmax) return BSM_ERR_INVALID_ARG;
  if (!aligned16(BL) || !aligned16(PhiL) || !aligned16(BR) || !aligned16(PhiR)) return BSM_ERR_INVALID_ARG;
  return from_cuda(ctx, bsm::launch_cost_wta(ctx, BL, PhiL, BR, PhiR, w, h, dmax, dispL, dispR, costL, costR,
                                             (cudaStream_t)stream));
}

bsm_status bsm_sgm(bsm_ctx *ctx, const uint16_t *cost, int32_t w, int32_t h, int32_t dmax, int32_t P1, int32_t P2,
                   int32_t paths, uint32_t *S, int32_t *disp, void *stream) {
  if (ctx == nullptr || cost == nullptr || S == nullptr || disp == nullptr) return BSM_ERR_INVALID_ARG;
  if (!size_ok(w, h) || dmax < 1 || dmax > ctx->p.dmax) return BSM_ERR_INVALID_ARG;
  if (P1 < 0 || P2 < P1 || P2 > 65535 || (paths != 4 && paths != 8)) return BSM_ERR_INVALID_ARG;
  if (((uintptr_t)cost & 1) != 0 || ((uintptr_t)S & 3) != 0 || ((uintptr_t)disp & 3) != 0) return BSM_ERR_INVALID_ARG;
  cudaError_t e = cudaSuccess;
  if (ctx->sgm_fork == nullptr) {
    e = cudaEventCreateWithFlags(&ctx->sgm_fork, cudaEventDisableTiming);
    for (int r = 0; r < 8 && e == cudaSuccess; ++r) {
      e = cudaStreamCreateWithFlags(&ctx->sgm_streams[r], cudaStreamNonBlocking);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->sgm_join[r], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return from_cuda(ctx, e);
  }
  const size_t need = bsm::sgm_scratch_bytes(w, h, dmax, paths);
  if (ctx->sgm_ws_bytes < need) {  // grows: earlier calls may still use the old planes
    e = cudaDeviceSynchronize();
    if (e == cudaSuccess) {
      cudaFree(ctx->sgm_ws);
      ctx->sgm_ws = nullptr;
      ctx->sgm_ws_bytes = 0;
      e = cudaMalloc(&ctx->sgm_ws, need);
      if (e == cudaSuccess) ctx->sgm_ws_bytes = need;
    }
    if (e != cudaSuccess) return from_cuda(ctx, e);
  }
  return from_cuda(ctx, bsm::launch_sgm(ctx, cost, w, h, dmax, P1, P2, paths, S, disp, (cudaStream_t)stream));
}

bsm_status bsm_refine(bsm_ctx *ctx, const uint8_t *rgbL_dev, int32_t pitch_bytes, const int32_t *dispL,
                      const int32_t *dispR, int32_t w, int32_t h, int32_t dmax, int32_t *out, void *stream) {
  if (ctx == nullptr || rgbL_dev == nullptr || dispL == nullptr || dispR == nullptr || out == nullptr)
    return BSM_ERR_INVALID_ARG;
  if (!size_ok(w, h) || pitch_bytes < 3 * w || dmax < 1 || dmax > ctx->p.dmax) return BSM_ERR_INVALID_ARG;
  // the context's colour-plane scratch holds the refinement words of the left view meanwhile
  const cudaError_t e = ensure_plane(ctx, (size_t)w * h);
  if (e != cudaSuccess) return from_cuda(ctx, e);
  return from_cuda(ctx, bsm::launch_refine(ctx, rgbL_dev, pitch_bytes, dispL, dispR, w, h, dmax, out, ctx->plane,
                                           (cudaStream_t)stream));
}

bsm_status bsm_match_host(bsm_ctx *ctx, const uint8_t *rgbL_host, const uint8_t *rgbR_host, int32_t w, int32_t h,
                          int32_t pitch_bytes, int32_t dmax, int32_t *out_host, void *stream) {
  if (ctx == nullptr || rgbL_host == nullptr || rgbR_host == nullptr || out_host == nullptr) return BSM_ERR_INVALID_ARG;
  if (!size_ok(w, h) || pitch_bytes < 3 * w || dmax < 1 || dmax > ctx->p.dmax) return BSM_ERR_INVALID_ARG;
  const size_t img = ((size_t)h * pitch_bytes + 255) & ~(size_t)255;
  const size_t plane = ((size_t)w * h * ctx->nw * 4 + 255) & ~(size_t)255;
  const size_t map = ((size_t)w * h * 4 + 255) & ~(size_t)255;
  const size_t need = 2 * img + 4 * plane + 3 * map;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = ensure_plane(ctx, (size_t)w * h);
  if (e != cudaSuccess) return from_cuda(e);
  if (ctx->ws_bytes < need) {
    e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
      cudaFree(ctx->ws);
      ctx->ws = nullptr;
      ctx->ws_bytes = 0;
      e = cudaMalloc(&ctx->ws, need);
      if (e == cudaSuccess) ctx->ws_bytes = need;
    }
    if (e != cudaSuccess) return from_cuda(e);
  }
  uint8_t *base = (uint8_t *)ctx->ws;
  uint8_t *dl = base, *dr = base + img;
  uint32_t *BL = (uint32_t *)(base + 2 * img), *PhiL = (uint32_t *)(base + 2 * img + plane);
  uint32_t *BR = (uint32_t *)(base + 2 * img + 2 * plane), *PhiR = (uint32_t *)(base + 2 * img + 3 * plane);
  int32_t *dispL = (int32_t *)(base + 2 * img + 4 * plane);
  int32_t *dispR = (int32_t *)(base + 2 * img + 4 * plane + map);
  int32_t *out = (int32_t *)(base + 2 * img + 4 * plane + 2 * map);
  if (ctx->copy_stream == nullptr) {
    e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->copy_after, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->copy_done, cudaEventDisableTiming);
    if (e != cudaSuccess) return from_cuda(e);
  }
  // the left view uploads first, alone on the host link; the right view then uploads on the context's copy
  // stream while the left view is described (both at once would share the link and delay the left view)
  e = cudaMemcpyAsync(dl, rgbL_host, (size_t)h * pitch_bytes, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->copy_after, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_after, 0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dr, rgbR_host, (size_t)h * pitch_bytes, cudaMemcpyHostToDevice, ctx->copy_stream);
  if (e == cudaSuccess) e = cudaEventRecord(ctx->copy_done, ctx->copy_stream);
  if (e == cudaSuccess) e = bsm::launch_describe(ctx, dl, w, h, pitch_bytes, ctx->plane, BL, PhiL, s);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->copy_done, 0);
  if (e == cudaSuccess) e = bsm::launch_describe(ctx, dr, w, h, pitch_bytes, ctx->plane, BR, PhiR, s);
  if (e == cudaSuccess)
    e = bsm::launch_cost_wta(ctx, BL, PhiL, BR, PhiR, w, h, dmax, dispL, dispR, nullptr, nullptr, s);
  if (e == cudaSuccess) e = bsm::launch_refine(ctx, dl, pitch_bytes, dispL, dispR, w, h, dmax, out, ctx->plane, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, out, (size_t)w * h * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return from_cuda(e);
}

bsm_status bsm_reserve(bsm_ctx *ctx, int32_t max_w, int32_t max_h) {
  if (ctx == nullptr || !size_ok(max_w, max_h)) return BSM_ERR_INVALID_ARG;
  return from_cuda(ensure_plane(ctx, (size_t)max_w * max_h));
}

bsm_status bsm_set_tuning(bsm_ctx *ctx, const bsm_tuning *t) {
  if (ctx == nullptr || t == nullptr) return BSM_ERR_INVALID_ARG;
  for (int i = 0; i < 2; ++i)
    if (t->reserved[i] != 0) return BSM_ERR_INVALID_ARG;
  if (t->describe_copies < 0 || t->describe_copies > bsm::kMaxTileCopies) return BSM_ERR_INVALID_ARG;
  if (t->describe_variant < 0 || t->describe_variant > 2) return BSM_ERR_INVALID_ARG;
  if (t->describe_variant == 1 && ctx->nw > 8) return BSM_ERR_UNSUPPORTED;
  if (t->describe_variant == 2 && ctx->nw % 2 != 0) return BSM_ERR_UNSUPPORTED;
  if (t->cost_variant < 0 || t->cost_variant > 3) return BSM_ERR_INVALID_ARG;
  if (t->cost_variant == 3 && !bsm::cost_tc_supported(ctx)) return BSM_ERR_UNSUPPORTED;
  if (t->cost_variant == 2 && ((ctx->nw != 4 && ctx->nw != 8) || ctx->p.mask_mode == BSM_MASK_BOTH))
    return BSM_ERR_UNSUPPORTED;
  if (t->cost_rows != 0 && (t->cost_rows < 8 || t->cost_rows > 512)) return BSM_ERR_INVALID_ARG;
  if (t->batch_rows != 0 && (t->batch_rows < 8 || t->batch_rows > 512)) return BSM_ERR_INVALID_ARG;
  if (t->cost_popc_plain < 0 || t->cost_popc_plain > 2) return BSM_ERR_INVALID_ARG;
  ctx->cost_rows = t->cost_rows;
  ctx->cost_plain_popc = t->cost_popc_plain;
  ctx->batch_rows = t->batch_rows;
  ctx->cost_variant = t->cost_variant;
  ctx->describe_variant = t->describe_variant;
  if (t->describe_copies != ctx->describe_copies) {
    ctx->describe_copies = t->describe_copies;
    ctx->warp_pt = bsm::warp_pair_table(ctx);
  }
  return BSM_OK;
}

bsm_status bsm_get_tuning(bsm_ctx *ctx, bsm_tuning *t) {
  if (ctx == nullptr || t == nullptr) return BSM_ERR_INVALID_ARG;
  std::memset(t, 0, sizeof(*t));
  t->cost_rows = ctx->cost_rows;
  t->cost_popc_plain = ctx->cost_plain_popc;
  t->batch_rows = ctx->batch_rows;
  t->cost_variant = ctx->cost_variant;
  t->describe_variant = ctx->describe_variant;
  t->describe_copies = ctx->describe_copies;
  return BSM_OK;
}

bsm_status bsm_describe_gather_plan(const int8_t *pairs, int32_t n_bits, int32_t copies, int32_t *pitch,
                                    int32_t *copies_used, int32_t *copy_base, int32_t *offsets, int32_t *wavefronts) {
  if (pairs == nullptr || n_bits < 32 || n_bits % 32 != 0 || n_bits > bsm::kMaxShortBits || copies < 1 ||
      copies > bsm::kMaxTileCopies)
    return BSM_ERR_INVALID_ARG;
  bsm::PairTable pt{};
  int tp = 0;
  const int used = bsm::plan_tile_gathers(pairs, n_bits, copies, &pt, &tp, wavefronts);
  if (used == 0) return BSM_ERR_INVALID_ARG;
  if (pitch != nullptr) *pitch = tp;
  if (copies_used != nullptr) *copies_used = used;
  for (int c = 0; copy_base != nullptr && c < used; ++c) copy_base[c] = pt.copy_base[c];
  for (int i = 0; offsets != nullptr && i < n_bits; ++i) {
    offsets[2 * i] = pt.off[i][0];
    offsets[2 * i + 1] = pt.off[i][1];
  }
  return BSM_OK;
}

bsm_status bsm_cost_plan(bsm_ctx *ctx, int32_t w, int32_t h, int32_t dmax, bsm_cost_plan_info *out) {
  if (ctx == nullptr || out == nullptr || !size_ok(w, h) || dmax < 1 || dmax > ctx->p.dmax) return BSM_ERR_INVALID_ARG;
  const bsm::CostPlan p = bsm::cost_plan(ctx, w, h, dmax);
  std::memset(out, 0, sizeof(*out));
  out->kernel = p.kernel;
  out->rows_per_band = p.rows;
  out->launches = p.launches;
  return BSM_OK;
}

bsm_status bsm_last_error(bsm_ctx *ctx) {
  if (ctx == nullptr) return BSM_ERR_INVALID_ARG;
  uint32_t v = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&v, ctx->status, sizeof(v), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ctx->status, 0, sizeof(uint32_t));
  if (e != cudaSuccess) return BSM_ERR_CUDA;
  return (bsm_status)v;
}

bsm_status bsm_debug_set(bsm_ctx *ctx, int32_t key, int32_t value) {
  if (ctx == nullptr) return BSM_ERR_INVALID_ARG;
  if (key == BSM_DEBUG_WITHHOLD_ARRIVALS && (value == 0 || value == 1)) {
    ctx->withhold_arrivals = value;
    return BSM_OK;
  }
  return BSM_ERR_INVALID_ARG;
}

const char *bsm_last_cuda_error(bsm_ctx *ctx) {
  if (ctx == nullptr || ctx->last_cuda == cudaSuccess) return "";
  return cudaGetErrorName(ctx->last_cuda);
}

bsm_status bsm_copy_color_table(bsm_ctx *ctx, uint32_t *dst_dev, void *stream) {
  if (ctx == nullptr || dst_dev == nullptr) return BSM_ERR_INVALID_ARG;
  return from_cuda(cudaMemcpyAsync(dst_dev, ctx->color_table, sizeof(uint32_t) << 24, cudaMemcpyDeviceToDevice,
                                   (cudaStream_t)stream));
}

}  // extern "C"
