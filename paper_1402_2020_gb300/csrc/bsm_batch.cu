// bsm_batch_run: many stereo pairs of uneven size and dmax through the whole path in four persistent
// launches (colour pre-pass, describe, cost/aggregation/WTA, refine); the first three are replayed from
// one CUDA graph.
//
// The host writes a ticket table (one BatchPair per pair plus per-stage ticket bases and totals) into
// a pinned buffer; the graph's first node copies it to the device, and every persistent CTA then
// takes tickets from the table's counters, which the copy resets to zero. Nothing in the graph
// depends on the batch's shape, so one graph, captured the first time, serves every later batch.
// Pairs of at least kTcAutoWork pixel-disparities take no cost tickets: where the context's parameters
// allow it they run the tensor-core cost kernel, one launch each, between the graph and the
// persistent refine launch (for them it is faster than the batched popcount kernel).
#include <algorithm>
#include <cstring>

#include "bsm_internal.cuh"

namespace bsm {
cudaError_t launch_color_plane_batch(const bsm_ctx *ctx, const BatchHeader *hdr, const BatchPair *pairs, int grid,
                                     cudaStream_t s);
cudaError_t launch_describe_batch(const bsm_ctx *ctx, BatchHeader *hdr, const BatchPair *pairs, int grid,
                                  cudaStream_t s);
cudaError_t launch_cost_batch(const bsm_ctx *ctx, BatchHeader *hdr, const BatchPair *pairs, int grid, cudaStream_t s);
cudaError_t launch_refine_batch(const bsm_ctx *ctx, BatchHeader *hdr, const BatchPair *pairs, int grid,
                                cudaStream_t s);

namespace {

constexpr int kDescTY = 4;           // rows per describe tile (describe kernel's CTA)
constexpr int kRefTX = kRefineTX, kRefTY = kRefineTY;
constexpr size_t kTableBytes = sizeof(BatchHeader) + sizeof(BatchPair) * kMaxBatch;

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

bsm_status fail(bsm_ctx *ctx, cudaError_t e) {
  ctx->last_cuda = e;
  return e == cudaErrorMemoryAllocation ? BSM_ERR_OUT_OF_MEMORY : BSM_ERR_CUDA;
}

cudaError_t ensure_batch_buffers(bsm_ctx *ctx, size_t plane_words) {
  cudaError_t e = cudaSuccess;
  if (ctx->batch_table_host == nullptr) {
    e = cudaHostAlloc(&ctx->batch_table_host, kTableBytes, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->batch_table_dev, kTableBytes);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->batch_copied, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->batch_capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) return e;
  }
  if (ctx->batch_plane_words < plane_words) {
    e = cudaDeviceSynchronize();  // earlier batches may still read the old planes
    if (e != cudaSuccess) return e;
    cudaFree(ctx->batch_plane);
    ctx->batch_plane = nullptr;
    ctx->batch_plane_words = 0;
    e = cudaMalloc(&ctx->batch_plane, plane_words * sizeof(uint32_t));
    if (e == cudaSuccess) ctx->batch_plane_words = plane_words;
  }
  return e;
}

// The kernel choices and the describe tile copies baked into the captured graph: a change of any of them
// means a new capture.
int graph_variant(const bsm_ctx *ctx) {
  return ctx->cost_plain_popc + 16 * ctx->describe_variant + 64 * ctx->warp_pt.copies;
}

cudaError_t capture_graph(bsm_ctx *ctx) {
  cudaStream_t cs = ctx->batch_capture;
  // Attributes and occupancy first: nothing but stream work may happen inside the capture.
  ctx->batch_grid[0] = ctx->sms * 8;
  cudaError_t p = prepare_describe_batch(ctx, &ctx->batch_grid[1]);
  if (p == cudaSuccess) p = prepare_cost_batch(ctx, &ctx->batch_grid[2]);
  if (p == cudaSuccess) p = prepare_refine_batch(ctx, &ctx->batch_grid[3]);
  if (p != cudaSuccess) return p;
  BatchHeader *hdr = reinterpret_cast<BatchHeader *>(ctx->batch_table_dev);
  const BatchPair *pairs = reinterpret_cast<const BatchPair *>(ctx->batch_table_dev + sizeof(BatchHeader));
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  cudaError_t k = cudaMemcpyAsync(ctx->batch_table_dev, ctx->batch_table_host, kTableBytes, cudaMemcpyHostToDevice, cs);
  // An external record node: the host waits on this event before it rewrites the pinned table.
  if (k == cudaSuccess) k = cudaEventRecordWithFlags(ctx->batch_copied, cs, cudaEventRecordExternal);
  if (k == cudaSuccess) k = launch_color_plane_batch(ctx, hdr, pairs, ctx->batch_grid[0], cs);
  if (k == cudaSuccess) k = launch_describe_batch(ctx, hdr, pairs, ctx->batch_grid[1], cs);
  if (k == cudaSuccess) k = launch_cost_batch(ctx, hdr, pairs, ctx->batch_grid[2], cs);
  cudaGraph_t graph = nullptr;
  e = cudaStreamEndCapture(cs, &graph);
  if (k != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return k;
  }
  if (e != cudaSuccess) return e;
  if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
  ctx->batch_graph = nullptr;
  e = cudaGraphInstantiate(&ctx->batch_graph, graph, 0);
  cudaGraphDestroy(graph);
  if (e == cudaSuccess) ctx->batch_graph_variant = graph_variant(ctx);
  return e;
}

}  // namespace
}  // namespace bsm

using namespace bsm;

extern "C" bsm_status bsm_batch_run(bsm_ctx *ctx, const bsm_pair_desc *descs, int32_t count, void *stream) {
  if (ctx == nullptr || descs == nullptr || count < 1 || count > kMaxBatch) return BSM_ERR_INVALID_ARG;
  // the batched kernels serve descriptors of up to 256 bits weighted by the reference pixel's mask
  if (ctx->nw > 8 || ctx->p.mask_mode == BSM_MASK_BOTH) return BSM_ERR_UNSUPPORTED;
  const int outc = 32 - 2 * (ctx->p.agg_window / 2);
  const int band = ctx->batch_rows > 0 ? ctx->batch_rows : 64;
  size_t plane_words = 0;
  for (int i = 0; i < count; ++i) {
    const bsm_pair_desc &d = descs[i];
    if (d.rgbL == nullptr || d.rgbR == nullptr || d.BL == nullptr || d.PhiL == nullptr || d.BR == nullptr ||
        d.PhiR == nullptr || d.dispL == nullptr || d.dispR == nullptr || d.out == nullptr)
      return BSM_ERR_INVALID_ARG;
    if (d.w < 1 || d.h < 1 || d.w > 16384 || d.h > 16384 || d.pitch_bytes < 3 * d.w) return BSM_ERR_INVALID_ARG;
    if (d.dmax < 1 || d.dmax > ctx->p.dmax) return BSM_ERR_INVALID_ARG;
    if (!aligned16(d.BL) || !aligned16(d.PhiL) || !aligned16(d.BR) || !aligned16(d.PhiR)) return BSM_ERR_INVALID_ARG;
    plane_words += 2 * (size_t)d.w * d.h;
  }
  cudaError_t e = ensure_batch_buffers(ctx, plane_words);
  if (e != cudaSuccess) return fail(ctx, e);
  // The previous batch's graph must have copied its table before the table is rewritten.
  e = cudaEventSynchronize(ctx->batch_copied);
  if (e != cudaSuccess) return fail(ctx, e);

  BatchHeader *hdr = reinterpret_cast<BatchHeader *>(ctx->batch_table_host);
  BatchPair *pairs = reinterpret_cast<BatchPair *>(ctx->batch_table_host + sizeof(BatchHeader));
  std::memset(hdr, 0, sizeof(BatchHeader));
  hdr->count = count;
  hdr->band_rows = band;
  size_t plane_off = 0;
  int t_pre = 0, t_desc = 0, t_cost = 0, t_ref = 0;
  // the tensor-core kernel, unless the tuning asks for a popcount form
  const bool tc_ok = cost_tc_supported(ctx) && (ctx->cost_variant == 0 || ctx->cost_variant == 3);
  for (int i = 0; i < count; ++i) {
    const bsm_pair_desc &d = descs[i];
    BatchPair &p = pairs[i];
    std::memset(&p, 0, sizeof(p));
    p.rgb[0] = d.rgbL; p.rgb[1] = d.rgbR;
    p.B[0] = d.BL; p.Phi[0] = d.PhiL; p.B[1] = d.BR; p.Phi[1] = d.PhiR;
    p.disp[0] = d.dispL; p.disp[1] = d.dispR; p.out = d.out;
    p.w = d.w; p.h = d.h; p.pitch = d.pitch_bytes; p.dmax = d.dmax;
    p.plane[0] = ctx->batch_plane + plane_off;
    p.plane[1] = ctx->batch_plane + plane_off + (size_t)d.w * d.h;
    plane_off += 2 * (size_t)d.w * d.h;
    p.desc_tx = (d.w + 31) / 32;
    p.desc_ty = (d.h + kDescTY - 1) / kDescTY;
    const bool tc = tc_ok && (long long)d.w * d.h * d.dmax >= kTcAutoWork;
    p.cost_cb = tc ? 0 : (d.w + outc - 1) / outc;  // no cost tickets: the pair's own tensor-core launch
    p.cost_bands = (d.h + band - 1) / band;
    p.cost_dr = (d.dmax + kBatchDisp - 1) / kBatchDisp;
    p.ref_tx = (d.w + kRefTX - 1) / kRefTX;
    p.ref_ty = (d.h + kRefTY - 1) / kRefTY;
    p.pre_base = t_pre;
    p.desc_base = t_desc;
    p.cost_base = t_cost;
    p.ref_base = t_ref;
    t_pre += 2 * d.h;
    t_desc += 2 * p.desc_tx * p.desc_ty;
    t_cost += 2 * p.cost_cb * p.cost_bands * p.cost_dr;
    t_ref += p.ref_tx * p.ref_ty;
  }
  hdr->total[0] = t_pre;
  hdr->total[1] = t_desc;
  hdr->total[2] = t_cost;
  hdr->total[3] = t_ref;

  if (ctx->batch_graph == nullptr || ctx->batch_graph_variant != graph_variant(ctx)) {
    e = capture_graph(ctx);
    if (e != cudaSuccess) return fail(ctx, e);
  }
  cudaStream_t s = (cudaStream_t)stream;
  e = cudaGraphLaunch(ctx->batch_graph, s);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    const bsm_pair_desc &d = descs[i];
    if (pairs[i].cost_cb == 0)
      e = launch_cost_tc(ctx, d.BL, d.PhiL, d.BR, d.PhiR, d.w, d.h, d.dmax, d.dispL, d.dispR, nullptr, nullptr, s);
  }
  BatchHeader *hdr_dev = reinterpret_cast<BatchHeader *>(ctx->batch_table_dev);
  const BatchPair *pairs_dev = reinterpret_cast<const BatchPair *>(ctx->batch_table_dev + sizeof(BatchHeader));
  if (e == cudaSuccess) e = launch_refine_batch(ctx, hdr_dev, pairs_dev, ctx->batch_grid[3], s);
  return e == cudaSuccess ? BSM_OK : fail(ctx, e);
}

extern "C" bsm_status bsm_reserve_batch(bsm_ctx *ctx, int64_t total_pixels) {
  if (ctx == nullptr || total_pixels < 1) return BSM_ERR_INVALID_ARG;
  const cudaError_t e = ensure_batch_buffers(ctx, 2 * (size_t)total_pixels);
  return e == cudaSuccess ? BSM_OK : fail(ctx, e);
}
