// Serving engine: continuous batching of stereo-matching requests on one GPU.
//
// A scheduler thread owns `lanes` execution lanes; each lane is a context (same parameters) with its
// own stream, so the batches of different lanes overlap on the device. Requests arrive from any thread
// (bsm_server_submit) into a FIFO queue. Whenever a lane is free, the scheduler admits queued requests
// in arrival order while the engine's device-memory budget allows (each request needs its two views,
// four descriptor planes and three maps; each lane keeps the colour-plane scratch its largest batch
// and largest per-pair request needed, and that scratch is charged to the budget when it grows),
// allocates their buffers
// from the engine's own stream-ordered memory pool, and enqueues on the lane's stream: the host-to-
// device copies of the views, one bsm_batch_run for the batch's small requests, the per-pair calls
// (describe, the tensor-core cost kernel where the parameters allow it, refine) for its large ones
// (w h dmax at least 1280 x 720 x 128: there a single pair fills the GPU and the per-pair kernels are
// the faster ones), the device-to-host copies of the refined maps, the frees, and a completion event. Requests that arrive while lanes are busy wait
// only until a lane and memory free up. Completed request ids (with a status each) are handed to
// bsm_server_poll. A request too large for the budget completes with BSM_ERR_INVALID_ARG; a batch
// whose launch fails completes every request of that batch with the failing status.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "bsm_internal.cuh"

namespace {

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

constexpr int64_t kPerPairWork = 1280LL * 720 * 128;  // w h dmax from which a request runs on its own

struct Pending {
  bsm_request req;
  size_t bytes;
  std::chrono::steady_clock::time_point t_submit;
};

struct InFlight {
  Pending p;
  uint8_t *mem = nullptr;  // one pool allocation per request
};

struct Lane {
  bsm_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  uint32_t *status_host = nullptr;  // pinned copy of the context's status word, written by each batch
  std::vector<InFlight> batch;  // empty when the lane is free
  int64_t plane_pixels = 0;     // batch scratch reserved on this lane's context (colour words)
  int64_t pair_pixels = 0;      // per-pair scratch reserved on this lane's context (colour words)
};

// Lane scratch a batch needs: the batch colour planes of its small requests, and the per-pair colour
// plane of its largest large request (4 bytes per pixel each).
struct LaneNeed {
  int64_t batch_px = 0, pair_px = 0;
  int32_t pair_w = 0, pair_h = 0;  // the largest per-pair request
  void add(const bsm_request &r) {
    const int64_t px = (int64_t)r.w * r.h;
    if ((int64_t)r.w * r.h * r.dmax < kPerPairWork) {
      batch_px += px;
    } else if (px > pair_px) {
      pair_px = px;
      pair_w = r.w;
      pair_h = r.h;
    }
  }
  size_t growth(const Lane &l) const {
    return 4 * (size_t)(std::max<int64_t>(0, batch_px - l.plane_pixels) + std::max<int64_t>(0, pair_px - l.pair_pixels));
  }
};

}  // namespace

struct bsm_server {
  bsm_params params{};
  int8_t pairs[bsm::kMaxBits * 4];
  bsm_server_config cfg{};
  int device = 0;
  cudaMemPool_t pool = nullptr;
  std::vector<Lane> lanes;
  size_t budget = 0;      // bytes of device memory the engine may hold (request buffers and lane scratch)
  size_t in_use = 0;      // bytes held by admitted requests
  size_t scratch = 0;     // bytes of lane scratch reserved so far (held until the engine is destroyed)
  std::mutex mu;
  std::condition_variable cv_work;  // submissions and shutdown
  std::condition_variable cv_done;  // completions
  std::deque<Pending> queue;
  std::deque<bsm_completion> completed;
  uint64_t submitted = 0, finished = 0;
  bool stop = false;
  std::thread worker;
  bsm_server_stats stats{};
};

namespace {

size_t request_bytes(const bsm_request &r, int nw) {
  const size_t px = (size_t)r.w * r.h;
  return 2 * round256((size_t)r.h * r.pitch_bytes) + 4 * round256(px * nw * 4) + 3 * round256(px * 4);
}

void complete(bsm_server *s, uint64_t id, bsm_status st, std::chrono::steady_clock::time_point t0) {
  // caller holds s->mu
  bsm_completion c{};
  c.id = id;
  c.status = st;
  c.latency_us = std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
  s->completed.push_back(c);
  ++s->finished;
  if (st == BSM_OK) ++s->stats.completed;
  else ++s->stats.failed;
}

// Launch one batch on a free lane. Called without the lock; `batch` already holds its budget.
bsm_status launch_batch(bsm_server *s, Lane &lane) {
  const int nw = s->params.n_bits / 32;
  cudaStream_t st = lane.stream;
  std::vector<bsm_pair_desc> descs(lane.batch.size());
  // the lane scratch the admission charged to the budget: reserved here, before any work is enqueued
  LaneNeed need;
  for (auto &f : lane.batch) need.add(f.p.req);
  if (need.batch_px > lane.plane_pixels) {
    const bsm_status r = bsm_reserve_batch(lane.ctx, need.batch_px);
    if (r != BSM_OK) return r;
    lane.plane_pixels = need.batch_px;
  }
  if (need.pair_px > lane.pair_pixels) {
    const bsm_status r = bsm_reserve(lane.ctx, need.pair_w, need.pair_h);
    if (r != BSM_OK) return r;
    lane.pair_pixels = need.pair_px;
  }
  if (cudaMemsetAsync(lane.ctx->status, 0, sizeof(uint32_t), st) != cudaSuccess) return BSM_ERR_CUDA;
  for (size_t i = 0; i < lane.batch.size(); ++i) {
    InFlight &f = lane.batch[i];
    const bsm_request &r = f.p.req;
    if (cudaMallocFromPoolAsync((void **)&f.mem, f.p.bytes, s->pool, st) != cudaSuccess) return BSM_ERR_OUT_OF_MEMORY;
    const size_t px = (size_t)r.w * r.h, img = round256((size_t)r.h * r.pitch_bytes), pl = round256(px * nw * 4),
                 mp = round256(px * 4);
    uint8_t *m = f.mem;
    bsm_pair_desc &d = descs[i];
    d.rgbL = m;
    d.rgbR = m + img;
    d.w = r.w;
    d.h = r.h;
    d.pitch_bytes = r.pitch_bytes;
    d.dmax = r.dmax;
    d.BL = (uint32_t *)(m + 2 * img);
    d.PhiL = (uint32_t *)(m + 2 * img + pl);
    d.BR = (uint32_t *)(m + 2 * img + 2 * pl);
    d.PhiR = (uint32_t *)(m + 2 * img + 3 * pl);
    d.dispL = (int32_t *)(m + 2 * img + 4 * pl);
    d.dispR = (int32_t *)(m + 2 * img + 4 * pl + mp);
    d.out = (int32_t *)(m + 2 * img + 4 * pl + 2 * mp);
    if (cudaMemcpyAsync((void *)d.rgbL, r.rgbL, (size_t)r.h * r.pitch_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync((void *)d.rgbR, r.rgbR, (size_t)r.h * r.pitch_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
      return BSM_ERR_CUDA;
  }
  std::vector<bsm_pair_desc> small;
  for (const bsm_pair_desc &d : descs)
    if ((int64_t)d.w * d.h * d.dmax < kPerPairWork) small.push_back(d);
  if (!small.empty()) {
    const bsm_status b = bsm_batch_run(lane.ctx, small.data(), (int32_t)small.size(), st);
    if (b != BSM_OK) return b;
  }
  for (const bsm_pair_desc &d : descs) {
    if ((int64_t)d.w * d.h * d.dmax < kPerPairWork) continue;
    bsm_status b = bsm_describe(lane.ctx, d.rgbL, d.w, d.h, d.pitch_bytes, d.BL, d.PhiL, st);
    if (b == BSM_OK) b = bsm_describe(lane.ctx, d.rgbR, d.w, d.h, d.pitch_bytes, d.BR, d.PhiR, st);
    if (b == BSM_OK)
      b = bsm_cost_aggregate_wta(lane.ctx, d.BL, d.PhiL, d.BR, d.PhiR, d.w, d.h, d.dmax, d.dispL, d.dispR, nullptr, st);
    if (b == BSM_OK) b = bsm_refine(lane.ctx, d.rgbL, d.pitch_bytes, d.dispL, d.dispR, d.w, d.h, d.dmax, d.out, st);
    if (b != BSM_OK) return b;
  }
  for (size_t i = 0; i < lane.batch.size(); ++i) {
    const bsm_request &r = lane.batch[i].p.req;
    if (cudaMemcpyAsync(r.out, descs[i].out, (size_t)r.w * r.h * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return BSM_ERR_CUDA;
    if (cudaFreeAsync(lane.batch[i].mem, st) != cudaSuccess) return BSM_ERR_CUDA;
    lane.batch[i].mem = nullptr;
  }
  // The context's status word (bounded device waits that gave up) travels with the batch, so the
  // scheduler reads it without synchronising the device.
  if (cudaMemcpyAsync(lane.status_host, lane.ctx->status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return BSM_ERR_CUDA;
  return cudaEventRecord(lane.done, st) == cudaSuccess ? BSM_OK : BSM_ERR_CUDA;
}

void worker_main(bsm_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    // 1. retire finished lanes
    bool any_busy = false;
    for (Lane &lane : s->lanes) {
      if (lane.batch.empty()) continue;
      const cudaError_t q = cudaEventQuery(lane.done);
      if (q == cudaErrorNotReady) {
        any_busy = true;
        continue;
      }
      bsm_status st = q == cudaSuccess ? BSM_OK : BSM_ERR_CUDA;
      if (st == BSM_OK && *lane.status_host != 0) st = (bsm_status)*lane.status_host;
      for (InFlight &f : lane.batch) {
        s->in_use -= f.p.bytes;
        complete(s, f.p.req.id, st, f.p.t_submit);
      }
      lane.batch.clear();
      s->cv_done.notify_all();
    }
    if (s->stop && s->queue.empty() && !any_busy) {
      bool idle = true;
      for (Lane &lane : s->lanes) idle = idle && lane.batch.empty();
      if (idle) return;
    }
    // 2. fill free lanes from the queue (arrival order) within the memory budget
    for (Lane &lane : s->lanes) {
      if (!lane.batch.empty() || s->queue.empty()) continue;
      int64_t work = 0;
      LaneNeed need;
      size_t grow = 0;  // lane scratch this batch adds (charged once, kept by the lane)
      while (!s->queue.empty() && (int)lane.batch.size() < s->cfg.max_batch) {
        Pending &p = s->queue.front();
        LaneNeed next = need;
        next.add(p.req);
        const size_t g = next.growth(lane);
        if (s->in_use + s->scratch + g + p.bytes > s->budget) break;  // waits for memory to free up
        const int64_t wk = (int64_t)p.req.w * p.req.h * p.req.dmax;
        if (!lane.batch.empty() && s->cfg.max_batch_work > 0 && work + wk > s->cfg.max_batch_work) break;
        work += wk;
        need = next;
        grow = g;
        s->in_use += p.bytes;
        lane.batch.push_back(InFlight{p, nullptr});
        s->queue.pop_front();
      }
      if (lane.batch.empty()) continue;  // the head needs memory that busy lanes hold, or another lane's scratch
      s->scratch += grow;
      ++s->stats.batches;
      s->stats.max_batch_seen = std::max<int64_t>(s->stats.max_batch_seen, (int64_t)lane.batch.size());
      lk.unlock();
      const bsm_status st = launch_batch(s, lane);
      lk.lock();
      if (st != BSM_OK) {
        cudaStreamSynchronize(lane.stream);
        for (InFlight &f : lane.batch) {
          if (f.mem) cudaFreeAsync(f.mem, lane.stream);
          s->in_use -= f.p.bytes;
          complete(s, f.p.req.id, st, f.p.t_submit);
        }
        cudaStreamSynchronize(lane.stream);
        lane.batch.clear();
        s->cv_done.notify_all();
      }
    }
    // 3. wait: briefly while batches are in flight (to retire them), else until work arrives
    bool busy = false;
    for (Lane &lane : s->lanes) busy = busy || !lane.batch.empty();
    if (!busy && !s->queue.empty()) {
      // every lane is idle and the head request still does not fit: the lanes' scratch leaves too
      // little of the budget for it, so it can never run
      Pending p = s->queue.front();
      s->queue.pop_front();
      complete(s, p.req.id, BSM_ERR_OUT_OF_MEMORY, p.t_submit);
      s->cv_done.notify_all();
      continue;
    }
    if (busy) s->cv_work.wait_for(lk, std::chrono::microseconds(50));
    else if (s->queue.empty() && !s->stop) s->cv_work.wait(lk);
  }
}

}  // namespace

extern "C" {

bsm_status bsm_server_create(const bsm_params *params, const bsm_server_config *cfg, bsm_server **out) {
  if (params == nullptr || cfg == nullptr || out == nullptr) return BSM_ERR_INVALID_ARG;
  if (cfg->lanes < 1 || cfg->lanes > 8 || cfg->max_batch < 1 || cfg->max_batch > bsm::kMaxBatch ||
      cfg->device_budget < 0 || cfg->max_batch_work < 0)
    return BSM_ERR_INVALID_ARG;
  const bsm_status v = bsm_validate_params(params);
  if (v != BSM_OK) return v;
  // served through bsm_batch_run
  if (params->n_bits > bsm::kMaxShortBits || params->mask_mode == BSM_MASK_BOTH) return BSM_ERR_UNSUPPORTED;
  bsm_server *s = new (std::nothrow) bsm_server();
  if (s == nullptr) return BSM_ERR_OUT_OF_MEMORY;
  s->params = *params;
  std::memcpy(s->pairs, params->pairs, (size_t)4 * params->n_bits);
  s->params.pairs = s->pairs;
  s->cfg = *cfg;
  cudaGetDevice(&s->device);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
    delete s;
    return BSM_ERR_CUDA;
  }
  s->budget = cfg->device_budget > 0 ? (size_t)cfg->device_budget : free_b / 2;
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = s->device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) {
    delete s;
    return BSM_ERR_CUDA;
  }
  uint64_t keep = UINT64_MAX;  // keep freed blocks in the pool: no allocation churn between batches
  cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep);
  s->lanes.resize(cfg->lanes);
  for (Lane &lane : s->lanes) {
    bsm_status st = bsm_create(&s->params, &lane.ctx);
    if (st == BSM_OK) {  // the per-pair requests use the tensor-core cost kernel where it is built
      bsm_tuning t{};
      t.cost_variant = 3;
      if (bsm_set_tuning(lane.ctx, &t) != BSM_OK) t.cost_variant = 0;
    }
    if (st == BSM_OK && cudaStreamCreateWithFlags(&lane.stream, cudaStreamNonBlocking) != cudaSuccess) st = BSM_ERR_CUDA;
    if (st == BSM_OK && cudaEventCreateWithFlags(&lane.done, cudaEventDisableTiming) != cudaSuccess) st = BSM_ERR_CUDA;
    if (st == BSM_OK && cudaHostAlloc(&lane.status_host, sizeof(uint32_t), cudaHostAllocDefault) != cudaSuccess)
      st = BSM_ERR_OUT_OF_MEMORY;
    if (st == BSM_OK) *lane.status_host = 0;
    if (st != BSM_OK) {
      for (Lane &l2 : s->lanes) {
        if (l2.status_host) cudaFreeHost(l2.status_host);
        if (l2.done) cudaEventDestroy(l2.done);
        if (l2.stream) cudaStreamDestroy(l2.stream);
        bsm_destroy(l2.ctx);
      }
      cudaMemPoolDestroy(s->pool);
      delete s;
      return st;
    }
  }
  s->worker = std::thread(worker_main, s);
  *out = s;
  return BSM_OK;
}

bsm_status bsm_server_submit(bsm_server *s, const bsm_request *r) {
  if (s == nullptr || r == nullptr) return BSM_ERR_INVALID_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  const bool ok = r->rgbL != nullptr && r->rgbR != nullptr && r->out != nullptr && r->w >= 1 && r->h >= 1 &&
                  r->w <= 16384 && r->h <= 16384 && r->pitch_bytes >= 3 * r->w && r->dmax >= 1 &&
                  r->dmax <= s->params.dmax;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return BSM_ERR_INVALID_ARG;
  ++s->submitted;
  ++s->stats.submitted;
  const size_t bytes = ok ? request_bytes(*r, s->params.n_bits / 32) : 0;
  // with its lane scratch (one colour word per pixel) it must fit the budget on its own
  if (!ok || bytes + 4 * (size_t)r->w * r->h > s->budget) {
    complete(s, r->id, BSM_ERR_INVALID_ARG, t0);  // malformed, or larger than the whole budget
    s->cv_done.notify_all();
    return BSM_ERR_INVALID_ARG;
  }
  s->queue.push_back(Pending{*r, bytes, t0});
  s->cv_work.notify_one();
  return BSM_OK;
}

int32_t bsm_server_poll(bsm_server *s, bsm_completion *out, int32_t max_out, int32_t timeout_us) {
  if (s == nullptr || out == nullptr || max_out < 1) return -1;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->completed.empty() && timeout_us != 0) {
    if (timeout_us < 0) s->cv_done.wait(lk, [&] { return !s->completed.empty(); });
    else s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return !s->completed.empty(); });
  }
  int32_t n = 0;
  while (n < max_out && !s->completed.empty()) {
    out[n++] = s->completed.front();
    s->completed.pop_front();
  }
  return n;
}

bsm_status bsm_server_drain(bsm_server *s, int32_t timeout_ms) {
  if (s == nullptr) return BSM_ERR_INVALID_ARG;
  std::unique_lock<std::mutex> lk(s->mu);
  const auto pred = [&] { return s->finished == s->submitted; };
  if (timeout_ms < 0) {
    s->cv_done.wait(lk, pred);
    return BSM_OK;
  }
  return s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred) ? BSM_OK : BSM_ERR_TIMEOUT;
}

bsm_status bsm_server_get_stats(bsm_server *s, bsm_server_stats *out) {
  if (s == nullptr || out == nullptr) return BSM_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->stats;
  out->queued = (int64_t)s->queue.size();
  out->bytes_in_use = (int64_t)s->in_use;
  out->scratch_bytes = (int64_t)s->scratch;
  out->budget = (int64_t)s->budget;
  return BSM_OK;
}

void bsm_server_destroy(bsm_server *s) {
  if (s == nullptr) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  s->worker.join();
  for (Lane &lane : s->lanes) {
    cudaStreamSynchronize(lane.stream);
    cudaFreeHost(lane.status_host);
    cudaEventDestroy(lane.done);
    cudaStreamDestroy(lane.stream);
    bsm_destroy(lane.ctx);
  }
  cudaMemPoolDestroy(s->pool);
  delete s;
}

}  // extern "C"
