// bsm_describe_noalloc: bsm_describe for callers that must not allocate device memory.
//
// bsm_describe keeps its colour-plane scratch in the context and grows it with cudaMalloc when a
// larger image arrives. Some callers cannot accept that: code that runs while a stream is being
// captured (an allocation is not a stream operation), code under a memory budget that was carved
// out up front (a serving process that owns all of its device memory through its own pool), and
// latency-bound loops where the implicit device synchronisation of cudaMalloc/cudaFree is not
// allowed. This entry point runs the same two kernels as bsm_describe, but the scratch plane is a
// fixed array in this file, reserved by the driver when it loads this file's module on a device (at
// the first symbol lookup below under lazy module loading) and held until the process exits. It calls
// no allocating routine.
#include <mutex>

#include "bsm_internal.cuh"

// The shared scratch plane: one packed colour word per pixel, BSM_NOALLOC_MAX_PIXELS pixels (16 MiB).
static __device__ __align__(256) uint32_t g_noalloc_plane[BSM_NOALLOC_MAX_PIXELS];

namespace {

constexpr int kMaxDevices = 64;

std::mutex g_setup_mu;
uint32_t *g_plane_addr[kMaxDevices] = {};  // device address of g_noalloc_plane, per device

// Host code may not use g_noalloc_plane's name as a device address: resolve it once per device,
// with that device current.
cudaError_t plane_for_current_device(uint32_t **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_plane_addr[dev] == nullptr) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_plane);
    if (e != cudaSuccess) return e;
    g_plane_addr[dev] = static_cast<uint32_t *>(p);
  }
  *out = g_plane_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" bsm_status bsm_describe_noalloc(bsm_ctx *ctx, const uint8_t *rgb_dev, int32_t w, int32_t h,
                                           int32_t pitch_bytes, uint32_t *B_dev, uint32_t *Phi_dev, void *stream) {
  if (ctx == nullptr || rgb_dev == nullptr || B_dev == nullptr || Phi_dev == nullptr) return BSM_ERR_INVALID_ARG;
  if (w < 1 || h < 1 || w > 16384 || h > 16384 || pitch_bytes < 3 * w) return BSM_ERR_INVALID_ARG;
  if (((uintptr_t)B_dev & 15u) != 0 || ((uintptr_t)Phi_dev & 15u) != 0) return BSM_ERR_INVALID_ARG;
  if ((int64_t)w * h > BSM_NOALLOC_MAX_PIXELS) return BSM_ERR_INVALID_ARG;  // larger than the fixed scratch
  uint32_t *plane = nullptr;
  cudaError_t e = plane_for_current_device(&plane);
  // The pre-pass writes every plane word that the describe kernel then reads, so nothing left by an
  // earlier call leaks into this one.
  if (e == cudaSuccess)
    e = bsm::launch_describe(ctx, rgb_dev, w, h, pitch_bytes, plane, B_dev, Phi_dev, (cudaStream_t)stream);
  if (e == cudaSuccess) return BSM_OK;
  ctx->last_cuda = e;  // as bsm_describe records it, for bsm_last_cuda_error
  return e == cudaErrorMemoryAllocation ? BSM_ERR_OUT_OF_MEMORY : BSM_ERR_CUDA;
}
