// Issue-rate probe of single integer and floating-point instructions on the GPU this library runs on.
//
// The integer rooflines of the cost and describe kernels divide their algorithmic operation counts by
// the rate at which one SM retires one instruction (lanes per clock). Those rates are properties of
// the silicon, so this probe measures them: one kernel per instruction, a full wave of 256-thread CTAs
// (eight per SM), every thread running eight independent dependency chains of the instruction in
// inline PTX for `iters` iterations. Each CTA records its SM, its first and last clock64 and the global
// timer; per SM the rate is the lane-instructions its CTAs retired over the span of their clocks, and
// the SM clock is the clock span over the global-timer span. Nothing waits on anything but the CTA's
// own arithmetic, and every store stays inside the arrays the host passes.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;

enum Op {
  OP_POPC = 0, OP_LOP3, OP_IADD3, OP_SHF, OP_PRMT, OP_IMAD, OP_VABSDIFF4, OP_DP4A, OP_IMNMX, OP_SHFL, OP_REDUX,
  OP_FFMA, OP_HFMA2, OP_MIN16X2, OP_COUNT
};

template <int OP>
__device__ __forceinline__ void step(uint32_t &r, uint32_t k1, uint32_t k2) {
  if constexpr (OP == OP_POPC) asm volatile("popc.b32 %0, %0;" : "+r"(r));
  else if constexpr (OP == OP_LOP3) asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(r) : "r"(k1), "r"(k2));
  else if constexpr (OP == OP_IADD3) asm volatile("add.u32 %0, %0, %1;" : "+r"(r) : "r"(k1));
  else if constexpr (OP == OP_SHF) asm volatile("shf.l.wrap.b32 %0, %0, %0, 3;" : "+r"(r));
  else if constexpr (OP == OP_PRMT) asm volatile("prmt.b32 %0, %0, %1, 0x5140;" : "+r"(r) : "r"(k1));
  else if constexpr (OP == OP_IMAD) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(r) : "r"(k1), "r"(k2));
  else if constexpr (OP == OP_VABSDIFF4)
    asm volatile("vabsdiff4.u32.u32.u32 %0, %0, %1, %2;" : "+r"(r) : "r"(k1), "r"(k2));
  else if constexpr (OP == OP_DP4A) asm volatile("dp4a.u32.u32 %0, %0, %1, %0;" : "+r"(r) : "r"(k1));
  else if constexpr (OP == OP_IMNMX) asm volatile("min.u32 %0, %0, %1;" : "+r"(r) : "r"(k1));
  else if constexpr (OP == OP_SHFL) asm volatile("shfl.sync.bfly.b32 %0, %0, 1, 0x1f, 0xffffffff;" : "+r"(r));
  else if constexpr (OP == OP_REDUX) asm volatile("redux.sync.min.u32 %0, %0, 0xffffffff;" : "+r"(r));
  else if constexpr (OP == OP_FFMA) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+r"(r) : "r"(k1), "r"(k2));
  else if constexpr (OP == OP_HFMA2) asm volatile("fma.rn.f16x2 %0, %0, %1, %2;" : "+r"(r) : "r"(k1), "r"(k2));
  else asm volatile("{\n.reg .b32 t;\nmin.u16x2 t, %0, %1;\nxor.b32 %0, t, %2;\n}" : "+r"(r) : "r"(k1), "r"(k2));
}

template <int OP>
__global__ void __launch_bounds__(kThreads) issue_kernel(int iters, uint32_t seed, uint32_t *sink,
                                                          long long *rec) {
  uint32_t r[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) r[j] = seed * (threadIdx.x + 1u) + 0x9E3779B9u * (j + 1u);
  // operands that keep the chains' values well defined (no NaN or infinity for the float forms)
  const uint32_t k1 = OP == OP_FFMA ? 0x3F7FFFF0u : OP == OP_HFMA2 ? 0x3BFF3BFFu : (seed | 1u);
  const uint32_t k2 = OP == OP_FFMA ? 0x3A800000u : OP == OP_HFMA2 ? 0x14001400u : (seed >> 3);
  if (OP == OP_FFMA || OP == OP_HFMA2) {
#pragma unroll
    for (int j = 0; j < kChains; ++j) r[j] = OP == OP_FFMA ? 0x3F800000u : 0x3C003C00u;
  }
  __syncthreads();
  uint32_t smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  long long c0 = clock64();
  unsigned long long g0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g0));
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) step<OP>(r[j], k1, k2);
    }
  }
  __syncthreads();
  long long c1 = clock64();
  unsigned long long g1;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(g1));
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < kChains; ++j) acc ^= r[j];
  if (acc == 0x12345678u) sink[blockIdx.x] = acc;  // keeps the chains live
  if (threadIdx.x == 0) {
    long long *o = rec + 5 * (size_t)blockIdx.x;
    o[0] = smid;
    o[1] = c0;
    o[2] = c1;
    o[3] = (long long)g0;
    o[4] = (long long)g1;
  }
}

template <int OP>
cudaError_t launch(int blocks, int iters, uint32_t *sink, long long *rec) {
  issue_kernel<OP><<<blocks, kThreads>>>(iters, 0x2545F491u, sink, rec);
  return cudaGetLastError();
}

cudaError_t launch_op(int op, int blocks, int iters, uint32_t *sink, long long *rec) {
  switch (op) {
    case OP_POPC: return launch<OP_POPC>(blocks, iters, sink, rec);
    case OP_LOP3: return launch<OP_LOP3>(blocks, iters, sink, rec);
    case OP_IADD3: return launch<OP_IADD3>(blocks, iters, sink, rec);
    case OP_SHF: return launch<OP_SHF>(blocks, iters, sink, rec);
    case OP_PRMT: return launch<OP_PRMT>(blocks, iters, sink, rec);
    case OP_IMAD: return launch<OP_IMAD>(blocks, iters, sink, rec);
    case OP_VABSDIFF4: return launch<OP_VABSDIFF4>(blocks, iters, sink, rec);
    case OP_DP4A: return launch<OP_DP4A>(blocks, iters, sink, rec);
    case OP_IMNMX: return launch<OP_IMNMX>(blocks, iters, sink, rec);
    case OP_SHFL: return launch<OP_SHFL>(blocks, iters, sink, rec);
    case OP_REDUX: return launch<OP_REDUX>(blocks, iters, sink, rec);
    case OP_FFMA: return launch<OP_FFMA>(blocks, iters, sink, rec);
    case OP_HFMA2: return launch<OP_HFMA2>(blocks, iters, sink, rec);
    case OP_MIN16X2: return launch<OP_MIN16X2>(blocks, iters, sink, rec);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

extern "C" {

// Number of instructions the probe knows (op indices 0 .. count - 1).
int bsm_probe_op_count(void) { return OP_COUNT; }

// Measures instruction `op`: lane-instructions retired per clock per SM (median over SMs) and the SM
// clock in MHz during the run (median over SMs). `ctas_per_sm` CTAs of 256 threads per SM, `iters`
// iterations of 32 instructions per thread. Returns 0, or a CUDA error code (nothing is written then).
int bsm_probe_issue_rate(int op, int ctas_per_sm, int iters, double *lanes_per_clk_per_sm, double *sm_mhz) {
  if (op < 0 || op >= OP_COUNT || ctas_per_sm < 1 || ctas_per_sm > 8 || iters < 1 || iters > (1 << 20) ||
      lanes_per_clk_per_sm == nullptr || sm_mhz == nullptr)
    return (int)cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return (int)e;
  const int blocks = sms * ctas_per_sm;
  uint32_t *sink = nullptr;
  long long *rec = nullptr;
  e = cudaMalloc(&sink, sizeof(uint32_t) * blocks);
  if (e == cudaSuccess) e = cudaMalloc(&rec, sizeof(long long) * 5 * blocks);
  if (e == cudaSuccess) e = launch_op(op, blocks, iters / 8 + 1, sink, rec);  // warm-up
  if (e == cudaSuccess) e = launch_op(op, blocks, iters, sink, rec);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  std::vector<long long> h((size_t)5 * blocks);
  if (e == cudaSuccess) e = cudaMemcpy(h.data(), rec, sizeof(long long) * 5 * blocks, cudaMemcpyDeviceToHost);
  cudaFree(sink);
  cudaFree(rec);
  if (e != cudaSuccess) return (int)e;
  // per SM: its CTAs' lane-instructions over the span of their clocks
  std::vector<long long> c_lo(sms, -1), c_hi(sms, -1), g_lo(sms, -1), g_hi(sms, -1);
  std::vector<int> n(sms, 0);
  for (int b = 0; b < blocks; ++b) {
    const long long *o = &h[(size_t)5 * b];
    const int s = (int)o[0];
    if (s < 0 || s >= sms) continue;
    c_lo[s] = n[s] ? std::min(c_lo[s], o[1]) : o[1];
    c_hi[s] = n[s] ? std::max(c_hi[s], o[2]) : o[2];
    g_lo[s] = n[s] ? std::min(g_lo[s], o[3]) : o[3];
    g_hi[s] = n[s] ? std::max(g_hi[s], o[4]) : o[4];
    ++n[s];
  }
  const double per_cta = (double)kThreads * iters * 4 * kChains;
  std::vector<double> rate, mhz;
  for (int s = 0; s < sms; ++s) {
    if (n[s] == 0 || c_hi[s] <= c_lo[s] || g_hi[s] <= g_lo[s]) continue;
    rate.push_back(per_cta * n[s] / (double)(c_hi[s] - c_lo[s]));
    mhz.push_back((double)(c_hi[s] - c_lo[s]) / (double)(g_hi[s] - g_lo[s]) * 1e3);
  }
  if (rate.empty()) return (int)cudaErrorUnknown;
  std::sort(rate.begin(), rate.end());
  std::sort(mhz.begin(), mhz.end());
  *lanes_per_clk_per_sm = rate[rate.size() / 2];
  *sm_mhz = mhz[mhz.size() / 2];
  return 0;
}

}  // extern "C"
