// Semi-global aggregation of a cost volume (the global optimisation the paper leaves to future work,
// Sec. 5), over Eq. 8's cost (box-aggregated or not) kept in HBM as [h][w][dmax] uint16.
//
// For each path direction r the path cost obeys
//   L_r(p, d) = C(p, d) + min(L_r(p-r, d), L_r(p-r, d-1) + P1, L_r(p-r, d+1) + P1, m + P2) - m,
//   m = min_k L_r(p-r, k),
// starting with L_r(p, d) = C(p, d) where p - r leaves the image; S = sum over the paths of L_r and
// the disparity is the smallest d reaching min_d S(p, d) (Eq. 1 applied to S).
//
// One warp walks one scanline of one direction; lane l holds disparities l*D .. l*D + D - 1
// (D = ceil(dmax / 32) rounded up to a power of two), so d - 1 and d + 1 are in the same lane or one
// shuffle away, and m is one warp-wide unsigned-min reduction. The loads of the next kPF pixels are
// in flight while a pixel is computed (a register ring, refilled as each slot is consumed), and move
// as 16-byte vectors when dmax allows. Every value is an exact integer: L_r <= C + P2 and
// S <= paths * (65535 + P2) < 2^24, so the (S << 8 | d) keys fit 32 bits.
//
// Two schedules, chosen on the device by the volume's largest cost (a first pass): where
// max C + P2 < 2^16 every L_r fits 16 bits, so all directions run at once (one launch each on the
// context's own streams, their scanlines filling the GPU together) and write L_r to 16-bit scratch
// planes, and one pass sums them into S and takes Eq. 1. Otherwise the directions run one after
// another on the caller's stream: the first writes S, the others add to it, the last also takes Eq. 1.
// Both are enqueued; each kernel of the schedule not chosen returns at once.
#include <algorithm>

#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr uint32_t kInf = 0x3FFFFFFFu;  // above any path cost; keeps + P2 free of overflow

struct SgmArgs {
  const uint16_t *C;
  uint32_t *S;
  int32_t *disp;
  int w, h, dmax;
  uint32_t P1, P2;
  int dx, dy;     // path direction r
  int nlines;
  int mode;       // 0: S = L, 1: S += L, 2: S += L and disparity, 3: L into Lr (16 bits)
  uint16_t *Lr;   // mode 3: this direction's path costs, [h][w][dmax]
  const uint32_t *cmax;  // the volume's largest cost; the kernel runs only when wide == (cmax + P2 >= 2^16)
  int wide;
};

__device__ __forceinline__ bool gate_open(const uint32_t *cmax, uint32_t P2, int wide) {
  return ((*cmax + P2) > 65535u) == (wide != 0);
}

// First pixel of scanline i for direction (dx, dy): every pixel whose predecessor p - r is outside.
__device__ __forceinline__ void line_start(const SgmArgs &a, int i, int &x, int &y) {
  if (a.dy == 0) {  // one line per row
    y = i;
    x = a.dx > 0 ? 0 : a.w - 1;
  } else if (a.dx == 0) {  // one line per column
    x = i;
    y = a.dy > 0 ? 0 : a.h - 1;
  } else if (i < a.w) {  // diagonals entering through the first row of the scan
    x = i;
    y = a.dy > 0 ? 0 : a.h - 1;
  } else {  // ... and through the first column of the scan (its corner pixel belongs to the row)
    const int j = i - a.w + 1;
    x = a.dx > 0 ? 0 : a.w - 1;
    y = a.dy > 0 ? j : a.h - 1 - j;
  }
}

// Pixels on the scanline that starts at (x, y): steps until p leaves the image.
__device__ __forceinline__ int line_length(const SgmArgs &a, int x, int y) {
  int n = 0x7FFFFFFF;
  if (a.dx > 0) n = min(n, a.w - x);
  if (a.dx < 0) n = min(n, x + 1);
  if (a.dy > 0) n = min(n, a.h - y);
  if (a.dy < 0) n = min(n, y + 1);
  return n;
}

// Costs and running sums of the lane's D disparities at one pixel. VEC: dmax is a multiple of D, so
// a lane's D values are all in range or all out, and they move as 2 D-byte / 4 D-byte vectors.
template <int D, bool VEC>
__device__ __forceinline__ void fetch(const SgmArgs &a, size_t base, int d0, uint32_t (&c)[D], uint32_t (&s)[D]) {
  if constexpr (VEC) {
    if (d0 < a.dmax) {
      const uint16_t *cp = a.C + base + d0;
      const uint32_t *sp = a.S + base + d0;
      uint32_t cw[D / 2 > 0 ? D / 2 : 1];
      if constexpr (D == 8) {
        const uint4 v = *reinterpret_cast<const uint4 *>(cp);
        cw[0] = v.x; cw[1] = v.y; cw[2] = v.z; cw[3] = v.w;
      } else if constexpr (D == 4) {
        const uint2 v = *reinterpret_cast<const uint2 *>(cp);
        cw[0] = v.x; cw[1] = v.y;
      } else if constexpr (D == 2) {
        cw[0] = *reinterpret_cast<const uint32_t *>(cp);
      }
      if constexpr (D == 1) {
        c[0] = cp[0];
      } else {
#pragma unroll
        for (int j = 0; j < D; ++j) c[j] = (cw[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
      }
      if (a.mode == 1 || a.mode == 2) {
#pragma unroll
        for (int j = 0; j < D; j += 4 <= D ? 4 : D) {
          if constexpr (D >= 4) {
            const uint4 v = *reinterpret_cast<const uint4 *>(sp + j);
            s[j] = v.x; s[j + 1] = v.y; s[j + 2] = v.z; s[j + 3] = v.w;
          } else if constexpr (D == 2) {
            const uint2 v = *reinterpret_cast<const uint2 *>(sp);
            s[0] = v.x; s[1] = v.y;
          } else {
            s[0] = sp[0];
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < D; ++j) s[j] = 0;
      }
    } else {
#pragma unroll
      for (int j = 0; j < D; ++j) c[j] = s[j] = 0;
    }
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j) {
      const int d = d0 + j;
      c[j] = d < a.dmax ? (uint32_t)a.C[base + d] : 0u;
      s[j] = ((a.mode == 1 || a.mode == 2) && d < a.dmax) ? a.S[base + d] : 0u;
    }
  }
}

template <int D, bool VEC>
__device__ __forceinline__ void store_s(const SgmArgs &a, size_t base, int d0, const uint32_t (&t)[D]) {
  if constexpr (VEC && D >= 4) {
    if (d0 < a.dmax) {
#pragma unroll
      for (int j = 0; j < D; j += 4)
        *reinterpret_cast<uint4 *>(a.S + base + d0 + j) = make_uint4(t[j], t[j + 1], t[j + 2], t[j + 3]);
    }
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (d0 + j < a.dmax) a.S[base + d0 + j] = t[j];
  }
}

// Mode 3: the lane's D path costs as 16-bit values (every L_r < 2^16 on this schedule).
template <int D, bool VEC>
__device__ __forceinline__ void store_l(const SgmArgs &a, size_t base, int d0, const uint32_t (&t)[D]) {
  if constexpr (VEC && D >= 2) {
    if (d0 < a.dmax) {
      uint32_t pk[D / 2];
#pragma unroll
      for (int j = 0; j < D / 2; ++j) pk[j] = t[2 * j] | (t[2 * j + 1] << 16);
      uint16_t *dst = a.Lr + base + d0;
      if constexpr (D == 8) *reinterpret_cast<uint4 *>(dst) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
      else if constexpr (D == 4) *reinterpret_cast<uint2 *>(dst) = make_uint2(pk[0], pk[1]);
      else *reinterpret_cast<uint32_t *>(dst) = pk[0];
    }
  } else {
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (d0 + j < a.dmax) a.Lr[base + d0 + j] = (uint16_t)t[j];
  }
}

// NARROW: the concurrent schedule (mode 3: 16-bit path costs out, no S). Its directions run side by
// side, so scanlines resident per SM count for more than load-ahead depth: a 2-pixel ring, 56 registers.
template <int D, bool VEC, bool NARROW>
__global__ void __launch_bounds__(128) sgm_path_kernel(const SgmArgs a) {
  constexpr int kPF = NARROW ? 2 : 3;  // pixels of the scanline whose loads are in flight ahead of the arithmetic
  const int lane = threadIdx.x & 31;
  const int line = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (line >= a.nlines || !gate_open(a.cmax, a.P2, a.wide)) return;
  int x0, y0;
  line_start(a, line, x0, y0);
  const int len = line_length(a, x0, y0);
  const int d0 = lane * D, dmax = a.dmax;
  auto pixel = [&](int k) { return ((size_t)(y0 + k * a.dy) * a.w + (x0 + k * a.dx)) * dmax; };

  uint32_t c[kPF][D], s[kPF][D], Lp[D];
#pragma unroll
  for (int u = 0; u < kPF; ++u)
    if (u < len) fetch<D, VEC>(a, pixel(u), d0, c[u], s[u]);

  for (int k0 = 0; k0 < len; k0 += kPF) {
#pragma unroll
    for (int u = 0; u < kPF; ++u) {
      const int k = k0 + u;
      if (k >= len) break;
      uint32_t L[D];
      if (k == 0) {
#pragma unroll
        for (int j = 0; j < D; ++j) L[j] = d0 + j < dmax ? c[u][j] : kInf;
      } else {
        uint32_t lmin = kInf;
#pragma unroll
        for (int j = 0; j < D; ++j) lmin = min(lmin, Lp[j]);
        const uint32_t m = __reduce_min_sync(0xFFFFFFFFu, lmin);
        const uint32_t below = __shfl_up_sync(0xFFFFFFFFu, Lp[D - 1], 1);  // L(p-r, d0 - 1)
        const uint32_t above = __shfl_down_sync(0xFFFFFFFFu, Lp[0], 1);    // L(p-r, d0 + D)
#pragma unroll
        for (int j = 0; j < D; ++j) {
          const uint32_t lo = j > 0 ? Lp[j - 1] : (lane > 0 ? below : kInf);
          const uint32_t hi = j < D - 1 ? Lp[j + 1] : (lane < 31 ? above : kInf);
          const uint32_t best = min(min(Lp[j], min(lo, hi) + a.P1), m + a.P2);
          L[j] = d0 + j < dmax ? c[u][j] + best - m : kInf;
        }
      }
      const size_t base = pixel(k);
      if constexpr (NARROW) {
        store_l<D, VEC>(a, base, d0, L);
#pragma unroll
        for (int j = 0; j < D; ++j) Lp[j] = L[j];
        if (k + kPF < len) fetch<D, VEC>(a, pixel(k + kPF), d0, c[u], s[u]);
        continue;
      }
      uint32_t tot[D];
#pragma unroll
      for (int j = 0; j < D; ++j) tot[j] = s[u][j] + L[j];
      store_s<D, VEC>(a, base, d0, tot);
      if (a.mode == 2) {
        uint32_t key = 0xFFFFFFFFu;
#pragma unroll
        for (int j = 0; j < D; ++j)
          if (d0 + j < dmax) key = min(key, (tot[j] << 8) | (uint32_t)(d0 + j));
        key = __reduce_min_sync(0xFFFFFFFFu, key);
        if (lane == 0) a.disp[base / dmax] = (int32_t)(key & 0xFFu);
      }
#pragma unroll
      for (int j = 0; j < D; ++j) Lp[j] = L[j];
      if (k + kPF < len) fetch<D, VEC>(a, pixel(k + kPF), d0, c[u], s[u]);  // refill this slot
    }
  }
}

constexpr int kDirs[8][2] = {{1, 0}, {-1, 0}, {0, 1}, {0, -1}, {1, 1}, {-1, 1}, {1, -1}, {-1, -1}};

// The volume's largest cost (grid-stride, one atomic per warp).
__global__ void __launch_bounds__(256) sgm_max_kernel(const uint16_t *__restrict__ C, size_t n, uint32_t *cmax) {
  uint32_t m = 0;
  const size_t n8 = ((uintptr_t)C % 16 == 0) ? n / 8 : 0;  // 16-byte vectors where the volume is aligned
  const uint4 *C8 = reinterpret_cast<const uint4 *>(C);
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x) {
    const uint4 v = __ldg(C8 + i);
    m = max(m, max(max(max(v.x & 0xFFFFu, v.x >> 16), max(v.y & 0xFFFFu, v.y >> 16)),
                   max(max(v.z & 0xFFFFu, v.z >> 16), max(v.w & 0xFFFFu, v.w >> 16))));
  }
  for (size_t i = n8 * 8 + blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = max(m, (uint32_t)C[i]);
  m = __reduce_max_sync(0xFFFFFFFFu, m);
  if ((threadIdx.x & 31) == 0) atomicMax(cmax, m);
}

// S(p, d) = sum over the directions of L_r(p, d) and Eq. 1, warp per pixel, lane D disparities.
template <int D, bool VEC>
__global__ void __launch_bounds__(256) sgm_sum_kernel(const SgmArgs a, const uint16_t *__restrict__ Lr, int paths,
                                                      size_t plane) {
  const int lane = threadIdx.x & 31;
  if (!gate_open(a.cmax, a.P2, 0)) return;
  const size_t npx = (size_t)a.w * a.h;
  const int d0 = lane * D, dmax = a.dmax;
  for (size_t px = blockIdx.x * (size_t)(blockDim.x >> 5) + (threadIdx.x >> 5); px < npx;
       px += (size_t)gridDim.x * (blockDim.x >> 5)) {
    const size_t base = px * dmax;
    uint32_t tot[D];
#pragma unroll
    for (int j = 0; j < D; ++j) tot[j] = 0;
    if (d0 < dmax) {
      for (int r = 0; r < paths; ++r) {
        const uint16_t *src = Lr + r * plane + base + d0;
        if constexpr (VEC && D >= 2) {
          uint32_t pk[D / 2];
          if constexpr (D == 8) {
            const uint4 v = *reinterpret_cast<const uint4 *>(src);
            pk[0] = v.x; pk[1] = v.y; pk[2] = v.z; pk[3] = v.w;
          } else if constexpr (D == 4) {
            const uint2 v = *reinterpret_cast<const uint2 *>(src);
            pk[0] = v.x; pk[1] = v.y;
          } else {
            pk[0] = *reinterpret_cast<const uint32_t *>(src);
          }
#pragma unroll
          for (int j = 0; j < D; ++j) tot[j] += (pk[j >> 1] >> (16 * (j & 1))) & 0xFFFFu;
        } else {
#pragma unroll
          for (int j = 0; j < D; ++j)
            if (d0 + j < dmax) tot[j] += src[j];
        }
      }
    }
    store_s<D, VEC>(a, base, d0, tot);
    uint32_t key = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < D; ++j)
      if (d0 + j < dmax) key = min(key, (tot[j] << 8) | (uint32_t)(d0 + j));
    key = __reduce_min_sync(0xFFFFFFFFu, key);
    if (lane == 0) a.disp[px] = (int32_t)(key & 0xFFu);
  }
}

template <int D, bool VEC>
cudaError_t launch_paths(bsm_ctx *ctx, SgmArgs a, int paths, cudaStream_t s) {
  const int warps = 4;
  auto lines = [&](int r) { return kDirs[r][1] == 0 ? a.h : (kDirs[r][0] == 0 ? a.w : a.w + a.h - 1); };
  // concurrent schedule (narrow costs): every direction on its own stream, then the sum
  cudaError_t e = cudaEventRecord(ctx->sgm_fork, s);
  const size_t plane = (size_t)a.w * a.h * a.dmax;
  for (int r = 0; r < paths && e == cudaSuccess; ++r) {
    SgmArgs b = a;
    b.dx = kDirs[r][0];
    b.dy = kDirs[r][1];
    b.nlines = lines(r);
    b.mode = 3;
    b.Lr = ctx->sgm_ws + r * plane;
    b.wide = 0;
    e = cudaStreamWaitEvent(ctx->sgm_streams[r], ctx->sgm_fork, 0);
    if (e == cudaSuccess)
      sgm_path_kernel<D, VEC, true><<<(b.nlines + warps - 1) / warps, warps * 32, 0, ctx->sgm_streams[r]>>>(b);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(ctx->sgm_join[r], ctx->sgm_streams[r]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ctx->sgm_join[r], 0);
  }
  if (e == cudaSuccess) {
    const int grid = ctx->sms * 8;
    sgm_sum_kernel<D, VEC><<<grid, 256, 0, s>>>(a, ctx->sgm_ws, paths, plane);
    e = cudaGetLastError();
  }
  // sequential schedule (wide costs): the directions one after another, accumulating into S
  for (int r = 0; r < paths && e == cudaSuccess; ++r) {
    SgmArgs b = a;
    b.dx = kDirs[r][0];
    b.dy = kDirs[r][1];
    b.nlines = lines(r);
    b.mode = r == 0 ? 0 : (r == paths - 1 ? 2 : 1);
    b.wide = 1;
    sgm_path_kernel<D, VEC, false><<<(b.nlines + warps - 1) / warps, warps * 32, 0, s>>>(b);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace

size_t sgm_scratch_bytes(int w, int h, int dmax, int paths) {
  return (size_t)paths * w * h * dmax * 2 + 256;
}

cudaError_t launch_sgm(bsm_ctx *ctx, const uint16_t *C, int w, int h, int dmax, int P1, int P2, int paths,
                       uint32_t *S, int32_t *disp, cudaStream_t s) {
  SgmArgs a{};
  a.C = C; a.S = S; a.disp = disp;
  a.w = w; a.h = h; a.dmax = dmax;
  a.P1 = (uint32_t)P1; a.P2 = (uint32_t)P2;
  // the largest cost sits after the 16-bit planes
  uint32_t *cmax = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(ctx->sgm_ws) +
                                                sgm_scratch_bytes(w, h, dmax, paths) - 256);
  a.cmax = cmax;
  cudaError_t e = cudaMemsetAsync(cmax, 0, 4, s);
  if (e != cudaSuccess) return e;
  const size_t n = (size_t)w * h * dmax;
  const int mgrid = (int)std::min<size_t>((size_t)ctx->sms * 8, (n / 8 + 255) / 256 + 1);
  sgm_max_kernel<<<mgrid, 256, 0, s>>>(C, n, cmax);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // vector loads need every pixel's row of dmax values to start on a 2 D-byte boundary
  const bool vec = ((uintptr_t)C % 16 == 0) && ((uintptr_t)S % 16 == 0);
  switch ((dmax + 31) / 32) {
    case 1: return vec ? launch_paths<1, true>(ctx, a, paths, s) : launch_paths<1, false>(ctx, a, paths, s);
    case 2:
      return vec && dmax % 2 == 0 ? launch_paths<2, true>(ctx, a, paths, s) : launch_paths<2, false>(ctx, a, paths, s);
    case 3: case 4:
      return vec && dmax % 4 == 0 ? launch_paths<4, true>(ctx, a, paths, s) : launch_paths<4, false>(ctx, a, paths, s);
    case 5: case 6: case 7: case 8:
      return vec && dmax % 8 == 0 ? launch_paths<8, true>(ctx, a, paths, s) : launch_paths<8, false>(ctx, a, paths, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsm
