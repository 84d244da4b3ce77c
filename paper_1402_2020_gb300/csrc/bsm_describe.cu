// Descriptor B(x) (Eq. 2-3) and binary mask Phi(x) (Eq. 5-7) for every pixel of one view.
//
// One CTA covers a 32 x kTY block of pixels; warp r owns row r of the block, lane l column l.
//  0. The CTA stages its block plus a halo of the pair table's largest |offset| in shared memory as
//     packed colour words (L, a+128, b+128, I), clamping coordinates to the image (border
//     replicate). One colour-table fetch per staged pixel.
//  1. Thread per pixel: for every sampling pair, tau = [I(p) > I(q)] goes into the descriptor word
//     held in a register; w = max(SAD(x, p), SAD(x, q)) (Eq. 5) is computed with byte-wise
//     absolute differences and a byte dot product, and stored as a 16-bit value in a per-warp
//     shared buffer. All 32 lanes read the same offset relative to their own pixel, so tile reads
//     are bank-conflict free.
//  2. Warp per pixel: lane l holds the weights of pairs l, l+32, l+64, ... . T (Eq. 6) is the
//     k-th smallest weight, found by bisection on the value range [0, 765] with one warp-wide
//     reduction per step; Phi's words are then __ballot_sync(w <= T) directly, because pair i sits
//     in lane i % 32.
//  3. The warp writes its 32 pixels' B and Phi words with coalesced stores.
#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kTY = 4;  // rows (warps) per CTA

struct DescribeArgs {
  const uint8_t *rgb;
  const uint32_t *table;
  uint32_t *B;
  uint32_t *Phi;
  int w, h, pitch;
  int k;      // mask rank
  int halo;   // tile halo
};

__device__ __forceinline__ uint32_t lab_sad(uint32_t a, uint32_t b) {
  // |dL| + |da| + |db|: byte 3 (intensity) has weight 0.
  return __dp4a(__vabsdiffu4(a, b), 0x00010101u, 0u);
}

// Shared-memory words per pixel of the weight buffer: NH groups of 32 words, each word holding the
// weights of pairs (64 m + s) in the low half and (64 m + 32 + s) in the high half. The +1 makes
// the pixel stride odd so that phase 1's column-wise stores are conflict free.
template <int NW>
struct WLayout {
  static constexpr int NH = (NW + 1) / 2;
  static constexpr int kStride = NH * 32 + 1;
};

template <int NW>
__global__ void __launch_bounds__(kTY * 32) describe_kernel(const DescribeArgs a, const __grid_constant__ PairTable pt) {
  using L = WLayout<NW>;
  extern __shared__ __align__(16) uint32_t smem[];
  const int halo = a.halo;
  const int tp = 32 + 2 * halo;
  const int th = kTY + 2 * halo;
  uint32_t *tile = smem;
  uint32_t *wbuf = tile + ((th * tp + 3) & ~3);
  uint32_t *stage = wbuf + kTY * 32 * L::kStride;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * kTY;

  // 0. colour tile with clamped coordinates
  for (int i = threadIdx.x; i < th * tp; i += blockDim.x) {
    const int ty = i / tp, tx = i - ty * tp;
    const int gx = min(max(x0 + tx - halo, 0), a.w - 1);
    const int gy = min(max(y0 + ty - halo, 0), a.h - 1);
    const uint8_t *px = a.rgb + (size_t)gy * a.pitch + 3 * gx;
    tile[i] = __ldg(a.table + (((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | (uint32_t)px[2]));
  }
  __syncthreads();

  const int y = y0 + warp;
  if (y >= a.h) return;  // whole warp; no CTA-wide barrier follows

  uint32_t *wb = wbuf + warp * 32 * L::kStride;
  uint32_t *stB = stage + warp * 2 * 32 * NW;
  uint32_t *stPhi = stB + 32 * NW;

  // 1. thread per pixel
  {
    const uint32_t *c = tile + (warp + halo) * tp + (lane + halo);
    const uint32_t cw = *c;
    uint32_t *wmine = wb + lane * L::kStride;
#pragma unroll
    for (int m = 0; m < L::NH; ++m) {
      uint32_t b0 = 0, b1 = 0;
#pragma unroll
      for (int s = 0; s < 32; ++s) {
        const int i0 = 64 * m + s;
        const uint32_t p0 = c[pt.off[i0][0]], q0 = c[pt.off[i0][1]];
        b0 |= (uint32_t)(p0 > (q0 | kLabMask)) << s;
        const uint32_t w0 = max(lab_sad(cw, p0), lab_sad(cw, q0));
        uint32_t w1 = 0x7FFu;  // padding slot: never <= T
        if (2 * m + 1 < NW) {
          const int i1 = i0 + 32;
          const uint32_t p1 = c[pt.off[i1][0]], q1 = c[pt.off[i1][1]];
          b1 |= (uint32_t)(p1 > (q1 | kLabMask)) << s;
          w1 = max(lab_sad(cw, p1), lab_sad(cw, q1));
        }
        wmine[m * 32 + s] = w0 | (w1 << 16);
      }
      stB[lane * NW + 2 * m] = b0;
      if (2 * m + 1 < NW) stB[lane * NW + 2 * m + 1] = b1;
    }
  }
  __syncwarp();

  // 2. warp per pixel
  const int npx = min(32, a.w - x0);
  for (int px = 0; px < npx; ++px) {
    uint32_t v[L::NH];
#pragma unroll
    for (int m = 0; m < L::NH; ++m) v[m] = wb[px * L::kStride + m * 32 + lane];
    int lo = 0, hi = kMaxSad;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      int cnt = 0;
#pragma unroll
      for (int m = 0; m < L::NH; ++m) cnt += ((int)(v[m] & 0xFFFFu) <= mid) + ((int)(v[m] >> 16) <= mid);
      cnt = (int)__reduce_add_sync(0xFFFFFFFFu, (unsigned)cnt);
      if (cnt >= a.k) hi = mid;
      else lo = mid + 1;
    }
#pragma unroll
    for (int m = 0; m < L::NH; ++m) {
      const uint32_t f0 = __ballot_sync(0xFFFFFFFFu, (int)(v[m] & 0xFFFFu) <= lo);
      const uint32_t f1 = __ballot_sync(0xFFFFFFFFu, (int)(v[m] >> 16) <= lo);
      if (lane == 0) {
        stPhi[px * NW + 2 * m] = f0;
        if (2 * m + 1 < NW) stPhi[px * NW + 2 * m + 1] = f1;
      }
    }
  }
  __syncwarp();

  // 3. coalesced write-out of the row segment
  uint32_t *gB = a.B + ((size_t)y * a.w + x0) * NW;
  uint32_t *gPhi = a.Phi + ((size_t)y * a.w + x0) * NW;
  for (int i = lane; i < npx * NW; i += 32) {
    gB[i] = stB[i];
    gPhi[i] = stPhi[i];
  }
}

template <int NW>
size_t describe_smem(int halo) {
  const int tp = 32 + 2 * halo, th = kTY + 2 * halo;
  return sizeof(uint32_t) * (size_t)(((th * tp + 3) & ~3) + kTY * 32 * WLayout<NW>::kStride + kTY * 2 * 32 * NW);
}

template <int NW>
cudaError_t launch_nw(const DescribeArgs &a, const PairTable &pt, cudaStream_t s) {
  const size_t smem = describe_smem<NW>(a.halo);
  cudaError_t e = cudaFuncSetAttribute(describe_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.w + 31) / 32, (a.h + kTY - 1) / kTY);
  describe_kernel<NW><<<grid, kTY * 32, smem, s>>>(a, pt);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_describe(const bsm_ctx *ctx, const uint8_t *rgb, int w, int h, int pitch, uint32_t *B,
                            uint32_t *Phi, cudaStream_t s) {
  DescribeArgs a{rgb, ctx->color_table, B, Phi, w, h, pitch, ctx->mask_rank, ctx->halo};
  const int tp = 32 + 2 * ctx->halo;
  PairTable pt{};
  for (int i = 0; i < ctx->p.n_bits; ++i) {
    const int8_t *q = ctx->pairs + 4 * i;
    pt.off[i][0] = q[1] * tp + q[0];
    pt.off[i][1] = q[3] * tp + q[2];
  }
  switch (ctx->nw) {
    case 1: return launch_nw<1>(a, pt, s);
    case 2: return launch_nw<2>(a, pt, s);
    case 3: return launch_nw<3>(a, pt, s);
    case 4: return launch_nw<4>(a, pt, s);
    case 5: return launch_nw<5>(a, pt, s);
    case 6: return launch_nw<6>(a, pt, s);
    case 7: return launch_nw<7>(a, pt, s);
    case 8: return launch_nw<8>(a, pt, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsm
