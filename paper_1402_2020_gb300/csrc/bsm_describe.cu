// Descriptor B(x) (Eq. 2-3) and binary mask Phi(x) (Eq. 5-7) for every pixel of one view.
//
// Pre-pass (color_plane_kernel): one thread per pixel turns the RGB8 image into a plane of packed
// colour words (L, a+128, b+128, I) with one colour-table fetch per pixel. The plane lives in the
// context's scratch memory.
//
// Describe (describe_kernel): one CTA covers a 32 x kTY block of pixels; warp r owns row r of the
// block, lane l column l.
//  0. The CTA copies its block plus a halo of the pair table's largest |offset| from the plane into
//     shared memory with 4-byte cp.async copies, clamping coordinates to the image (border
//     replicate).
//  1. Thread per pixel: for every sampling pair, tau = [I(p) > I(q)] goes into the descriptor word
//     held in a register; w = max(SAD(x, p), SAD(x, q)) (Eq. 5) is computed with byte-wise
//     absolute differences and a byte dot product, and stored as a 16-bit value in a per-warp
//     shared buffer. All 32 lanes read the same offset relative to their own pixel, so tile reads
//     are bank-conflict free. The finished descriptor goes straight to HBM (two 16-byte stores).
//  2. Warp per pixel: lane l holds the weights of pairs l, l+32, l+64, ... . T (Eq. 6) is the
//     k-th smallest weight, found by bisection between the smallest and the largest weight with
//     one warp-wide reduction per step. The weights are stored as fp16 bit patterns of 1024 + w
//     (exact: every integer below 2048 is an fp16 value), so one fp16x2 compare tests two weights
//     and the per-lane counts run on the FMA pipe; the bisections of kG pixels are interleaved so
//     that their reductions overlap. Phi's words are then __ballot_sync(w <= T) directly, because
//     pair i sits in lane i % 32, and lanes 0..n/32-1 store them.
#include <cuda_fp16.h>

#include <algorithm>
#include <cstdlib>
#include <vector>

#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kTY = 4;  // rows (warps) per CTA
constexpr int kG = 4;   // pixels whose T searches are interleaved in phase 2
constexpr uint32_t kHalfBias = 0x64006400u;  // fp16 1024.0 in both halves

struct DescribeArgs {
  const uint32_t *plane;  // packed colour words, w * h
  uint32_t *B;
  uint32_t *Phi;
  int w, h;
  int k;      // mask rank
  int halo;   // tile halo
};

__device__ __forceinline__ uint32_t lab_sad(uint32_t a, uint32_t b) {
  // |dL| + |da| + |db|: byte 3 (intensity) has weight 0.
  return __dp4a(__vabsdiffu4(a, b), 0x00010101u, 0u);
}

// The same SAD plus 1024 in the fp16 bit pattern (0x6400 | SAD for SAD < 1024): the weight's fp16 form
// without a separate bias.
__device__ __forceinline__ uint32_t lab_sad_h(uint32_t a, uint32_t b) {
  return __dp4a(__vabsdiffu4(a, b), 0x00010101u, 0x6400u);
}

__global__ void __launch_bounds__(256) color_plane_kernel(const uint8_t *__restrict__ rgb, int w, int h, int pitch,
                                                          const uint32_t *__restrict__ table,
                                                          uint32_t *__restrict__ plane) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= w) return;
  const uint8_t *px = rgb + (size_t)y * pitch + 3 * x;
  plane[(size_t)y * w + x] = __ldg(table + (((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | (uint32_t)px[2]));
}

// Shared-memory words per pixel of the weight buffer: NH groups of 32 words, each word holding the
// weights of pairs (64 m + s) in the low half and (64 m + 32 + s) in the high half. The +1 makes
// the pixel stride odd so that phase 1's column-wise stores are conflict free.
template <int NW>
struct WLayout {
  static constexpr int NH = (NW + 1) / 2;
  static constexpr int kStride = NH * 32 + 1;
};

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

// One 32 x kTY block of pixels with top-left corner (x0, y0). Contains one CTA-wide barrier, which
// every thread of the CTA reaches.
template <int NW>
__device__ __forceinline__ void describe_tile(const DescribeArgs &a, const PairTable &pt, int x0, int y0,
                                              uint32_t *smem) {
  using L = WLayout<NW>;
  const int halo = a.halo;
  const int tp = 32 + 2 * halo;
  const int th = kTY + 2 * halo;
  uint32_t *tile = smem;
  uint32_t *wbuf = tile + ((th * tp + 3) & ~3);

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // 0. colour tile with clamped coordinates
  for (int i = threadIdx.x; i < th * tp; i += blockDim.x) {
    const int ty = i / tp, tx = i - ty * tp;
    const int gx = min(max(x0 + tx - halo, 0), a.w - 1);
    const int gy = min(max(y0 + ty - halo, 0), a.h - 1);
    cp_async4(tile + i, a.plane + (size_t)gy * a.w + gx);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();

  const int y = y0 + warp;
  if (y >= a.h) return;  // whole warp; no CTA-wide barrier follows in this tile
  uint32_t *wb = wbuf + warp * 32 * L::kStride;
  const int x = x0 + lane;

  // 1. thread per pixel
  {
    const uint32_t *c = tile + (warp + halo) * tp + (lane + halo);
    const uint32_t cw = *c;
    uint32_t *wmine = wb + lane * L::kStride;
    uint32_t bw[NW];
#pragma unroll
    for (int m = 0; m < L::NH; ++m) {
      uint32_t b0 = 0, b1 = 0;
#pragma unroll
      for (int s = 0; s < 32; ++s) {
        const int i0 = 64 * m + s;
        const uint32_t p0 = c[pt.off[i0][0]], q0 = c[pt.off[i0][1]];
        b0 |= (uint32_t)(p0 > (q0 | kLabMask)) << s;
        const uint32_t w0 = max(lab_sad(cw, p0), lab_sad(cw, q0));
        uint32_t w1 = 0x3FFu;  // padding slot: 1024 + 1023 as fp16, above every T
        if (2 * m + 1 < NW) {
          const int i1 = i0 + 32;
          const uint32_t p1 = c[pt.off[i1][0]], q1 = c[pt.off[i1][1]];
          b1 |= (uint32_t)(p1 > (q1 | kLabMask)) << s;
          w1 = max(lab_sad(cw, p1), lab_sad(cw, q1));
        }
        wmine[m * 32 + s] = (w0 | (w1 << 16)) | kHalfBias;
      }
      bw[2 * m] = b0;
      if (2 * m + 1 < NW) bw[2 * m + 1] = b1;
    }
    if (x < a.w) {
      uint32_t *gB = a.B + ((size_t)y * a.w + x) * NW;
      if constexpr (NW % 4 == 0) {
#pragma unroll
        for (int j = 0; j < NW; j += 4)
          *reinterpret_cast<uint4 *>(gB + j) = make_uint4(bw[j], bw[j + 1], bw[j + 2], bw[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < NW; ++j) gB[j] = bw[j];
      }
    }
  }
  __syncwarp();

  // 2. warp per pixel, kG pixels at a time
  const int npx = min(32, a.w - x0);
  for (int px0 = 0; px0 < npx; px0 += kG) {
    __half2 v[kG][L::NH];
    uint32_t lo[kG], hi[kG];
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      const int px = min(px0 + g, npx - 1);
#pragma unroll
      for (int m = 0; m < L::NH; ++m) {
        const uint32_t word = wb[px * L::kStride + m * 32 + lane];
        v[g][m] = *reinterpret_cast<const __half2 *>(&word);
      }
      __half2 mn = v[g][0], mx = v[g][0];
#pragma unroll
      for (int m = 1; m < L::NH; ++m) {
        mn = __hmin2(mn, v[g][m]);
        mx = __hmax2(mx, v[g][m]);
      }
      const uint32_t mnb = *reinterpret_cast<const uint32_t *>(&mn), mxb = *reinterpret_cast<const uint32_t *>(&mx);
      lo[g] = __reduce_min_sync(0xFFFFFFFFu, min(mnb & 0xFFFFu, mnb >> 16)) & 0x3FFu;
      hi[g] = __reduce_max_sync(0xFFFFFFFFu, max(mxb & 0xFFFFu, mxb >> 16)) & 0x3FFu;
    }
    // T lies in [lo, hi] and count(w <= hi) >= k; every step halves the interval.
    bool open = false;
#pragma unroll
    for (int g = 0; g < kG; ++g) open |= lo[g] < hi[g];
    while (open) {
      uint32_t mid[kG], cnt[kG];
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        mid[g] = (lo[g] + hi[g]) >> 1;
        const uint32_t tb = (0x6400u | mid[g]) * 0x10001u;
        const __half2 t2 = *reinterpret_cast<const __half2 *>(&tb);
        __half2 acc = __hle2(v[g][0], t2);
#pragma unroll
        for (int m = 1; m < L::NH; ++m) acc = __hadd2(acc, __hle2(v[g][m], t2));
        const __half c = __hadd(__hadd(__low2half(acc), __high2half(acc)), __ushort_as_half((unsigned short)0x6400));
        cnt[g] = (uint32_t)__half_as_ushort(c) & 0x3FFu;  // 1024 + count, count <= 2 NH
      }
#pragma unroll
      for (int g = 0; g < kG; ++g) cnt[g] = __reduce_add_sync(0xFFFFFFFFu, cnt[g]);
      open = false;
#pragma unroll
      for (int g = 0; g < kG; ++g) {
        if (lo[g] < hi[g]) {
          if ((int)cnt[g] >= a.k) hi[g] = mid[g];
          else lo[g] = mid[g] + 1;
        }
        open |= lo[g] < hi[g];
      }
    }
#pragma unroll
    for (int g = 0; g < kG; ++g) {
      if (px0 + g >= npx) break;
      const uint32_t tb = 0x6400u | lo[g];
      uint32_t mine = 0;
#pragma unroll
      for (int m = 0; m < L::NH; ++m) {
        const uint32_t word = *reinterpret_cast<const uint32_t *>(&v[g][m]);
        const uint32_t f0 = __ballot_sync(0xFFFFFFFFu, (word & 0xFFFFu) <= tb);
        const uint32_t f1 = __ballot_sync(0xFFFFFFFFu, (word >> 16) <= tb);
        mine = lane == 2 * m ? f0 : mine;
        mine = lane == 2 * m + 1 ? f1 : mine;
      }
      if (lane < NW) a.Phi[((size_t)y * a.w + x0 + px0 + g) * NW + lane] = mine;
    }
  }
}

template <int NW>
__global__ void __launch_bounds__(kTY * 32) describe_kernel(const DescribeArgs a, const __grid_constant__ PairTable pt) {
  extern __shared__ __align__(16) uint32_t smem[];
  describe_tile<NW>(a, pt, blockIdx.x * 32, blockIdx.y * kTY, smem);
}

// Warp per pixel for n <= 256 (NW = 2, 4, 8 words): lane l evaluates pairs l, l + 32, ..., keeping
// their tile offsets in registers for the whole CTA. Descriptor word j is __ballot_sync of its 32 tau
// bits (Eq. 3) and lands in lane j; the lane's NW weights (Eq. 5) are packed two per register as fp16
// 1024 + w, T (Eq. 6) is found by bisection with one warp-wide sum per step (each step's per-lane count
// from fp16x2 compares that yield 0xFFFF per true half, summed as integers), and Phi's words are ballots
// of w <= T (Eq. 7). One warp covers a row of 32 pixels, one pixel at a time, four pixels' chains
// interleaved.
constexpr int kWY = 4;  // rows (warps) per CTA of describe_warp_kernel

// One 32 x kWY block with top-left corner (x0, y0). Contains one CTA-wide barrier, which every thread
// of the CTA reaches.
template <int NW, int UNR>
__device__ __forceinline__ void describe_warp_tile(const DescribeArgs &a, const PairTable &pt, int x0, int y0,
                                                   uint32_t *smem) {
  constexpr int NH = NW / 2;
  const int halo = a.halo, tp = 32 + 2 * halo, th = kWY + 2 * halo;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *tile = smem;
  // every copy of the tile (at pt.copy_base[c]; copy 0 at 0): rows by warp, columns by lane
  for (int c = 0; c < pt.copies; ++c) {
    uint32_t *dst = tile + pt.copy_base[c];
    for (int ty = warp; ty < th; ty += kWY) {
      const uint32_t *src = a.plane + (size_t)min(max(y0 + ty - halo, 0), a.h - 1) * a.w;
      for (int tx = lane; tx < tp; tx += 32) cp_async4(dst + ty * tp + tx, src + min(max(x0 + tx - halo, 0), a.w - 1));
    }
  }
  // The offsets differ per lane, so a constant-bank read of them is serialised across the warp: read
  // them once per tile, through an opaque move that keeps them in registers instead of re-read.
  int op[NW], oq[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) {
    asm volatile("mov.b32 %0, %1;" : "=r"(op[j]) : "r"(pt.off[32 * j + lane][0]));
    asm volatile("mov.b32 %0, %1;" : "=r"(oq[j]) : "r"(pt.off[32 * j + lane][1]));
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  const int y = y0 + warp;
  if (y >= a.h) return;
  const int npx = min(32, a.w - x0);
  const uint32_t *row = tile + (warp + halo) * tp + halo;
  const int kbr = (a.k + 31) / 32 - 1;  // the per-lane rank that brackets T (see below)
#pragma unroll UNR  // UNR pixels' ballot and reduction chains overlap
  for (int px = 0; px < npx; ++px) {
    const uint32_t *c = row + px;  // the same for every lane
    const uint32_t cw = *c;
    uint32_t bw[NW], w[NW];  // the descriptor words are warp-wide ballots: every lane holds all of them
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      const uint32_t pw = c[op[j]], qw = c[oq[j]];
      bw[j] = __ballot_sync(0xFFFFFFFFu, pw > (qw | kLabMask));
      w[j] = max(lab_sad_h(cw, pw), lab_sad_h(cw, qw));  // fp16 bits of 1024 + w
    }
    uint32_t wv[NH];
#pragma unroll
    for (int m = 0; m < NH; ++m) wv[m] = __byte_perm(w[2 * m], w[2 * m + 1], 0x5410);
    // Bracket for T: with a = ceil(k / 32) - 1 and s_a(l) lane l's a-th smallest weight (0-based), fewer
    // than k weights lie below min_l s_a(l) (at most a per lane) and at least k at or below max_l s_a(l)
    // (a + 1 per lane), so T is in [min_l s_a, max_l s_a]. Built for a = 0 and, at NW = 8, a = 1; other
    // ranks bracket with the smallest and the largest weight.
    uint32_t lo, hi;
    if (kbr == 0 || (NW == 8 && kbr == 1)) {
      __half2 h1, h2;  // per half (pairs 2m / 2m + 1): the smallest and the second smallest of its NW / 2 weights
      if constexpr (NW == 8) {
        const __half2 w0 = *reinterpret_cast<const __half2 *>(&wv[0]), w1 = *reinterpret_cast<const __half2 *>(&wv[1]);
        const __half2 w2 = *reinterpret_cast<const __half2 *>(&wv[2]), w3 = *reinterpret_cast<const __half2 *>(&wv[3]);
        const __half2 a = __hmin2(w0, w1), A = __hmax2(w0, w1), b = __hmin2(w2, w3), B = __hmax2(w2, w3);
        h1 = __hmin2(a, b);
        h2 = __hmin2(__hmax2(a, b), __hmin2(A, B));
      } else if constexpr (NW == 4) {
        const __half2 w0 = *reinterpret_cast<const __half2 *>(&wv[0]), w1 = *reinterpret_cast<const __half2 *>(&wv[1]);
        h1 = __hmin2(w0, w1);
        h2 = __hmax2(w0, w1);
      } else {
        h1 = h2 = *reinterpret_cast<const __half2 *>(&wv[0]);
      }
      // a = 0: the lane's smallest weight; a = 1: its second smallest (min of the larger first and the smaller
      // second), both halves alike, so the u32 order of the pattern is the order of the weight
      const __half2 h1s = __lowhigh2highlow(h1), h2s = __lowhigh2highlow(h2);
      const __half2 s2 = kbr == 0 ? __hmin2(h1, h1s) : __hmin2(__hmax2(h1, h1s), __hmin2(h2, h2s));
      const uint32_t sab = *reinterpret_cast<const uint32_t *>(&s2);
      lo = __reduce_min_sync(0xFFFFFFFFu, sab) & 0x3FFu;
      hi = __reduce_max_sync(0xFFFFFFFFu, sab) & 0x3FFu;
    } else {
      __half2 mn = *reinterpret_cast<const __half2 *>(&wv[0]), mx = mn;
#pragma unroll
      for (int m = 1; m < NH; ++m) {
        mn = __hmin2(mn, *reinterpret_cast<const __half2 *>(&wv[m]));
        mx = __hmax2(mx, *reinterpret_cast<const __half2 *>(&wv[m]));
      }
      const uint32_t mnb = *reinterpret_cast<const uint32_t *>(&mn), mxb = *reinterpret_cast<const uint32_t *>(&mx);
      lo = __reduce_min_sync(0xFFFFFFFFu, min(mnb & 0xFFFFu, mnb >> 16)) & 0x3FFu;
      hi = __reduce_max_sync(0xFFFFFFFFu, max(mxb & 0xFFFFu, mxb >> 16)) & 0x3FFu;
    }
    while (lo < hi) {  // T in [lo, hi] with count(w <= hi) >= k; every step halves the interval
      const uint32_t mid = (lo + hi) >> 1;
      // (1024 + mid + 1) - (1024 + w) saturated to [0, 1] is 1 exactly where w <= mid (integers below 2048
      // are exact in fp16); the lane's sum starts at 1024, so its bits are 0x6400 + the count of each half
      const uint32_t tb = (mid + 1) * 0x10001u + kHalfBias;
      const __half2 t2 = *reinterpret_cast<const __half2 *>(&tb);
      __half2 c[NH];
#pragma unroll
      for (int m = 0; m < NH; ++m) c[m] = __hsub2_sat(t2, *reinterpret_cast<const __half2 *>(&wv[m]));
      const uint32_t bias = kHalfBias;
      __half2 sum = *reinterpret_cast<const __half2 *>(&bias);
#pragma unroll
      for (int m = 0; m < NH; ++m) sum = __hadd2(sum, c[m]);
      // over the warp: 32 (0x6400 (1 + 2^16)) + C_lo + C_hi 2^16 mod 2^32, both counts below 2^16
      const uint32_t tot = __reduce_add_sync(0xFFFFFFFFu, *reinterpret_cast<const uint32_t *>(&sum)) - 0x800C8000u;
      if ((tot & 0xFFFFu) + (tot >> 16) >= (uint32_t)a.k) hi = mid;
      else lo = mid + 1;
    }
    const uint32_t tb = lo * 0x10001u + kHalfBias;  // fp16 1024 + T in both halves
    uint32_t fw[NW];
#pragma unroll
    for (int m = 0; m < NH; ++m)  // one fp16x2 compare sets the predicates of pairs 2 m (low) and 2 m + 1
      asm("{\n.reg .pred p, q;\nsetp.le.f16x2 p|q, %2, %3;\nvote.sync.ballot.b32 %0, p, 0xffffffff;\n"
          "vote.sync.ballot.b32 %1, q, 0xffffffff;\n}"
          : "=r"(fw[2 * m]), "=r"(fw[2 * m + 1])
          : "r"(wv[m]), "r"(tb));
    if (lane == 0) {  // the pixel's NW words of B and of Phi as vector stores (the planes are 16-byte aligned)
      uint32_t *ob = a.B + ((size_t)y * a.w + x0 + px) * NW, *of = a.Phi + ((size_t)y * a.w + x0 + px) * NW;
      if constexpr (NW == 2) {
        *reinterpret_cast<uint2 *>(ob) = make_uint2(bw[0], bw[1]);
        *reinterpret_cast<uint2 *>(of) = make_uint2(fw[0], fw[1]);
      } else {
#pragma unroll
        for (int v = 0; v < NW / 4; ++v) {
          reinterpret_cast<uint4 *>(ob)[v] = make_uint4(bw[4 * v], bw[4 * v + 1], bw[4 * v + 2], bw[4 * v + 3]);
          reinterpret_cast<uint4 *>(of)[v] = make_uint4(fw[4 * v], fw[4 * v + 1], fw[4 * v + 2], fw[4 * v + 3]);
        }
      }
    }
  }
}

// 12 CTAs per SM: 40 registers a thread (a few bytes spill; measured faster than 8 CTAs at 64 registers)
template <int NW>
__global__ void __launch_bounds__(kWY * 32, 12) describe_warp_kernel(const DescribeArgs a, const __grid_constant__ PairTable pt) {
  extern __shared__ __align__(16) uint32_t smem[];
  describe_warp_tile<NW, 8>(a, pt, blockIdx.x * 32, blockIdx.y * kWY, smem);
}

// Words between the bases of consecutive tile copies: the tile rounded up to whole 32-word rows of banks,
// plus one such row for the copy's bank shift.
int copy_stride(int halo) { return (((kWY + 2 * halo) * (32 + 2 * halo) + 31) & ~31) + 32; }

size_t describe_warp_smem(int halo, int copies) {
  return copies <= 1 ? 4 * (size_t)(kWY + 2 * halo) * (32 + 2 * halo) : 4 * (size_t)copies * copy_stride(halo);
}

template <int NW>
cudaError_t launch_warp_nw(const DescribeArgs &a, const PairTable &pt, cudaStream_t s) {
  const size_t smem = describe_warp_smem(a.halo, pt.copies);
  cudaError_t e = cudaFuncSetAttribute(describe_warp_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.w + 31) / 32, (a.h + kWY - 1) / kWY);
  describe_warp_kernel<NW><<<grid, kWY * 32, smem, s>>>(a, pt);
  return cudaGetLastError();
}

// Binary search: the last pair whose first ticket of the stage is <= tk.
template <typename F>
__device__ __forceinline__ int find_pair(const BatchPair *pairs, int count, int tk, F base) {
  int lo = 0, hi = count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (base(pairs[mid]) <= tk) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Batched pre-pass: every row of every view of the batch (grid-stride). Also sets the pair's WTA
// key buffers to all ones, ready for the batched cost kernel's atomicMin merge.
__global__ void __launch_bounds__(256) color_plane_batch_kernel(const BatchHeader *hdr, const BatchPair *pairs,
                                                                const uint32_t *__restrict__ table) {
  const int total = hdr->total[0], count = hdr->count;
  for (int tk = blockIdx.x; tk < total; tk += gridDim.x) {
    const int i = find_pair(pairs, count, tk, [](const BatchPair &p) { return p.pre_base; });
    const BatchPair &p = pairs[i];
    const int r = tk - p.pre_base, view = r / p.h, y = r - view * p.h;
    const uint8_t *row = p.rgb[view] + (size_t)y * p.pitch;
    uint32_t *plane = p.plane[view] + (size_t)y * p.w;
    int32_t *keys = p.disp[view] + (size_t)y * p.w;
    for (int x = threadIdx.x; x < p.w; x += blockDim.x) {
      const uint8_t *px = row + 3 * x;
      plane[x] = __ldg(table + (((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | (uint32_t)px[2]));
      keys[x] = -1;
    }
  }
}

// Batched describe: persistent CTAs take (pair, view, tile) tickets.
template <int NW>
__global__ void __launch_bounds__(kTY * 32) describe_batch_kernel(BatchHeader *hdr, const BatchPair *pairs, int k,
                                                                  int halo, const __grid_constant__ PairTable pt) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_ticket;
  const int total = hdr->total[1], count = hdr->count;
  for (;;) {
    __syncthreads();  // the previous tile is done with shared memory
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&hdr->counters[1], 1u);
    __syncthreads();
    const int tk = s_ticket;
    if (tk >= total) return;
    const BatchPair &p = pairs[find_pair(pairs, count, tk, [](const BatchPair &q) { return q.desc_base; })];
    int r = tk - p.desc_base;
    const int per_view = p.desc_tx * p.desc_ty;
    const int view = r / per_view;
    r -= view * per_view;
    const int ty = r / p.desc_tx, tx = r - ty * p.desc_tx;
    const DescribeArgs a{p.plane[view], p.B[view], p.Phi[view], p.w, p.h, k, halo};
    describe_tile<NW>(a, pt, tx * 32, ty * kTY, smem);
  }
}

// Batched describe, warp per pixel: persistent CTAs take (pair, view, tile) tickets of the same tiling.
template <int NW>
__global__ void __launch_bounds__(kWY * 32) describe_warp_batch_kernel(BatchHeader *hdr, const BatchPair *pairs, int k,
                                                                       int halo, const __grid_constant__ PairTable pt) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_ticket;
  const int total = hdr->total[1], count = hdr->count;
  for (;;) {
    __syncthreads();  // the previous tile is done with shared memory
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&hdr->counters[1], 1u);
    __syncthreads();
    const int tk = s_ticket;
    if (tk >= total) return;
    const BatchPair &p = pairs[find_pair(pairs, count, tk, [](const BatchPair &q) { return q.desc_base; })];
    int r = tk - p.desc_base;
    const int per_view = p.desc_tx * p.desc_ty;
    const int view = r / per_view;
    r -= view * per_view;
    const int ty = r / p.desc_tx, tx = r - ty * p.desc_tx;
    const DescribeArgs a{p.plane[view], p.B[view], p.Phi[view], p.w, p.h, k, halo};
    describe_warp_tile<NW, 4>(a, pt, tx * 32, ty * kWY, smem);  // 8 would spill with the ticket loop's registers
  }
}

template <int NW>
size_t describe_smem(int halo) {
  const int tp = 32 + 2 * halo, th = kTY + 2 * halo;
  return sizeof(uint32_t) * (size_t)(((th * tp + 3) & ~3) + kTY * 32 * WLayout<NW>::kStride);
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

static_assert(kWY == kTY, "the batched describe kernels share one tiling");

template <int NW, bool WARP>
cudaError_t prepare_batch_nw(int halo, int copies, int sms, int *grid) {
  size_t smem;
  void (*kern)(BatchHeader *, const BatchPair *, int, int, const PairTable);
  if constexpr (WARP) {
    smem = describe_warp_smem(halo, copies);
    kern = describe_warp_batch_kernel<NW>;
  } else {
    smem = describe_smem<NW>(halo);
    kern = describe_batch_kernel<NW>;
  }
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTY * 32, smem);
  *grid = max(1, per_sm) * sms;
  return e;
}

template <int NW, bool WARP>
cudaError_t launch_batch_nw(BatchHeader *hdr, const BatchPair *pairs, int k, int halo, const PairTable &pt, int grid,
                            cudaStream_t s) {
  if constexpr (WARP)
    describe_warp_batch_kernel<NW><<<grid, kTY * 32, describe_warp_smem(halo, pt.copies), s>>>(hdr, pairs, k, halo, pt);
  else
    describe_batch_kernel<NW><<<grid, kTY * 32, describe_smem<NW>(halo), s>>>(hdr, pairs, k, halo, pt);
  return cudaGetLastError();
}

// The batched describe follows the per-pair choice: warp per pixel for n = 256 unless told otherwise.
bool batch_warp(const bsm_ctx *ctx) {
  return ctx->nw % 2 == 0 && (ctx->describe_variant == 2 || (ctx->describe_variant == 0 && ctx->nw == 8));
}

// One tile copy at base 0 (the thread-per-pixel kernels: every lane reads the same offset from its own
// pixel, so a load touches 32 consecutive words).
PairTable make_pair_table(const bsm_ctx *ctx) {
  const int tp = 32 + 2 * ctx->halo;
  PairTable pt{};
  for (int i = 0; i < ctx->p.n_bits && i < kMaxShortBits; ++i) {
    const int8_t *q = ctx->pairs + 4 * i;
    pt.off[i][0] = q[1] * tp + q[0];
    pt.off[i][1] = q[3] * tp + q[2];
  }
  pt.copies = 1;
  return pt;
}

// ---------------------------------------------------------------- gather plan of the warp-per-pixel kernel
//
// Lane l of a warp reads, for descriptor word j, the two samples of pair 32 j + l from the tile (one load
// instruction per word and sample). The offsets of a word's 32 pairs are arbitrary, so with one tile the 32
// addresses fall in the 32 banks at random and the load replays (about 3.3 wavefronts per load at n = 256,
// S = 31). The kernel therefore keeps several copies of the tile whose bases lie in different banks: a
// sample may be read from any copy, and the host picks, per load, a copy for every distinct offset so that
// the fewest offsets share a bank (a matching of offsets to banks with a capacity L per bank, found by
// augmenting paths, L raised until one exists). The copies' bank shifts are chosen among a fixed list of
// candidates by the total wavefronts of all loads. Which lane reads which pair is unchanged, so word j's
// bit l is still pair 32 j + l's (Eq. 3), and the samples' values are the same in every copy.
constexpr int kDescribeCopies = 1;    // default tile copies (measured: with 2-4 copies the kernel is slower)
constexpr int kMaxCopyWords = 16384;  // shared memory the copies of one tile may take (64 KB)
constexpr int kShiftCandidates = 64;

int bank_of(int word) { return ((word % 32) + 32) % 32; }

struct LoadMatch {
  int items = 0;       // distinct in-copy offsets of the load
  int offs[32];
  int choice[32];      // copy of each offset
  int nb[32];          // offsets placed in each bank
  int slot[32][32];    // ... and which
  const int *base = nullptr;
  int C = 1, L = 1;

  bool place(int i, uint32_t &seen) {
    for (int c = 0; c < C; ++c) {
      const int b = bank_of(base[c] + offs[i]);
      if ((seen >> b) & 1u) continue;
      seen |= 1u << b;
      if (nb[b] < L) {
        slot[b][nb[b]++] = i;
        choice[i] = c;
        return true;
      }
      for (int k = 0; k < nb[b]; ++k) {
        if (place(slot[b][k], seen)) {  // the occupant moved to another bank
          slot[b][k] = i;
          choice[i] = c;
          return true;
        }
      }
    }
    return false;
  }

  // The smallest capacity with a complete placement (the load's wavefronts); choice[] holds that placement.
  int solve(const int *bases, int copies) {
    base = bases;
    C = copies;
    for (L = 1; L <= 32; ++L) {
      for (int b = 0; b < 32; ++b) nb[b] = 0;
      bool ok = true;
      for (int i = 0; i < items && ok; ++i) {
        uint32_t seen = 0;
        ok = place(i, seen);
      }
      if (ok) return L;
    }
    return 32;  // not reached: one bank holds at most 32 offsets
  }
};

}  // namespace

int plan_tile_gathers(const int8_t *pairs, int n_bits, int copies, PairTable *pt, int *pitch, int *wavefronts) {
  if (pairs == nullptr || pt == nullptr || n_bits < 32 || n_bits % 32 != 0 || n_bits > kMaxShortBits || copies < 1 ||
      copies > kMaxTileCopies)
    return 0;
  int halo = 0;
  for (int i = 0; i < 4 * n_bits; ++i) halo = std::max(halo, std::abs((int)pairs[i]));
  if (halo > kMaxHalo) return 0;
  const int tp = 32 + 2 * halo, stride = copy_stride(halo), nl = 2 * (n_bits / 32);
  while (copies > 1 && copies * stride > kMaxCopyWords) --copies;
  // the loads: lane l of load 2 j + s reads sample s of pair 32 j + l; item[l] indexes its distinct offset
  std::vector<LoadMatch> loads(nl);
  std::vector<int> item((size_t)nl * 32);
  for (int ld = 0; ld < nl; ++ld) {
    LoadMatch &m = loads[ld];
    for (int l = 0; l < 32; ++l) {
      const int8_t *q = pairs + 4 * (32 * (ld >> 1) + l) + 2 * (ld & 1);
      const int off = q[1] * tp + q[0];
      int k = 0;
      while (k < m.items && m.offs[k] != off) ++k;
      if (k == m.items) m.offs[m.items++] = off;
      item[(size_t)ld * 32 + l] = k;
    }
  }
  // candidate bank shifts of copies 1 .. C-1 (copy 0, which holds the centre, at shift 0): evenly spaced,
  // then sets drawn by a fixed linear congruential generator
  int best_shift[kMaxTileCopies] = {0, 0, 0, 0}, best_total = 1 << 30;
  uint32_t rng = 12345u;
  for (int cand = 0; cand < (copies > 1 ? kShiftCandidates : 1); ++cand) {
    int shift[kMaxTileCopies] = {0, 0, 0, 0};
    for (int c = 1; c < copies; ++c) {
      if (cand == 0) {
        shift[c] = 32 * c / copies;
        continue;
      }
      for (;;) {
        rng = rng * 1664525u + 1013904223u;
        const int v = 1 + (int)((rng >> 8) % 31u);
        bool dup = false;
        for (int d = 1; d < c; ++d) dup = dup || shift[d] == v;
        if (!dup) {
          shift[c] = v;
          break;
        }
      }
    }
    int base[kMaxTileCopies];
    for (int c = 0; c < copies; ++c) base[c] = c * stride + shift[c];
    int total = 0;
    for (int ld = 0; ld < nl; ++ld) total += loads[ld].solve(base, copies);
    if (total < best_total) {
      best_total = total;
      for (int c = 0; c < copies; ++c) best_shift[c] = shift[c];
    }
  }
  *pt = PairTable{};
  pt->copies = copies;
  for (int c = 0; c < copies; ++c) pt->copy_base[c] = copies > 1 ? c * stride + best_shift[c] : 0;
  for (int ld = 0; ld < nl; ++ld) {
    LoadMatch &m = loads[ld];
    const int w = m.solve(pt->copy_base, copies);
    if (wavefronts != nullptr) wavefronts[ld] = w;
    for (int l = 0; l < 32; ++l) {
      const int k = item[(size_t)ld * 32 + l];
      pt->off[32 * (ld >> 1) + l][ld & 1] = pt->copy_base[m.choice[k]] + m.offs[k];
    }
  }
  if (pitch != nullptr) *pitch = tp;
  return copies;
}

PairTable warp_pair_table(const bsm_ctx *ctx) {
  PairTable pt{};
  const int copies = ctx->describe_copies > 0 ? ctx->describe_copies : kDescribeCopies;
  if (ctx->p.n_bits <= kMaxShortBits && plan_tile_gathers(ctx->pairs, ctx->p.n_bits, copies, &pt, nullptr, nullptr) > 0)
    return pt;
  return make_pair_table(ctx);
}

cudaError_t launch_color_plane_batch(const bsm_ctx *ctx, const BatchHeader *hdr, const BatchPair *pairs, int grid,
                                     cudaStream_t s) {
  color_plane_batch_kernel<<<grid, 256, 0, s>>>(hdr, pairs, ctx->color_table);
  return cudaGetLastError();
}

cudaError_t prepare_describe_batch(const bsm_ctx *ctx, int *grid) {
  const bool wp = batch_warp(ctx);
  const int hl = ctx->halo, cp = ctx->warp_pt.copies, sm = ctx->sms;
  switch (ctx->nw) {
    case 1: return prepare_batch_nw<1, false>(hl, 1, sm, grid);
    case 2: return wp ? prepare_batch_nw<2, true>(hl, cp, sm, grid) : prepare_batch_nw<2, false>(hl, 1, sm, grid);
    case 4: return wp ? prepare_batch_nw<4, true>(hl, cp, sm, grid) : prepare_batch_nw<4, false>(hl, 1, sm, grid);
    case 8: return wp ? prepare_batch_nw<8, true>(hl, cp, sm, grid) : prepare_batch_nw<8, false>(hl, 1, sm, grid);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_describe_batch(const bsm_ctx *ctx, BatchHeader *hdr, const BatchPair *pairs, int grid,
                                  cudaStream_t s) {
  const bool wp = batch_warp(ctx);
  const PairTable pt = wp ? ctx->warp_pt : make_pair_table(ctx);
  const int k = ctx->mask_rank, hl = ctx->halo;
  switch (ctx->nw) {
    case 1: return launch_batch_nw<1, false>(hdr, pairs, k, hl, pt, grid, s);
    case 2: return wp ? launch_batch_nw<2, true>(hdr, pairs, k, hl, pt, grid, s) : launch_batch_nw<2, false>(hdr, pairs, k, hl, pt, grid, s);
    case 4: return wp ? launch_batch_nw<4, true>(hdr, pairs, k, hl, pt, grid, s) : launch_batch_nw<4, false>(hdr, pairs, k, hl, pt, grid, s);
    case 8: return wp ? launch_batch_nw<8, true>(hdr, pairs, k, hl, pt, grid, s) : launch_batch_nw<8, false>(hdr, pairs, k, hl, pt, grid, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_color_plane(const bsm_ctx *ctx, const uint8_t *rgb, int w, int h, int pitch, uint32_t *plane,
                               cudaStream_t s) {
  dim3 grid((w + 255) / 256, h);
  color_plane_kernel<<<grid, 256, 0, s>>>(rgb, w, h, pitch, ctx->color_table, plane);
  return cudaGetLastError();
}

cudaError_t launch_describe_plane(const bsm_ctx *ctx, const uint32_t *plane, int w, int h, uint32_t *B,
                                  uint32_t *Phi, cudaStream_t s) {
  if (ctx->nw > 8) return launch_describe_wide(ctx, plane, w, h, B, Phi, s);
  DescribeArgs a{plane, B, Phi, w, h, ctx->mask_rank, ctx->halo};
  // warp per pixel: chosen, or automatic from n = 256 on (measured faster there; thread per pixel below)
  if (ctx->describe_variant == 2 || (ctx->describe_variant == 0 && ctx->nw == 8)) {
    switch (ctx->nw) {
      case 2: return launch_warp_nw<2>(a, ctx->warp_pt, s);
      case 4: return launch_warp_nw<4>(a, ctx->warp_pt, s);
      case 8: return launch_warp_nw<8>(a, ctx->warp_pt, s);
      default: return cudaErrorInvalidValue;
    }
  }
  const PairTable pt = make_pair_table(ctx);
  switch (ctx->nw) {
    case 1: return launch_nw<1>(a, pt, s);
    case 2: return launch_nw<2>(a, pt, s);
    case 4: return launch_nw<4>(a, pt, s);
    case 8: return launch_nw<8>(a, pt, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_describe(const bsm_ctx *ctx, const uint8_t *rgb, int w, int h, int pitch, uint32_t *plane,
                            uint32_t *B, uint32_t *Phi, cudaStream_t s) {
  cudaError_t e = launch_color_plane(ctx, rgb, w, h, pitch, plane, s);
  if (e != cudaSuccess) return e;
  return launch_describe_plane(ctx, plane, w, h, B, Phi, s);
}

}  // namespace bsm
