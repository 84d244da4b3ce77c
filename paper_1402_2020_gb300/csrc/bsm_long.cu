// Long descriptors (n = 512 ... 4096 bits; the paper's experiments use n = 4096, Sec. 4.1).
//
// describe_wide_kernel (Eq. 2-3, 5-7): one warp per pixel for both phases. Lane l takes the pairs
// l, l + 32, l + 64, ...: tau of pair 32 j + l is bit l of descriptor word j, so each word is one
// __ballot_sync; the lane keeps its n/32 weights in registers as fp16 pairs (1024 + w, exact), and T is
// found by the same bisection as for short descriptors with one warp-wide reduction per step. The
// pairs' tile offsets come from a shared-memory table (n can exceed what fits in kernel parameters).
//
// cost_long_kernel (Eq. 8 + box aggregation + Eq. 1): one column per lane and 8 disparities per warp,
// as for short descriptors, but each row is staged and consumed in chunks of 8 descriptor words
// (32 bytes per pixel) with 16-byte cp.async copies, double-buffered over the sequence of (row, chunk);
// the masked popcounts accumulate over the chunks, and the out-of-image cost, the box sums and the
// argmin follow a row's last chunk. n * window^2 <= 65535 keeps two costs per 32-bit register.
// The same kernel serves the mask ablation that also ANDs the matched pixel's Phi (template MM), for
// any n that is a multiple of 256 bits: the other view's Phi is then staged beside its B.
#include <cuda_fp16.h>

#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kWTY = 4;  // rows (warps) per CTA of describe_wide_kernel

__device__ __forceinline__ uint32_t lab_sad(uint32_t a, uint32_t b) {
  return __dp4a(__vabsdiffu4(a, b), 0x00010101u, 0u);
}

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

struct WideArgs {
  const uint32_t *plane;   // packed colour words
  const int32_t *offs;     // n entries: (q offset << 16) | (p offset & 0xFFFF), tile-relative
  uint32_t *B, *Phi;
  int w, h, k, halo;
};

template <int NW>
__global__ void __launch_bounds__(kWTY * 32) describe_wide_kernel(const WideArgs a) {
  constexpr int NH = NW / 2;  // fp16 pairs per lane: pairs 32 j + l and 32 (j + 1) + l share a register
  extern __shared__ __align__(16) uint32_t smem[];
  const int halo = a.halo, tp = 32 + 2 * halo, th = kWTY + 2 * halo;
  int32_t *soffs = reinterpret_cast<int32_t *>(smem);  // [NW][32]
  uint32_t *tile = smem + NW * 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x0 = blockIdx.x * 32, y0 = blockIdx.y * kWTY;

  for (int i = threadIdx.x; i < NW * 32; i += blockDim.x) soffs[i] = __ldg(a.offs + i);
  for (int i = threadIdx.x; i < th * tp; i += blockDim.x) {
    const int ty = i / tp, tx = i - ty * tp;
    const int gx = min(max(x0 + tx - halo, 0), a.w - 1);
    const int gy = min(max(y0 + ty - halo, 0), a.h - 1);
    cp_async4(tile + i, a.plane + (size_t)gy * a.w + gx);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();

  const int y = y0 + warp;
  if (y >= a.h) return;
  const int npx = min(32, a.w - x0);
  for (int px = 0; px < npx; ++px) {
    const uint32_t *c = tile + (warp + halo) * tp + (px + halo);
    const uint32_t cw = *c;
    uint32_t wv[NH];
    constexpr int NL = (NW + 31) / 32;  // descriptor words kept per lane (word j lives in lane j % 32)
    uint32_t bwords[NL], fwords[NL];
#pragma unroll
    for (int m = 0; m < NL; ++m) bwords[m] = fwords[m] = 0;
    // phase 1: lane l, pairs 32 j + l (fully unrolled: the register arrays need constant indices)
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      const int32_t o = soffs[j * 32 + lane];
      const int op = (int)(int16_t)(o & 0xFFFF), oq = o >> 16;
      const uint32_t pw = c[op], qw = c[oq];
      const uint32_t bits = __ballot_sync(0xFFFFFFFFu, pw > (qw | kLabMask));
      if (lane == (j & 31)) bwords[j >> 5] = bits;
      const uint32_t wt = max(lab_sad(cw, pw), lab_sad(cw, qw)) | 0x6400u;  // fp16 bits of 1024 + w
      if (j & 1) wv[j >> 1] |= wt << 16;
      else wv[j >> 1] = wt;
    }
    // phase 2: T by bisection between the smallest and the largest weight
    __half2 mn = *reinterpret_cast<const __half2 *>(&wv[0]), mx = mn;
#pragma unroll
    for (int m = 1; m < NH; ++m) {
      const __half2 v = *reinterpret_cast<const __half2 *>(&wv[m]);
      mn = __hmin2(mn, v);
      mx = __hmax2(mx, v);
    }
    const uint32_t mnb = *reinterpret_cast<const uint32_t *>(&mn), mxb = *reinterpret_cast<const uint32_t *>(&mx);
    uint32_t lo = __reduce_min_sync(0xFFFFFFFFu, min(mnb & 0xFFFFu, mnb >> 16)) & 0x3FFu;
    uint32_t hi = __reduce_max_sync(0xFFFFFFFFu, max(mxb & 0xFFFFu, mxb >> 16)) & 0x3FFu;
    while (lo < hi) {
      const uint32_t mid = (lo + hi) >> 1;
      const uint32_t tb = (0x6400u | mid) * 0x10001u;
      const __half2 t2 = *reinterpret_cast<const __half2 *>(&tb);
      // per-lane count <= n / 32 <= 128: exact in fp16; the pairwise sums keep each partial small
      __half2 acc = __hle2(*reinterpret_cast<const __half2 *>(&wv[0]), t2);
#pragma unroll
      for (int m = 1; m < NH; ++m) acc = __hadd2(acc, __hle2(*reinterpret_cast<const __half2 *>(&wv[m]), t2));
      const __half cnt = __hadd(__hadd(__low2half(acc), __high2half(acc)), __ushort_as_half((unsigned short)0x6400));
      const int total = (int)__reduce_add_sync(0xFFFFFFFFu, (uint32_t)__half_as_ushort(cnt) & 0x3FFu);
      if (total >= a.k) hi = mid;
      else lo = mid + 1;
    }
    const uint32_t tb = 0x6400u | lo;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
      const uint32_t wt = (j & 1) ? (wv[j >> 1] >> 16) : (wv[j >> 1] & 0xFFFFu);
      const uint32_t bits = __ballot_sync(0xFFFFFFFFu, wt <= tb);
      if (lane == (j & 31)) fwords[j >> 5] = bits;
    }
    const size_t base = ((size_t)y * a.w + x0 + px) * NW;
#pragma unroll
    for (int m = 0; m < NL; ++m) {
      if (32 * m + lane < NW) {
        a.B[base + 32 * m + lane] = bwords[m];
        a.Phi[base + 32 * m + lane] = fwords[m];
      }
    }
  }
}

template <int NW>
cudaError_t launch_wide_nw(const WideArgs &a, cudaStream_t s) {
  const int tp = 32 + 2 * a.halo, th = kWTY + 2 * a.halo;
  const size_t smem = 4 * ((size_t)NW * 32 + (size_t)th * tp);
  cudaError_t e = cudaFuncSetAttribute(describe_wide_kernel<NW>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.w + 31) / 32, (a.h + kWTY - 1) / kWTY);
  describe_wide_kernel<NW><<<grid, kWTY * 32, smem, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- chunked cost kernel

constexpr int kDC = 8, kDP = 4, kChunkWords = 8;

struct LongArgs {
  const uint32_t *B[2], *Phi[2], *O[2], *OPhi[2];
  int32_t *disp[2];
  uint16_t *cost[2];  // optional aggregated cost volume per reference view
  int w, h, dmax, rows, nw;
};

__device__ __forceinline__ uint32_t lop3_xor3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t lop3_maj(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t r;
  asm("lop3.b32 %0, %1, %2, %3, 0xE8;" : "=r"(r) : "r"(a), "r"(b), "r"(c));
  return r;
}
__device__ __forceinline__ uint32_t lop3_xor_and(uint32_t a, uint32_t b, uint32_t m) {
  uint32_t r;
  asm("lop3.b32 %0, %1, %2, %3, 0x28;" : "=r"(r) : "r"(a), "r"(b), "r"(m));
  return r;
}

__device__ __forceinline__ void load8(const uint32_t *p, int q, uint32_t (&v)[8]) {
  const uint4 a = *reinterpret_cast<const uint4 *>(p + 4 * q);
  const uint4 b = *reinterpret_cast<const uint4 *>(p + 4 * (1 - q));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// popcount of 8 masked words through carry-save adders (4 POPC)
__device__ __forceinline__ uint32_t masked_hamming8(const uint32_t (&b)[8], const uint32_t (&o)[8],
                                                    const uint32_t (&m)[8]) {
  uint32_t v[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = lop3_xor_and(b[j], o[j], m[j]);
  const uint32_t s1 = lop3_xor3(v[0], v[1], v[2]), c1 = lop3_maj(v[0], v[1], v[2]);
  const uint32_t s2 = lop3_xor3(v[3], v[4], v[5]), c2 = lop3_maj(v[3], v[4], v[5]);
  const uint32_t s3 = lop3_xor3(s1, s2, v[6]), c3 = lop3_maj(s1, s2, v[6]);
  const uint32_t s4 = lop3_xor3(c1, c2, c3), c4 = lop3_maj(c1, c2, c3);
  return (uint32_t)__popc(s3) + (uint32_t)__popc(v[7]) + 2u * (uint32_t)__popc(s4) + 4u * (uint32_t)__popc(c4);
}

// the same with both views' masks: popcount((b ^ o) & m & mo)
__device__ __forceinline__ uint32_t masked2_hamming8(const uint32_t (&b)[8], const uint32_t (&o)[8],
                                                     const uint32_t (&m)[8], const uint32_t (&mo)[8]) {
  uint32_t mm[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) mm[j] = m[j] & mo[j];
  return masked_hamming8(b, o, mm);
}

template <int WIN, int DIR, int MM>
__device__ __forceinline__ void cost_long_body(const LongArgs &a, uint8_t *smem_raw) {
  constexpr int R = WIN / 2, OUTC = 32 - 2 * R;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nd = nwarps * kDC, ocols = 32 + nd - 1;
  const int stage_words = 64 * kChunkWords + (MM + 1) * ocols * kChunkWords;
  uint32_t *stages = reinterpret_cast<uint32_t *>(smem_raw);
  uint32_t *keys = stages + 2 * stage_words;  // [2][nwarps][32]
  uint4 *ring = reinterpret_cast<uint4 *>(keys + 2 * nwarps * 32);

  const uint32_t *__restrict__ Bref = a.B[DIR];
  const uint32_t *__restrict__ Phiref = a.Phi[DIR];
  const uint32_t *__restrict__ Both = a.O[DIR];
  const uint32_t *__restrict__ Phioth = a.OPhi[DIR];
  int32_t *__restrict__ disp = a.disp[DIR];
  const int w = a.w, h = a.h, dmax = a.dmax, nw = a.nw, nch = nw / kChunkWords;
  const uint32_t nbits = 32u * (uint32_t)nw;
  const int x0 = (int)blockIdx.x * OUTC - R, x = x0 + lane;
  const int yb = (int)blockIdx.y * a.rows, ye = min(h, yb + a.rows);
  const int d0 = warp * kDC;
  const int ox0 = DIR == 0 ? x0 - (nd - 1) : x0;
  const bool col_in = x >= 0 && x < w;
  const bool out_lane = lane >= R && lane < 32 - R && col_in;
  const int q = (lane >> 2) & 1;
  const int y_first = yb - R, n_it = (ye + R) - y_first;

  auto issue = [&](int f, int s) {  // stage chunk f % nch of row y_first + f / nch into buffer s
    const int y = y_first + f / nch, ch = f % nch;
    if (y < 0 || y >= h) return;
    uint32_t *st = stages + s * stage_words;
    const int nref = 2 * 32 * 2, noth = ocols * 2;  // 16-byte halves of each pixel's chunk
    for (int i = tid; i < nref + (MM + 1) * noth; i += blockDim.x) {
      if (i < nref) {
        const int plane = i >> 6, j = (i >> 1) & 31, half = i & 1;
        const int gx = x0 + j;
        if (gx >= 0 && gx < w)
          cp_async16(st + plane * 32 * kChunkWords + j * kChunkWords + 4 * half,
                     (plane ? Phiref : Bref) + ((size_t)y * w + gx) * nw + ch * kChunkWords + 4 * half);
      } else {
        const int r0 = i - nref, plane = r0 >= noth ? 1 : 0, r = r0 - plane * noth, p = r >> 1, half = r & 1;
        const int gx = ox0 + p;
        if (gx >= 0 && gx < w)
          cp_async16(st + 64 * kChunkWords + (plane * ocols + p) * kChunkWords + 4 * half,
                     (plane ? Phioth : Both) + ((size_t)y * w + gx) * nw + ch * kChunkWords + 4 * half);
      }
    }
  };
  auto reduce_keys = [&](int it) {
    const int yo = y_first + it - R;
    const uint32_t *kb = keys + (it & 1) * nwarps * 32;
    uint32_t best = kb[lane];
    for (int k = 1; k < nwarps; ++k) best = min(best, kb[k * 32 + lane]);
    if (out_lane) disp[(size_t)yo * w + x] = (int32_t)(best & 1023u);
  };

  if constexpr (WIN > 1) {
    for (int s = 0; s < WIN; ++s) ring[s * blockDim.x + tid] = make_uint4(0, 0, 0, 0);
  }
  issue(0, 0);
  asm volatile("cp.async.commit_group;" ::: "memory");
  uint32_t V[kDP] = {0, 0, 0, 0}, C[kDP] = {0, 0, 0, 0};
  const int nf = n_it * nch;
  for (int f = 0; f < nf; ++f) {
    const int it = f / nch, ch = f - it * nch, y = y_first + it, s = f & 1;
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    if (f + 1 < nf) issue(f + 1, s ^ 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (ch == 0) {
      if (warp == 0 && it >= 1 && y - 1 - R >= yb) reduce_keys(it - 1);
#pragma unroll
      for (int j = 0; j < kDP; ++j) C[j] = 0;
    }
    const bool row_in = y >= 0 && y < h;
    if (row_in && col_in && d0 < dmax) {
      const uint32_t *st = stages + s * stage_words;
      uint32_t b[8], m[8];
      load8(st + lane * kChunkWords, q, b);
      load8(st + 32 * kChunkWords + lane * kChunkWords, q, m);
      const uint32_t *ob = st + 64 * kChunkWords + (DIR == 0 ? lane + nd - 1 - d0 : lane + d0) * kChunkWords;
#pragma unroll
      for (int dd = 0; dd < kDC; ++dd) {
        uint32_t o[8];
        load8(ob + (DIR == 0 ? -dd : dd) * kChunkWords, q, o);
        if constexpr (MM) {
          uint32_t mo[8];
          load8(ob + (ocols + (DIR == 0 ? -dd : dd)) * kChunkWords, q, mo);
          C[dd >> 1] += masked2_hamming8(b, o, m, mo) << (16 * (dd & 1));
        } else {
          C[dd >> 1] += masked_hamming8(b, o, m) << (16 * (dd & 1));
        }
      }
    }
    if (ch != nch - 1) continue;

    // the row is complete: out-of-image matches cost n, columns outside the image contribute 0
    if (row_in) {
#pragma unroll
      for (int dd = 0; dd < kDC; ++dd) {
        const int d = d0 + dd;
        const bool match_in = DIR == 0 ? x - d >= 0 : x + d < w;
        const uint32_t sh = 16 * (dd & 1), mask = 0xFFFFu << sh;
        uint32_t cv = (C[dd >> 1] >> sh) & 0xFFFFu;
        cv = !col_in ? 0u : (match_in ? cv : nbits);
        C[dd >> 1] = (C[dd >> 1] & ~mask) | (cv << sh);
      }
    }
    if constexpr (WIN > 1) {
      uint4 *slot = ring + (it % WIN) * blockDim.x + tid;
      const uint4 old = *slot;
      *slot = make_uint4(C[0], C[1], C[2], C[3]);
      V[0] += C[0] - old.x; V[1] += C[1] - old.y; V[2] += C[2] - old.z; V[3] += C[3] - old.w;
    } else {
#pragma unroll
      for (int j = 0; j < kDP; ++j) V[j] = C[j];
    }
    const int yo = y - R;
    if (yo >= yb) {
      uint32_t key = 0xFFFFFFFFu;
#pragma unroll
      for (int j = 0; j < kDP; ++j) {
        uint32_t A = V[j];
#pragma unroll
        for (int u = 1; u <= R; ++u)
          A += __shfl_up_sync(0xFFFFFFFFu, V[j], u) + __shfl_down_sync(0xFFFFFFFFu, V[j], u);
        const int de = d0 + 2 * j;
        const uint32_t ae = A & 0xFFFFu, ao = A >> 16;
        if (de < dmax) key = min(key, (ae << 10) | (uint32_t)de);
        if (de + 1 < dmax) key = min(key, (ao << 10) | (uint32_t)(de + 1));
        if (a.cost[DIR] != nullptr && out_lane) {
          uint16_t *cp = a.cost[DIR] + ((size_t)yo * w + x) * dmax;
          if (de < dmax) cp[de] = (uint16_t)ae;
          if (de + 1 < dmax) cp[de + 1] = (uint16_t)ao;
        }
      }
      keys[(it & 1) * nwarps * 32 + warp * 32 + lane] = key;
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (warp == 0 && y_first + n_it - 1 - R >= yb) reduce_keys(n_it - 1);
}

template <int WIN, int MM>
__global__ void __launch_bounds__(1024, 1) cost_long_kernel(const LongArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  if (blockIdx.z == 0) cost_long_body<WIN, 0, MM>(a, smem_raw);
  else cost_long_body<WIN, 1, MM>(a, smem_raw);
}

template <int WIN, int MM>
cudaError_t launch_long_t(const LongArgs &a, cudaStream_t s) {
  constexpr int OUTC = 32 - 2 * (WIN / 2);
  const int nwarps = (a.dmax + kDC - 1) / kDC, nd = nwarps * kDC, nt = nwarps * 32;
  const size_t stage_words = 64 * kChunkWords + (size_t)(MM + 1) * (32 + nd - 1) * kChunkWords;
  size_t smem = 4 * (2 * stage_words + 2 * (size_t)nwarps * 32);
  if (WIN > 1) smem += (size_t)WIN * nt * 16;
  cudaError_t e =
      cudaFuncSetAttribute(cost_long_kernel<WIN, MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.w + OUTC - 1) / OUTC, (a.h + a.rows - 1) / a.rows, 2);
  cost_long_kernel<WIN, MM><<<grid, nt, smem, s>>>(a);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_long_win(int win, const LongArgs &a, cudaStream_t s) {
  switch (win) {
    case 1: return launch_long_t<1, MM>(a, s);
    case 3: return launch_long_t<3, MM>(a, s);
    case 5: return launch_long_t<5, MM>(a, s);
    case 7: return launch_long_t<7, MM>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_describe_wide(const bsm_ctx *ctx, const uint32_t *plane, int w, int h, uint32_t *B, uint32_t *Phi,
                                 cudaStream_t s) {
  const WideArgs a{plane, ctx->wide_offs, B, Phi, w, h, ctx->mask_rank, ctx->halo};
  switch (ctx->nw) {
    case 2: return launch_wide_nw<2>(a, s);
    case 4: return launch_wide_nw<4>(a, s);
    case 8: return launch_wide_nw<8>(a, s);
    case 16: return launch_wide_nw<16>(a, s);
    case 32: return launch_wide_nw<32>(a, s);
    case 64: return launch_wide_nw<64>(a, s);
    case 128: return launch_wide_nw<128>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

// Tile-relative pair offsets of the wide describe kernel, for its tile pitch 32 + 2 * halo.
void wide_offsets(const bsm_ctx *ctx, int32_t *out) {
  const int tp = 32 + 2 * ctx->halo;
  for (int i = 0; i < ctx->p.n_bits; ++i) {
    const int8_t *q = ctx->pairs + 4 * i;
    const int op = q[1] * tp + q[0], oq = q[3] * tp + q[2];
    out[i] = (int32_t)(((uint32_t)oq << 16) | ((uint32_t)op & 0xFFFFu));
  }
}

int cost_long_rows(const bsm_ctx *ctx, int w, int h, int dmax) {
  (void)w;
  (void)dmax;
  return ctx->cost_rows > 0 ? ctx->cost_rows : (h >= 256 ? 64 : 16);
}

cudaError_t launch_cost_long(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                             const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *costL,
                             uint16_t *costR, cudaStream_t s) {
  LongArgs a{};
  a.B[0] = BL; a.Phi[0] = PhiL; a.O[0] = BR; a.OPhi[0] = PhiR; a.disp[0] = dL;
  a.B[1] = BR; a.Phi[1] = PhiR; a.O[1] = BL; a.OPhi[1] = PhiL; a.disp[1] = dR;
  a.cost[0] = costL; a.cost[1] = costR;
  a.w = w; a.h = h; a.dmax = dmax; a.nw = ctx->nw;
  a.rows = cost_long_rows(ctx, w, h, dmax);
  if (a.nw % kChunkWords != 0) return cudaErrorInvalidValue;
  return ctx->p.mask_mode == BSM_MASK_BOTH ? launch_long_win<1>(ctx->p.agg_window, a, s)
                                           : launch_long_win<0>(ctx->p.agg_window, a, s);
}

}  // namespace bsm
