// Fused Eq. 8 cost + box aggregation + Eq. 1, two columns per lane (n = 128 or 256).
//
// Same computation as bsm_cost.cu; a different mapping that halves the shared-memory traffic of the
// other view's descriptors and trims the horizontal halo:
//   - lane l of every warp owns columns x0 + 2l and x0 + 2l + 1 (a warp covers 64 columns, 64 - 2r of
//     them outputs); warp k owns disparities dbase + 8k .. dbase + 8k + 7;
//   - the descriptor the second column needs at disparity d is the one the first column needed at
//     d - 1 (left reference) or d + 1 (right reference), so each step loads one new descriptor for two
//     (x, d): 9 loads serve the 16 (x, d) of a thread's row;
//   - the rows are staged with 16-byte cp.async copies into shared memory laid out by pixel parity,
//     so the stride-2 reads of a warp fall on consecutive 32-byte slots (bank-conflict free with the
//     lane-dependent order of the two 16-byte halves);
//   - a CTA of up to 16 warps covers up to 128 disparities; a larger dmax is split into disparity
//     ranges (blockIdx.z), whose minima merge into the disparity buffer with atomicMin on
//     (A << 10 | d) keys; a last elementwise pass keeps the low 10 bits.
// Copies are cp.async groups completed by the issuing threads; there is no spin-wait in this kernel.
#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kDC = 8;
constexpr int kDP = kDC / 2;
constexpr int kMaxWarps = 16;

struct Cost2Args {
  const uint32_t *B[2], *Phi[2], *O[2];
  int32_t *disp[2];
  uint16_t *cost[2];  // optional aggregated cost volume per reference view
  int w, h, dmax, rows, ndr;  // ndr: disparity ranges per (column block, band, view)
};

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}

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
__device__ __forceinline__ uint32_t vmin_u16x2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}
__device__ __forceinline__ uint32_t lop3_xor_and(uint32_t a, uint32_t b, uint32_t m) {
  uint32_t r;
  asm("lop3.b32 %0, %1, %2, %3, 0x28;" : "=r"(r) : "r"(a), "r"(b), "r"(m));
  return r;
}

// Popcount forms of the masked words (results identical): 0 = carry-save tree over all 8 words
// (4 POPC), 1 = one POPC per word, 2 = two 3-word carry-save adders and 2 plain words (6 POPC).
template <int NW, int PM>
__device__ __forceinline__ uint32_t masked_hamming(const uint32_t (&b)[NW], const uint32_t (&o)[NW],
                                                   const uint32_t (&m)[NW]) {
  uint32_t v[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) v[j] = lop3_xor_and(b[j], o[j], m[j]);
  if constexpr (PM == 0 && NW == 8) {
    const uint32_t s1 = lop3_xor3(v[0], v[1], v[2]), c1 = lop3_maj(v[0], v[1], v[2]);
    const uint32_t s2 = lop3_xor3(v[3], v[4], v[5]), c2 = lop3_maj(v[3], v[4], v[5]);
    const uint32_t s3 = lop3_xor3(s1, s2, v[6]), c3 = lop3_maj(s1, s2, v[6]);
    const uint32_t s4 = lop3_xor3(c1, c2, c3), c4 = lop3_maj(c1, c2, c3);
    return (uint32_t)__popc(s3) + (uint32_t)__popc(v[7]) + 2u * (uint32_t)__popc(s4) + 4u * (uint32_t)__popc(c4);
  } else if constexpr (PM == 2 && NW == 8) {
    const uint32_t s1 = lop3_xor3(v[0], v[1], v[2]), c1 = lop3_maj(v[0], v[1], v[2]);
    const uint32_t s2 = lop3_xor3(v[3], v[4], v[5]), c2 = lop3_maj(v[3], v[4], v[5]);
    return (uint32_t)__popc(s1) + (uint32_t)__popc(s2) + (uint32_t)__popc(v[6]) + (uint32_t)__popc(v[7]) +
           2u * ((uint32_t)__popc(c1) + (uint32_t)__popc(c2));
  } else {
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) c += (uint32_t)__popc(v[j]);
    return c;
  }
}

// A descriptor in shared memory; for n = 256 the two 16-byte halves are read in a lane-dependent order.
template <int NW>
__device__ __forceinline__ void load_desc(const uint32_t *p, int q, uint32_t (&v)[NW]) {
  if constexpr (NW == 8) {
    const uint4 a = *reinterpret_cast<const uint4 *>(p + 4 * q);
    const uint4 b = *reinterpret_cast<const uint4 *>(p + 4 * (1 - q));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
    const uint4 a = *reinterpret_cast<const uint4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  }
}

// Shared layout of one stage: reference B and Phi for the 64 columns, and the other view's staged
// columns, each split into an even-pixel and an odd-pixel half.
template <int NW>
struct Stage {
  int ocols;        // staged other-view columns
  int ohalf;        // pixels per parity half of the other row
  int words;        // one stage
  __device__ __host__ explicit Stage(int nd) {
    ocols = 64 + nd - 1;
    ohalf = (ocols + 1) / 2;
    words = 2 * 64 * NW + 2 * ohalf * NW;
  }
  __device__ __forceinline__ static uint32_t *ref(uint32_t *st, int plane, int j) {  // column j of 64
    return st + plane * 64 * NW + ((j & 1) * 32 + (j >> 1)) * NW;
  }
  __device__ __forceinline__ uint32_t *oth(uint32_t *st, int p) const {  // staged other-view pixel p
    return st + 2 * 64 * NW + ((p & 1) * ohalf + (p >> 1)) * NW;
  }
};

template <int NW>
size_t cost2_smem_bytes(int nd, int win, int nthreads) {
  const Stage<NW> S(nd);
  size_t b = 2 * (size_t)S.words * 4;               // two stages
  b += 2 * (size_t)(nthreads / 32) * 64 * 4;        // keys, double-buffered
  if (win > 1) b += (size_t)win * nthreads * 32;    // vertical ring: 8 packed words per thread per row
  return b;
}

template <int NW, int WIN, int DIR, int PM, bool SPLIT, bool PK>
__device__ __forceinline__ void cost2_body(const Cost2Args &a, uint8_t *smem_raw) {
  constexpr int R = WIN / 2;
  constexpr int OUTC = 64 - 2 * R;
  constexpr int NBITS = 32 * NW;
  constexpr int CH = NW / 4;  // 16-byte chunks per descriptor
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nd = nwarps * kDC;
  const Stage<NW> S(nd);
  uint32_t *stages = reinterpret_cast<uint32_t *>(smem_raw);
  uint32_t *keys = stages + 2 * S.words;  // [2][nwarps][64]
  uint4 *ring = reinterpret_cast<uint4 *>(keys + 2 * nwarps * 64);

  const int dr = (int)blockIdx.x % a.ndr;  // sibling disparity ranges run side by side and share L2
  const uint32_t *__restrict__ Bref = a.B[DIR];
  const uint32_t *__restrict__ Phiref = a.Phi[DIR];
  const uint32_t *__restrict__ Both = a.O[DIR];
  int32_t *__restrict__ disp = a.disp[DIR];
  const int w = a.w, h = a.h, dmax = a.dmax;
  const int x0 = (int)(blockIdx.x / a.ndr) * OUTC - R;  // column of lane 0's first column
  const int xa = x0 + 2 * lane, xb = xa + 1;       // this lane's two columns
  const int yb = (int)blockIdx.y * a.rows, ye = min(h, yb + a.rows);
  const int dbase = dr * nd;
  const int d0 = dbase + warp * kDC;
  const int ox0 = DIR == 0 ? x0 - (dbase + nd - 1) : x0 + dbase;  // first staged other-view column
  const bool ina = xa >= 0 && xa < w, inb = xb >= 0 && xb < w;
  const int q = NW == 8 ? (lane >> 2) & 1 : 0;
  const int y_first = yb - R, n_it = (ye + R) - y_first;
  const bool fast = DIR == 0 ? (x0 >= d0 + kDC - 1 && x0 + 63 < w) : (x0 >= 0 && x0 + 63 + d0 + kDC - 1 < w);

  auto issue = [&](int y, int s) {  // all threads: 16-byte copies of row y into stage s
    if (y < 0 || y >= h) return;
    uint32_t *st = stages + s * S.words;
    const int nref = 2 * 64 * CH, noth = S.ocols * CH;
    for (int i = tid; i < nref + noth; i += blockDim.x) {
      if (i < nref) {
        const int plane = i / (64 * CH), r = i - plane * 64 * CH, j = r / CH, c = r - j * CH;
        const int gx = x0 + j;
        if (gx >= 0 && gx < w) {
          const uint32_t *src = (plane ? Phiref : Bref) + ((size_t)y * w + gx) * NW + 4 * c;
          cp_async16(Stage<NW>::ref(st, plane, j) + 4 * c, src);
        }
      } else {
        const int r = i - nref, p = r / CH, c = r - p * CH;
        const int gx = ox0 + p;
        if (gx >= 0 && gx < w) cp_async16(S.oth(st, p) + 4 * c, Both + ((size_t)y * w + gx) * NW + 4 * c);
      }
    }
  };
  auto reduce_keys = [&](int it) {  // warp 0: minimum over the warps for the 64 columns of a row
    const int yo = y_first + it - R;
    const uint32_t *kb = keys + (it & 1) * nwarps * 64;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int j = lane + 32 * half;
      uint32_t best = kb[j];
      for (int k = 1; k < nwarps; ++k) best = min(best, kb[k * 64 + j]);
      const int x = x0 + j;
      if (j >= R && j < 64 - R && x >= 0 && x < w) {
        if constexpr (SPLIT) atomicMin(reinterpret_cast<unsigned *>(disp) + (size_t)yo * w + x, best);
        else disp[(size_t)yo * w + x] = (int32_t)(best & 1023u);
      }
    }
  };

  if constexpr (WIN > 1) {
    for (int s = 0; s < WIN; ++s) {
      ring[(s * blockDim.x + tid) * 2] = make_uint4(0, 0, 0, 0);
      ring[(s * blockDim.x + tid) * 2 + 1] = make_uint4(0, 0, 0, 0);
    }
  }
  issue(y_first, 0);
  asm volatile("cp.async.commit_group;" ::: "memory");

  uint32_t Va[kDP] = {0, 0, 0, 0}, Vb[kDP] = {0, 0, 0, 0};
  for (int it = 0; it < n_it; ++it) {
    const int y = y_first + it, s = it & 1;
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();  // row y is in stage s; every thread is done with iteration it - 1
    if (it + 1 < n_it) issue(y + 1, s ^ 1);
    asm volatile("cp.async.commit_group;" ::: "memory");
    if (warp == 0 && it >= 1 && y - 1 - R >= yb) reduce_keys(it - 1);

    uint32_t *st = stages + s * S.words;
    uint32_t Ca[kDP] = {0, 0, 0, 0}, Cb[kDP] = {0, 0, 0, 0};
    if (y >= 0 && y < h && d0 < dmax) {
      uint32_t ba[NW], ma[NW], bb[NW], mb[NW];
      load_desc<NW>(Stage<NW>::ref(st, 0, 2 * lane), q, ba);
      load_desc<NW>(Stage<NW>::ref(st, 1, 2 * lane), q, ma);
      load_desc<NW>(Stage<NW>::ref(st, 0, 2 * lane + 1), q, bb);
      load_desc<NW>(Stage<NW>::ref(st, 1, 2 * lane + 1), q, mb);
      // staged pixel of the first column's match at step dd: p(dd); the second column's is p(dd) + 1
      const int pbase = DIR == 0 ? 2 * lane + nd - 1 - warp * kDC : 2 * lane + warp * kDC;
      uint32_t o_keep[NW];
      load_desc<NW>(S.oth(st, DIR == 0 ? pbase + 1 : pbase), q, o_keep);
#pragma unroll
      for (int dd = 0; dd < kDC; ++dd) {
        uint32_t o_new[NW];
        uint32_t ca, cb;
        if constexpr (DIR == 0) {
          load_desc<NW>(S.oth(st, pbase - dd), q, o_new);  // first column at d; second reuses d - 1's
          ca = masked_hamming<NW, PM>(ba, o_new, ma);
          cb = masked_hamming<NW, PM>(bb, o_keep, mb);
        } else {
          load_desc<NW>(S.oth(st, pbase + dd + 1), q, o_new);  // second column at d; first reuses it
          ca = masked_hamming<NW, PM>(ba, o_keep, ma);
          cb = masked_hamming<NW, PM>(bb, o_new, mb);
        }
#pragma unroll
        for (int j = 0; j < NW; ++j) o_keep[j] = o_new[j];
        if (!fast) {
          const int d = d0 + dd;
          const bool ma_in = DIR == 0 ? xa - d >= 0 : xa + d < w;
          const bool mb_in = DIR == 0 ? xb - d >= 0 : xb + d < w;
          ca = ina ? (ma_in ? ca : (uint32_t)NBITS) : 0u;
          cb = inb ? (mb_in ? cb : (uint32_t)NBITS) : 0u;
        }
        Ca[dd >> 1] += ca << (16 * (dd & 1));
        Cb[dd >> 1] += cb << (16 * (dd & 1));
      }
    }

    if constexpr (WIN > 1) {
      uint4 *slot = ring + ((it % WIN) * blockDim.x + tid) * 2;
      const uint4 oa = slot[0], ob = slot[1];
      slot[0] = make_uint4(Ca[0], Ca[1], Ca[2], Ca[3]);
      slot[1] = make_uint4(Cb[0], Cb[1], Cb[2], Cb[3]);
      Va[0] += Ca[0] - oa.x; Va[1] += Ca[1] - oa.y; Va[2] += Ca[2] - oa.z; Va[3] += Ca[3] - oa.w;
      Vb[0] += Cb[0] - ob.x; Vb[1] += Cb[1] - ob.y; Vb[2] += Cb[2] - ob.z; Vb[3] += Cb[3] - ob.w;
    } else {
#pragma unroll
      for (int j = 0; j < kDP; ++j) {
        Va[j] = Ca[j];
        Vb[j] = Cb[j];
      }
    }

    const int yo = y - R;
    if (yo >= yb) {
      uint32_t ka = 0xFFFFFFFFu, kb = 0xFFFFFFFFu;
      uint32_t pa = 0xFFFFFFFFu, pb = 0xFFFFFFFFu;  // packed 16-bit keys (A << 3 | dd) when PK
#pragma unroll
      for (int j = 0; j < kDP; ++j) {
        // Column 2l sums offsets -R..R of 2l, column 2l+1 those of 2l+1. Lane l-t holds columns
        // 2l-2t and 2l-2t+1, lane l+t holds 2l+2t and 2l+2t+1; each joins a sum if its offset
        // from that output column is at most R.
        uint32_t Aa = Va[j] + (R >= 1 ? Vb[j] : 0u), Ab = Vb[j] + (R >= 1 ? Va[j] : 0u);
#pragma unroll
        for (int t = 1; t <= (R + 1) / 2; ++t) {
          const uint32_t ua = __shfl_up_sync(0xFFFFFFFFu, Va[j], t), ub = __shfl_up_sync(0xFFFFFFFFu, Vb[j], t);
          const uint32_t da = __shfl_down_sync(0xFFFFFFFFu, Va[j], t), db = __shfl_down_sync(0xFFFFFFFFu, Vb[j], t);
          if (2 * t <= R) {  // offsets -2t, +2t of column 2l and of column 2l+1
            Aa += ua + da;
            Ab += ub + db;
          }
          if (2 * t - 1 <= R) {  // offset -2t+1 of column 2l, +2t-1 of column 2l+1
            Aa += ub;
            Ab += da;
          }
          if (2 * t + 1 <= R) {  // offset +2t+1 of column 2l, -2t-1 of column 2l+1
            Aa += db;
            Ab += ua;
          }
        }
        const int de = d0 + 2 * j;
        const uint32_t a_lo = Aa & 0xFFFFu, a_hi = Aa >> 16, b_lo = Ab & 0xFFFFu, b_hi = Ab >> 16;
        if constexpr (PK) {
          // A < 2^13, so A << 3 | dd fits a 16-bit half; one multiply-add forms both halves' keys
          const uint32_t dd2 = (uint32_t)(2 * j) | ((uint32_t)(2 * j + 1) << 16);
          uint32_t ea = Aa * 8u + dd2, eb = Ab * 8u + dd2;
          if (de >= dmax) { ea |= 0xFFFFu; eb |= 0xFFFFu; }
          if (de + 1 >= dmax) { ea |= 0xFFFF0000u; eb |= 0xFFFF0000u; }
          pa = vmin_u16x2(pa, ea);
          pb = vmin_u16x2(pb, eb);
        } else {
          if (de < dmax) {
            ka = min(ka, (a_lo << 10) | (uint32_t)de);
            kb = min(kb, (b_lo << 10) | (uint32_t)de);
          }
          if (de + 1 < dmax) {
            ka = min(ka, (a_hi << 10) | (uint32_t)(de + 1));
            kb = min(kb, (b_hi << 10) | (uint32_t)(de + 1));
          }
        }
        if (a.cost[DIR] != nullptr) {
          if (2 * lane >= R && 2 * lane < 64 - R && ina) {
            uint16_t *cp = a.cost[DIR] + ((size_t)yo * w + xa) * dmax;
            if (de < dmax) cp[de] = (uint16_t)a_lo;
            if (de + 1 < dmax) cp[de + 1] = (uint16_t)a_hi;
          }
          if (2 * lane + 1 >= R && 2 * lane + 1 < 64 - R && inb) {
            uint16_t *cp = a.cost[DIR] + ((size_t)yo * w + xb) * dmax;
            if (de < dmax) cp[de] = (uint16_t)b_lo;
            if (de + 1 < dmax) cp[de + 1] = (uint16_t)b_hi;
          }
        }
      }
      if constexpr (PK) {
        const uint32_t a16 = min(pa & 0xFFFFu, pa >> 16), b16 = min(pb & 0xFFFFu, pb >> 16);
        ka = a16 == 0xFFFFu ? 0xFFFFFFFFu : ((a16 >> 3) << 10) | (uint32_t)(d0 + (a16 & 7u));
        kb = b16 == 0xFFFFu ? 0xFFFFFFFFu : ((b16 >> 3) << 10) | (uint32_t)(d0 + (b16 & 7u));
      }
      keys[(it & 1) * nwarps * 64 + warp * 64 + 2 * lane] = ka;
      keys[(it & 1) * nwarps * 64 + warp * 64 + 2 * lane + 1] = kb;
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  if (warp == 0 && y_first + n_it - 1 - R >= yb) reduce_keys(n_it - 1);
}

template <int NW, int WIN, int PM, bool SPLIT, bool PK>
__global__ void __launch_bounds__(512, 1) cost2_kernel(const Cost2Args a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  if (blockIdx.z == 0) cost2_body<NW, WIN, 0, PM, SPLIT, PK>(a, smem_raw);
  else cost2_body<NW, WIN, 1, PM, SPLIT, PK>(a, smem_raw);
}

__global__ void __launch_bounds__(256) keep_disparity_bits(int32_t *a, int32_t *b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    a[i] &= 1023;
    b[i] &= 1023;
  }
}

template <int NW, int WIN, int PM, bool SPLIT>
cudaError_t launch_t(const Cost2Args &a, int nwarps, cudaStream_t s) {
  constexpr int OUTC = 64 - 2 * (WIN / 2);
  constexpr bool PK = 32 * NW * WIN * WIN < 8192;  // aggregated costs fit 13 bits: packed argmin
  const size_t smem = cost2_smem_bytes<NW>(nwarps * kDC, WIN, nwarps * 32);
  cudaError_t e = cudaFuncSetAttribute(cost2_kernel<NW, WIN, PM, SPLIT, PK>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(((a.w + OUTC - 1) / OUTC) * a.ndr, (a.h + a.rows - 1) / a.rows, 2);
  cost2_kernel<NW, WIN, PM, SPLIT, PK><<<grid, nwarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NW, int PM, bool SPLIT>
cudaError_t launch_win(int win, const Cost2Args &a, int nwarps, cudaStream_t s) {
  switch (win) {
    case 1: return launch_t<NW, 1, PM, SPLIT>(a, nwarps, s);
    case 3: return launch_t<NW, 3, PM, SPLIT>(a, nwarps, s);
    case 5: return launch_t<NW, 5, PM, SPLIT>(a, nwarps, s);
    case 7: return launch_t<NW, 7, PM, SPLIT>(a, nwarps, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int NW, int PM>
cudaError_t launch_split(bool split, int win, const Cost2Args &a, int nwarps, cudaStream_t s) {
  return split ? launch_win<NW, PM, true>(win, a, nwarps, s) : launch_win<NW, PM, false>(win, a, nwarps, s);
}

int pick_rows2(int w, int h, int win, int ctas_z) {
  const int outc = 64 - 2 * (win / 2);
  const long cols = (w + outc - 1) / outc;
  const long target = 2L * 152;
  long rows = 128;
  while (rows > 8 && cols * ((h + rows - 1) / rows) * ctas_z < target) rows /= 2;
  return (int)rows;
}

}  // namespace

bool cost2_supported(const bsm_ctx *ctx) { return ctx->nw == 4 || ctx->nw == 8; }

int cost2_rows(const bsm_ctx *ctx, int w, int h, int dmax) {
  const int need = (dmax + kDC - 1) / kDC;
  const int nwarps = min(kMaxWarps, need);
  const int ndr = (need + nwarps - 1) / nwarps;
  return ctx->cost_rows > 0 ? ctx->cost_rows : pick_rows2(w, h, ctx->p.agg_window, 2 * ndr);
}

cudaError_t launch_cost2(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                         const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *costL,
                         uint16_t *costR, cudaStream_t s) {
  Cost2Args a{};
  a.B[0] = BL; a.Phi[0] = PhiL; a.O[0] = BR; a.disp[0] = dL;
  a.B[1] = BR; a.Phi[1] = PhiR; a.O[1] = BL; a.disp[1] = dR;
  a.cost[0] = costL; a.cost[1] = costR;
  a.w = w; a.h = h; a.dmax = dmax;
  const int need = (dmax + kDC - 1) / kDC;
  const int nwarps = min(kMaxWarps, need);
  a.ndr = (need + nwarps - 1) / nwarps;
  a.rows = cost2_rows(ctx, w, h, dmax);
  const bool split = a.ndr > 1;
  cudaError_t e = cudaSuccess;
  if (split) {
    e = cudaMemsetAsync(dL, 0xFF, (size_t)w * h * 4, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(dR, 0xFF, (size_t)w * h * 4, s);
    if (e != cudaSuccess) return e;
  }
  const int win = ctx->p.agg_window;
  if (ctx->nw == 8) {
    switch (ctx->cost_plain_popc) {
      case 1: e = launch_split<8, 1>(split, win, a, nwarps, s); break;
      case 2: e = launch_split<8, 2>(split, win, a, nwarps, s); break;
      default: e = launch_split<8, 0>(split, win, a, nwarps, s); break;
    }
  } else if (ctx->nw == 4) {
    e = launch_split<4, 1>(split, win, a, nwarps, s);
  } else {
    return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess || !split) return e;
  keep_disparity_bits<<<152 * 4, 256, 0, s>>>(dL, dR, (size_t)w * h);
  return cudaGetLastError();
}

}  // namespace bsm
