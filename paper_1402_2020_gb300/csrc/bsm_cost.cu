// Fused Eq. 8 cost + square-window box aggregation + Eq. 1 winner-take-all, for both views.
//
// blockIdx.z selects the reference view: 0 = left (match x - d), 1 = right (match x + d).
// A CTA owns 32 - 2r consecutive output columns (r = WIN / 2) and a band of rows; lane l of every
// warp owns column x0 + l (the outer r lanes on each side only feed the horizontal window), and warp
// k owns disparities [8k, 8k + 8). The CTA walks down its band one row at a time:
//   - the reference row's B and Phi for the 32 columns and the other view's B row for the
//     32 + dmax - 1 columns any of them can match are contiguous in HBM; one thread stages them in
//     shared memory with bulk asynchronous copies (TMA, cp.async.bulk) completing on an mbarrier,
//     double-buffered so that row y + 1 is in flight while row y is computed; every wait is bounded
//     and a wait that gives up latches BSM_ERR_TIMEOUT in the status word;
//   - each thread computes C(x, y, d) = popc((B_ref ^ B_other) & Phi_ref) for its 8 disparities (a
//     match outside the image costs n), two 16-bit costs per 32-bit register. For n = 256 the eight
//     masked words go through a carry-save adder tree (Harley-Seal), so 4 POPC replace 8;
//   - vertical box sums: V += C_new - C_old, the last WIN rows of C kept per thread in a shared ring;
//   - the horizontal box sum takes V from the neighbouring lanes with warp shuffles;
//   - each thread reduces its 8 aggregated costs to a key (A << 10 | d); warp 0 takes the minimum over
//     the warps one row later, which gives the smallest d with the minimum cost. The cost volume never
//     reaches HBM unless the caller asks for it.
// For n = 256 a lane reads the two 16-byte halves of a descriptor in an order that depends on bit 2
// of its lane index (for the reference and the other view alike), which keeps every 128-bit shared
// load conflict free; the popcount sum does not depend on word order.
#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kDC = 8;   // disparities per thread
constexpr int kDP = kDC / 2;
constexpr int kPad = 8;  // guard columns on both sides of the staged other-view row
constexpr long long kWaitCycles = 1LL << 31;  // about one second at the GB300 clock

struct CostArgs {
  const uint32_t *B[2];    // reference descriptors per direction
  const uint32_t *Phi[2];  // reference masks per direction
  const uint32_t *O[2];    // other view's descriptors per direction
  int32_t *disp[2];
  uint16_t *cost[2];       // optional aggregated cost volume per reference view
  uint32_t *status;
  int w, h, dmax, rows;
  int withhold;            // test hook: skip the mbarrier arrivals so the bounded waits run out
};

// ---------------------------------------------------------------- TMA bulk copies and mbarriers

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: false after about a second without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(bar))
               : "memory");
}

// ---------------------------------------------------------------- per-pixel masked Hamming cost

template <int NW>
__device__ __forceinline__ void load_desc(const uint32_t *p, int q, uint32_t (&v)[NW]) {
  if constexpr (NW == 8) {
    const uint4 a = *reinterpret_cast<const uint4 *>(p + 4 * q);
    const uint4 b = *reinterpret_cast<const uint4 *>(p + 4 * (1 - q));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else if constexpr (NW == 4) {
    const uint4 a = *reinterpret_cast<const uint4 *>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  } else if constexpr (NW == 2) {
    const uint2 a = *reinterpret_cast<const uint2 *>(p);
    v[0] = a.x; v[1] = a.y;
  } else {
#pragma unroll
    for (int j = 0; j < NW; ++j) v[j] = p[j];
  }
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
// (a ^ b) & m
__device__ __forceinline__ uint32_t lop3_xor_and(uint32_t a, uint32_t b, uint32_t m) {
  uint32_t r;
  asm("lop3.b32 %0, %1, %2, %3, 0x28;" : "=r"(r) : "r"(a), "r"(b), "r"(m));
  return r;
}

// popcount over NW words of (b ^ o) & m (Eq. 8).
template <int NW, bool CSA>
__device__ __forceinline__ uint32_t masked_hamming(const uint32_t (&b)[NW], const uint32_t (&o)[NW],
                                                   const uint32_t (&m)[NW]) {
  uint32_t v[NW];
#pragma unroll
  for (int j = 0; j < NW; ++j) v[j] = lop3_xor_and(b[j], o[j], m[j]);
  if constexpr (CSA && NW == 8) {
    // Carry-save adders: every bit position's count of ones across the 8 words, in binary.
    const uint32_t s1 = lop3_xor3(v[0], v[1], v[2]), c1 = lop3_maj(v[0], v[1], v[2]);
    const uint32_t s2 = lop3_xor3(v[3], v[4], v[5]), c2 = lop3_maj(v[3], v[4], v[5]);
    const uint32_t s3 = lop3_xor3(s1, s2, v[6]), c3 = lop3_maj(s1, s2, v[6]);
    const uint32_t s4 = lop3_xor3(c1, c2, c3), c4 = lop3_maj(c1, c2, c3);
    return (uint32_t)__popc(s3) + (uint32_t)__popc(v[7]) + 2u * (uint32_t)__popc(s4) + 4u * (uint32_t)__popc(c4);
  } else {
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) c += (uint32_t)__popc(v[j]);
    return c;
  }
}

// ---------------------------------------------------------------- kernel

template <int NW>
struct Layout {
  static constexpr bool kTma = NW >= 4;  // 16-byte granules: every row segment is a legal bulk copy
  int ocols;                             // staged other-view columns including guards
  int stage_words;                       // one stage: ref B, ref Phi, other row
  __device__ __host__ explicit Layout(int nd) {
    ocols = 32 + nd - 1 + 2 * kPad;
    stage_words = (2 * 32 * NW + ocols * NW + 3) & ~3;  // 16-byte multiple: every stage stays aligned
  }
};

template <int NW>
size_t cost_smem_bytes(int nd, int win, int nthreads) {
  const Layout<NW> L(nd);
  size_t b = 2 * sizeof(uint64_t);                 // mbarriers
  b += 2 * (size_t)L.stage_words * 4;              // two stages
  b += 2 * 32 * 32 * 4;                            // keys, double-buffered
  if (win > 1) b += (size_t)win * nthreads * 16;   // vertical ring (uint4 per thread per row)
  return b;
}

// One band of one reference view: output rows [yb, ye) of the columns whose lane is an output lane
// (lane 0 sits at column x0), for the disparities [dbase, dbase + 8 * warps).
struct CostTask {
  const uint32_t *Bref, *Phiref, *Both;
  int32_t *disp;
  uint16_t *cost;  // optional cost volume (left reference only), or nullptr
  int w, h, dmax;
  int x0, yb, ye, dbase;
};

// Runs one task. `g` counts the rows this CTA has staged so far (it selects the stage buffer and the
// mbarrier phase, and carries over between the tasks of a persistent CTA). Returns false, in every
// thread, if a bounded wait gave up.
template <int NW, int WIN, int DIR, bool CSA, bool ATOMIC>
__device__ __forceinline__ bool cost_task(const CostTask &t, uint8_t *smem_raw, uint32_t &g, uint32_t *status,
                                          int withhold = 0) {
  constexpr int R = WIN / 2;
  constexpr int NBITS = 32 * NW;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  const int nd = nwarps * kDC;
  const Layout<NW> L(nd);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
  uint32_t *stages = reinterpret_cast<uint32_t *>(smem_raw + 16);
  uint32_t *keys = stages + 2 * L.stage_words;     // [2][32][32]
  uint4 *ring = reinterpret_cast<uint4 *>(keys + 2 * 32 * 32);

  const uint32_t *__restrict__ Bref = t.Bref;
  const uint32_t *__restrict__ Phiref = t.Phiref;
  const uint32_t *__restrict__ Both = t.Both;
  const int w = t.w, h = t.h, dmax = t.dmax;
  const int x0 = t.x0, x = x0 + lane;
  const int yb = t.yb, ye = t.ye;
  const int d0 = t.dbase + warp * kDC;               // this warp's first disparity
  // first staged other-view column (before guards) and the count of staged columns
  const int ox0 = DIR == 0 ? x0 - (t.dbase + nd - 1) : x0 + t.dbase;
  const int nocols = 32 + nd - 1;
  const bool col_in = x >= 0 && x < w;
  const bool out_lane = lane >= R && lane < 32 - R && col_in;
  const int q = NW == 8 ? (lane >> 2) & 1 : 0;
  const int y_first = yb - R, n_it = (ye + R) - y_first;
  // warp-uniform: every lane's x is in the image and every one of the warp's d matches in the image
  const bool fast_cols =
      DIR == 0 ? (x0 >= d0 + kDC - 1 && x0 + 31 < w) : (x0 >= 0 && x0 + 31 + d0 + kDC - 1 < w);

  auto issue = [&](int y, int s) {  // one thread: stage row y into buffer s
    uint32_t *st = stages + s * L.stage_words;
    if (withhold) return;  // test hook: no arrival, so the phase never completes
    if (y >= 0 && y < h) {
      const int c0 = max(x0, 0), c1 = min(x0 + 32, w);
      const int o0 = max(ox0, 0), o1 = min(ox0 + nocols, w);
      uint32_t bytes = 0;
      if (c1 > c0) bytes += 2u * (uint32_t)((c1 - c0) * NW * 4);
      if (o1 > o0) bytes += (uint32_t)((o1 - o0) * NW * 4);
      mbar_arrive_expect_tx(&full[s], bytes);
      if (c1 > c0) {
        const uint32_t nb = (uint32_t)((c1 - c0) * NW * 4);
        bulk_g2s(st + (c0 - x0) * NW, Bref + ((size_t)y * w + c0) * NW, nb, &full[s]);
        bulk_g2s(st + 32 * NW + (c0 - x0) * NW, Phiref + ((size_t)y * w + c0) * NW, nb, &full[s]);
      }
      if (o1 > o0)
        bulk_g2s(st + 64 * NW + (kPad + o0 - ox0) * NW, Both + ((size_t)y * w + o0) * NW,
                 (uint32_t)((o1 - o0) * NW * 4), &full[s]);
    } else {
      mbar_arrive_expect_tx(&full[s], 0);
    }
  };
  auto load_plain = [&](int y, int s) {  // all threads: stage row y into buffer s with plain loads
    uint32_t *st = stages + s * L.stage_words;
    if (y < 0 || y >= h) return;
    for (int i = tid; i < 64 * NW; i += blockDim.x) {
      const int half = i / (32 * NW), j = i - half * 32 * NW;
      const int gx = x0 + j / NW;
      const uint32_t *src = half ? Phiref : Bref;
      if (gx >= 0 && gx < w) st[i] = __ldg(src + (size_t)y * w * NW + (ptrdiff_t)x0 * NW + j);
    }
    for (int i = tid; i < nocols * NW; i += blockDim.x) {
      const int gx = ox0 + i / NW;
      if (gx >= 0 && gx < w)
        st[64 * NW + kPad * NW + i] = __ldg(Both + (size_t)y * w * NW + (ptrdiff_t)ox0 * NW + i);
    }
  };
  auto reduce_keys = [&](int it) {  // warp 0: minimum key over the warps -> the row's result
    const int yo = y_first + it - R;
    const uint32_t *kb = keys + (it & 1) * 1024;
    uint32_t best = kb[lane];
    for (int k = 1; k < nwarps; ++k) best = min(best, kb[k * 32 + lane]);
    if (out_lane) {
      if constexpr (ATOMIC) atomicMin(reinterpret_cast<unsigned *>(t.disp) + (size_t)yo * w + x, best);
      else t.disp[(size_t)yo * w + x] = (int32_t)(best & 1023u);
    }
  };

  if constexpr (WIN > 1) {
    for (int s = 0; s < WIN; ++s) ring[s * blockDim.x + tid] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();  // the previous task is done with every buffer
  if constexpr (Layout<NW>::kTma) {
    if (tid == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(y_first, g & 1);
    }
  } else {
    load_plain(y_first, g & 1);
  }

  uint32_t V[kDP] = {0, 0, 0, 0};
  for (int it = 0; it < n_it; ++it) {
    const int y = y_first + it;
    const uint32_t G = g + (uint32_t)it;
    const int s = (int)(G & 1u);
    bool ok = true;
    if constexpr (Layout<NW>::kTma) ok = mbar_wait(&full[s], (G >> 1) & 1u);
    if (!__syncthreads_and(ok)) {
      if (tid == 0) {
        atomicCAS(status, 0u, (uint32_t)BSM_ERR_TIMEOUT);
        if (Layout<NW>::kTma) mbar_wait(&full[s], (G >> 1) & 1u);  // let the late copy land
      }
      return false;
    }
    // Every thread finished iteration it - 1: its buffer and its keys may be reused.
    if (it + 1 < n_it) {
      if constexpr (Layout<NW>::kTma) {
        if (tid == 0) {
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          issue(y + 1, s ^ 1);
        }
      } else {
        load_plain(y + 1, s ^ 1);
      }
    }
    if (warp == 0 && it >= 1 && y - 1 - R >= yb) reduce_keys(it - 1);

    const uint32_t *st = stages + s * L.stage_words;
    uint32_t C[kDP] = {0, 0, 0, 0};
    const bool row_in = y >= 0 && y < h;
    if (row_in && (col_in || !fast_cols)) {
      uint32_t b[NW], m[NW];
      load_desc<NW>(st + lane * NW, q, b);
      load_desc<NW>(st + 32 * NW + lane * NW, q, m);
      const uint32_t *ob =
          st + 64 * NW + (kPad + (DIR == 0 ? lane + nd - 1 - warp * kDC : lane + warp * kDC)) * NW;
      if (fast_cols) {
#pragma unroll
        for (int dd = 0; dd < kDC; ++dd) {
          uint32_t o[NW];
          load_desc<NW>(ob + (DIR == 0 ? -dd : dd) * NW, q, o);
          const uint32_t c = masked_hamming<NW, CSA>(b, o, m);
          C[dd >> 1] += c << (16 * (dd & 1));
        }
      } else {
#pragma unroll
        for (int dd = 0; dd < kDC; ++dd) {
          uint32_t o[NW];
          load_desc<NW>(ob + (DIR == 0 ? -dd : dd) * NW, q, o);
          uint32_t c = masked_hamming<NW, CSA>(b, o, m);
          const int d = d0 + dd;
          const bool match_in = DIR == 0 ? x - d >= 0 : x + d < w;
          c = col_in ? (match_in ? c : (uint32_t)NBITS) : 0u;
          C[dd >> 1] += c << (16 * (dd & 1));
        }
      }
    }

    // vertical box sum over the last WIN rows
    if constexpr (WIN > 1) {
      uint4 *slot = ring + (it % WIN) * blockDim.x + tid;
      const uint4 old = *slot;
      *slot = make_uint4(C[0], C[1], C[2], C[3]);
      V[0] += C[0] - old.x;
      V[1] += C[1] - old.y;
      V[2] += C[2] - old.z;
      V[3] += C[3] - old.w;
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
        if constexpr (R == 2) {
          const uint32_t s1 = V[j] + __shfl_down_sync(0xFFFFFFFFu, V[j], 1);  // V(x) + V(x+1)
          A = __shfl_up_sync(0xFFFFFFFFu, s1, 2) + s1 + __shfl_down_sync(0xFFFFFFFFu, V[j], 2);
        } else {
#pragma unroll
          for (int u = 1; u <= R; ++u)
            A += __shfl_up_sync(0xFFFFFFFFu, V[j], u) + __shfl_down_sync(0xFFFFFFFFu, V[j], u);
        }
        const int de = d0 + 2 * j;
        const uint32_t ae = A & 0xFFFFu, ao = A >> 16;
        if (de < dmax) key = min(key, (ae << 10) | (uint32_t)de);
        if (de + 1 < dmax) key = min(key, (ao << 10) | (uint32_t)(de + 1));
        if (t.cost != nullptr && out_lane) {
          uint16_t *cp = t.cost + ((size_t)yo * w + x) * dmax;
          if (de < dmax) cp[de] = (uint16_t)ae;
          if (de + 1 < dmax) cp[de + 1] = (uint16_t)ao;
        }
      }
      keys[(it & 1) * 1024 + warp * 32 + lane] = key;
    }
  }
  __syncthreads();
  if (warp == 0 && y_first + n_it - 1 - R >= yb) reduce_keys(n_it - 1);
  g += (uint32_t)n_it;
  return true;
}

__device__ __forceinline__ void init_barriers(uint8_t *smem_raw) {
  if (threadIdx.x == 0) {
    uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw);
    mbar_init(&full[0], 1);
    mbar_init(&full[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
}

// One CTA per (column block, row band, reference view); its warps cover all of [0, dmax).
template <int NW, int WIN, bool CSA>
__global__ void __launch_bounds__(1024, 1) cost_wta_kernel(const CostArgs a) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  constexpr int OUTC = 32 - 2 * (WIN / 2);
  init_barriers(smem_raw);
  const int dir = blockIdx.z;
  CostTask t;
  t.Bref = dir == 0 ? a.B[0] : a.B[1];
  t.Phiref = dir == 0 ? a.Phi[0] : a.Phi[1];
  t.Both = dir == 0 ? a.O[0] : a.O[1];
  t.disp = dir == 0 ? a.disp[0] : a.disp[1];
  t.cost = dir == 0 ? a.cost[0] : a.cost[1];
  t.w = a.w; t.h = a.h; t.dmax = a.dmax;
  t.x0 = blockIdx.x * OUTC - WIN / 2;
  t.yb = blockIdx.y * a.rows;
  t.ye = min(a.h, t.yb + a.rows);
  t.dbase = 0;
  uint32_t g = 0;
  if (dir == 0) cost_task<NW, WIN, 0, CSA, false>(t, smem_raw, g, a.status, a.withhold);
  else cost_task<NW, WIN, 1, CSA, false>(t, smem_raw, g, a.status, a.withhold);
}

// Persistent batch kernel: 8 warps (64 disparities) per CTA; every CTA takes tasks
// (pair, reference view, row band, column block, disparity range) from the batch's ticket counter and
// merges its partial minimum into the pair's disparity buffers with atomicMin on (A << 10 | d) keys.
template <int NW, int WIN, bool CSA>
__global__ void __launch_bounds__(256, 2) cost_batch_kernel(BatchHeader *hdr, const BatchPair *pairs,
                                                             uint32_t *status) {
  extern __shared__ __align__(16) uint8_t smem_raw[];
  constexpr int OUTC = 32 - 2 * (WIN / 2);
  __shared__ int s_ticket;
  init_barriers(smem_raw);
  const int total = hdr->total[2], count = hdr->count, band = hdr->band_rows;
  uint32_t g = 0;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&hdr->counters[2], 1u);
    __syncthreads();
    const int tk = s_ticket;
    if (tk >= total) break;
    int lo = 0, hi = count - 1;  // last pair whose first ticket <= tk
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pairs[mid].cost_base <= tk) lo = mid;
      else hi = mid - 1;
    }
    const BatchPair &p = pairs[lo];
    int r = tk - p.cost_base;
    const int dr = r % p.cost_dr; r /= p.cost_dr;
    const int cb = r % p.cost_cb; r /= p.cost_cb;
    const int bd = r % p.cost_bands; r /= p.cost_bands;
    const int dir = r;
    CostTask t;
    t.Bref = p.B[dir]; t.Phiref = p.Phi[dir]; t.Both = p.B[1 - dir];
    t.disp = p.disp[dir]; t.cost = nullptr;
    t.w = p.w; t.h = p.h; t.dmax = p.dmax;
    t.x0 = cb * OUTC - WIN / 2;
    t.yb = bd * band;
    t.ye = min(p.h, t.yb + band);
    t.dbase = dr * 8 * (int)(blockDim.x >> 5);
    const bool ok = dir == 0 ? cost_task<NW, WIN, 0, CSA, true>(t, smem_raw, g, status)
                             : cost_task<NW, WIN, 1, CSA, true>(t, smem_raw, g, status);
    if (!ok) return;
  }
}

template <int NW, int WIN, bool CSA>
cudaError_t launch_t(const CostArgs &a, cudaStream_t s) {
  constexpr int OUTC = 32 - 2 * (WIN / 2);
  const int nwarps = (a.dmax + kDC - 1) / kDC;
  const size_t smem = cost_smem_bytes<NW>(nwarps * kDC, WIN, nwarps * 32);
  cudaError_t e = cudaFuncSetAttribute(cost_wta_kernel<NW, WIN, CSA>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.w + OUTC - 1) / OUTC, (a.h + a.rows - 1) / a.rows, 2);
  cost_wta_kernel<NW, WIN, CSA><<<grid, nwarps * 32, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NW, int WIN, bool CSA>
cudaError_t launch_batch_t(BatchHeader *hdr, const BatchPair *pairs, uint32_t *status, int grid, bool prepare,
                           int *grid_out, cudaStream_t s) {
  constexpr int kThreads = kBatchDisp / kDC * 32;
  const size_t smem = cost_smem_bytes<NW>(kBatchDisp, WIN, kThreads);
  if (prepare) {
    cudaError_t e = cudaFuncSetAttribute(cost_batch_kernel<NW, WIN, CSA>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cost_batch_kernel<NW, WIN, CSA>, kThreads, smem);
    *grid_out = max(1, per_sm) * grid;  // `grid` carries the SM count when preparing
    return e;
  }
  cost_batch_kernel<NW, WIN, CSA><<<grid, kThreads, smem, s>>>(hdr, pairs, status);
  return cudaGetLastError();
}

template <int NW, bool CSA>
cudaError_t launch_win(int win, const CostArgs &a, cudaStream_t s) {
  switch (win) {
    case 1: return launch_t<NW, 1, CSA>(a, s);
    case 3: return launch_t<NW, 3, CSA>(a, s);
    case 5: return launch_t<NW, 5, CSA>(a, s);
    case 7: return launch_t<NW, 7, CSA>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int NW, bool CSA>
cudaError_t launch_batch_win(int win, BatchHeader *hdr, const BatchPair *pairs, uint32_t *status, int grid,
                             bool prepare, int *grid_out, cudaStream_t s) {
  switch (win) {
    case 1: return launch_batch_t<NW, 1, CSA>(hdr, pairs, status, grid, prepare, grid_out, s);
    case 3: return launch_batch_t<NW, 3, CSA>(hdr, pairs, status, grid, prepare, grid_out, s);
    case 5: return launch_batch_t<NW, 5, CSA>(hdr, pairs, status, grid, prepare, grid_out, s);
    case 7: return launch_batch_t<NW, 7, CSA>(hdr, pairs, status, grid, prepare, grid_out, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t cost_batch_dispatch(const bsm_ctx *ctx, BatchHeader *hdr, const BatchPair *pairs, int grid, bool prepare,
                                int *grid_out, cudaStream_t s) {
  const int win = ctx->p.agg_window;
  switch (ctx->nw) {
    case 1: return launch_batch_win<1, false>(win, hdr, pairs, ctx->status, grid, prepare, grid_out, s);
    case 2: return launch_batch_win<2, false>(win, hdr, pairs, ctx->status, grid, prepare, grid_out, s);
    case 4: return launch_batch_win<4, false>(win, hdr, pairs, ctx->status, grid, prepare, grid_out, s);
    case 8:
      return ctx->cost_plain_popc == 1
                 ? launch_batch_win<8, false>(win, hdr, pairs, ctx->status, grid, prepare, grid_out, s)
                 : launch_batch_win<8, true>(win, hdr, pairs, ctx->status, grid, prepare, grid_out, s);
    default: return cudaErrorInvalidValue;
  }
}

// Rows per CTA: long bands amortise the 2r halo rows, short bands give small images enough CTAs.
int pick_rows(int w, int h, int win, int dmax) {
  const int outc = 32 - 2 * (win / 2);
  const long cols = (w + outc - 1) / outc;
  const int nwarps = (dmax + kDC - 1) / kDC;
  const long ctas_per_sm = nwarps >= 16 ? 1 : (nwarps >= 8 ? 2 : 4);
  const long target = 2L * 152 * ctas_per_sm;  // two full waves of both directions
  long rows = 128;
  while (rows > 8 && cols * ((h + rows - 1) / rows) * 2 < target) rows /= 2;
  return (int)rows;
}

}  // namespace

int cost1_rows(const bsm_ctx *ctx, int w, int h, int dmax) {
  return ctx->cost_rows > 0 ? ctx->cost_rows : pick_rows(w, h, ctx->p.agg_window, dmax);
}

CostPlan cost_plan(const bsm_ctx *ctx, int w, int h, int dmax) {
  if (ctx->nw > 8 || ctx->p.mask_mode == BSM_MASK_BOTH) return {4, cost_long_rows(ctx, w, h, dmax), 1};
  // tensor cores when asked for, and by default for pairs large enough to fill the GPU with them; the
  // two-column kernel has no staging wait to withhold, so the failure-detection hook keeps the
  // one-column kernel unless the tensor-core kernel was asked for
  const bool tc = ctx->cost_variant == 3 || (ctx->cost_variant == 0 && (long long)w * h * dmax >= kTcAutoWork);
  if (tc && cost_tc_supported(ctx) && (!ctx->withhold_arrivals || ctx->cost_variant == 3))
    return {3, cost_tc_rows(ctx, w, h, dmax), 1};
  if (ctx->cost_variant != 1 && cost2_supported(ctx) && !ctx->withhold_arrivals) {
    const bool split = (dmax + 7) / 8 > 16;  // more 8-disparity groups than the two-column kernel's 16 warps
    return {2, cost2_rows(ctx, w, h, dmax), split ? 2 : 1};
  }
  return {1, cost1_rows(ctx, w, h, dmax), 1};
}

cudaError_t launch_cost_wta(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                            const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *costL,
                            uint16_t *costR, cudaStream_t s) {
  const CostPlan plan = cost_plan(ctx, w, h, dmax);
  if (plan.kernel == 4) return launch_cost_long(ctx, BL, PhiL, BR, PhiR, w, h, dmax, dL, dR, costL, costR, s);
  if (plan.kernel == 3) return launch_cost_tc(ctx, BL, PhiL, BR, PhiR, w, h, dmax, dL, dR, costL, costR, s);
  if (plan.kernel == 2) return launch_cost2(ctx, BL, PhiL, BR, PhiR, w, h, dmax, dL, dR, costL, costR, s);
  CostArgs a{};
  a.B[0] = BL; a.Phi[0] = PhiL; a.O[0] = BR; a.disp[0] = dL;
  a.B[1] = BR; a.Phi[1] = PhiR; a.O[1] = BL; a.disp[1] = dR;
  a.cost[0] = costL; a.cost[1] = costR;
  a.status = ctx->status;
  a.w = w; a.h = h; a.dmax = dmax;
  a.rows = plan.rows;
  a.withhold = ctx->withhold_arrivals;
  switch (ctx->nw) {
    case 1: return launch_win<1, false>(ctx->p.agg_window, a, s);
    case 2: return launch_win<2, false>(ctx->p.agg_window, a, s);
    case 4: return launch_win<4, false>(ctx->p.agg_window, a, s);
    case 8:
      return ctx->cost_plain_popc == 1 ? launch_win<8, false>(ctx->p.agg_window, a, s)
                                  : launch_win<8, true>(ctx->p.agg_window, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t prepare_cost_batch(const bsm_ctx *ctx, int *grid) {
  return cost_batch_dispatch(ctx, nullptr, nullptr, ctx->sms, true, grid, nullptr);
}

cudaError_t launch_cost_batch(const bsm_ctx *ctx, BatchHeader *hdr, const BatchPair *pairs, int grid, cudaStream_t s) {
  return cost_batch_dispatch(ctx, hdr, pairs, grid, false, nullptr, s);
}

}  // namespace bsm
