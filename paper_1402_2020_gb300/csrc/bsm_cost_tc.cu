// Fused Eq. 8 cost + box aggregation + Eq. 1 on the 5th-generation tensor cores (n = 256).
//
// Eq. 8 as a contraction. With s_i(x) = Phi_i(x) (1 - 2 B_i(x)) in {-1, 0, 1} and o_i the other view's
// bits, popcount((B(x) XOR O) AND Phi(x)) = popcount(Phi(x) AND B(x)) + sum_i s_i(x) o_i exactly, so the
// costs of 128 reference columns (TMEM lanes) against the band of other-view columns their
// disparities reach (TMEM columns) are one product S O^T. The window's vertical sum is a running
// accumulator: every input row adds [s(new row) | -s(old row)] . [o(new row) | o(old row)] (K = 2n)
// with tcgen05.mma kind::f8f6f4, E4M3 operands +-2^-6 and 2^-6, fp32 accumulation in TMEM: every value
// is an integer times 2^-12 below 2^11, so the products and sums are exact.
//
// Per input row (one CTA: 128 columns, a band of rows, one reference view):
//   1. the K dimension is expanded from bits to E4M3 bytes in 64-byte chunks, double-buffered in the
//      no-swizzle K-major canonical layout (8-row x 16-byte core matrices; rows 16 bytes apart, K
//      groups of 16 bytes one operand height apart): 128 threads build the A rows from the reference
//      B / Phi words, 384 threads the B rows from the other view's words (read through L1, which
//      keeps each pixel's 32 bytes for the row's four chunks); after each chunk one thread issues its
//      MMAs (2 k-steps x up to 2 N-blocks) and commits them to the chunk buffer's mbarrier;
//   2. once the row's MMAs are done, every warp reads its lane quadrant of the accumulator
//      (tcgen05.ld 32x32b.x32) and writes term(x, d) = V(x, x_d) + the window's popcount(Phi AND B)
//      of column x (or the out-of-image sentinel n per in-image row) into a shared [x][d] table with
//      one fused multiply-add and one store per value;
//   3. one warp per run of 8 output columns, 8 disparities per lane: the horizontal box sum slides
//      along x on packed 16-bit pairs (128-bit table reads), (A << 3 | d % 8) keys reduce with
//      min.u16x2, and one warp-wide unsigned minimum of (A << 8 | d) gives Eq. 1's smallest d.
// Every wait is bounded; a wait that gives up latches BSM_ERR_TIMEOUT and the CTA stops.
#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kTM = 128;         // reference columns per CTA: MMA M, TMEM lanes
constexpr int kNB = 384;         // rows of the B operand buffer: the band of 128 + 256 - 1 other columns
constexpr int kChunk = 64;       // K bytes per operand chunk (= descriptor bits)
constexpr int kThreads = 512;    // 128 threads build A rows, 384 build B rows
constexpr int kTP = 264;         // u16 pitch of the term table T[x][d] (rows 16-byte aligned)
constexpr int kAB = kTM * kChunk;        // A chunk bytes
constexpr int kBB = kNB * kChunk;        // B chunk bytes
constexpr int kOpB = kAB + kBB;          // one operand buffer
constexpr int kOffOp = 0;
constexpr int kOffT = kOffOp + 2 * kOpB;
constexpr int kOffC0 = kOffT + kTM * kTP * 2;
constexpr int kOffMisc = kOffC0 + kTM * 4;
constexpr int kSmem = kOffMisc + 64;
static_assert(kSmem <= 232448, "shared memory of one CTA");
static_assert(kOffT % 16 == 0 && kOffMisc % 16 == 0 && (kTP * 2) % 16 == 0, "alignment");
constexpr long long kWait = 1LL << 31;  // about one second at the GB300 clock

struct TcArgs {
  const uint32_t *B[2], *Phi[2], *O[2];
  int32_t *disp[2];
  uint16_t *cost[2];
  uint32_t *status;
  int w, h, dmax, rows;
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok) : "r"(saddr(bar)), "r"(parity) : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > kWait) return false;
  return true;
}

// Shared-memory matrix descriptor: no swizzle, K-major; lbo = bytes between K groups of 16 bytes,
// sbo = bytes between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f8f6f4: E4M3 x E4M3 -> F32, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t instr_desc(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

__device__ __forceinline__ void mma_f8(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}"
               ::"r"(tmem), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                 "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                 "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                 "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Byte k (k = 0..3) of output word q takes bit 8k + q of w, placed at bit `pos` of the byte: the
// expansion's K order is a fixed permutation of the descriptor bits, the same for both operands.
template <int Q, int POS>
__device__ __forceinline__ uint32_t spread(uint32_t w) {
  constexpr int sh = POS - Q;
  constexpr uint32_t mask = 0x01010101u << POS;
  if constexpr (sh >= 0) return (w << sh) & mask;
  else return (w >> (-sh)) & mask;
}

// 32 K bytes of the A operand from one reference word pair: +-2^-6 (0x08 / 0x88) where the mask bit
// is set, the sign from the descriptor bit (negated for the row that leaves the window).
__device__ __forceinline__ void expand_a(uint32_t b, uint32_t m, bool neg, uint8_t *dst_g0, uint8_t *dst_g1) {
  const uint32_t sb = m & (neg ? ~b : b);
  uint32_t o[8];
  o[0] = spread<0, 3>(m) | spread<0, 7>(sb);
  o[1] = spread<1, 3>(m) | spread<1, 7>(sb);
  o[2] = spread<2, 3>(m) | spread<2, 7>(sb);
  o[3] = spread<3, 3>(m) | spread<3, 7>(sb);
  o[4] = spread<4, 3>(m) | spread<4, 7>(sb);
  o[5] = spread<5, 3>(m) | spread<5, 7>(sb);
  o[6] = spread<6, 3>(m) | spread<6, 7>(sb);
  o[7] = spread<7, 3>(m) | spread<7, 7>(sb);
  *reinterpret_cast<uint4 *>(dst_g0) = make_uint4(o[0], o[1], o[2], o[3]);
  *reinterpret_cast<uint4 *>(dst_g1) = make_uint4(o[4], o[5], o[6], o[7]);
}

// 32 K bytes of the B operand from one other-view word: 2^-6 (0x08) where the bit is set.
__device__ __forceinline__ void expand_b(uint32_t o, uint8_t *dst_g0, uint8_t *dst_g1) {
  *reinterpret_cast<uint4 *>(dst_g0) =
      make_uint4(spread<0, 3>(o), spread<1, 3>(o), spread<2, 3>(o), spread<3, 3>(o));
  *reinterpret_cast<uint4 *>(dst_g1) =
      make_uint4(spread<4, 3>(o), spread<5, 3>(o), spread<6, 3>(o), spread<7, 3>(o));
}

__device__ __forceinline__ uint32_t vmin_u16x2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

template <int WIN, int DIR>
__device__ __forceinline__ void cost_tc_body(const TcArgs &a, uint8_t *smem) {
  constexpr int R = WIN / 2, OUTC = kTM - 2 * R;
  constexpr bool PK = 256 * WIN * WIN < 8192;  // aggregated costs below 2^13: 16-bit (A << 3 | dd) keys
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t *__restrict__ Bref = DIR ? a.B[1] : a.B[0];
  const uint32_t *__restrict__ Phiref = DIR ? a.Phi[1] : a.Phi[0];
  const uint32_t *__restrict__ Both = DIR ? a.O[1] : a.O[0];
  int32_t *__restrict__ disp = DIR ? a.disp[1] : a.disp[0];
  uint16_t *cost = DIR ? a.cost[1] : a.cost[0];
  const int w = a.w, h = a.h, dmax = a.dmax;
  const int D = (dmax + 31) & ~31;             // band depth: disparities per reference column
  const int ntot = kTM + D;                    // band columns, the MMA's N in total
  const int nb0 = ntot < 256 ? ntot : 256, nb1 = ntot - nb0;
  const uint32_t ncols = ntot <= 256 ? 256u : 512u;
  const int X0 = (int)blockIdx.x * OUTC - R;   // column of TMEM lane 0
  const int xb0 = DIR == 0 ? X0 - D + 1 : X0;  // other-view column of band column 0
  const int yb = (int)blockIdx.y * a.rows, ye = min(h, yb + a.rows);
  const int y_first = yb - R, n_it = (ye + R) - y_first;
  // every column of the tile is in the image and every match of it lies inside the other view
  const bool fast = X0 >= 0 && X0 + kTM <= w && (DIR == 0 ? X0 >= D - 1 : X0 + kTM - 1 + D - 1 < w);

  uint64_t *mbar = reinterpret_cast<uint64_t *>(smem + kOffMisc);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(smem + kOffMisc + 16);
  uint16_t *T = reinterpret_cast<uint16_t *>(smem + kOffT);
  int32_t *c0v = reinterpret_cast<int32_t *>(smem + kOffC0);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&mbar[1])));
  }
  if (tid < kTM) c0v[tid] = 0;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // this thread's operand row: A row `arow` (tid < 128) or B row `brow`
  const bool is_a = tid < kTM;
  const int arow = tid, brow = tid - kTM;
  const int xa = X0 + arow, xo = xb0 + brow;
  const bool row_ok = is_a ? (xa >= 0 && xa < w) : (brow < ntot && xo >= 0 && xo < w);
  const size_t pix_col = is_a ? (size_t)xa : (size_t)xo;

  uint32_t uses0 = 0, uses1 = 0;  // commits made to each operand buffer's mbarrier (uniform)
  int last_buf = -1;              // buffer of the newest commit not yet waited for
  bool acc_init = false, ok = true;
  uint32_t nchunk = 0;

  for (int i = 0; i < n_it && ok; ++i) {
    const int yn = y_first + i, yold = yn - (2 * R + 1), yout = yn - R;
    const bool has_new = yn >= 0 && yn < h, has_old = i >= 2 * R + 1 && yold >= 0 && yold < h;
    int c0acc = 0;
    for (int c = 0; c < 8; ++c) {
      const bool is_new = c < 4;
      if (!(is_new ? has_new : has_old)) continue;
      const int j0 = 2 * (c & 3);
      // this chunk's two words of the thread's pixel (an L1 hit after the row's first chunk)
      uint2 bw = make_uint2(0u, 0u), mw = make_uint2(0u, 0u);
      if (row_ok) {
        const size_t off = ((size_t)(is_new ? yn : yold) * w + pix_col) * 8 + j0;
        if (is_a) {
          bw = __ldg(reinterpret_cast<const uint2 *>(Bref + off));
          mw = __ldg(reinterpret_cast<const uint2 *>(Phiref + off));
        } else {
          bw = __ldg(reinterpret_cast<const uint2 *>(Both + off));
        }
      }
      const int bb = (int)(nchunk & 1u);
      const uint32_t ub = bb ? uses1 : uses0;
      if (ub > 0) ok = mbar_wait(&mbar[bb], (ub - 1) & 1u);  // the MMAs two chunks back
      ok = __syncthreads_and(ok) != 0;
      if (!ok) break;
      uint8_t *opA = smem + kOffOp + bb * kOpB, *opB = opA + kAB;
      if (is_a) {
        expand_a(bw.x, mw.x, !is_new, opA + 0 * (kTM * 16) + arow * 16, opA + 1 * (kTM * 16) + arow * 16);
        expand_a(bw.y, mw.y, !is_new, opA + 2 * (kTM * 16) + arow * 16, opA + 3 * (kTM * 16) + arow * 16);
        const int pc = __popc(bw.x & mw.x) + __popc(bw.y & mw.y);
        c0acc += is_new ? pc : -pc;
      } else if (brow < ntot) {
        expand_b(bw.x, opB + 0 * (kNB * 16) + brow * 16, opB + 1 * (kNB * 16) + brow * 16);
        expand_b(bw.y, opB + 2 * (kNB * 16) + brow * 16, opB + 3 * (kNB * 16) + brow * 16);
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      __syncthreads();
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint64_t ad = smem_desc(saddr(opA) + ks * 2 * (kTM * 16), kTM * 16, 128);
          const uint32_t acc = (acc_init || ks > 0) ? 1u : 0u;
          mma_f8(tmem, ad, smem_desc(saddr(opB) + ks * 2 * (kNB * 16), kNB * 16, 128), instr_desc(nb0), acc);
          if (nb1 > 0)
            mma_f8(tmem + 256, ad, smem_desc(saddr(opB) + ks * 2 * (kNB * 16) + 256 * 16, kNB * 16, 128),
                   instr_desc(nb1), acc);
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         saddr(&mbar[bb]))
                     : "memory");
      }
      acc_init = true;
      if (bb) ++uses1;
      else ++uses0;
      last_buf = bb;
      ++nchunk;
    }
    if (!ok) break;
    if (is_a) c0v[arow] += c0acc;  // the window's popcount(Phi AND B) per reference column
    if (yout < yb) {
      __syncthreads();
      continue;  // the window is not full yet
    }

    // ---- the accumulator holds V(x, x_d) for output row yout
    if (last_buf >= 0) {
      ok = mbar_wait(&mbar[last_buf], ((last_buf ? uses1 : uses0) - 1) & 1u);
      last_buf = -1;
    }
    ok = __syncthreads_and(ok) != 0;  // also publishes c0v
    if (!ok) break;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    {
      int nh = 0;
#pragma unroll
      for (int v = -R; v <= R; ++v) nh += (yout + v >= 0 && yout + v < h) ? 1 : 0;
      const int q = warp & 3, g = warp >> 2, r = 32 * q + lane, xr = X0 + r;
      const float base = (float)c0v[r] + 12582912.0f;  // 1.5 * 2^23: the sum's integer sits in the low bits
      uint16_t *Trow = T + r * kTP;
      const int nck = D / 32 + 1;
      for (int k = g; k < nck; k += 4) {
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * q + 32 * k), v);
        // band column 32 q + 32 k + t is disparity d = DIR ? rel : D - 1 - rel, rel = 32 k + t - lane
        if (fast && k > 0 && k < nck - 1) {
          uint16_t *p0 = DIR == 0 ? Trow + (D - 1 - 32 * k + lane) : Trow + (32 * k - lane);
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            const uint32_t val = __float_as_uint(fmaf(__uint_as_float(v[t]), 4096.0f, base));
            if (DIR == 0) p0[-t] = (uint16_t)val;
            else p0[t] = (uint16_t)val;
          }
        } else {
          const bool col_in = xr >= 0 && xr < w;
          const uint32_t sentinel = (uint32_t)nh * 256u;
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            const int rel = 32 * k + t - lane;
            if (rel < 0 || rel >= D) continue;
            const int d = DIR == 0 ? D - 1 - rel : rel;
            uint32_t val = __float_as_uint(fmaf(__uint_as_float(v[t]), 4096.0f, base));
            const bool match_in = DIR == 0 ? xr - d >= 0 : xr + d < w;
            if (!match_in) val = sentinel;
            Trow[d] = (uint16_t)(col_in ? val : 0u);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // T complete; the accumulator may be overwritten by the next row's MMAs

    {  // warp: output columns rr0 .. rr1 - 1; lane: disparities 8 lane .. 8 lane + 7
      const int rr0 = R + 8 * warp, rr1 = min(rr0 + 8, kTM - R);
      const int d8 = 8 * lane;
      if (rr0 < rr1) {
        const bool lane_on = d8 < D;
        uint32_t s4[4] = {0, 0, 0, 0};
        if (lane_on) {
#pragma unroll
          for (int u = -R; u <= R; ++u) {
            const uint4 t4 = *reinterpret_cast<const uint4 *>(T + (rr0 + u) * kTP + d8);
            s4[0] += t4.x; s4[1] += t4.y; s4[2] += t4.z; s4[3] += t4.w;
          }
        }
        // halves holding a disparity at or above dmax never win
        uint32_t inval[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          inval[j] = (d8 + 2 * j < dmax ? 0u : 0xFFFFu) | (d8 + 2 * j + 1 < dmax ? 0u : 0xFFFF0000u);
        for (int rr = rr0; rr < rr1; ++rr) {
          if (rr > rr0 && lane_on) {
            const uint4 tn = *reinterpret_cast<const uint4 *>(T + (rr + R) * kTP + d8);
            const uint4 to = *reinterpret_cast<const uint4 *>(T + (rr - R - 1) * kTP + d8);
            s4[0] += tn.x - to.x; s4[1] += tn.y - to.y; s4[2] += tn.z - to.z; s4[3] += tn.w - to.w;
          }
          uint32_t key;
          if constexpr (PK) {
            uint32_t m = 0xFFFFFFFFu;
#pragma unroll
            for (int j = 0; j < 4; ++j)
              m = vmin_u16x2(m, (s4[j] * 8u + ((uint32_t)(2 * j) | ((uint32_t)(2 * j + 1) << 16))) | inval[j]);
            const uint32_t m16 = min(m & 0xFFFFu, m >> 16);
            key = (m16 == 0xFFFFu || !lane_on) ? 0xFFFFFFFFu : ((m16 >> 3) << 8) | (uint32_t)(d8 + (m16 & 7u));
          } else {
            key = 0xFFFFFFFFu;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              if (d8 + 2 * j < dmax) key = min(key, ((s4[j] & 0xFFFFu) << 8) | (uint32_t)(d8 + 2 * j));
              if (d8 + 2 * j + 1 < dmax) key = min(key, ((s4[j] >> 16) << 8) | (uint32_t)(d8 + 2 * j + 1));
            }
          }
          key = __reduce_min_sync(0xFFFFFFFFu, key);
          const int x = X0 + rr;
          if (x >= 0 && x < w) {
            if (lane == 0) disp[(size_t)yout * w + x] = (int32_t)(key & 0xFFu);
            if (cost != nullptr && lane_on) {
              uint16_t *cp = cost + ((size_t)yout * w + x) * dmax;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                if (d8 + 2 * j < dmax) cp[d8 + 2 * j] = (uint16_t)(s4[j] & 0xFFFFu);
                if (d8 + 2 * j + 1 < dmax) cp[d8 + 2 * j + 1] = (uint16_t)(s4[j] >> 16);
              }
            }
          }
        }
      }
    }
    __syncthreads();  // every warp is done with T
  }

  if (!ok && tid == 0) atomicCAS(a.status, 0u, (uint32_t)BSM_ERR_TIMEOUT);
  if (ok && last_buf >= 0) ok = mbar_wait(&mbar[last_buf], ((last_buf ? uses1 : uses0) - 1) & 1u);  // in flight
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols));
}

template <int WIN>
__global__ void __launch_bounds__(kThreads, 1) cost_tc_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  if (blockIdx.z == 0) cost_tc_body<WIN, 0>(a, smem);
  else cost_tc_body<WIN, 1>(a, smem);
}

template <int WIN>
cudaError_t launch_tc_t(const TcArgs &a, cudaStream_t s) {
  constexpr int OUTC = kTM - 2 * (WIN / 2);
  cudaError_t e = cudaFuncSetAttribute(cost_tc_kernel<WIN>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.w + OUTC - 1) / OUTC, (a.h + a.rows - 1) / a.rows, 2);
  cost_tc_kernel<WIN><<<grid, kThreads, kSmem, s>>>(a);
  return cudaGetLastError();
}

// Row bands so that the grid is about three waves of one CTA per SM.
int pick_rows_tc(int w, int h, int win) {
  const int outc = kTM - 2 * (win / 2);
  const int ntx = (w + outc - 1) / outc;
  int bands = (3 * 152 + 2 * ntx - 1) / (2 * ntx);
  bands = max(1, min(bands, h));
  return (h + bands - 1) / bands;
}

}  // namespace

bool cost_tc_supported(const bsm_ctx *ctx) { return ctx->nw == 8 && ctx->p.mask_mode != BSM_MASK_BOTH; }

cudaError_t launch_cost_tc(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                           const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *costL,
                           uint16_t *costR, cudaStream_t s) {
  TcArgs a{};
  a.B[0] = BL; a.Phi[0] = PhiL; a.O[0] = BR; a.disp[0] = dL; a.cost[0] = costL;
  a.B[1] = BR; a.Phi[1] = PhiR; a.O[1] = BL; a.disp[1] = dR; a.cost[1] = costR;
  a.status = ctx->status;
  a.w = w; a.h = h; a.dmax = dmax;
  a.rows = ctx->cost_rows > 0 ? ctx->cost_rows : pick_rows_tc(w, h, ctx->p.agg_window);
  switch (ctx->p.agg_window) {
    case 1: return launch_tc_t<1>(a, s);
    case 3: return launch_tc_t<3>(a, s);
    case 5: return launch_tc_t<5>(a, s);
    case 7: return launch_tc_t<7>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsm
