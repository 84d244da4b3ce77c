// Fused Eq. 8 cost + box aggregation + Eq. 1 on the 5th-generation tensor cores (n = 256).
//
// Eq. 8 as a contraction. With s_i(x) = Phi_i(x) (1 - 2 B_i(x)) in {-1, 0, 1} and o_i the other view's
// bits, popcount((B(x) XOR O) AND Phi(x)) = popcount(Phi(x) AND B(x)) + sum_i s_i(x) o_i exactly, so the
// costs of 128 reference columns (TMEM lanes) against the band of other-view columns their
// disparities reach (TMEM columns) are one product S O^T. The window's vertical sum is a running
// accumulator: every input row adds s(entering row) . o(entering row) and, with the A operand negated
// by the instruction descriptor, subtracts s(leaving row) . o(leaving row); tcgen05.mma kind::f8f6f4,
// E4M3 operands whose every product is 0 or +-2^-2 (the encoding is below), fp32 accumulation in
// TMEM: every value is an integer times 2^-2 below 2^9, so the products and sums are exact.
//
// One launch, cost_tc_kernel, one CTA per (128 reference columns, band of rows, reference view), 20 warps;
// the K order within a 32-bit descriptor word is a fixed permutation of its bits (byte k of operand word
// q is bit 8k + q), the same for both operands:
//    - warp 0 (producer) loads, by TMA, the other view's descriptor words of the entering and the
//      leaving row (32 bytes per band column); the tensor maps fill columns outside the image with zeros;
//    - warps 2..7 (builders) form each 64-byte K chunk's operands in shared memory: A (4 groups x 128
//      reference columns of s bytes, nonzero where the mask bit is set, from the reference view's B and
//      Phi words, read from global memory one row half ahead) and B (4 groups x up to 384 band columns
//      of o bytes, nonzero where the bit is set, from the TMA'd words); they also keep each column's
//      window popcount(Phi AND B) and publish it per input row in a small ring;
//    - warp 1 owns the TMEM accumulator and issues the MMAs (2 k-steps x 2 N-blocks per chunk), commits
//      each chunk to its buffer's "empty" barrier and each finished output row to "acc_full"; before the
//      next row's MMAs it waits until the epilogue has read the accumulator;
//    - warps 8..19 (epilogue) read their lane quadrant of the accumulator (tcgen05.ld 32x32b.x32) into
//      registers as 16-bit term(x, d) = V(x, x_d) + the window's popcount(Phi AND B) of column x (or the
//      sentinel n per in-image row when the match leaves the image), release the accumulator, write the
//      terms into a shared [x][d] table, then slide the horizontal box sum along x on packed 16-bit pairs
//      and reduce (A << 3 | d % 8) keys with min.u16x2 and one warp-wide minimum of (A << 8 | d): Eq. 1's
//      smallest d. This overlaps the next row's MMAs.
// Every wait is bounded; a wait that gives up latches BSM_ERR_TIMEOUT and the CTA winds down. The
// failure-detection hook (withhold) makes the producer issue no copies, so every wait runs out.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <type_traits>

#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kTM = 128;          // reference columns per CTA: MMA M, TMEM lanes
constexpr int kNB = 384;          // B operand rows: the band of 128 + 256 - 1 other-view columns
constexpr int kChunk = 64;        // K bytes per operand chunk: 2 descriptor words (2 MMA k-steps of 32)
constexpr int kBuf = 4;           // operand buffers: A in TMEM, B in shared memory
constexpr int kBW = 4;            // operand builder warps (warps 2 .. kBW + 1)
constexpr int kE0 = 2 + kBW;      // first epilogue warp
constexpr int kWarps = kE0 + 12;  // producer, MMA, builders, 12 epilogue warps (3 per TMEM lane quadrant)
constexpr int kThreads = 32 * kWarps;
constexpr int kXpd = kBW * 32;    // operand builder threads
// Builder warp w (2 .. 5) forms the A rows of TMEM lane quadrant w % 4 (the quadrant its tcgen05.st
// reaches) and, with its thread index bt = tid - 64, the band columns bt + kBT j of the B operand; the
// hardware places warps 2 .. 5 on schedulers 2, 3, 0, 1, one builder per scheduler. (Six builder
// warps, the A rows on four of them, measured slower.)
constexpr int kBT = kXpd;                // band-column threads
constexpr int kBC = kNB / kBT;
static_assert(kXpd == kTM && kBT * kBC == kNB, "one A row and kBC band columns per builder thread");
constexpr int kEpi = 12 * 32;     // epilogue threads (warps kE0 .. kE0 + 11)
constexpr int kTP = 288;          // u16 pitch of the term table T[x][d] (rows 16-byte aligned)
constexpr int kTPad = 32;         // u16 in front of row 0; row r's band terms past d = 255 land in row r + 1's first 32
constexpr int kBB = kNB * kChunk;         // B chunk: 4 groups x 384 rows x 16 bytes (24 KB)
constexpr int kRawRow = kNB * 32;         // other-view words of one row of the band (8 words per column)
constexpr int kOffOp = 0;
constexpr int kOffRaw = kOffOp + kBuf * kBB;           // 2 slots x (entering, leaving) rows
constexpr int kOffT = kOffRaw + 2 * 2 * kRawRow;
constexpr int kOffC0 = kOffT + (kTM * kTP + kTPad) * 2;
constexpr int kC0Ring = 8;        // rows of window popcounts in flight between builders and epilogue
constexpr int kOffRing = kOffC0 + kTM * 4;
constexpr int kOffMisc = kOffRing + kC0Ring * kTM * 4;
constexpr int kSmem = kOffMisc + 256;
static_assert(kSmem <= 232448, "shared memory of one CTA");
static_assert(kOffRaw % 1024 == 0 && kOffT % 1024 == 0 && kOffC0 % 16 == 0 && kOffMisc % 16 == 0 && (kTP * 2) % 16 == 0 &&
                  (kTPad * 2) % 16 == 0 && kTP >= 256 + kTPad,
              "alignment");
// TMEM: 512 columns; the accumulator takes columns 0 .. 383, A buffer b columns kACol + 16 b .. + 15
// (16 32-bit columns hold a row's 64 E4M3 K bytes of one chunk)
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kACol = 384;
static_assert(kACol + 16 * kBuf <= kTmemCols, "A buffers beside the accumulator");
constexpr long long kWait = 1LL << 31;  // about one second at the GB300 clock

struct TcArgs {
  CUtensorMap bmap0[2];   // descriptor plane of the other view, box 32 bytes x 256 columns x 1 row
  CUtensorMap bmap1[2];   // the same, box 32 bytes x 128 columns x 1 row
  const uint32_t *Bv[2];  // descriptor plane of the reference view, [h][w][8], per reference view
  const uint32_t *Pv[2];  // mask plane of the reference view
  int32_t *disp[2];
  uint16_t *cost[2];
  uint32_t *status;
  int w, h, dmax, rows;
  int withhold;           // test hook: the producer issues no copies, so every wait on them runs out
};

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// One try of a phase wait. A thread whose phase is not complete sleeps in the barrier hardware until the
// phase completes or about 20 microseconds pass (the suspend-time hint), so waiting warps take few issue
// slots from the working ones.
__device__ __forceinline__ bool mbar_try(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok) : "r"(saddr(bar)), "r"(parity), "r"(20000u) : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(bar, parity))
    if (clock64() - t0 > kWait) return false;
  return true;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}

// 3-D tile copy (16 bytes x columns x K groups) of an operand plane into shared memory.
__device__ __forceinline__ void tma_load3(void *dst, const CUtensorMap *map, int x, int row, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(saddr(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(x), "r"(row), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void epi_sync() {  // named barrier of the epilogue warps
  asm volatile("bar.sync 1, %0;" ::"r"(kEpi) : "memory");
}

// The same barrier, returning whether every epilogue thread passed `ok`.
__device__ __forceinline__ bool epi_sync_and(bool ok) {
  uint32_t r;
  asm volatile("{\n.reg .pred p, q;\nsetp.ne.u32 q, %1, 0;\nbarrier.cta.red.and.pred p, 1, %2, q;\nselp.u32 %0, 1, 0, p;\n}"
               : "=r"(r) : "r"((uint32_t)ok), "r"(kEpi) : "memory");
  return r != 0;
}

// Shared-memory matrix descriptor: no swizzle, K-major; lbo = bytes between K groups of 16 bytes,
// sbo = bytes between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f8f6f4: E4M3 x E4M3 -> F32, both K-major, M = 128, N = n; bit 13
// negates A.
__device__ __forceinline__ uint32_t instr_desc(int n, bool neg_a) {
  return (1u << 4) | (neg_a ? (1u << 13) : 0u) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTM >> 4) << 24);
}

// D (TMEM) += or = A (TMEM, K-major: row m in lane m, 4 K bytes per 32-bit column) x B^T (shared memory).
__device__ __forceinline__ void mma_f8_ta(uint32_t tmem_d, uint32_t tmem_a, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f8f6f4 [%0], [%1], %2, %3, p;\n}"
               ::"r"(tmem_d), "r"(tmem_a), "l"(bd), "r"(idesc), "r"(acc));
}

// 16 consecutive TMEM columns of the warp's lane quadrant from 16 registers per thread.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
               ::"r"(taddr), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                 "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
               : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// 32 consecutive accumulator columns of the warp's 32 TMEM lanes into r, asynchronously: the registers
// hold the values only after tmem_wait_ld().
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                 "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                 "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
                 "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
                 "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
               : "r"(taddr)
               : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ uint32_t vmin_u16x2(uint32_t a, uint32_t b) {
  uint32_t r;
  asm("min.u16x2 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(b));
  return r;
}

// Operand bytes. Byte k (k = 0..3) of operand word q holds bit 8k + q of a descriptor word; the same K
// permutation for both operands. The other view's bit o becomes the byte o << q as it stands (one AND
// per word), except bit 7, which moves to 0x40 (0x80 would be E4M3's -0): so bit q of a byte carries the
// E4M3 value v_q = 2^-9, 2^-8, 2^-7, 2^-6, 2^-5, 2^-3, 2^1, 2^1 for q = 0 .. 7 (q < 3 are subnormals).
// The reference byte carries s = Phi (1 - 2 B) times a_q = 2^-2 / v_q = 2^7, 2^6, 2^5, 2^4, 2^3, 2^1,
// 2^-3, 2^-3 (E4M3 codes 0x70, 0x68, 0x60, 0x58, 0x50, 0x40, 0x20, 0x20, sign 0x80), so every product is
// s o 2^-2 exactly and the accumulator holds 2^-2 sum_i s_i o_i.

// 32 K bytes of the B operand from one other-view word o.
__device__ __forceinline__ void expand_b(uint32_t o, uint8_t *dst_g0, uint8_t *dst_g1) {
  *reinterpret_cast<uint4 *>(dst_g0) = make_uint4(o & 0x01010101u, o & 0x02020202u, o & 0x04040404u, o & 0x08080808u);
  *reinterpret_cast<uint4 *>(dst_g1) =
      make_uint4(o & 0x10101010u, o & 0x20202020u, o & 0x40404040u, (o >> 1) & 0x40404040u);
}

// Operand word q < 6 of the A operand: (m & M_q) (P_q / 2^q) puts the magnitude code P_q in every byte
// whose mask bit is set, (s & M_q) 2^(7 - q) the sign where the descriptor bit is set too (s = m & b).
template <int Q>
__device__ __forceinline__ uint32_t a_word(uint32_t m, uint32_t sb) {
  constexpr uint32_t M = 0x01010101u << Q;
  constexpr uint32_t P[6] = {0x70u, 0x68u, 0x60u, 0x58u, 0x50u, 0x40u};
  return (m & M) * (P[Q] >> Q) + (sb & M) * (0x80u >> Q);
}

// 32 K bytes (8 words, from word o of `out`) of the A operand from one descriptor word b and mask word m
// of the reference column.
__device__ __forceinline__ void expand_a(uint32_t b, uint32_t m, uint32_t (&out)[16], int o) {
  const uint32_t sb = m & b;
  out[o + 0] = a_word<0>(m, sb);
  out[o + 1] = a_word<1>(m, sb);
  out[o + 2] = a_word<2>(m, sb);
  out[o + 3] = a_word<3>(m, sb);
  out[o + 4] = a_word<4>(m, sb);
  out[o + 5] = a_word<5>(m, sb);
  out[o + 6] = ((m >> 1) & 0x20202020u) | ((sb << 1) & 0x80808080u);
  out[o + 7] = ((m >> 2) & 0x20202020u) | (sb & 0x80808080u);
}

// ---------------------------------------------------------------- cost kernel

template <int WIN, int DIR, bool WC>
__device__ __forceinline__ void cost_tc_body(const TcArgs &a, uint8_t *smem) {
  constexpr int R = WIN / 2, OUTC = kTM - 2 * R;
  constexpr bool PK = 256 * WIN * WIN < 8192;  // aggregated costs below 2^13: 16-bit (A << 3 | dd) keys
  constexpr int kHC = (OUTC + 11) / 12;        // output columns per epilogue warp in the horizontal pass
  // With 16-bit keys the term table holds 8 x each term, so a column's packed window sums are directly
  // (A << 3 | d % 8) once the disparity's low bits are added at the window's start.
  constexpr uint32_t kTS = PK ? 8u : 1u;
  static_assert(WIN + 1 <= kC0Ring, "the popcount ring holds the rows the builders may run ahead");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const CUtensorMap *bmap0 = &a.bmap0[DIR], *bmap1 = &a.bmap1[DIR];
  const uint32_t *__restrict__ Bref = DIR ? a.Bv[1] : a.Bv[0];
  const uint32_t *__restrict__ Pref = DIR ? a.Pv[1] : a.Pv[0];
  int32_t *__restrict__ disp = DIR ? a.disp[1] : a.disp[0];
  uint16_t *cost = WC ? (DIR ? a.cost[1] : a.cost[0]) : nullptr;  // WC: the cost volume is written
  const int w = a.w, h = a.h, dmax = a.dmax;
  const int D = (dmax + 31) & ~31;             // band depth: disparities per reference column
  const int ntot = kTM + D;                    // band columns, the MMA's N in total
  const int nb0 = ntot < 256 ? ntot : 256, nb1 = ntot - nb0;
  const int X0 = (int)blockIdx.x * OUTC - R;   // column of TMEM lane 0
  const int xb0 = DIR == 0 ? X0 - D + 1 : X0;  // other-view column of band column 0
  const int yb = (int)blockIdx.y * a.rows, ye = min(h, yb + a.rows);
  const int y_first = yb - R, n_it = (ye + R) - y_first;
  // every column of the tile is in the image and every match of it lies inside the other view
  const bool fast = X0 >= 0 && X0 + kTM <= w && (DIR == 0 ? X0 >= D - 1 : X0 + kTM - 1 + D - 1 < w);

  uint64_t *full = reinterpret_cast<uint64_t *>(smem + kOffMisc);  // [kBuf]
  uint64_t *empty = full + kBuf;                                    // [kBuf]
  uint64_t *raw_full = empty + kBuf, *raw_empty = raw_full + 2;     // [2] each
  uint64_t *acc_full = raw_empty + 2, *acc_empty = acc_full + 1;
  uint64_t *c0_full = acc_empty + 1;                                // [kC0Ring]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(c0_full + kC0Ring);
  uint32_t *abort_flag = tmem_slot + 1;
  uint16_t *T = reinterpret_cast<uint16_t *>(smem + kOffT) + kTPad;
  int32_t *c0v = reinterpret_cast<int32_t *>(smem + kOffC0);
  int32_t *ring = reinterpret_cast<int32_t *>(smem + kOffRing);  // [kC0Ring][kTM]

  if (tid == 0) {
    for (int b = 0; b < kBuf; ++b) {
      mbar_init(&full[b], kXpd / 32);  // every builder warp
      mbar_init(&empty[b], 1);
    }
    for (int k = 0; k < 2; ++k) {
      mbar_init(&raw_full[k], 1);
      mbar_init(&raw_empty[k], kXpd / 32);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, kEpi / 32);
    for (int k = 0; k < kC0Ring; ++k) mbar_init(&c0_full[k], kXpd / 32);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(tmem_slot)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  auto row_new = [&](int i) { const int y = y_first + i; return y >= 0 && y < h; };
  auto row_old = [&](int i) { const int y = y_first + i - (2 * R + 1); return i >= 2 * R + 1 && y >= 0 && y < h; };

  if (warp == 0) {
    // ---- producer: per input row the other view's words, per chunk the A operand, in order
    if (lane == 0 && !a.withhold) {
      const uint32_t rowbytes = (uint32_t)(256 * 32 + (nb1 > 0 ? 128 * 32 : 0));
      bool ok = true;
      int last = -1;  // the last input row whose copies were issued
      for (int i = 0; i < n_it && ok; ++i) {
        const int rs = i & 1;
        if (i >= 2) ok = mbar_wait(&raw_empty[rs], ((i >> 1) - 1) & 1u);
        if (!ok) break;
        const bool hn = row_new(i), ho = row_old(i);
        uint8_t *raw = smem + kOffRaw + rs * 2 * kRawRow;
        if (hn || ho) {
          mbar_expect_tx(&raw_full[rs], (hn ? rowbytes : 0u) + (ho ? rowbytes : 0u));
          for (int k = 0; k < 2; ++k) {
            if (!(k == 0 ? hn : ho)) continue;
            const int y = k == 0 ? y_first + i : y_first + i - (2 * R + 1);
            tma_load3(raw + k * kRawRow, bmap0, xb0, y, &raw_full[rs]);
            if (nb1 > 0) tma_load3(raw + k * kRawRow + 256 * 32, bmap1, xb0 + 256, y, &raw_full[rs]);
          }
          last = i;
        } else {
          mbar_arrive(&raw_full[rs]);
        }
      }
      if (!ok) atomicExch(abort_flag, 1u);
      if (!ok && last >= 0) mbar_wait(&raw_full[last & 1], (last >> 1) & 1u);  // let the copies land
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      uint32_t slot = 0, outs = 0;
      bool ok = true, acc_init = false, pending = false;
      for (int i = 0; i < n_it && ok; ++i) {
        if (pending) {  // the epilogue has read the previous output row's accumulator
          ok = mbar_wait(acc_empty, (outs - 1) & 1u);
          pending = false;
          if (!ok) break;
        }
        for (int c = 0; c < 8 && ok; ++c) {
          const bool is_new = c < 4;
          if (!(is_new ? row_new(i) : row_old(i))) continue;
          const int b = (int)(slot % kBuf);
          ok = mbar_wait(&full[b], (slot / kBuf) & 1u);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t op = saddr(smem + kOffOp + b * kBB);
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t ta = tmem + kACol + 16 * b + 8 * ks;  // A of this k-step: 8 columns of 4 K bytes
            const uint32_t acc = (acc_init || ks > 0) ? 1u : 0u;
            mma_f8_ta(tmem, ta, smem_desc(op + ks * 2 * (kNB * 16), kNB * 16, 128), instr_desc(nb0, !is_new), acc);
            if (nb1 > 0)
              mma_f8_ta(tmem + 256, ta, smem_desc(op + ks * 2 * (kNB * 16) + 256 * 16, kNB * 16, 128),
                        instr_desc(nb1, !is_new), acc);
          }
          mma_commit(&empty[b]);
          acc_init = true;
          ++slot;
        }
        if (ok && y_first + i - R >= yb) {  // an output row: hand the accumulator to the epilogue
          mma_commit(acc_full);
          ++outs;
          pending = true;
        }
      }
      if (!ok) atomicExch(abort_flag, 1u);
    }
  } else if (warp < kE0) {
    // ---- operand builders: per chunk, the A operand's row ra of this warp's TMEM lane quadrant (the s
    // bytes of reference column X0 + ra, from its descriptor and mask words), written to TMEM, and the B
    // operand's band columns bt + kXpd j in shared memory
    const int ra = 32 * (warp & 3) + lane, xa = X0 + ra, bt = tid - 64;
    constexpr bool has_a = true, has_b = true;
    const bool a_in = xa >= 0 && xa < w;
    const uint32_t ta_lane = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's lane quadrant
    auto present = [&](int ii, int hh) { return hh == 0 ? row_new(ii) : row_old(ii); };
    // the reference words of the next (row, half) with an image row are loaded one half ahead
    auto load_ref = [&](int ii, int hh, uint4(&q)[4]) {
      if (a_in) {
        const int y = hh == 0 ? y_first + ii : y_first + ii - (2 * R + 1);
        const size_t o = ((size_t)y * w + xa) * 8;
        q[0] = __ldg(reinterpret_cast<const uint4 *>(Bref + o));
        q[1] = __ldg(reinterpret_cast<const uint4 *>(Bref + o + 4));
        q[2] = __ldg(reinterpret_cast<const uint4 *>(Pref + o));
        q[3] = __ldg(reinterpret_cast<const uint4 *>(Pref + o + 4));
      } else {
        q[0] = q[1] = q[2] = q[3] = make_uint4(0u, 0u, 0u, 0u);  // columns off the image: s = 0
      }
    };
    int ni = 0, nh = 0;
    auto advance = [&]() {
      do {
        nh ^= 1;
        if (nh == 0) ++ni;
      } while (ni < n_it && !present(ni, nh));
    };
    if (!present(0, 0)) advance();
    int c0run = 0;  // the window's popcount(Phi AND B) of column X0 + ra
    uint4 nxt[4];
    if (ni < n_it) load_ref(ni, nh, nxt);
    uint32_t slot = 0;
    bool ok = true;
    for (int i = 0; i < n_it && ok; ++i) {
      const int rs = i & 1;
      const bool hn = row_new(i), ho = row_old(i);
      ok = mbar_wait(&raw_full[rs], (i >> 1) & 1u);
      if (!ok) break;
      const uint8_t *raw = smem + kOffRaw + rs * 2 * kRawRow;
      // per row half (entering, leaving): the 8 words of each of the thread's band columns, read once
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        if (!ok || !(half == 0 ? hn : ho)) continue;
        uint4 cur[4];  // this half's reference words: B 0..3, B 4..7, Phi 0..3, Phi 4..7
#pragma unroll
        for (int k = 0; k < 4; ++k) cur[k] = nxt[k];
        advance();
        if (ni < n_it) load_ref(ni, nh, nxt);
        {
          const int pc = __popc(cur[0].x & cur[2].x) + __popc(cur[0].y & cur[2].y) + __popc(cur[0].z & cur[2].z) +
                         __popc(cur[0].w & cur[2].w) + __popc(cur[1].x & cur[3].x) + __popc(cur[1].y & cur[3].y) +
                         __popc(cur[1].z & cur[3].z) + __popc(cur[1].w & cur[3].w);
          c0run += half == 0 ? pc : -pc;
        }
        const uint32_t *rw = reinterpret_cast<const uint32_t *>(raw + half * kRawRow);
        uint4 qw[kBC];  // words 4 (cc / 2) .. 4 (cc / 2) + 3 of each of the thread's band columns
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) {  // chunk cc: descriptor words 2 cc and 2 cc + 1
          if (!ok) break;
          if ((cc & 1) == 0) {
#pragma unroll
            for (int k = 0; k < kBC; ++k) {
              const int r = bt + kBT * k;
              if (has_b)
                qw[k] = r < ntot ? *reinterpret_cast<const uint4 *>(rw + r * 8 + 2 * cc) : make_uint4(0u, 0u, 0u, 0u);
            }
          }
          const int b = (int)(slot % kBuf);
          if (slot >= kBuf) ok = mbar_wait(&empty[b], ((slot / kBuf) - 1) & 1u);
          if (!ok) break;
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");  // the MMAs that read buffer b are done
          if (has_a) {
            const uint4 &bq = cur[cc >> 1], &mq = cur[2 + (cc >> 1)];
            uint32_t av[16];
            expand_a((cc & 1) ? bq.z : bq.x, (cc & 1) ? mq.z : mq.x, av, 0);
            expand_a((cc & 1) ? bq.w : bq.y, (cc & 1) ? mq.w : mq.y, av, 8);
            tmem_st16(ta_lane + kACol + 16 * b, av);
          }
          uint8_t *opB = smem + kOffOp + b * kBB;
#pragma unroll
          for (int k = 0; k < kBC; ++k) {
            const int r = bt + kBT * k;
            if (has_b && r < ntot) {
              const uint4 &qq = qw[k];
              expand_b((cc & 1) ? qq.z : qq.x, opB + 0 * (kNB * 16) + r * 16, opB + 1 * (kNB * 16) + r * 16);
              expand_b((cc & 1) ? qq.w : qq.y, opB + 2 * (kNB * 16) + r * 16, opB + 3 * (kNB * 16) + r * 16);
            }
          }
          if (has_a) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(&full[b]);
          ++slot;
        }
      }
      __syncwarp();
      if (lane == 0 && ok) mbar_arrive(&raw_empty[rs]);  // this row's words are no longer needed
      if (ok) {  // the window's popcount after input row i, for the epilogue
        if (has_a) ring[(i & (kC0Ring - 1)) * kTM + ra] = c0run;
        __syncwarp();
        if (lane == 0) mbar_arrive(&c0_full[i & (kC0Ring - 1)]);
      }
    }
    if (!ok) atomicExch(abort_flag, 1u);
  } else {
    // ---- epilogue: warps kE0 .. kE0 + 11; lane quadrant q = warp % 4, g = its index among the quadrant's warps
    const int q = warp & 3, g = (warp - kE0) >> 2, ew = warp - kE0, r = 32 * q + lane, xr = X0 + r;
    const bool col_in = xr >= 0 && xr < w;
    uint32_t outs = 0;
    bool ok = true;
    for (int i = 0; i < n_it && ok; ++i) {
      const int yout = y_first + i - R;
      if (yout < yb) continue;
      bool okc = true;
      if (g == 0) {  // the builders' window popcount of column r after input row i
        okc = mbar_wait(&c0_full[i & (kC0Ring - 1)], (uint32_t)(i / kC0Ring) & 1u);
        c0v[r] = col_in ? ring[(i & (kC0Ring - 1)) * kTM + r] : 0;
      }
      ok = mbar_wait(acc_full, outs & 1u) && okc;
      if (*reinterpret_cast<volatile uint32_t *>(abort_flag) != 0) ok = false;  // the other roles gave up
      ++outs;
      // c0v published; the previous row's horizontal pass is done with T; all agree on ok
      ok = epi_sync_and(ok);
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      int nh = 0;
#pragma unroll
      for (int v = -R; v <= R; ++v) nh += (yout + v >= 0 && yout + v < h) ? 1 : 0;
      {
        const float base = (float)(kTS * c0v[r]) + 12582912.0f;  // 1.5 * 2^23: the sum's integer in the low bits
        const int nck = D / 32 + 1;
        const uint32_t sentinel = col_in ? kTS * (uint32_t)nh * 256u : 0u;
        // Element t of chunk k is disparity c - t (left reference) or c + t (right); its terms are
        // consecutive 16-bit entries of row r from u16 index a0 = r kTP + c down (left) or up (right),
        // written as 32-bit words: where a0 sits mid-word, 15 whole words and two single entries. Terms
        // of d outside [0, D) land in row padding that is never read. The first chunk is written at
        // once; the other two are held in registers until the accumulator is released.
        uint32_t *T32 = reinterpret_cast<uint32_t *>(T);
        uint32_t wd[2][16];
        auto put = [&](int a0, bool al, const uint32_t(&wk)[16]) {
          if (DIR == 0) {
            uint32_t *wp = T32 + ((a0 - 1) >> 1);
#pragma unroll
            for (int p = 0; p < 16; ++p)
              if (p < 15 || al) wp[-p] = wk[p];
          } else {
            uint32_t *wp = T32 + ((a0 + 1) >> 1);
#pragma unroll
            for (int p = 0; p < 16; ++p)
              if (p < 15 || al) wp[p] = wk[p];
          }
        };
        auto chunk_a0 = [&](int k) { return r * kTP + (DIR == 0 ? D - 1 - 32 * k + lane : 32 * k - lane); };
        auto whole = [&](int a0) { return DIR == 0 ? (a0 & 1) != 0 : (a0 & 1) == 0; };  // 16 whole words
        // chunk kk of this warp (k = g + 3 kk): convert to 16-bit terms and pack them as words
        auto process = [&](uint32_t(&v)[32], int k, uint32_t(&wk)[16]) {
#pragma unroll
          for (int t = 0; t < 32; ++t) v[t] = __float_as_uint(fmaf(__uint_as_float(v[t]), 4.0f * kTS, base));
          const int a0 = chunk_a0(k);
          if (!fast) {  // the sentinel where the match leaves the other view; 0 for columns off the image
            const int c = a0 - r * kTP;
            const int cut = DIR == 0 ? (col_in ? c - xr : 64) : (col_in ? w - xr - c : -1);
#pragma unroll
            for (int t = 0; t < 32; ++t) v[t] = (DIR == 0 ? t >= cut : t < cut) ? v[t] : sentinel;
          }
          const bool al = whole(a0);
          const uint32_t sel = (al == (DIR == 0)) ? 0x5410u : 0x1054u;
#pragma unroll
          for (int p = 0; p < 16; ++p)
            wk[p] = __byte_perm(v[2 * p + 1], al ? v[2 * p] : v[2 * p + 2 < 32 ? 2 * p + 2 : 31], sel);
          if (!al) {
            T[a0] = (uint16_t)v[0];
            T[DIR == 0 ? a0 - 31 : a0 + 31] = (uint16_t)v[31];
          }
        };
        auto col_addr = [&](int k) { return tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(32 * q + 32 * k); };
        // one chunk at a time (two in flight need 32 more live registers: at 18 warps, five share a
        // scheduler, which caps a thread at 96 and would spill)
        const int k0 = g, k1 = g + 3, k2 = g + 6;
        {
          uint32_t va[32];
          if (k0 < nck) {
            tmem_ld32_async(col_addr(k0), va);
            tmem_wait_ld();
            uint32_t wk[16];
            process(va, k0, wk);
            put(chunk_a0(k0), whole(chunk_a0(k0)), wk);
          }
          if (k1 < nck) {
            tmem_ld32_async(col_addr(k1), va);
            tmem_wait_ld();
            process(va, k1, wd[0]);
          }
          if (k2 < nck) {
            tmem_ld32_async(col_addr(k2), va);
            tmem_wait_ld();
            process(va, k2, wd[1]);
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(acc_empty);  // the next row's MMAs may start; the stores below overlap them
#pragma unroll
        for (int kk = 1; kk < 3; ++kk) {
          const int k = g + 3 * kk;
          if (k < nck) {
            const int a0 = chunk_a0(k);
            put(a0, whole(a0), wd[kk - 1]);
          }
        }
      }
      epi_sync();  // T complete

      // horizontal box sum + Eq. 1: warp ew takes output columns rr0 .. rr0 + ncol - 1, lane 8 disparities;
      // the lane keeps the window's 2R + 1 rows of T in a register ring, so each column reads one new row
      const int rr0 = R + kHC * ew, ncol = min(kHC, OUTC - kHC * ew);
      const int d8 = 8 * lane;
      if (ncol > 0) {
        const bool lane_on = d8 < D;
        auto trow = [&](int rr) {
          return lane_on ? *reinterpret_cast<const uint4 *>(T + rr * kTP + d8) : make_uint4(0u, 0u, 0u, 0u);
        };
        uint4 ring[2 * R + 1];
        uint32_t s4[4];  // with 16-bit keys: 8 x the window sums of disparities d8 + 2 j (low), + 2 j + 1 (high), plus 2 j, 2 j + 1
#pragma unroll
        for (int j = 0; j < 4; ++j) s4[j] = PK ? ((uint32_t)(2 * j) | ((uint32_t)(2 * j + 1) << 16)) : 0u;
#pragma unroll
        for (int u = 0; u < 2 * R + 1; ++u) {
          ring[u] = trow(rr0 - R + u);
          s4[0] += ring[u].x; s4[1] += ring[u].y; s4[2] += ring[u].z; s4[3] += ring[u].w;
        }
        uint32_t inval[4];  // halves holding a disparity at or above dmax never win
#pragma unroll
        for (int j = 0; j < 4; ++j)
          inval[j] = (d8 + 2 * j < dmax ? 0u : 0xFFFFu) | (d8 + 2 * j + 1 < dmax ? 0u : 0xFFFF0000u);
        const uint32_t lane_d = (uint32_t)d8;  // bits 3 .. 7 of every key of this lane
        // FULL: dmax = 256, so every lane's 8 disparities are below dmax: no invalid halves to mask
        auto columns = [&](auto full_tag) {
          constexpr bool FULL = decltype(full_tag)::value;
          int32_t mydisp = 0;
          uint4 tn = ncol > 1 ? trow(rr0 + R + 1) : make_uint4(0u, 0u, 0u, 0u);  // next column's entering row
#pragma unroll
          for (int c = 0; c < kHC; ++c) {
            if (c >= ncol) break;
            const int rr = rr0 + c;
            if (c > 0) {  // slide: the entering row replaces the leaving one in the ring
              uint4 &old = ring[(c - 1) % (2 * R + 1)];
              s4[0] += tn.x - old.x; s4[1] += tn.y - old.y; s4[2] += tn.z - old.z; s4[3] += tn.w - old.w;
              old = tn;
              if (c + 1 < ncol) tn = trow(rr + R + 1);
            }
            uint32_t key;
            if constexpr (PK) {
              uint32_t m;
              if constexpr (FULL) {
                m = vmin_u16x2(vmin_u16x2(s4[0], s4[1]), vmin_u16x2(s4[2], s4[3]));
              } else {
                m = vmin_u16x2(vmin_u16x2(s4[0] | inval[0], s4[1] | inval[1]),
                               vmin_u16x2(s4[2] | inval[2], s4[3] | inval[3]));
              }
              m = vmin_u16x2(m, __byte_perm(m, 0u, 0x1032));  // both halves: the lane's smallest (A << 3 | d % 8)
              key = (((m & 0xFFF8u) << 5) | lane_d) | (m & 7u);  // A << 8 | d
              if constexpr (!FULL) key = ((m & 0xFFFFu) == 0xFFFFu || !lane_on) ? 0xFFFFFFFFu : key;
            } else {
              key = 0xFFFFFFFFu;
#pragma unroll
              for (int j = 0; j < 4; ++j) {
                if (d8 + 2 * j < dmax) key = min(key, ((s4[j] & 0xFFFFu) << 8) | (uint32_t)(d8 + 2 * j));
                if (d8 + 2 * j + 1 < dmax) key = min(key, ((s4[j] >> 16) << 8) | (uint32_t)(d8 + 2 * j + 1));
              }
            }
            key = __reduce_min_sync(0xFFFFFFFFu, key);
            mydisp = lane == c ? (int32_t)(key & 0xFFu) : mydisp;
            const int x = X0 + rr;
            if (WC && lane_on && x >= 0 && x < w) {
              uint16_t *cp = cost + ((size_t)yout * w + x) * dmax;
#pragma unroll
              for (int j = 0; j < 4; ++j) {  // the window sums themselves (the 16-bit keys' sums are 8 x, plus d % 8)
                if (d8 + 2 * j < dmax) cp[d8 + 2 * j] = (uint16_t)((s4[j] & 0xFFFFu) / kTS);
                if (d8 + 2 * j + 1 < dmax) cp[d8 + 2 * j + 1] = (uint16_t)((s4[j] >> 16) / kTS);
              }
            }
          }
          // lane c holds column rr0 + c's disparity: one store for the warp's columns
          const int xo = X0 + rr0 + lane;
          if (lane < ncol && xo >= 0 && xo < w) disp[(size_t)yout * w + xo] = mydisp;
        };
        if (dmax == 256) columns(std::true_type{});
        else columns(std::false_type{});
      }
    }
    if (!ok && tid == kE0 * 32) atomicCAS(a.status, 0u, (uint32_t)BSM_ERR_TIMEOUT);
  }
  if (tid == 0 && *abort_flag != 0) atomicCAS(a.status, 0u, (uint32_t)BSM_ERR_TIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
}

// WC: the launch writes cost volumes (a separate instance, so that the disparity-only kernel does not
// carry the volume path's registers).
template <int WIN, bool WC>
__global__ void __launch_bounds__(kThreads, 1) cost_tc_kernel(const __grid_constant__ TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  if (blockIdx.z == 0) cost_tc_body<WIN, 0, WC>(a, smem);
  else cost_tc_body<WIN, 1, WC>(a, smem);
}

template <int WIN, bool WC>
cudaError_t launch_tc_wc(const TcArgs &a, cudaStream_t s) {
  constexpr int OUTC = kTM - 2 * (WIN / 2);
  cudaError_t e = cudaFuncSetAttribute(cost_tc_kernel<WIN, WC>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.w + OUTC - 1) / OUTC, (a.h + a.rows - 1) / a.rows, 2);
  cost_tc_kernel<WIN, WC><<<grid, kThreads, kSmem, s>>>(a);
  return cudaGetLastError();
}

template <int WIN>
cudaError_t launch_tc_t(const TcArgs &a, cudaStream_t s) {
  return (a.cost[0] != nullptr || a.cost[1] != nullptr) ? launch_tc_wc<WIN, true>(a, s) : launch_tc_wc<WIN, false>(a, s);
}

// Row bands: one CTA per SM (all of TMEM), so the launch takes ceil(CTAs / SMs) waves of about
// (band rows + the window's halo) input rows each. The band count that minimises that product.
int pick_rows_tc(int w, int h, int win, int sms) {
  const int outc = kTM - 2 * (win / 2);
  const long ntx = (w + outc - 1) / outc;
  long best_cost = -1;
  int best_rows = h;
  for (int bands = 1; bands <= h; ++bands) {
    const int rows = (h + bands - 1) / bands;
    if (bands > 1 && rows == (h + bands - 2) / (bands - 1)) continue;  // same rows as fewer bands
    const long waves = (2 * ntx * bands + sms - 1) / sms;
    const long cost = waves * (rows + 2 * (win / 2));
    if (best_cost < 0 || cost < best_cost) {
      best_cost = cost;
      best_rows = rows;
    }
  }
  return best_rows;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (fn == nullptr) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// Descriptor plane [h][w][8 words] as a 3-D byte tensor (32, w, h); box 32 x cols x 1.
bool desc_map(CUtensorMap *map, const void *base, int w, int h, int cols) {
  auto fn = encode_fn();
  if (fn == nullptr) return false;
  const cuuint64_t dims[3] = {32, (cuuint64_t)w, (cuuint64_t)h};
  const cuuint64_t strides[2] = {32, (cuuint64_t)32 * w};
  const cuuint32_t box[3] = {32, (cuuint32_t)cols, 1};
  const cuuint32_t elem[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, const_cast<void *>(base), dims, strides, box, elem,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool cost_tc_supported(const bsm_ctx *ctx) { return ctx->nw == 8 && ctx->p.mask_mode != BSM_MASK_BOTH; }

int cost_tc_rows(const bsm_ctx *ctx, int w, int h, int dmax) {
  (void)dmax;
  return ctx->cost_rows > 0 ? ctx->cost_rows : pick_rows_tc(w, h, ctx->p.agg_window, ctx->sms > 0 ? ctx->sms : 152);
}

cudaError_t launch_cost_tc(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                           const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *costL,
                           uint16_t *costR, cudaStream_t s) {
  TcArgs a{};
  // left reference: A from the left view's planes, B from the right view's descriptors; right reference the other way
  if (!desc_map(&a.bmap0[0], BR, w, h, 256) || !desc_map(&a.bmap0[1], BL, w, h, 256) ||
      !desc_map(&a.bmap1[0], BR, w, h, 128) || !desc_map(&a.bmap1[1], BL, w, h, 128))
    return cudaErrorInvalidValue;
  a.Bv[0] = BL; a.Pv[0] = PhiL;
  a.Bv[1] = BR; a.Pv[1] = PhiR;
  a.disp[0] = dL; a.disp[1] = dR;
  a.cost[0] = costL; a.cost[1] = costR;
  a.status = ctx->status;
  a.w = w; a.h = h; a.dmax = dmax;
  a.rows = cost_tc_rows(ctx, w, h, dmax);
  a.withhold = ctx->withhold_arrivals;
  switch (ctx->p.agg_window) {
    case 1: return launch_tc_t<1>(a, s);
    case 3: return launch_tc_t<3>(a, s);
    case 5: return launch_tc_t<5>(a, s);
    case 7: return launch_tc_t<7>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsm
