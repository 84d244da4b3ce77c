// Left/right check and voting refinement of the left disparity map (Sec. 3, Eq. 9-10).
//
// Every pixel is summarised in one refinement word: byte 0 = L | v << 7 (v: the pixel passes the
// left/right check; CIELAB L is at most 100, so bit 7 is free), byte 1 = a + 128, byte 2 = b + 128,
// byte 3 = the pixel's disparity when v, else the no-vote fallback of Eq. 10's row rule (the smaller of
// the nearest valid disparities to its left and right on the row, whichever exists, else 0). A pre-pass
// (refine_words_kernel, one warp per row) forms the words; the batched form builds them while staging,
// with byte 3 = 0 for invalid pixels, and scans the row for the fallback instead.
//
// One CTA (16 warps) covers a 32 x 32 block of output pixels (32 x 8 on small images). The pre-pass also
// counts each block's invalid pixels, and the blocks are taken in decreasing order of that count: invalid
// pixels cluster (occlusions), so a few blocks carry most of the votes, and started last they would set
// the kernel's tail. The CTA stages the words of the block plus a halo of R pixels, together with the two
// integer vote tables. Valid pixels keep their disparity. Invalid pixels are collected into a list that
// the CTA's warps share: a warp takes one invalid pixel at a time and walks the window's valid voters,
// summing each one's vote floor(Ec[c] * Es[e2] / 2^15) in a register while consecutive voters share a
// disparity and adding the run to a per-warp shared histogram over d when the disparity changes
// (disparities are piecewise smooth, so runs are long and shared atomics few). The warp then takes the
// smallest d with the largest weight (Eq. 9), scanning only the bins between the smallest and largest
// disparity it added to, or the fallback when no vote is positive.
//
// The batched form reads the colour words from the batch's colour planes, and its disparity inputs
// are the batched cost kernel's keys (A << 10 | d): every read keeps the low 10 bits, and each CTA
// writes its block's final disparities back over the keys. A key and its disparity agree in the low
// 10 bits, so reads by other CTAs see the same disparity before and after that write.
#include "bsm_internal.cuh"

namespace bsm {
namespace {

// A CTA of kWarps warps refines a kTX x kTY block (kTX x kShortTY on small images, below). Its staged tile
// adds the window's R-pixel halo on every side, so the block is square-ish: at R = 15 a 32 x 32 block
// stages 3.75 entries per output pixel (a 32 x 8 block stages 9.2).
constexpr int kTX = kRefineTX, kTY = kRefineTY;
constexpr int kWarps = 16;  // a block's invalid pixels spread over more warps (the heaviest blocks set the tail)
constexpr int kThreadsR = 32 * kWarps;
constexpr uint32_t kDispMask = 1023u;

struct RefineArgs {
  const uint8_t *rgb;      // RGB view (when plane == nullptr)
  const uint32_t *plane;   // packed colour words, or nullptr
  const uint32_t *table;
  int32_t *dL;             // WTA maps (or keys, see above)
  int32_t *dR;
  int32_t *out;
  int w, h, pitch, dmax, tol, R;
  int hist_stride;         // shared histogram bins per warp (>= dmax)
  bool finalize;           // write the masked disparities back into dL and dR
  const uint32_t *words;   // the refinement words of the view (with the row fallback), or nullptr to form
                           // them while staging and scan the row for the fallback
  int *tile_cnt;           // per block: its invalid pixels (counted by the pre-pass), or nullptr
  const int *tile_order;   // the blocks in the order CTAs take them (most invalid pixels first), or nullptr
  int tile_h;              // rows of a block (kTY or kShortTY)
};

constexpr uint32_t kValidBit = 0x80u;

// The refinement word of a pixel with colour word `colour`, check result `ok` and byte 3 `d`.
__device__ __forceinline__ uint32_t refine_word(uint32_t colour, bool ok, uint32_t d) {
  return (colour & kLabMask) | (ok ? kValidBit : 0u) | (d << 24);
}

__device__ __forceinline__ uint32_t lab_sad(uint32_t a, uint32_t b) {
  return __dp4a(__vabsdiffu4(a, b), 0x00010101u, 0u);
}

__device__ __forceinline__ int disp_at(const int32_t *m, size_t i) {
  return (int)((uint32_t)__ldcg(m + i) & kDispMask);
}

__device__ __forceinline__ bool lr_valid(const RefineArgs &a, int x, int y, int d) {
  const int xr = x - d;
  if (xr < 0 || xr >= a.w) return false;
  return abs(d - disp_at(a.dR, (size_t)y * a.w + xr)) <= a.tol;
}

__host__ __device__ size_t table_words(int R) { return (kMaxSad + 1) + (size_t)(2 * R * R + 1); }

__device__ __forceinline__ void load_vote_tables(const uint32_t *Ec, const uint32_t *Es, int R, uint32_t *smem) {
  const int ne = 2 * R * R + 1;
  for (int i = threadIdx.x; i <= kMaxSad; i += blockDim.x) smem[i] = __ldg(Ec + i);
  for (int i = threadIdx.x; i < ne; i += blockDim.x) smem[kMaxSad + 1 + i] = __ldg(Es + i);
}

// The shared memory a CTA's tile takes after the vote tables, as byte offsets in carve-up order: the
// staged words (th x tp), the warps' histograms, the invalid-pixel count and list (kTX x ty), the row
// bitmaps (2 words a tile row) and the warps' voter lists (32 x (2R + 1) entries each). refine_tile takes
// its pointers from here and the launch sizes the allocation from `bytes`, so the two cannot disagree.
struct TileLayout {
  size_t hist, count, list, vbits, vlist, bytes;
};

__host__ __device__ __forceinline__ TileLayout tile_layout(int R, int hist_stride, int ty) {
  const size_t tp = kTX + 2 * R, th = ty + 2 * R;
  TileLayout l;
  l.hist = th * tp * 4;
  l.count = l.hist + (size_t)kWarps * hist_stride * 4;
  l.list = l.count + 4;
  l.vbits = l.list + (size_t)kTX * ty * 2;  // a multiple of 4: the list has kTX * ty = 32 ty entries
  l.vlist = l.vbits + th * 2 * 4;
  l.bytes = l.vlist + (size_t)kWarps * 32 * (2 * R + 1) * 2;
  return l;
}

// One kTX x TY block with top-left corner (x0, y0); `tabs` holds the vote tables, `work` the tile.
// Every thread of the CTA reaches its two CTA-wide barriers. RT > 0: the window radius is RT (the
// window's 2 RT + 1 <= 32 columns are lanes and its rows an unrolled loop, so every shared-memory
// address is a per-lane base plus a constant); RT == 0: any radius, a.R.
template <int RT, int TY>
__device__ __forceinline__ void refine_tile(const RefineArgs &a, int x0, int y0, const uint32_t *tabs,
                                            uint32_t *work) {
  static_assert(RT == 0 || 2 * RT + 1 <= 32, "one lane per window column");
  const int R = RT > 0 ? RT : a.R, side = 2 * R + 1;
  const int tp = kTX + 2 * R, th = TY + 2 * R;
  const uint32_t *sEc = tabs;
  const uint32_t *sEs = tabs + (kMaxSad + 1);
  const TileLayout lay = tile_layout(R, a.hist_stride, TY);
  uint8_t *base = reinterpret_cast<uint8_t *>(work);
  uint32_t *slab = work;                                                // th * tp refinement words
  uint32_t *shist = reinterpret_cast<uint32_t *>(base + lay.hist);     // kWarps * hist_stride
  int *s_count = reinterpret_cast<int *>(base + lay.count);
  int16_t *s_list = reinterpret_cast<int16_t *>(base + lay.list);      // kTX * TY
  // RT > 0: per tile row, the validity of its tp <= 64 columns as two bit words; per warp, the list of
  // an invalid pixel's voters (window row << 5 | window column)
  uint32_t *vbits = reinterpret_cast<uint32_t *>(base + lay.vbits);    // 2 th
  uint16_t *vlist = reinterpret_cast<uint16_t *>(base + lay.vlist);    // kWarps * 32 * (2 RT + 1)

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) *s_count = 0;
  // Staging, kSG entries per thread at a time. From the pre-pass: one word per entry. Otherwise each
  // level of dependent loads (colour bytes and dL, then the colour table and dR) is issued for all of them
  // before any result is used. Outside the image: an invalid word.
  constexpr int kSG = 4;
  for (int i0 = threadIdx.x; a.words != nullptr && i0 < th * tp; i0 += kSG * (int)blockDim.x) {
    uint32_t v[kSG];
#pragma unroll
    for (int u = 0; u < kSG; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      const int ty = i / tp, tx = i - ty * tp;
      const int gx = x0 + tx - R, gy = y0 + ty - R;
      v[u] = 0u;
      if (i < th * tp && gx >= 0 && gx < a.w && gy >= 0 && gy < a.h) v[u] = __ldg(a.words + (size_t)gy * a.w + gx);
    }
#pragma unroll
    for (int u = 0; u < kSG; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      if (i < th * tp) slab[i] = v[u];
    }
  }
  for (int i0 = threadIdx.x; a.words == nullptr && i0 < th * tp; i0 += kSG * (int)blockDim.x) {
    int gx[kSG], gy[kSG], d[kSG];
    bool in[kSG];
    uint32_t key[kSG];
#pragma unroll
    for (int u = 0; u < kSG; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      const int ty = i / tp, tx = i - ty * tp;
      gx[u] = x0 + tx - R;
      gy[u] = y0 + ty - R;
      in[u] = i < th * tp && gx[u] >= 0 && gx[u] < a.w && gy[u] >= 0 && gy[u] < a.h;
      key[u] = 0;
      d[u] = a.dmax;
      if (in[u]) {
        const size_t o = (size_t)gy[u] * a.w + gx[u];
        if (a.plane != nullptr) {
          key[u] = __ldg(a.plane + o);
        } else {
          const uint8_t *px = a.rgb + (size_t)gy[u] * a.pitch + 3 * gx[u];
          key[u] = ((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | (uint32_t)px[2];
        }
        d[u] = disp_at(a.dL, o);
      }
    }
    bool ok[kSG];
#pragma unroll
    for (int u = 0; u < kSG; ++u) {
      ok[u] = in[u] && d[u] < a.dmax && lr_valid(a, gx[u], gy[u], d[u]);
      if (in[u] && a.plane == nullptr) key[u] = __ldg(a.table + key[u]);
    }
#pragma unroll
    for (int u = 0; u < kSG; ++u) {
      const int i = i0 + u * (int)blockDim.x;
      if (i < th * tp) slab[i] = refine_word(key[u], ok[u], ok[u] ? (uint32_t)d[u] : 0u);
    }
  }
  __syncthreads();
  if constexpr (RT > 0) {  // the validity bitmaps of the tile rows (read after the next barrier)
    static_assert(kTX + 2 * RT <= 64, "a tile row in two bit words");
    for (int r = warp; r < th; r += kWarps) {
      const uint32_t b0 = __ballot_sync(0xFFFFFFFFu, lane < tp && (slab[r * tp + lane] & kValidBit));
      const uint32_t b1 = __ballot_sync(0xFFFFFFFFu, 32 + lane < tp && (slab[r * tp + 32 + lane] & kValidBit));
      if (lane == 0) {
        vbits[2 * r] = b0;
        vbits[2 * r + 1] = b1;
      }
    }
  }

  for (int p = threadIdx.x; p < kTX * TY; p += blockDim.x) {
    const int tx = p & (kTX - 1), ty = p / kTX;
    const int x = x0 + tx, y = y0 + ty;
    if (x < a.w && y < a.h) {
      const size_t i = (size_t)y * a.w + x;
      const uint32_t wv = slab[(ty + R) * tp + tx + R];
      if (wv & kValidBit) a.out[i] = (int)(wv >> 24);
      else s_list[atomicAdd(s_count, 1)] = (int16_t)p;
    }
  }
  __syncthreads();

  const int count = *s_count;
  uint32_t *hist = shist + warp * a.hist_stride;
  // the warp's histogram is cleared once here; after each pixel only the bins it touched are cleared again
  for (int d = lane; d < a.dmax; d += 32) hist[d] = 0;
  __syncwarp();
  for (int it = warp; it < count; it += kWarps) {
    const int t = s_list[it];
    const int tx = t & (kTX - 1), ty = t / kTX;
    const int x = x0 + tx, y = y0 + ty;
    // a run of equal disparity goes to the histogram with one atomic; [dlo, dhi] holds the bins the lane touched
    uint32_t dlo = 0xFFFFu, dhi = 0u;
    auto add_run = [&](int d, uint32_t v) {
      atomicAdd(&hist[d], v);
      dlo = min(dlo, (uint32_t)d);
      dhi = max(dhi, (uint32_t)d);
    };
    const uint32_t wx0 = slab[(ty + R) * tp + tx + R];  // the invalid pixel's own word
    const uint32_t labx = wx0 | kValidBit;  // every voter has the bit: it drops out of the CIELAB SAD
    if constexpr (RT > 0) {
      // Only valid neighbours vote, and around an invalid pixel most are invalid (they cluster): lane wy
      // takes window row wy's validity bits from the row bitmap, a warp prefix sum of their counts lays
      // the voters out as one list, and each lane then walks a contiguous stretch of it, so neighbouring
      // voters (mostly the same disparity) share one histogram add.
      constexpr int W = 2 * RT + 1;
      uint16_t *wl = vlist + warp * (32 * W);
      uint32_t m = 0;
      if (lane < W) {
        const int r = ty + lane;  // tile row of window row `lane`; window columns are tile columns tx .. tx + 2 RT
        const uint64_t bits = ((uint64_t)vbits[2 * r + 1] << 32) | vbits[2 * r];
        m = (uint32_t)(bits >> tx) & ((1u << W) - 1u);
      }
      const int cnt = __popc(m);
      int incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int n = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += n;
      }
      const int total = __shfl_sync(0xFFFFFFFFu, incl, 31);
      for (int p = incl - cnt; m; m &= m - 1u, ++p) wl[p] = (uint16_t)((lane << 5) | (__ffs(m) - 1));
      __syncwarp();
      const int per = (total + 31) >> 5;
      const int s0 = min(total, lane * per), s1 = min(total, s0 + per);
      int run_d = -1;
      uint32_t run = 0;
      for (int q = s0; q < s1; ++q) {
        const int pos = wl[q], wy = pos >> 5, wx = pos & 31;
        const uint32_t wv = slab[(ty + wy) * tp + tx + wx];
        const int dv = (int)(wv >> 24);
        const uint32_t v = (sEc[lab_sad(labx, wv)] * sEs[(wx - RT) * (wx - RT) + (wy - RT) * (wy - RT)]) >> kVoteShift;
        if (dv != run_d) {
          if (run) add_run(run_d, run);
          run_d = dv;
          run = 0;
        }
        run += v;
      }
      if (run) add_run(run_d, run);
    }
    for (int wx = lane; RT == 0 && wx < side; wx += 32) {
      const int dx2 = (wx - R) * (wx - R);
      const uint32_t *lcol = slab + ty * tp + tx + wx;  // window row 0 of this column
      int run_d = -1;
      uint32_t run = 0;
      for (int wy = 0; wy < side; ++wy) {
        const uint32_t wv = lcol[wy * tp];
        if (wv & kValidBit) {
          const int dv = (int)(wv >> 24);
          const int dy = wy - R;
          const uint32_t c = lab_sad(labx, wv);
          const uint32_t v = (sEc[c] * sEs[dx2 + dy * dy]) >> kVoteShift;
          if (dv != run_d) {
            if (run) add_run(run_d, run);
            run_d = dv;
            run = 0;
          }
          run += v;
        }
      }
      if (run) add_run(run_d, run);
    }
    __syncwarp();
    // the argmax scans only the bins some lane touched (no pixel's votes span many disparities)
    const int rlo = (int)__reduce_min_sync(0xFFFFFFFFu, dlo), rhi = (int)__reduce_max_sync(0xFFFFFFFFu, dhi);
    uint32_t bv = 0;
    int bd = 0x7FFFFFFF;
    for (int d = rlo + lane; d <= rhi; d += 32) {
      const uint32_t hv = hist[d];
      if (hv > bv) {
        bv = hv;
        bd = d;
      }
    }
    const uint32_t gmax = __reduce_max_sync(0xFFFFFFFFu, bv);
    for (int d = rlo + lane; d <= rhi; d += 32) hist[d] = 0;  // every lane's reads fed the reduction above
    int best;
    if (gmax > 0) {
      best = (int)__reduce_min_sync(0xFFFFFFFFu, (unsigned)(bv == gmax ? bd : 0x7FFFFFFF));
    } else if (a.words != nullptr) {
      best = (int)(wx0 >> 24);  // no positive vote: the pre-pass's row fallback
    } else {
      // no positive vote: nearest valid disparities on the row
      int left = -1, right = -1;
      for (int xs = x - 1; xs >= 0; xs -= 32) {
        const int xi = xs - lane;
        int d = -1;
        if (xi >= 0) d = disp_at(a.dL, (size_t)y * a.w + xi);
        const bool ok = xi >= 0 && d < a.dmax && lr_valid(a, xi, y, d);
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, ok);
        if (m) {
          left = __shfl_sync(0xFFFFFFFFu, d, __ffs(m) - 1);
          break;
        }
      }
      for (int xs = x + 1; xs < a.w; xs += 32) {
        const int xi = xs + lane;
        int d = -1;
        if (xi < a.w) d = disp_at(a.dL, (size_t)y * a.w + xi);
        const bool ok = xi < a.w && d < a.dmax && lr_valid(a, xi, y, d);
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, ok);
        if (m) {
          right = __shfl_sync(0xFFFFFFFFu, d, __ffs(m) - 1);
          break;
        }
      }
      if (left >= 0 && right >= 0) best = min(left, right);
      else if (left >= 0) best = left;
      else if (right >= 0) best = right;
      else best = 0;
    }
    if (lane == 0) a.out[(size_t)y * a.w + x] = best;
    __syncwarp();
  }

  if (a.finalize) {
    for (int p = threadIdx.x; p < kTX * TY; p += blockDim.x) {
      const int tx = p & (kTX - 1), ty = p / kTX;
      const int x = x0 + tx, y = y0 + ty;
      if (x < a.w && y < a.h) {
        const size_t i = (size_t)y * a.w + x;
        a.dL[i] = disp_at(a.dL, i);
        a.dR[i] = disp_at(a.dR, i);
      }
    }
  }
}

size_t tile_bytes(int R, int hist_stride, int ty) { return tile_layout(R, hist_stride, ty).bytes; }

// Refinement words of a view (the plain form's pre-pass): one warp per row walks it in 32-pixel segments,
// left to right and then right to left. Left to right: each pixel's colour word (its RGB through the
// colour table), WTA disparity and left/right check give its word; an invalid pixel's byte 3 holds the
// nearest valid disparity to its left (0 before the row's first valid pixel, whose position the warp
// keeps). Right to left: an invalid pixel's byte 3 becomes the fallback of that value and the nearest
// valid disparity to its right, carried along the row and, inside a segment, taken from the ballot of the
// segment's valid lanes. Each lane reads back only the words it wrote. The loads (and left/right checks)
// of kNS segments are issued together.
constexpr int kNS = 8;

__global__ void __launch_bounds__(256) refine_words_kernel(const RefineArgs a, uint32_t *words) {
  const int lane = threadIdx.x & 31;
  const int y = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (y >= a.h) return;
  const size_t row = (size_t)y * a.w;
  const uint8_t *rgb = a.rgb + (size_t)y * a.pitch;
  int carry = -1;   // the last valid disparity left of the segment
  int first = a.w;  // the row's first valid pixel
  for (int xb = 0; xb < a.w; xb += 32 * kNS) {
    int d[kNS];
    uint32_t key[kNS];
    bool ok[kNS];
#pragma unroll
    for (int u = 0; u < kNS; ++u) {
      const int x = xb + 32 * u + lane;
      d[u] = a.dmax;
      key[u] = 0u;
      if (x < a.w) {
        d[u] = disp_at(a.dL, row + x);
        key[u] = ((uint32_t)rgb[3 * x] << 16) | ((uint32_t)rgb[3 * x + 1] << 8) | (uint32_t)rgb[3 * x + 2];
      }
    }
#pragma unroll
    for (int u = 0; u < kNS; ++u) {
      const int x = xb + 32 * u + lane;
      ok[u] = d[u] < a.dmax && lr_valid(a, x, y, d[u]);  // d == dmax outside the row
      if (x < a.w) key[u] = __ldg(a.table + key[u]);
    }
#pragma unroll
    for (int u = 0; u < kNS; ++u) {
      const int x = xb + 32 * u + lane;
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, ok[u]);
      const uint32_t below = m & ((1u << lane) - 1u);  // valid lanes strictly left of this one
      const int dl = __shfl_sync(0xFFFFFFFFu, d[u], below ? 31 - __clz(below) : 0);
      const int left = below ? dl : carry;
      if (m != 0u && first == a.w) first = xb + 32 * u + __ffs(m) - 1;
      if (a.tile_cnt != nullptr) {  // the segment's invalid pixels, to the count of its block
        const int nbad = __popc(__ballot_sync(0xFFFFFFFFu, x < a.w) & ~m);
        if (lane == 0 && nbad > 0)
          atomicAdd(a.tile_cnt + (y / a.tile_h) * ((a.w + kTX - 1) / kTX) + (xb + 32 * u) / kTX, nbad);
      }
      if (x < a.w) words[row + x] = refine_word(key[u], ok[u], (uint32_t)(ok[u] ? d[u] : max(left, 0)));
      if (m) carry = __shfl_sync(0xFFFFFFFFu, d[u], 31 - __clz(m));
    }
  }
  carry = -1;  // the first valid disparity right of the segment
  for (int xb = ((a.w - 1) / (32 * kNS)) * (32 * kNS); xb >= 0; xb -= 32 * kNS) {
    uint32_t wv[kNS];
#pragma unroll
    for (int u = 0; u < kNS; ++u) {
      const int x = xb + 32 * u + lane;
      wv[u] = x < a.w ? words[row + x] : 0u;
    }
#pragma unroll
    for (int u = kNS - 1; u >= 0; --u) {
      const int x = xb + 32 * u + lane;
      const bool valid = (wv[u] & kValidBit) != 0u;
      const int vd = (int)(wv[u] >> 24);
      const uint32_t m = __ballot_sync(0xFFFFFFFFu, valid);
      const uint32_t above = lane == 31 ? 0u : m & (0xFFFFFFFEu << lane);  // valid lanes strictly right
      const int dr = __shfl_sync(0xFFFFFFFFu, vd, above ? __ffs(above) - 1 : 0);
      const int right = above ? dr : carry;
      if (x < a.w && !valid) {
        const bool has_left = x > first;  // vd is the nearest valid disparity to the left
        const int f = has_left && right >= 0 ? min(vd, right) : has_left ? vd : right >= 0 ? right : 0;
        words[row + x] = (wv[u] & kLabMask) | ((uint32_t)f << 24);
      }
      if (m) carry = __shfl_sync(0xFFFFFFFFu, vd, __ffs(m) - 1);
    }
  }
}

constexpr int kRFast = 15;  // the radius with an unrolled window walk (the paper's setting)

// Blocks of kTX x TY: 32 rows where the grid fills the GPU (fewer staged halo entries per output pixel),
// kShortTY rows on images too small for that (more CTAs).
constexpr int kShortTY = 8;

// The blocks in decreasing order of their invalid pixels (buckets of 8; any order within a bucket): CTAs
// are dispatched in index order, so the blocks that take longest start first instead of setting the tail.
// Every block appears exactly once. One CTA.
constexpr int kOrderBuckets = kTX * kTY / 8 + 1;

__global__ void __launch_bounds__(1024) order_tiles_kernel(const int *cnt, int n, int *order) {
  __shared__ int hist[kOrderBuckets], base[kOrderBuckets];
  for (int i = threadIdx.x; i < kOrderBuckets; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) atomicAdd(&hist[min(cnt[i] >> 3, kOrderBuckets - 1)], 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    int run = 0;
    for (int b = kOrderBuckets - 1; b >= 0; --b) {
      base[b] = run;
      run += hist[b];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) order[atomicAdd(&base[min(cnt[i] >> 3, kOrderBuckets - 1)], 1)] = i;
}

template <int RT, int TY>
__global__ void __launch_bounds__(kThreadsR) refine_kernel(const RefineArgs a, const uint32_t *Ec, const uint32_t *Es) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int lin = (int)(blockIdx.y * gridDim.x + blockIdx.x);
  const int t = a.tile_order != nullptr ? a.tile_order[lin] : lin;
  load_vote_tables(Ec, Es, a.R, smem);
  refine_tile<RT, TY>(a, (t % (int)gridDim.x) * kTX, (t / (int)gridDim.x) * TY, smem, smem + table_words(a.R));
}

template <int TY>
cudaError_t launch_refine_ty(const RefineArgs &a, const bsm_ctx *ctx, cudaStream_t s) {
  const size_t smem = table_words(a.R) * 4 + tile_bytes(a.R, a.hist_stride, TY);
  auto kern = a.R == kRFast ? refine_kernel<kRFast, TY> : refine_kernel<0, TY>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.w + kTX - 1) / kTX, (a.h + TY - 1) / TY);
  kern<<<grid, kThreadsR, smem, s>>>(a, ctx->vote_ec, ctx->vote_es);
  return cudaGetLastError();
}

// Batched refinement: persistent CTAs take (pair, block) tickets.
template <int RT>
__global__ void __launch_bounds__(kThreadsR) refine_batch_kernel(BatchHeader *hdr, const BatchPair *pairs,
                                                               const uint32_t *Ec, const uint32_t *Es,
                                                               const uint32_t *table, int tol, int R,
                                                               int hist_stride) {
  extern __shared__ __align__(16) uint32_t smem[];
  __shared__ int s_ticket;
  load_vote_tables(Ec, Es, R, smem);
  const int total = hdr->total[3], count = hdr->count;
  for (;;) {
    __syncthreads();  // the previous block is done with shared memory
    if (threadIdx.x == 0) s_ticket = (int)atomicAdd(&hdr->counters[3], 1u);
    __syncthreads();
    const int tk = s_ticket;
    if (tk >= total) return;
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (pairs[mid].ref_base <= tk) lo = mid;
      else hi = mid - 1;
    }
    const BatchPair &p = pairs[lo];
    const int r = tk - p.ref_base, ty = r / p.ref_tx, tx = r - ty * p.ref_tx;
    RefineArgs a{p.rgb[0], p.plane[0], table, p.disp[0], p.disp[1], p.out, p.w, p.h, p.pitch, p.dmax,
                 tol, R, hist_stride, true, nullptr};
    refine_tile<RT, kTY>(a, tx * kTX, ty * kTY, smem, smem + table_words(R));
  }
}

}  // namespace

cudaError_t launch_refine(const bsm_ctx *ctx, const uint8_t *rgb, int pitch, const int32_t *dL, const int32_t *dR,
                          int w, int h, int dmax, int32_t *out, uint32_t *words, cudaStream_t s) {
  // The plain form never writes dL or dR (finalize is off), so the const inputs stay untouched.
  RefineArgs a{rgb, nullptr, ctx->color_table, const_cast<int32_t *>(dL), const_cast<int32_t *>(dR), out, w, h, pitch,
               dmax, ctx->p.lr_tol, ctx->p.vote_radius, dmax, false, words, nullptr, nullptr, kTY};
  const int tiles_x = (w + kTX - 1) / kTX;
  const bool tall = (long long)tiles_x * ((h + kTY - 1) / kTY) >= 4LL * ctx->sms;
  a.tile_h = tall ? kTY : kShortTY;
  const int ntiles = tiles_x * ((h + a.tile_h - 1) / a.tile_h);
  if (words != nullptr) {
    if (ctx->refine_tiles != nullptr && ntiles <= kMaxRefineTiles) {
      a.tile_cnt = ctx->refine_tiles;
      cudaError_t e0 = cudaMemsetAsync(a.tile_cnt, 0, sizeof(int) * (size_t)ntiles, s);
      if (e0 != cudaSuccess) return e0;
    }
    refine_words_kernel<<<(h + 7) / 8, 256, 0, s>>>(a, words);
    cudaError_t e0 = cudaGetLastError();
    if (e0 != cudaSuccess) return e0;
    if (a.tile_cnt != nullptr) {
      int *order = ctx->refine_tiles + kMaxRefineTiles;
      order_tiles_kernel<<<1, 1024, 0, s>>>(a.tile_cnt, ntiles, order);
      e0 = cudaGetLastError();
      if (e0 != cudaSuccess) return e0;
      a.tile_order = order;
    }
  }
  return tall ? launch_refine_ty<kTY>(a, ctx, s) : launch_refine_ty<kShortTY>(a, ctx, s);
}

cudaError_t prepare_refine_batch(const bsm_ctx *ctx, int *grid) {
  const int R = ctx->p.vote_radius, hs = ctx->p.dmax;
  const size_t smem = table_words(R) * 4 + tile_bytes(R, hs, kTY);
  auto kern = R == kRFast ? refine_batch_kernel<kRFast> : refine_batch_kernel<0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreadsR, smem);
  *grid = max(1, per_sm) * ctx->sms;
  return e;
}

cudaError_t launch_refine_batch(const bsm_ctx *ctx, BatchHeader *hdr, const BatchPair *pairs, int grid,
                                cudaStream_t s) {
  const int R = ctx->p.vote_radius, hs = ctx->p.dmax;
  const size_t smem = table_words(R) * 4 + tile_bytes(R, hs, kTY);
  auto kern = R == kRFast ? refine_batch_kernel<kRFast> : refine_batch_kernel<0>;
  kern<<<grid, kThreadsR, smem, s>>>(hdr, pairs, ctx->vote_ec, ctx->vote_es, ctx->color_table, ctx->p.lr_tol, R, hs);
  return cudaGetLastError();
}

}  // namespace bsm
