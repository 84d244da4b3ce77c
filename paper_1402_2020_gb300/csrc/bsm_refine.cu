// Left/right check and voting refinement of the left disparity map (Sec. 3, Eq. 9-10).
//
// One CTA covers a 32 x 8 block of output pixels. It stages, for the block plus a halo of R pixels,
// each pixel's CIELAB word (from the colour table) and its disparity if that pixel passes the
// left/right check (-1 otherwise), together with the two integer vote tables. Valid pixels keep
// their disparity. Invalid pixels are collected into a list that the CTA's warps share: a warp takes
// one invalid pixel at a time; lane l owns window column l (and l + 32 when 2R+1 > 32) and walks
// down its rows, summing each valid neighbour's vote floor(Ec[c] * Es[e2] / 2^15) in a register
// while consecutive voters share a disparity and adding the run to a per-warp shared histogram over
// d when the disparity changes (disparities are piecewise smooth, so runs are long and shared
// atomics few). The warp then takes the smallest d with the largest weight (Eq. 9). When no vote
// is positive the warp scans the row outward, 32 positions per step, for the nearest valid pixels
// on each side.
#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kTX = 32, kTY = 8;
constexpr int kWarps = kTX * kTY / 32;

struct RefineArgs {
  const uint8_t *rgb;
  const uint32_t *table;
  const int32_t *dL;
  const int32_t *dR;
  const uint32_t *Ec;
  const uint32_t *Es;
  int32_t *out;
  int w, h, pitch, dmax, tol, R;
};

__device__ __forceinline__ uint32_t lab_sad(uint32_t a, uint32_t b) {
  return __dp4a(__vabsdiffu4(a, b), 0x00010101u, 0u);
}

__device__ __forceinline__ bool lr_valid(const RefineArgs &a, int x, int y, int d) {
  const int xr = x - d;
  if (xr < 0 || xr >= a.w) return false;
  const int dr = __ldg(a.dR + (size_t)y * a.w + xr);
  return abs(d - dr) <= a.tol;
}

__global__ void __launch_bounds__(kTX *kTY) refine_kernel(const RefineArgs a) {
  extern __shared__ __align__(16) uint32_t smem[];
  const int R = a.R, side = 2 * R + 1;
  const int tp = kTX + 2 * R, th = kTY + 2 * R;
  const int ne = 2 * R * R + 1;
  uint32_t *sEc = smem;                              // kMaxSad + 1
  uint32_t *sEs = sEc + (kMaxSad + 1);               // ne
  uint32_t *slab = sEs + ne;                         // th * tp
  uint32_t *shist = slab + th * tp;                  // kWarps * dmax
  int16_t *sd = reinterpret_cast<int16_t *>(shist + kWarps * a.dmax);  // th * tp
  __shared__ int s_count;
  __shared__ int16_t s_list[kTX * kTY];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int x0 = blockIdx.x * kTX, y0 = blockIdx.y * kTY;
  if (threadIdx.x == 0) s_count = 0;
  for (int i = threadIdx.x; i <= kMaxSad; i += blockDim.x) sEc[i] = __ldg(a.Ec + i);
  for (int i = threadIdx.x; i < ne; i += blockDim.x) sEs[i] = __ldg(a.Es + i);
  for (int i = threadIdx.x; i < th * tp; i += blockDim.x) {
    const int ty = i / tp, tx = i - ty * tp;
    const int gx = x0 + tx - R, gy = y0 + ty - R;
    int16_t dv = -1;
    uint32_t lab = 0;
    if (gx >= 0 && gx < a.w && gy >= 0 && gy < a.h) {
      const uint8_t *px = a.rgb + (size_t)gy * a.pitch + 3 * gx;
      lab = __ldg(a.table + (((uint32_t)px[0] << 16) | ((uint32_t)px[1] << 8) | (uint32_t)px[2])) & kLabMask;
      const int d = __ldg(a.dL + (size_t)gy * a.w + gx);
      if (d >= 0 && d < a.dmax && lr_valid(a, gx, gy, d)) dv = (int16_t)d;
    }
    slab[i] = lab;
    sd[i] = dv;
  }
  __syncthreads();

  {
    const int tx = threadIdx.x & (kTX - 1), ty = threadIdx.x / kTX;
    const int x = x0 + tx, y = y0 + ty;
    if (x < a.w && y < a.h) {
      const int dv = sd[(ty + R) * tp + tx + R];
      if (dv >= 0) a.out[(size_t)y * a.w + x] = dv;
      else s_list[atomicAdd(&s_count, 1)] = (int16_t)threadIdx.x;
    }
  }
  __syncthreads();

  const int count = s_count;
  uint32_t *hist = shist + warp * a.dmax;
  for (int it = warp; it < count; it += kWarps) {
    const int t = s_list[it];
    const int tx = t & (kTX - 1), ty = t / kTX;
    const int x = x0 + tx, y = y0 + ty;
    for (int d = lane; d < a.dmax; d += 32) hist[d] = 0;
    __syncwarp();
    const uint32_t labx = slab[(ty + R) * tp + tx + R];
    for (int wx = lane; wx < side; wx += 32) {
      const int dx2 = (wx - R) * (wx - R);
      const int16_t *dcol = sd + ty * tp + tx + wx;     // window row 0 of this column
      const uint32_t *lcol = slab + ty * tp + tx + wx;
      int run_d = -1;
      uint32_t run = 0;
      for (int wy = 0; wy < side; ++wy) {
        const int dv = dcol[wy * tp];
        if (dv >= 0) {
          const int dy = wy - R;
          const uint32_t c = lab_sad(labx, lcol[wy * tp]);
          const uint32_t v = (sEc[c] * sEs[dx2 + dy * dy]) >> kVoteShift;
          if (dv != run_d) {
            if (run) atomicAdd(&hist[run_d], run);
            run_d = dv;
            run = 0;
          }
          run += v;
        }
      }
      if (run) atomicAdd(&hist[run_d], run);
    }
    __syncwarp();
    uint32_t bv = 0;
    int bd = 0x7FFFFFFF;
    for (int d = lane; d < a.dmax; d += 32) {
      const uint32_t hv = hist[d];
      if (hv > bv) {
        bv = hv;
        bd = d;
      }
    }
    const uint32_t gmax = __reduce_max_sync(0xFFFFFFFFu, bv);
    int best;
    if (gmax > 0) {
      best = (int)__reduce_min_sync(0xFFFFFFFFu, (unsigned)(bv == gmax ? bd : 0x7FFFFFFF));
    } else {
      // no positive vote: nearest valid disparities on the row
      int left = -1, right = -1;
      for (int xs = x - 1; xs >= 0; xs -= 32) {
        const int xi = xs - lane;
        int d = -1;
        if (xi >= 0) d = __ldg(a.dL + (size_t)y * a.w + xi);
        const bool ok = xi >= 0 && d >= 0 && d < a.dmax && lr_valid(a, xi, y, d);
        const uint32_t m = __ballot_sync(0xFFFFFFFFu, ok);
        if (m) {
          left = __shfl_sync(0xFFFFFFFFu, d, __ffs(m) - 1);
          break;
        }
      }
      for (int xs = x + 1; xs < a.w; xs += 32) {
        const int xi = xs + lane;
        int d = -1;
        if (xi < a.w) d = __ldg(a.dL + (size_t)y * a.w + xi);
        const bool ok = xi < a.w && d >= 0 && d < a.dmax && lr_valid(a, xi, y, d);
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
}

}  // namespace

size_t refine_smem_bytes(int R, int dmax) {
  const int tp = kTX + 2 * R, th = kTY + 2 * R;
  const size_t words = (kMaxSad + 1) + (2 * R * R + 1) + (size_t)th * tp + (size_t)kWarps * dmax;
  return words * 4 + (size_t)th * tp * 2;
}

cudaError_t launch_refine(const bsm_ctx *ctx, const uint8_t *rgb, int pitch, const int32_t *dL, const int32_t *dR,
                          int w, int h, int dmax, int32_t *out, cudaStream_t s) {
  RefineArgs a{rgb, ctx->color_table, dL, dR, ctx->vote_ec, ctx->vote_es, out, w, h, pitch, dmax,
               ctx->p.lr_tol, ctx->p.vote_radius};
  const size_t smem = refine_smem_bytes(a.R, dmax);
  cudaError_t e = cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((w + kTX - 1) / kTX, (h + kTY - 1) / kTY);
  refine_kernel<<<grid, kTX * kTY, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace bsm
