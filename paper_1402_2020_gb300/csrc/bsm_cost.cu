// Fused Eq. 8 cost + square-window box aggregation + Eq. 1 winner-take-all, for both views.
//
// blockIdx.z selects the reference view: 0 = left (match x - d), 1 = right (match x + d).
// A CTA owns 32 - 2r consecutive output columns (r = WIN / 2) and a band of rows; lane l of every
// warp owns column x0 + l (the outer r lanes on each side only feed the horizontal window), and warp
// k owns disparities [8k, 8k + 8). The CTA walks down its band one row at a time:
//   - the reference row's B and Phi for the 32 columns and the other view's B row for the
//     32 + dmax - 1 columns any of them can match are staged in shared memory;
//   - each thread computes C(x, y, d) = popc((B_ref ^ B_other) & Phi_ref) for its 8 disparities
//     (a match outside the image costs n), two 16-bit costs per 32-bit register;
//   - vertical box sums run in registers over a ring of the last WIN rows (V += C_new - C_old);
//   - the horizontal box sum takes V from the neighbouring lanes with warp shuffles;
//   - each thread reduces its 8 aggregated costs to a key (A << 10 | d), whose minimum over the
//     warps gives the smallest d with the minimum cost; the cost volume never reaches HBM unless
//     the caller asks for it.
// For n = 256 a lane reads the two 16-byte halves of a descriptor in an order that depends on bit 2
// of its lane index (both for the reference and the other view), which keeps every 128-bit shared
// load conflict free; the popcount sum does not depend on word order.
#include "bsm_internal.cuh"

namespace bsm {
namespace {

constexpr int kDC = 8;  // disparities per thread
constexpr int kDP = kDC / 2;

struct CostArgs {
  const uint32_t *B[2];    // reference descriptors per direction
  const uint32_t *Phi[2];  // reference masks per direction
  const uint32_t *O[2];    // other view's descriptors per direction
  int32_t *disp[2];
  uint16_t *cost;          // optional, direction 0 only
  int w, h, dmax, rows;
};

template <int NW>
__device__ __forceinline__ void load_desc(const uint32_t *p, int lane, uint32_t (&v)[NW]) {
  if constexpr (NW == 8) {
    const int q = (lane >> 2) & 1;
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

template <int NW, int WIN>
__global__ void __launch_bounds__(1024, 1) cost_wta_kernel(const CostArgs a) {
  constexpr int R = WIN / 2;
  constexpr int OUTC = 32 - 2 * R;
  constexpr int NBITS = 32 * NW;
  __shared__ __align__(16) uint32_t sref[2][32 * NW];
  __shared__ __align__(16) uint32_t soth[(32 + kMaxDmax - 1) * NW];
  __shared__ uint32_t skey[32][32];

  const int dir = blockIdx.z;
  const uint32_t *__restrict__ Bref = dir == 0 ? a.B[0] : a.B[1];
  const uint32_t *__restrict__ Phiref = dir == 0 ? a.Phi[0] : a.Phi[1];
  const uint32_t *__restrict__ Both = dir == 0 ? a.O[0] : a.O[1];
  int32_t *__restrict__ disp = dir == 0 ? a.disp[0] : a.disp[1];
  const int w = a.w, h = a.h, dmax = a.dmax;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int x0 = blockIdx.x * OUTC - R;  // column of lane 0
  const int x = x0 + lane;
  const int yb = blockIdx.y * a.rows;
  const int ye = min(h, yb + a.rows);
  const int d0 = warp * kDC;
  const int ox0 = dir == 0 ? x0 - (dmax - 1) : x0;  // first staged column of the other view
  const int nocols = 32 + dmax - 1;
  const bool col_in = x >= 0 && x < w;
  const bool out_lane = lane >= R && lane < 32 - R && col_in;

  uint32_t ring[WIN > 1 ? WIN : 1][kDP];
  uint32_t V[kDP];
#pragma unroll
  for (int j = 0; j < kDP; ++j) {
    V[j] = 0;
#pragma unroll
    for (int s = 0; s < (WIN > 1 ? WIN : 1); ++s) ring[s][j] = 0;
  }

  for (int y = yb - R; y < ye + R; ++y) {
    const bool row_in = y >= 0 && y < h;
    __syncthreads();
    if (row_in) {
      const uint32_t *rB = Bref + (size_t)y * w * NW;
      const uint32_t *rP = Phiref + (size_t)y * w * NW;
      for (int i = threadIdx.x; i < 32 * NW; i += blockDim.x) {
        const int gx = x0 + i / NW;
        const bool in = gx >= 0 && gx < w;
        sref[0][i] = in ? __ldg(rB + (ptrdiff_t)x0 * NW + i) : 0u;
        sref[1][i] = in ? __ldg(rP + (ptrdiff_t)x0 * NW + i) : 0u;
      }
      const uint32_t *rO = Both + (size_t)y * w * NW;
      for (int i = threadIdx.x; i < nocols * NW; i += blockDim.x) {
        const int gx = ox0 + i / NW;
        soth[i] = (gx >= 0 && gx < w) ? __ldg(rO + (ptrdiff_t)ox0 * NW + i) : 0u;
      }
    }
    __syncthreads();

    uint32_t C[kDP];
#pragma unroll
    for (int j = 0; j < kDP; ++j) C[j] = 0;
    if (row_in && col_in) {
      uint32_t b[NW], m[NW];
      load_desc<NW>(&sref[0][lane * NW], lane, b);
      load_desc<NW>(&sref[1][lane * NW], lane, m);
#pragma unroll
      for (int dd = 0; dd < kDC; ++dd) {
        const int d = d0 + dd;
        if (d < dmax) {
          const int idx = dir == 0 ? lane + (dmax - 1) - d : lane + d;
          uint32_t o[NW];
          load_desc<NW>(&soth[idx * NW], lane, o);
          uint32_t c = 0;
#pragma unroll
          for (int j = 0; j < NW; ++j) c += __popc((b[j] ^ o[j]) & m[j]);
          const int xo = dir == 0 ? x - d : x + d;
          if (xo < 0 || xo >= w) c = NBITS;
          C[dd >> 1] |= c << (16 * (dd & 1));
        }
      }
    }

    // vertical box sum over the last WIN rows
    if constexpr (WIN > 1) {
#pragma unroll
      for (int j = 0; j < kDP; ++j) {
        V[j] = V[j] + C[j] - ring[0][j];
#pragma unroll
        for (int s = 0; s < WIN - 1; ++s) ring[s][j] = ring[s + 1][j];
        ring[WIN - 1][j] = C[j];
      }
    } else {
#pragma unroll
      for (int j = 0; j < kDP; ++j) V[j] = C[j];
    }

    const int yo = y - R;
    if (yo >= yb) {
      uint32_t A[kDP];
#pragma unroll
      for (int j = 0; j < kDP; ++j) {
        A[j] = V[j];
#pragma unroll
        for (int s = 1; s <= R; ++s)
          A[j] += __shfl_up_sync(0xFFFFFFFFu, V[j], s) + __shfl_down_sync(0xFFFFFFFFu, V[j], s);
      }
      uint32_t key = 0xFFFFFFFFu;
#pragma unroll
      for (int dd = 0; dd < kDC; ++dd) {
        const int d = d0 + dd;
        if (d < dmax) {
          const uint32_t av = (A[dd >> 1] >> (16 * (dd & 1))) & 0xFFFFu;
          key = min(key, (av << 10) | (uint32_t)d);
          if (dir == 0 && a.cost != nullptr && out_lane) a.cost[((size_t)yo * w + x) * dmax + d] = (uint16_t)av;
        }
      }
      skey[warp][lane] = key;
      __syncthreads();
      if (warp == 0) {
        uint32_t best = skey[0][lane];
        for (int k = 1; k < nwarps; ++k) best = min(best, skey[k][lane]);
        if (out_lane) disp[(size_t)yo * w + x] = (int32_t)(best & 1023u);
      }
    }
  }
}

template <int NW, int WIN>
cudaError_t launch_t(const CostArgs &a, cudaStream_t s) {
  constexpr int OUTC = 32 - 2 * (WIN / 2);
  const int nwarps = (a.dmax + kDC - 1) / kDC;
  dim3 grid((a.w + OUTC - 1) / OUTC, (a.h + a.rows - 1) / a.rows, 2);
  cost_wta_kernel<NW, WIN><<<grid, nwarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <int NW>
cudaError_t launch_win(int win, const CostArgs &a, cudaStream_t s) {
  switch (win) {
    case 1: return launch_t<NW, 1>(a, s);
    case 3: return launch_t<NW, 3>(a, s);
    case 5: return launch_t<NW, 5>(a, s);
    case 7: return launch_t<NW, 7>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_cost_wta(const bsm_ctx *ctx, const uint32_t *BL, const uint32_t *PhiL, const uint32_t *BR,
                            const uint32_t *PhiR, int w, int h, int dmax, int32_t *dL, int32_t *dR, uint16_t *cost,
                            cudaStream_t s) {
  CostArgs a{};
  a.B[0] = BL; a.Phi[0] = PhiL; a.O[0] = BR; a.disp[0] = dL;
  a.B[1] = BR; a.Phi[1] = PhiR; a.O[1] = BL; a.disp[1] = dR;
  a.cost = cost;
  a.w = w; a.h = h; a.dmax = dmax;
  a.rows = h >= 512 ? 64 : 32;
  switch (ctx->nw) {
    case 1: return launch_win<1>(ctx->p.agg_window, a, s);
    case 2: return launch_win<2>(ctx->p.agg_window, a, s);
    case 4: return launch_win<4>(ctx->p.agg_window, a, s);
    case 8: return launch_win<8>(ctx->p.agg_window, a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace bsm
