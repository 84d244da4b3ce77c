// Colour table: for every 24-bit RGB colour, integer CIELAB (the colour space of Eq. 5's SAD) and
// the intensity I of Eq. 3, packed into one word so that the describe and refine kernels fetch both
// with a single load per pixel.
//
// Definition: sRGB with the IEC 61966-2-1 transfer curve, the sRGB -> XYZ matrix for D65, the D65
// white taken as that matrix's row sums, CIE 1976 f(t) with the (6/29)^3 break,
// L = 116 f(Y) - 16, a = 500 (f(X) - f(Y)), b = 200 (f(Y) - f(Z)), each rounded half away from
// zero. The transfer curve's 256 values arrive precomputed from the host; every other operation is
// written with explicit round-to-nearest intrinsics so that no fused multiply-add changes a result.
#include "bsm_internal.cuh"

namespace bsm {
namespace {

__device__ __forceinline__ double cie_f(double t) {
  const double delta = 6.0 / 29.0;
  const double delta3 = __dmul_rn(__dmul_rn(delta, delta), delta);
  if (t > delta3) return cbrt(t);
  const double slope = __dmul_rn(__dmul_rn(3.0, delta), delta);
  return __dadd_rn(__ddiv_rn(t, slope), 4.0 / 29.0);
}

__device__ __forceinline__ double mix3(double c0, double x0, double c1, double x1, double c2, double x2) {
  return __dadd_rn(__dadd_rn(__dmul_rn(c0, x0), __dmul_rn(c1, x1)), __dmul_rn(c2, x2));
}

__global__ void __launch_bounds__(256) color_table_kernel(uint32_t *__restrict__ table,
                                                          const double *__restrict__ lin) {
  const uint32_t idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (1u << 24)) return;
  const int R = (int)(idx >> 16), G = (int)((idx >> 8) & 255u), B = (int)(idx & 255u);
  const double r = lin[R], g = lin[G], b = lin[B];
  const double X = mix3(0.4124564, r, 0.3575761, g, 0.1804375, b);
  const double Y = mix3(0.2126729, r, 0.7151522, g, 0.0721750, b);
  const double Z = mix3(0.0193339, r, 0.1191920, g, 0.9503041, b);
  const double Xn = 0.4124564 + 0.3575761 + 0.1804375;
  const double Yn = 0.2126729 + 0.7151522 + 0.0721750;
  const double Zn = 0.0193339 + 0.1191920 + 0.9503041;
  const double fx = cie_f(__ddiv_rn(X, Xn));
  const double fy = cie_f(__ddiv_rn(Y, Yn));
  const double fz = cie_f(__ddiv_rn(Z, Zn));
  const long L = lround(__dsub_rn(__dmul_rn(116.0, fy), 16.0));
  const long A = lround(__dmul_rn(500.0, __dsub_rn(fx, fy)));
  const long Bb = lround(__dmul_rn(200.0, __dsub_rn(fy, fz)));
  const uint32_t I = (uint32_t)((77 * R + 150 * G + 29 * B + 128) >> 8);
  table[idx] = (uint32_t)L | ((uint32_t)(A + 128) << 8) | ((uint32_t)(Bb + 128) << 16) | (I << 24);
}

}  // namespace

cudaError_t build_color_table(uint32_t *table, const double *lin256, cudaStream_t s) {
  color_table_kernel<<<(1u << 24) / 256, 256, 0, s>>>(table, lin256);
  return cudaGetLastError();
}

}  // namespace bsm
