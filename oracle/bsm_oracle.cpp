// Oracle for Binary Stereo Matching (Zhang, Li, Li, Hu, Sun, Yang, "Binary Stereo Matching", Sec. 3).
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, single-threaded CPU statement of what the
// method computes, written from the paper's equations. Only the test suite, the package smoke check
// and the benchmark's CPU-baseline leg may load it. It shares no code, header, table or constant
// generator with the CUDA library, and the library never calls it.
//
// Every function follows the definition directly: direct loops, no sliding sums, no blocking, no
// reordering beyond what the equation states. A library primitive (std::sort, std::exp, std::cbrt,
// std::pow, __builtin_popcount) may serve as one step.
//
// Readings of what the paper leaves open (each one is listed with its reason in the design notes):
//   R1  intensity I(x) of Eq. 3 is integer luma Y = (77 R + 150 G + 29 B + 128) >> 8;
//   R2  CIELAB of Eq. 5 is sRGB (IEC 61966-2-1 transfer curve), the sRGB->XYZ D65 matrix, the D65
//       white given by that matrix's row sums, the CIE f(t) with the (6/29)^3 break, each of L, a, b
//       rounded to the nearest integer with halves away from zero;
//   R3  sampling positions outside the image are clamped to the border (replicate);
//   R4  T of Eq. 6 ("quarter smallest value") is the k-th smallest weight, 1-based, k = n/4 by default;
//   R5  Eq. 8 is read as (B(x) XOR B(x_d)) AND Phi(x), the mask of the reference pixel only;
//       a match position outside the image costs n;
//   R6  window aggregation (not in the paper; window 1 is the identity) is the sum over in-image
//       neighbours of a square window;
//   R7  Eq. 1 keeps the smallest d on ties;
//   R8  the left/right check accepts |d_L(x) - d_R(x - d_L(x))| <= tol with x - d_L(x) >= 0;
//   R9  Eq. 10 uses integer votes floor(Ec[c] * Es[e2] / 2^15) with Ec[c] = round(32768 exp(-c/lambda_c)),
//       Es[e2] = round(32768 exp(-sqrt(e2)/lambda_e)), c the CIELAB SAD of Eq. 5, e2 = dx^2 + dy^2,
//       over valid pixels of a (2R+1)^2 window; Eq. 9 keeps the smallest d on ties; if no vote is
//       positive the nearest valid disparities to the left and right on the row are used (their
//       minimum; the one that exists; else 0).
//   R10 the global optimisation the paper names as future work (Sec. 5) is read as semi-global
//       aggregation of the cost volume along straight image paths with penalties P1 (disparity change
//       of 1) and P2 (larger change), the disparity being the smallest d with the minimum path sum.
//
// Parity against the paper's own numbers is unpinned for every function here: the paper prints no
// worked example or intermediate value. Each function is pinned instead by closed forms, invariants,
// special cases and brute force in the test suite.

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

namespace {

// Sec. 3 / Eq. 3: I(x). Reading R1.
inline int intensity(const uint8_t *px) {
  return (77 * px[0] + 150 * px[1] + 29 * px[2] + 128) >> 8;
}

// sRGB transfer curve, IEC 61966-2-1, for one 8-bit channel.
double srgb_to_linear(int v) {
  const double c = v / 255.0;
  if (c <= 0.04045) return c / 12.92;
  return std::pow((c + 0.055) / 1.055, 2.4);
}

// CIE 1976 f(t) with the (6/29)^3 break.
double cie_f(double t) {
  const double delta = 6.0 / 29.0;
  if (t > delta * delta * delta) return std::cbrt(t);
  return t / (3.0 * delta * delta) + 4.0 / 29.0;
}

// Eq. 5 needs pixels in CIELAB. Reading R2.
void lab_of(int R, int G, int B, int out[3]) {
  const double r = srgb_to_linear(R);
  const double g = srgb_to_linear(G);
  const double b = srgb_to_linear(B);
  const double X = 0.4124564 * r + 0.3575761 * g + 0.1804375 * b;
  const double Y = 0.2126729 * r + 0.7151522 * g + 0.0721750 * b;
  const double Z = 0.0193339 * r + 0.1191920 * g + 0.9503041 * b;
  const double Xn = 0.4124564 + 0.3575761 + 0.1804375;
  const double Yn = 0.2126729 + 0.7151522 + 0.0721750;
  const double Zn = 0.0193339 + 0.1191920 + 0.9503041;
  const double fx = cie_f(X / Xn), fy = cie_f(Y / Yn), fz = cie_f(Z / Zn);
  out[0] = (int)std::lround(116.0 * fy - 16.0);
  out[1] = (int)std::lround(500.0 * (fx - fy));
  out[2] = (int)std::lround(200.0 * (fy - fz));
}

// SAD of Eq. 5 between two CIELAB pixels: sum over L, a, b of absolute differences.
inline int lab_sad(const int *u, const int *v) {
  return std::abs(u[0] - v[0]) + std::abs(u[1] - v[1]) + std::abs(u[2] - v[2]);
}

inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

inline int popcount32(uint32_t v) { return __builtin_popcount(v); }

// Eq. 8 for one (x, y, d): popcount((B_ref(x) XOR B_oth(x_d)) AND Phi_ref(x)); reading R5.
// dir 0: left view is the reference and x_d = x - d; dir 1: right view is the reference, x_d = x + d.
// Phioth, when given, is the other view's mask plane: the ablation that also weights by the matched
// pixel's mask, popcount((B_ref XOR B_oth) AND Phi_ref(x) AND Phi_oth(x_d)) (not the paper's Eq. 8).
uint32_t cost_at(const uint32_t *Bref, const uint32_t *Phiref, const uint32_t *Both, int w, int nw,
                 int x, int y, int d, int dir, const uint32_t *Phioth = nullptr) {
  const int xd = dir == 0 ? x - d : x + d;
  if (xd < 0 || xd >= w) return (uint32_t)(32 * nw);
  const uint32_t *b = Bref + ((size_t)y * w + x) * nw;
  const uint32_t *m = Phiref + ((size_t)y * w + x) * nw;
  const uint32_t *o = Both + ((size_t)y * w + xd) * nw;
  uint32_t c = 0;
  if (Phioth == nullptr) {
    for (int j = 0; j < nw; ++j) c += (uint32_t)popcount32((b[j] ^ o[j]) & m[j]);
  } else {
    const uint32_t *mo = Phioth + ((size_t)y * w + xd) * nw;
    for (int j = 0; j < nw; ++j) c += (uint32_t)popcount32((b[j] ^ o[j]) & m[j] & mo[j]);
  }
  return c;
}

// Window aggregation of Eq. 8's cost at (x, y, d); reading R6.
uint32_t aggregated_at(const uint32_t *Bref, const uint32_t *Phiref, const uint32_t *Both, int w, int h,
                       int nw, int win, int x, int y, int d, int dir, const uint32_t *Phioth = nullptr) {
  const int r = win / 2;
  uint32_t s = 0;
  for (int dy = -r; dy <= r; ++dy)
    for (int dx = -r; dx <= r; ++dx) {
      const int xx = x + dx, yy = y + dy;
      if (xx < 0 || xx >= w || yy < 0 || yy >= h) continue;
      s += cost_at(Bref, Phiref, Both, w, nw, xx, yy, d, dir, Phioth);
    }
  return s;
}

}  // namespace

extern "C" {

int oracle_abi_version(void) { return 1; }

// Intensity I(x) of Eq. 3 for one RGB pixel (reading R1).
int oracle_intensity(int R, int G, int B) {
  const uint8_t px[3] = {(uint8_t)R, (uint8_t)G, (uint8_t)B};
  return intensity(px);
}

// CIELAB of one RGB pixel (reading R2): out = {L, a, b}.
void oracle_lab(int R, int G, int B, int32_t *out) {
  int v[3];
  lab_of(R, G, B, v);
  out[0] = v[0];
  out[1] = v[1];
  out[2] = v[2];
}

// CIELAB (reading R2) and intensity (reading R1) of every 24-bit colour, index (R << 16) | (G << 8) | B.
void oracle_lab_all(int8_t *L, int8_t *A, int8_t *Bc, uint8_t *I) {
  for (int R = 0; R < 256; ++R)
    for (int G = 0; G < 256; ++G)
      for (int B = 0; B < 256; ++B) {
        const size_t i = ((size_t)R << 16) | ((size_t)G << 8) | (size_t)B;
        int v[3];
        lab_of(R, G, B, v);
        L[i] = (int8_t)v[0];
        A[i] = (int8_t)v[1];
        Bc[i] = (int8_t)v[2];
        const uint8_t px[3] = {(uint8_t)R, (uint8_t)G, (uint8_t)B};
        I[i] = (uint8_t)intensity(px);
      }
}

// Eq. 2-3 (descriptor B) and Eq. 5-7 (mask Phi) for every pixel of rows [y0, y1) of one view.
// rgb: h rows of pitch bytes, pixel = 3 bytes R, G, B. pairs: n entries (px, py, qx, qy), offsets from x.
// B, Phi: full-image planes [h][w][n/32]; pair i (0-based) is bit i % 32 of word i / 32, which is the
// weight 2^(i-1) of the paper's 1-based sum. Only rows [y0, y1) are written.
// Returns 0, or -1 on an argument error.
int oracle_describe(const uint8_t *rgb, int w, int h, int pitch, const int8_t *pairs, int n, int k, int y0,
                    int y1, uint32_t *B, uint32_t *Phi) {
  if (w <= 0 || h <= 0 || n <= 0 || n % 32 != 0 || k < 1 || k > n || y0 < 0 || y1 > h || y0 > y1) return -1;
  const int nw = n / 32;
  // Rows that the band's sampling pairs can reach (clamped to the image).
  int ry0 = y0, ry1 = y1 - 1;
  for (int i = 0; i < n; ++i) {
    ry0 = std::min(ry0, y0 + std::min((int)pairs[4 * i + 1], (int)pairs[4 * i + 3]));
    ry1 = std::max(ry1, y1 - 1 + std::max((int)pairs[4 * i + 1], (int)pairs[4 * i + 3]));
  }
  ry0 = clampi(ry0, 0, h - 1);
  ry1 = clampi(ry1, 0, h - 1);
  std::vector<int> lab((size_t)w * h * 3);
  std::vector<int> gray((size_t)w * h);
  for (int y = ry0; y <= ry1 && y0 < y1; ++y)
    for (int x = 0; x < w; ++x) {
      const uint8_t *px = rgb + (size_t)y * pitch + 3 * x;
      lab_of(px[0], px[1], px[2], &lab[((size_t)y * w + x) * 3]);
      gray[(size_t)y * w + x] = intensity(px);
    }
  std::vector<int> wgt(n), sorted(n);
  for (int y = y0; y < y1; ++y)
    for (int x = 0; x < w; ++x) {
      uint32_t *b = B + ((size_t)y * w + x) * nw;
      uint32_t *m = Phi + ((size_t)y * w + x) * nw;
      for (int j = 0; j < nw; ++j) b[j] = m[j] = 0;
      const int *lx = &lab[((size_t)y * w + x) * 3];
      for (int i = 0; i < n; ++i) {
        // Sampling positions p_i, q_i around x, clamped to the image (reading R3).
        const int px = clampi(x + pairs[4 * i + 0], 0, w - 1), py = clampi(y + pairs[4 * i + 1], 0, h - 1);
        const int qx = clampi(x + pairs[4 * i + 2], 0, w - 1), qy = clampi(y + pairs[4 * i + 3], 0, h - 1);
        // Eq. 3: tau = 1 iff I(p_i) > I(q_i).
        if (gray[(size_t)py * w + px] > gray[(size_t)qy * w + qx]) b[i / 32] |= 1u << (i % 32);
        // Eq. 5: w = max(SAD(x, p_i), SAD(x, q_i)).
        const int sp = lab_sad(lx, &lab[((size_t)py * w + px) * 3]);
        const int sq = lab_sad(lx, &lab[((size_t)qy * w + qx) * 3]);
        wgt[i] = std::max(sp, sq);
      }
      // T: the k-th smallest weight (reading R4).
      sorted = wgt;
      std::sort(sorted.begin(), sorted.end());
      const int T = sorted[k - 1];
      // Eq. 6-7: delta = 1 iff w <= T.
      for (int i = 0; i < n; ++i)
        if (wgt[i] <= T) m[i / 32] |= 1u << (i % 32);
    }
  return 0;
}

// Eq. 8 (with reading R5) for one (x, y, d).
uint32_t oracle_cost_at(const uint32_t *Bref, const uint32_t *Phiref, const uint32_t *Both, int w, int h, int n,
                        int x, int y, int d, int dir, const uint32_t *Phioth) {
  (void)h;
  return cost_at(Bref, Phiref, Both, w, n / 32, x, y, d, dir, Phioth);
}

// Aggregated cost A(x, y, d) for every pixel of the region [x0, x1) x [y0, y1) and d in [0, dmax):
// A is written as [y1-y0][x1-x0][dmax] (d fastest). With win = 1 this is Eq. 8's cost itself.
int oracle_aggregate(const uint32_t *Bref, const uint32_t *Phiref, const uint32_t *Both, int w, int h, int n,
                     int dmax, int win, int dir, int x0, int x1, int y0, int y1, uint32_t *A,
                     const uint32_t *Phioth) {
  if (n % 32 != 0 || win < 1 || win % 2 == 0 || dmax < 1 || x0 < 0 || x1 > w || y0 < 0 || y1 > h) return -1;
  const int nw = n / 32;
  for (int y = y0; y < y1; ++y)
    for (int x = x0; x < x1; ++x)
      for (int d = 0; d < dmax; ++d)
        A[(((size_t)(y - y0)) * (x1 - x0) + (x - x0)) * dmax + d] =
            aggregated_at(Bref, Phiref, Both, w, h, nw, win, x, y, d, dir, Phioth);
  return 0;
}

// Eq. 1 (winner-take-all, reading R7) on the aggregated cost, for the region [x0, x1) x [y0, y1).
// disp is [y1-y0][x1-x0].
int oracle_wta(const uint32_t *Bref, const uint32_t *Phiref, const uint32_t *Both, int w, int h, int n, int dmax,
               int win, int dir, int x0, int x1, int y0, int y1, int32_t *disp, const uint32_t *Phioth) {
  if (n % 32 != 0 || win < 1 || win % 2 == 0 || dmax < 1 || x0 < 0 || x1 > w || y0 < 0 || y1 > h) return -1;
  const int nw = n / 32;
  for (int y = y0; y < y1; ++y)
    for (int x = x0; x < x1; ++x) {
      uint32_t best = 0xffffffffu;
      int arg = 0;
      for (int d = 0; d < dmax; ++d) {
        const uint32_t a = aggregated_at(Bref, Phiref, Both, w, h, nw, win, x, y, d, dir, Phioth);
        if (a < best) {
          best = a;
          arg = d;
        }
      }
      disp[((size_t)(y - y0)) * (x1 - x0) + (x - x0)] = arg;
    }
  return 0;
}

// Left/right consistency check (Sec. 3, reading R8) for the left map: valid[y][x] in {0, 1}.
int oracle_lr_check(const int32_t *dL, const int32_t *dR, int w, int h, int tol, uint8_t *valid) {
  if (w <= 0 || h <= 0 || tol < 0) return -1;
  for (int y = 0; y < h; ++y)
    for (int x = 0; x < w; ++x) {
      const int d = dL[(size_t)y * w + x];
      const int xr = x - d;
      int ok = 0;
      if (xr >= 0 && xr < w) ok = std::abs(d - dR[(size_t)y * w + xr]) <= tol;
      valid[(size_t)y * w + x] = (uint8_t)ok;
    }
  return 0;
}

// Integer vote tables of reading R9: Ec[c] for c in [0, nc), Es[e2] for e2 in [0, ne).
void oracle_vote_tables(double lambda_c, double lambda_e, int nc, int ne, uint32_t *Ec, uint32_t *Es) {
  for (int c = 0; c < nc; ++c) Ec[c] = (uint32_t)std::lround(32768.0 * std::exp(-(double)c / lambda_c));
  for (int e = 0; e < ne; ++e) Es[e] = (uint32_t)std::lround(32768.0 * std::exp(-std::sqrt((double)e) / lambda_e));
}

// Eq. 9-10: voting refinement of the invalid pixels of the left map (reading R9), for the output
// region [x0, x1) x [y0, y1). rgb is the left view; dL the left WTA map; valid from the left/right
// check (both full-image); out[y - y0][x - x0] receives the refined map of the region.
int oracle_refine_region(const uint8_t *rgb, int pitch, const int32_t *dL, const uint8_t *valid, int w, int h,
                         int dmax, int R, double lambda_c, double lambda_e, int x0, int x1, int y0, int y1,
                         int32_t *out) {
  if (w <= 0 || h <= 0 || dmax < 1 || R < 0 || x0 < 0 || x1 > w || y0 < 0 || y1 > h || x0 > x1 || y0 > y1) return -1;
  // CIELAB of every pixel a window of the region can reach.
  const int lx0 = std::max(0, x0 - R), lx1 = std::min(w, x1 + R), ly0 = std::max(0, y0 - R), ly1 = std::min(h, y1 + R);
  const int lw = std::max(0, lx1 - lx0);
  std::vector<int> lab((size_t)lw * std::max(0, ly1 - ly0) * 3);
  for (int y = ly0; y < ly1; ++y)
    for (int x = lx0; x < lx1; ++x) {
      const uint8_t *px = rgb + (size_t)y * pitch + 3 * x;
      lab_of(px[0], px[1], px[2], &lab[((size_t)(y - ly0) * lw + (x - lx0)) * 3]);
    }
  auto lab_at = [&](int x, int y) { return &lab[((size_t)(y - ly0) * lw + (x - lx0)) * 3]; };
  const int nc = 3 * 255 + 1, ne = 2 * R * R + 1;
  std::vector<uint32_t> Ec(nc), Es(ne);
  oracle_vote_tables(lambda_c, lambda_e, nc, ne, Ec.data(), Es.data());
  std::vector<uint32_t> W(dmax);
  for (int y = y0; y < y1; ++y)
    for (int x = x0; x < x1; ++x) {
      const size_t i = (size_t)y * w + x;
      int32_t &o = out[(size_t)(y - y0) * (x1 - x0) + (x - x0)];
      if (valid[i]) {
        o = dL[i];
        continue;
      }
      std::fill(W.begin(), W.end(), 0u);
      for (int yy = std::max(0, y - R); yy <= std::min(h - 1, y + R); ++yy)
        for (int xx = std::max(0, x - R); xx <= std::min(w - 1, x + R); ++xx) {
          const size_t j = (size_t)yy * w + xx;
          if (!valid[j]) continue;
          const int c = lab_sad(lab_at(x, y), lab_at(xx, yy));
          const int e2 = (xx - x) * (xx - x) + (yy - y) * (yy - y);
          const uint32_t v = (uint32_t)(((uint64_t)Ec[c] * Es[e2]) >> 15);
          const int d = dL[j];
          if (d >= 0 && d < dmax) W[d] += v;
        }
      // Eq. 9: argmax over d, smallest d on ties.
      uint32_t best = 0;
      int arg = -1;
      for (int d = 0; d < dmax; ++d)
        if (W[d] > best) {
          best = W[d];
          arg = d;
        }
      if (arg < 0) {
        // No positive vote: nearest valid disparities on the row.
        int left = -1, right = -1;
        for (int xx = x - 1; xx >= 0; --xx)
          if (valid[(size_t)y * w + xx]) {
            left = dL[(size_t)y * w + xx];
            break;
          }
        for (int xx = x + 1; xx < w; ++xx)
          if (valid[(size_t)y * w + xx]) {
            right = dL[(size_t)y * w + xx];
            break;
          }
        if (left >= 0 && right >= 0) arg = std::min(left, right);
        else if (left >= 0) arg = left;
        else if (right >= 0) arg = right;
        else arg = 0;
      }
      o = arg;
    }
  return 0;
}

// Reading R10: semi-global aggregation of the cost volume C[y][x][d] along the directions
// dirs[2 i], dirs[2 i + 1] (dx, dy), i < ndirs. For each direction, pixels are visited so that p - r
// comes before p, and
//   L(p, d) = C(p, d) + min(L(p-r, d), L(p-r, d-1) + P1, L(p-r, d+1) + P1, min_k L(p-r, k) + P2)
//             - min_k L(p-r, k),
// with L(p, d) = C(p, d) where p - r is outside the image. S = sum of L over the directions (written
// to S when it is not null); disp = the smallest d with the minimum S(p, d).
int oracle_sgm(const uint16_t *C, int w, int h, int dmax, int P1, int P2, const int *dirs, int ndirs, uint32_t *S,
               int32_t *disp) {
  if (w <= 0 || h <= 0 || dmax < 1 || P1 < 0 || P2 < 0 || ndirs < 1) return -1;
  const size_t npx = (size_t)w * h;
  std::vector<int64_t> sum(npx * dmax, 0), L(npx * dmax);
  for (int r = 0; r < ndirs; ++r) {
    const int dx = dirs[2 * r], dy = dirs[2 * r + 1];
    if ((dx == 0 && dy == 0) || dx < -1 || dx > 1 || dy < -1 || dy > 1) return -1;
    for (int yi = 0; yi < h; ++yi) {
      const int y = dy >= 0 ? yi : h - 1 - yi;
      for (int xi = 0; xi < w; ++xi) {
        const int x = dx >= 0 ? xi : w - 1 - xi;
        const size_t p = (size_t)y * w + x;
        const int px = x - dx, py = y - dy;
        if (px < 0 || px >= w || py < 0 || py >= h) {
          for (int d = 0; d < dmax; ++d) L[p * dmax + d] = C[p * dmax + d];
          continue;
        }
        const int64_t *prev = &L[((size_t)py * w + px) * dmax];
        int64_t m = prev[0];
        for (int k = 1; k < dmax; ++k) m = std::min(m, prev[k]);
        for (int d = 0; d < dmax; ++d) {
          int64_t best = std::min(prev[d], m + P2);
          if (d > 0) best = std::min(best, prev[d - 1] + P1);
          if (d < dmax - 1) best = std::min(best, prev[d + 1] + P1);
          L[p * dmax + d] = C[p * dmax + d] + best - m;
        }
      }
    }
    for (size_t i = 0; i < npx * dmax; ++i) sum[i] += L[i];
  }
  for (size_t p = 0; p < npx; ++p) {
    int arg = 0;
    for (int d = 1; d < dmax; ++d)
      if (sum[p * dmax + d] < sum[p * dmax + arg]) arg = d;
    disp[p] = arg;
    if (S != nullptr)
      for (int d = 0; d < dmax; ++d) S[p * dmax + d] = (uint32_t)sum[p * dmax + d];
  }
  return 0;
}

// Eq. 9-10 over the whole image.
int oracle_refine(const uint8_t *rgb, int pitch, const int32_t *dL, const uint8_t *valid, int w, int h, int dmax,
                  int R, double lambda_c, double lambda_e, int32_t *out) {
  return oracle_refine_region(rgb, pitch, dL, valid, w, h, dmax, R, lambda_c, lambda_e, 0, w, 0, h, out);
}

}  // extern "C"
