// tet_math.cuh -- exact and filtered per-tetrahedron arithmetic of the voxelizer.
//
// Notation.  A tetrahedron V0..V3 (lattice coordinates, |X| <= 2^21) is first
// oriented so that its signed volume V6 = det[V1-V0, V2-V0, V3-V0] (Lemma 1.1's
// det(AB, AC, AD)) is positive, by swapping V2 and V3 if needed.  For a point P
// the four orientation values
//
//   lam_0 = orient(P, V1, V2, V3)   lam_1 = orient(V0, P, V2, V3)
//   lam_2 = orient(V0, V1, P, V3)   lam_3 = orient(V0, V1, V2, P)
//
// (orient(A,B,C,D) = det[B-A, C-A, D-A]) are affine in P and sum to V6.  They
// equal Theorem 1's determinants up to sign: lam_0 = D_a, lam_1 = -D_b,
// lam_2 = D_c, lam_3 = -D_d (Section 4; a row transposition flips a
// determinant's sign), so Theorem 1's closed test for a positively oriented tet
// is "all lam_m >= 0" and its strict test "all lam_m > 0".
//
// With e_m = V_m - V0 and n1 = e2 x e3, n2 = e3 x e1, n3 = e1 x e2:
//   lam_m(P) = (P - V0) . n_m            for m = 1, 2, 3
//   lam_0(P) = V6 - lam_1 - lam_2 - lam_3
// On the sample lattice P = P0 + 2s (a, b, c), where P0 is the lowest sample of
// the tet's bounding box, so lam_m = L_m + Dx_m a + Dy_m b + Dz_m c with
// L_m = lam_m(P0) and D_m = 2s n_m (n_0 = -(n1 + n2 + n3)).
//
// Bit widths.  Let E be the tet's largest coordinate extent.  Every |n| <= 2E^2
// and, for points inside the vertex bounding box, |lam| <= 6E^3.  With
// E <= 2^20 every true intermediate is below 1.5 * 2^62, so 64-bit integers are
// exact (sums that may wrap transiently are formed in unsigned arithmetic and
// are exact modulo 2^64, hence exact).  Wider tets use 128-bit integers.
#pragma once
#include <stdint.h>

namespace voxtet {

constexpr int kLatticeBits = 20;
constexpr int kCoordLimit = 1 << 21;
constexpr int kNarrowExtent = 1 << 20;  // E <= this: 64-bit exact path

// Error bits recorded in the workspace header.
constexpr int kErrIndex = 1;
constexpr int kErrRange = 2;
constexpr int kErrNan = 4;

typedef long long i64;
typedef unsigned long long u64;
typedef __int128 i128;

struct Box {
  int i0, j0, l0;  // lowest sample index per axis
  int na, nb, nc;  // sample counts per axis (all > 0 when live)
};

// Sample-index box of one axis: samples (2i+1)s with mn <= (2i+1)s <= mx, clamped to
// [lo_lim, hi_lim] (the grid's samples on that axis, or a z-slab of them).  The
// lattice step is 2s = 1 << sh per voxel (sh = 20 - K, K = ceil(log2 of the grid's
// longest side)) and s = 1 << (sh - 1); arithmetic shifts give floor division for
// negative operands.
__device__ __forceinline__ void axis_box(int mn, int mx, int sh, int lo_lim, int hi_lim, int &lo, int &n) {
  const int s = 1 << (sh - 1);
  int a = (mn + s - 1) >> sh;  // ceil((mn - s) / 2s)
  int b = (mx - s) >> sh;      // floor((mx - s) / 2s)
  a = a < lo_lim ? lo_lim : a;
  b = b > hi_lim ? hi_lim : b;
  lo = a;
  n = b - a + 1;
}

__device__ __forceinline__ int imin4(int a, int b, int c, int d) { return min(min(a, b), min(c, d)); }
__device__ __forceinline__ int imax4(int a, int b, int c, int d) { return max(max(a, b), max(c, d)); }

// Bounding box of the samples of an (oriented or not) tet within a grid of rx x ry
// samples per slice and slices z0 <= l < z1; returns the extent E.
__device__ __forceinline__ int tet_box(const int3 V[4], int sh, int rx, int ry, int z0, int z1, Box &bx) {
  int mnx = imin4(V[0].x, V[1].x, V[2].x, V[3].x), mxx = imax4(V[0].x, V[1].x, V[2].x, V[3].x);
  int mny = imin4(V[0].y, V[1].y, V[2].y, V[3].y), mxy = imax4(V[0].y, V[1].y, V[2].y, V[3].y);
  int mnz = imin4(V[0].z, V[1].z, V[2].z, V[3].z), mxz = imax4(V[0].z, V[1].z, V[2].z, V[3].z);
  axis_box(mnx, mxx, sh, 0, rx - 1, bx.i0, bx.na);
  axis_box(mny, mxy, sh, 0, ry - 1, bx.j0, bx.nb);
  axis_box(mnz, mxz, sh, z0, z1 - 1, bx.l0, bx.nc);
  return max(max(mxx - mnx, mxy - mny), mxz - mnz);
}

// Sign of V6 = det[V1-V0, V2-V0, V3-V0], exact.  E is the tet's extent.
__device__ __forceinline__ int v6_sign(const int3 V[4], int E) {
  const int e1x = V[1].x - V[0].x, e1y = V[1].y - V[0].y, e1z = V[1].z - V[0].z;
  const int e2x = V[2].x - V[0].x, e2y = V[2].y - V[0].y, e2z = V[2].z - V[0].z;
  const int e3x = V[3].x - V[0].x, e3y = V[3].y - V[0].y, e3z = V[3].z - V[0].z;
  if (E <= kNarrowExtent) {
    // |e| <= 2^20: cross terms <= 2^41, the triple product <= 1.5 * 2^62
    const i64 cx = (i64)e2y * e3z - (i64)e2z * e3y;
    const i64 cy = (i64)e2z * e3x - (i64)e2x * e3z;
    const i64 cz = (i64)e2x * e3y - (i64)e2y * e3x;
    const i64 v = (i64)e1x * cx + (i64)e1y * cy + (i64)e1z * cz;
    return (v > 0) - (v < 0);
  }
  const i128 cx = (i128)e2y * e3z - (i128)e2z * e3y;
  const i128 cy = (i128)e2z * e3x - (i128)e2x * e3z;
  const i128 cz = (i128)e2x * e3y - (i128)e2y * e3x;
  const i128 v = (i128)e1x * cx + (i128)e1y * cy + (i128)e1z * cz;
  return (v > 0) - (v < 0);
}

// Exact affine data of the four lam_m over the sample lattice, for a positively
// oriented tet.  T = i64 requires E <= 2^20; T = i128 is exact for every input.
template <typename T>
struct Exact {
  T L[4], Dx[4], Dy[4], Dz[4];
};

template <typename T>
__device__ __forceinline__ T wrap_sub(T a, T b) {
  return a - b;
}
template <>
__device__ __forceinline__ i64 wrap_sub<i64>(i64 a, i64 b) {
  return (i64)((u64)a - (u64)b);
}

template <typename T>
__device__ __forceinline__ void exact_setup(const int3 V[4], const Box &bx, int sh, Exact<T> &X) {
  const int s = 1 << (sh - 1);
  const T e1x = V[1].x - V[0].x, e1y = V[1].y - V[0].y, e1z = V[1].z - V[0].z;
  const T e2x = V[2].x - V[0].x, e2y = V[2].y - V[0].y, e2z = V[2].z - V[0].z;
  const T e3x = V[3].x - V[0].x, e3y = V[3].y - V[0].y, e3z = V[3].z - V[0].z;
  const T n1x = e2y * e3z - e2z * e3y, n1y = e2z * e3x - e2x * e3z, n1z = e2x * e3y - e2y * e3x;
  const T n2x = e3y * e1z - e3z * e1y, n2y = e3z * e1x - e3x * e1z, n2z = e3x * e1y - e3y * e1x;
  const T n3x = e1y * e2z - e1z * e2y, n3y = e1z * e2x - e1x * e2z, n3z = e1x * e2y - e1y * e2x;
  const T v6 = e1x * n1x + e1y * n1y + e1z * n1z;
  // P0 - V0, with P0 = ((2 i0 + 1) s, ...) inside the vertex bounding box
  const T qx = (T)(s + (bx.i0 << sh)) - V[0].x;
  const T qy = (T)(s + (bx.j0 << sh)) - V[0].y;
  const T qz = (T)(s + (bx.l0 << sh)) - V[0].z;
  const T l1 = qx * n1x + qy * n1y + qz * n1z;
  const T l2 = qx * n2x + qy * n2y + qz * n2z;
  const T l3 = qx * n3x + qy * n3y + qz * n3z;
  X.L[1] = l1;
  X.L[2] = l2;
  X.L[3] = l3;
  X.L[0] = wrap_sub<T>(wrap_sub<T>(wrap_sub<T>(v6, l1), l2), l3);
  const T n0x = wrap_sub<T>(wrap_sub<T>(wrap_sub<T>((T)0, n1x), n2x), n3x);
  const T n0y = wrap_sub<T>(wrap_sub<T>(wrap_sub<T>((T)0, n1y), n2y), n3y);
  const T n0z = wrap_sub<T>(wrap_sub<T>(wrap_sub<T>((T)0, n1z), n2z), n3z);
  const T two_s = (T)1 << sh;
  X.Dx[0] = n0x * two_s; X.Dy[0] = n0y * two_s; X.Dz[0] = n0z * two_s;
  X.Dx[1] = n1x * two_s; X.Dy[1] = n1y * two_s; X.Dz[1] = n1z * two_s;
  X.Dx[2] = n2x * two_s; X.Dy[2] = n2y * two_s; X.Dz[2] = n2z * two_s;
  X.Dx[3] = n3x * two_s; X.Dy[3] = n3y * two_s; X.Dz[3] = n3z * two_s;
}

// Exact affine data of constraint m alone (64-bit, requires E <= 2^20), so that a
// caller can process one face at a time.  Face m is opposite vertex m:
//   m = 1, 2, 3:  lam_m(P) = (P - V0) . n_m with n1 = e2 x e3, n2 = e3 x e1, n3 = e1 x e2
//   m = 0:        lam_0(P) = (V1 - P) . ((V2 - V1) x (V3 - V1))
// (the same four values as exact_setup; lam_0 is formed directly instead of as
// V6 - lam_1 - lam_2 - lam_3).
template <int M>
__device__ __forceinline__ void slot_exact(const int3 V[4], const Box &bx, int sh, i64 &L, i64 &Dx, i64 &Dy,
                                           i64 &Dz) {
  const int s = 1 << (sh - 1);
  const int3 A = M == 0 ? V[1] : V[0];
  const int3 U = M == 0 ? V[2] : (M == 1 ? V[2] : (M == 2 ? V[3] : V[1]));
  const int3 W = M == 0 ? V[3] : (M == 1 ? V[3] : (M == 2 ? V[1] : V[2]));
  const i64 ux = U.x - A.x, uy = U.y - A.y, uz = U.z - A.z;
  const i64 wx = W.x - A.x, wy = W.y - A.y, wz = W.z - A.z;
  i64 nx = uy * wz - uz * wy, ny = uz * wx - ux * wz, nz = ux * wy - uy * wx;
  if (M == 0) {
    nx = -nx;
    ny = -ny;
    nz = -nz;
  }
  const i64 qx = (i64)(s + (bx.i0 << sh)) - A.x;
  const i64 qy = (i64)(s + (bx.j0 << sh)) - A.y;
  const i64 qz = (i64)(s + (bx.l0 << sh)) - A.z;
  L = qx * nx + qy * ny + qz * nz;
  const i64 two_s = (i64)1 << sh;
  Dx = nx * two_s;
  Dy = ny * two_s;
  Dz = nz * two_s;
}

// Slot of each constraint: first those with Dx < 0 (upper bounds on a), then
// Dx > 0 (lower bounds), then Dx == 0 (whole-row conditions).  slot[m] is the
// position of constraint m; nup / nlo count the first two groups.
template <typename T>
__device__ __forceinline__ void slot_order(const Exact<T> &X, int slot[4], int &nup, int &nlo) {
  int up = 0, lo = 0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    up += X.Dx[m] < 0;
    lo += X.Dx[m] > 0;
  }
  int cu = 0, cl = up, cz = up + lo;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    if (X.Dx[m] < 0) slot[m] = cu++;
    else if (X.Dx[m] > 0) slot[m] = cl++;
    else slot[m] = cz++;
  }
  nup = up;
  nlo = lo;
}

// Permute X into slot order (register-friendly: fully unrolled selects).
template <typename T>
__device__ __forceinline__ void permute_slots(Exact<T> &X, const int slot[4]) {
  Exact<T> Y;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    Y.L[q] = 0; Y.Dx[q] = 0; Y.Dy[q] = 0; Y.Dz[q] = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m)
      if (slot[m] == q) {
        Y.L[q] = X.L[m]; Y.Dx[q] = X.Dx[m]; Y.Dy[q] = X.Dy[m]; Y.Dz[q] = X.Dz[m];
      }
  }
  X = Y;
}

template <bool STRICT, typename T>
__device__ __forceinline__ bool lam_ok(T v) {
  return STRICT ? (v > 0) : (v >= 0);
}

// Exact sample interval [lo, hi] (0-based within the box's x-extent na) of row (b, c);
// returns false if the row has no sample.  Each bound is found by bisection on the
// monotone exact lam(a) = H + Dx a, probing only a in [0, na-1] (inside the box).
template <bool STRICT, typename T>
__device__ __forceinline__ bool exact_row(const Exact<T> &X, int nup, int nlo, int na, int b, int c, int &lo_out,
                                       int &hi_out) {
  int lo = 0, hi = na - 1;
#pragma unroll 1
  for (int m = 0; m < 4; ++m) {
    const T H = X.L[m] + X.Dz[m] * (T)c + X.Dy[m] * (T)b;
    if (m < nup) {  // lam decreasing in a: largest a in [-1, na-1] with lam(a) ok
      int x = -1, y = na - 1;
      while (x < y) {
        const int mid = (x + y + 1) >> 1;
        if (lam_ok<STRICT>(H + X.Dx[m] * (T)mid)) x = mid;
        else y = mid - 1;
      }
      hi = min(hi, x);
    } else if (m < nup + nlo) {  // lam increasing in a: smallest a in [0, na] with lam(a) ok
      int x = 0, y = na;
      while (x < y) {
        const int mid = (x + y) >> 1;
        if (lam_ok<STRICT>(H + X.Dx[m] * (T)mid)) y = mid;
        else x = mid + 1;
      }
      lo = max(lo, x);
    } else if (!lam_ok<STRICT>(H)) {
      return false;
    }
    if (lo > hi) return false;
  }
  lo_out = lo;
  hi_out = hi;
  return true;
}

// The same interval as exact_row for a 64-bit tet, faces in any order (no slot order
// needed).  Each bound starts from a single-precision estimate of the root of
// lam(a) = H + Dx a, clamped to the box, and is then moved to the exact bound by exact
// probes: lam is monotone in a, so stepping while the test still fails (or still holds one
// step further) ends on the bound whatever the estimate; with the estimate within one of
// the root, one or two probes per face.  Probes stay in [0, na-1] like the bisection's.
template <bool STRICT>
__device__ __forceinline__ bool exact_row_probe(const Exact<i64> &X, int na, int b, int c, int &lo_out,
                                                int &hi_out) {
  int lo = 0, hi = na - 1;
  bool empty = false;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const i64 H = X.L[m] + X.Dz[m] * (i64)c + X.Dy[m] * (i64)b;
    const i64 Dx = X.Dx[m];
    if (Dx == 0) {
      empty |= !lam_ok<STRICT>(H);
      continue;
    }
    const float r = fminf(fmaxf(__fdividef(-__ll2float_rn(H), __ll2float_rn(Dx)), -1.f), (float)na);
    int x = (int)floorf(r);  // in [-1, na]
    if (Dx < 0) {  // lam decreasing in a: largest a in [-1, na-1] with lam(a) ok
      x = min(x, na - 1);
      while (x >= 0 && !lam_ok<STRICT>(H + Dx * (i64)x)) --x;
      while (x + 1 <= na - 1 && lam_ok<STRICT>(H + Dx * (i64)(x + 1))) ++x;
      hi = min(hi, x);
    } else {  // lam increasing in a: smallest a in [0, na] with lam(a) ok
      x = max(x, 0);
      while (x <= na - 1 && !lam_ok<STRICT>(H + Dx * (i64)x)) ++x;
      while (x - 1 >= 0 && lam_ok<STRICT>(H + Dx * (i64)(x - 1))) --x;
      lo = max(lo, x);
    }
  }
  if (empty || lo > hi) return false;
  lo_out = lo;
  hi_out = hi;
  return true;
}

// Single-precision filter data of one 64-bit-exact tet, slot order as in Exact.
// For slot m with Dx != 0, the real root of lam_m along the row is
//   a*(b, c) = -(L + Dy b + Dz c) / Dx,
// and we keep t(b, c) = (L + Dy b + Dz c) / |Dx| = alpha + beta b + gamma c, so that
// upper slots (Dx < 0) need a <= t and lower slots (Dx > 0) need a >= -t.
//
// Error bound.  alpha~ = fl(fl(L) * fl(1/|fl(Dx)|)) carries at most four
// roundings (u = 2^-24): |alpha~ - alpha| <= 4.0001 u |alpha|, likewise beta and
// gamma.  A row evaluates t~ = fma(beta~, b, fma(gamma~, c, alpha~)) with two
// more roundings, so |t~ - t| <= 6.001 u S~ with S~ = |alpha~| + |beta~| b +
// |gamma~| c.  delta = 8u * Smax (Smax bounds S~ over the box, rounded up)
// therefore brackets t: t is in [t~ - delta, t~ + delta], evaluated with
// downward/upward rounding.  A bound is certified when floor (closed) or ceil
// (strict) agrees at both ends of that bracket; otherwise the row is solved
// exactly by exact_row.

// Filter data of one slot with Dx != 0 (L, Dx, Dy, Dz exact 64-bit values).
__device__ __forceinline__ void filter_slot(i64 L, i64 Dx, i64 Dy, i64 Dz, float fb, float fc, float &alpha,
                                            float &beta, float &gamma, float &delta) {
  const float fL = __ll2float_rn(L);
  const float fDx = __ll2float_rn(Dx);
  const float fDy = __ll2float_rn(Dy);
  const float fDz = __ll2float_rn(Dz);
  const float r = __frcp_rn(fabsf(fDx));
  const float a = __fmul_rn(fL, r), bb = __fmul_rn(fDy, r), g = __fmul_rn(fDz, r);
  const float S = __fmaf_ru(fabsf(g), fc, __fmaf_ru(fabsf(bb), fb, fabsf(a)));
  alpha = a;
  beta = bb;
  gamma = g;
  delta = __fmul_ru(S, 0x1p-21f);  // 8u
}

}  // namespace voxtet
