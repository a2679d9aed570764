// voxtet_slices.cu -- the slice-unit kernel of the voxelizer (scanline step and OR writes).
//
// The operation is the same as the span kernel's (voxtet.cu): every voxel-centre sample
// of a tet's bounding box that passes the closed (or strict) point-in-tetrahedron test of
// Section 4, Theorem 1 is set, the samples of one x-row solved at once as an interval
// (Section 3, "Voxelization", per row instead of per sample).  Only the distribution of
// the work differs.  A block takes a tile of kSuBlock tets, one per thread, and
//   (1) sets each tet up once: checked load, sample box, exact orientation from the
//       64-bit face normals, the four faces' single-precision filter data (a record in
//       shared memory), and for every z-slice of the box the exact range of candidate
//       rows (the cross-section's y-extent, narrowed exactly by faces parallel to x);
//   (2) counting-sorts the tile's (tet, slice) units by their row count, so the 32 lanes
//       of a warp walk units of the same length and stay in step (a block-wide exclusive
//       scan over per-warp bucket counters is the work distributor);
//   (3) walks each unit's rows: per row the four face bounds, the tightest upper and
//       lower bound certified once each (the filter's bracket of Section 4's orientation
//       values, see tet_math.cuh), and the interval ORed into the grid's words.
// Tets this kernel does not take -- zero volume (skipped), wider than 2^20 lattice
// units or use_filter = 0 (exact kernel), or more than kSuSlices slices or kSuRows rows
// per slice (listed at the back of the tet queue for the span kernel) -- are counted or
// queued exactly as the span kernel would.  Rows the filter cannot certify go to the
// same row queue, solved afterwards by the exact kernel.
#include <cuda_runtime.h>

#include <atomic>

#include "voxtet.h"
#include "tet_math.cuh"
#include "voxtet_device.cuh"
#include "voxtet_slices.cuh"

namespace voxtet {

constexpr int kSuWarps = kSuBlock / 32;
constexpr int kSuBuckets = 64;                           // row counts 1..63 one bucket each, >= 64 together
constexpr int kSuCounters = kSuBuckets * kSuWarps;       // bucket-major, one counter per warp of each bucket
constexpr int kSuRec = 28;  // floats per tet record: 24 used; 7 groups of 16 bytes, an odd number,
                            // so that lanes loading records of random slots spread over all banks
constexpr int kSuStage = 64;                             // staged uncertain rows per block (about 5 per tile)
constexpr uint32_t kSuEmpty = 0xFFFFFFFFu;               // a slice without candidate rows
static_assert(kSuBlock == 128 && kSuSlices <= 32 && kSuRows == 1024, "unit fields: 7 + 5 bits; rows in 10 bits");

// Tet record (kSuRec floats per slot).  The faces bounding a from above (Dx < 0) fill slots
// U0..U2 and those bounding it from below (Dx > 0) slots L0..L2, unused slots a neutral face
// (alpha = +inf, beta = gamma = 0: its bound is +inf and never the smallest).  Each U/L pair
// is adjacent.  Fields: alpha U0 L0 U1 L1 U2 L2 | beta (same order) | gamma (same order) |
// bracket of the upper side, of the lower side | na - 1 | i0 (int bits) | 64-bit grid word
// offset of the box's row (b, c) = (0, 0).
constexpr int kRecAl = 0, kRecBe = 6, kRecGa = 12, kRecDU = 18, kRecDL = 19, kRecHi = 20, kRecI0 = 21, kRecBase = 22;

// Shared memory of one block (dynamic), for tets of at most SL slices.
template <int SL>
struct SuSmem {
  float rec[kSuBlock * kSuRec];
  // per tet slot, slice k of its tet: b_lo | (n - 1) << 10, or kSuEmpty
  uint32_t slice[SL][kSuBlock];
  // the tile's units sorted by row count, longest first: slot | k << 7
  uint16_t unit[kSuBlock * SL];
  uint32_t hist[kSuCounters];
  uint32_t cur[kSuCounters + 1];
  uint32_t warp_tot[kSuWarps];
  RowStageN<kSuStage> stage;
  long long tile;
};

// 16-slice tiles fit 7 blocks per SM (228 KB, 1 KB reserved per block), 32-slice tiles 5
static_assert(sizeof(SuSmem<kSuSlicesSmall>) <= 31 * 1024, "slice-unit kernel shared memory: seven blocks per SM");
static_assert(sizeof(SuSmem<kSuSlices>) <= 44 * 1024, "slice-unit kernel shared memory: five blocks per SM");

// Counter of a unit with n rows emitted by warp w: longer units first.
__device__ __forceinline__ int su_counter(int n, int w) {
  return (kSuBuckets - min(n, kSuBuckets)) * kSuWarps + w;
}

// Edges of a tet for the per-slice row range, its vertices sorted by z (z0 <= z1 <= z2 <=
// z3): edge e = (p, q) meets the plane at height Z at y = yp + (Z - zp) k, k = (yq - yp) /
// (zq - zp) (0 for a horizontal edge, whose end points other edges reach).  Z - zp and the
// integer differences are exact in float; k comes from __fdividef (at most 2 ulp off for
// divisors in [1, 2^22]), so a crossing point is within 4u 2^22 + u 2^22 = 1.25 lattice
// units of the true one, inside the 2 units the range is widened by.
// Order: 01 02 03 12 13 23.  Slices below z1 cross 01 02 03, slices in [z1, z2] cross
// 02 03 12 13, above z2 03 13 23.  A horizontal edge (k = 0) yields only its first end
// point, so in [z1, z2] vertex 2 is added at Z = z2 (02 and 12 are both horizontal when
// z0 = z1 = z2, and 23, which starts there, belongs to the slices above); vertex 1 always
// comes from 12 and 13, which start at it.
struct SuEdges {
  float zp[6], yp[6], k[6];
  int z1, z2;
};

__device__ __forceinline__ void su_edges(const int3 V[4], SuEdges &E) {
  int z[4] = {V[0].z, V[1].z, V[2].z, V[3].z};
  int y[4] = {V[0].y, V[1].y, V[2].y, V[3].y};
#define VOXTET_CSWAP(a, b)                                  \
  if (z[b] < z[a]) {                                        \
    const int tz = z[a], ty = y[a];                         \
    z[a] = z[b]; y[a] = y[b]; z[b] = tz; y[b] = ty;         \
  }
  VOXTET_CSWAP(0, 1)
  VOXTET_CSWAP(2, 3)
  VOXTET_CSWAP(0, 2)
  VOXTET_CSWAP(1, 3)
  VOXTET_CSWAP(1, 2)
#undef VOXTET_CSWAP
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const int pi = e < 3 ? 0 : (e < 5 ? 1 : 2);
    const int qi = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
    const int dz = z[qi] - z[pi];
    E.zp[e] = (float)z[pi];
    E.yp[e] = (float)y[pi];
    E.k[e] = dz != 0 ? __fdividef((float)(y[qi] - y[pi]), (float)dz) : 0.f;
  }
  E.z1 = z[1];
  E.z2 = z[2];
}

// Phase (1) for tet t of this thread (t < 0: none).  Returns the slices whose entries it
// wrote to sm.slice (0 if the tet has no unit here); counts each unit in its counter (no
// rank is needed here, so the count does not wait on the shared-memory atomic).
template <bool STRICT, bool CULL, int SL>
__device__ __forceinline__ int su_setup(const Params &p, long long t, SuSmem<SL> &sm, TileCounters &ctr) {
  const int tid = threadIdx.x, warp = tid >> 5;
  if (t < 0) return 0;
  int3 V[4];
  if (!load_tet(p, t, V, ctr.err)) return 0;
  Box bx;
  const int E = tet_box(V, p.sh, p.rx, p.ry, p.z0, p.z1, bx);
  const bool empty = bx.na <= 0 || bx.nb <= 0 || bx.nc <= 0;
  if (E > kNarrowExtent) {  // wider than 2^20 lattice units: 128-bit sign, exact kernel
    if (v6_sign(V, E) == 0) {
      ++ctr.degenerate;
      return 0;
    }
    if (empty) return 0;
    ++ctr.wide;
    const unsigned k = atomicAdd(&p.hdr->tetq_count, 1u);
    p.tetq[k] = (uint32_t)t;
    return 0;
  }
  // E <= 2^20: edges below 2^21, normals below 2^43, V6 and every face value below 1.5 * 2^62
  const int e1x = V[1].x - V[0].x, e1y = V[1].y - V[0].y, e1z = V[1].z - V[0].z;
  const int e2x = V[2].x - V[0].x, e2y = V[2].y - V[0].y, e2z = V[2].z - V[0].z;
  const int e3x = V[3].x - V[0].x, e3y = V[3].y - V[0].y, e3z = V[3].z - V[0].z;
  i64 n1x = (i64)e2y * e3z - (i64)e2z * e3y, n1y = (i64)e2z * e3x - (i64)e2x * e3z, n1z = (i64)e2x * e3y - (i64)e2y * e3x;
  i64 n2x = (i64)e3y * e1z - (i64)e3z * e1y, n2y = (i64)e3z * e1x - (i64)e3x * e1z, n2z = (i64)e3x * e1y - (i64)e3y * e1x;
  i64 n3x = (i64)e1y * e2z - (i64)e1z * e2y, n3y = (i64)e1z * e2x - (i64)e1x * e2z, n3z = (i64)e1x * e2y - (i64)e1y * e2x;
  i64 v6 = (i64)e1x * n1x + (i64)e1y * n1y + (i64)e1z * n1z;
  if (v6 == 0) {
    ++ctr.degenerate;
    return 0;
  }
  if (empty) return 0;
  if (p.exact_all || bx.nb > kMaxFilterRows) {
    const unsigned k = atomicAdd(&p.hdr->tetq_count, 1u);
    p.tetq[k] = (uint32_t)t;
    return 0;
  }
  if (bx.nc > SL || bx.nb > kSuRows) {  // the span kernel takes it (list mode)
    const unsigned k = atomicAdd(&p.hdr->listq_count, 1u);
    p.tetq[p.n_tets - 1 - k] = (uint32_t)t;
    return 0;
  }
  // Orientation (Lemma 1.1): for V6 < 0 every orientation value of an inside point is <= 0,
  // so negating the normals (and V6) gives the positively oriented form of the same faces.
  if (v6 < 0) {
    n1x = -n1x; n1y = -n1y; n1z = -n1z;
    n2x = -n2x; n2y = -n2y; n2z = -n2z;
    n3x = -n3x; n3y = -n3y; n3z = -n3z;
    v6 = -v6;
  }
  // lam_m at the box's lowest sample P0 (tet_math.cuh): lam_m = (P0 - V0) . n_m for m = 1..3,
  // lam_0 = V6 - lam_1 - lam_2 - lam_3 with n_0 = -(n_1 + n_2 + n_3); sums that may wrap
  // transiently are formed in unsigned arithmetic (exact modulo 2^64, and the result fits)
  const int s = 1 << (p.sh - 1);
  const i64 qx = (i64)(s + (bx.i0 << p.sh)) - V[0].x;
  const i64 qy = (i64)(s + (bx.j0 << p.sh)) - V[0].y;
  const i64 qz = (i64)(s + (bx.l0 << p.sh)) - V[0].z;
  i64 L[4], Nx[4], Ny[4], Nz[4];
  L[1] = qx * n1x + qy * n1y + qz * n1z;
  L[2] = qx * n2x + qy * n2y + qz * n2z;
  L[3] = qx * n3x + qy * n3y + qz * n3z;
  L[0] = wrap_sub<i64>(wrap_sub<i64>(wrap_sub<i64>(v6, L[1]), L[2]), L[3]);
  Nx[1] = n1x; Ny[1] = n1y; Nz[1] = n1z;
  Nx[2] = n2x; Ny[2] = n2y; Nz[2] = n2z;
  Nx[3] = n3x; Ny[3] = n3y; Nz[3] = n3z;
  Nx[0] = wrap_sub<i64>(wrap_sub<i64>(wrap_sub<i64>(0, n1x), n2x), n3x);
  Ny[0] = wrap_sub<i64>(wrap_sub<i64>(wrap_sub<i64>(0, n1y), n2y), n3y);
  Nz[0] = wrap_sub<i64>(wrap_sub<i64>(wrap_sub<i64>(0, n1z), n2z), n3z);
  // Filter data per face (lam = L + D . (a, b, c) with D = 2s n) into the record's upper or
  // lower slots; a face parallel to x (Dx = 0) is an exact condition on the rows of each
  // slice below instead (at most two such faces).  Every live tet has a face with Dx < 0
  // and one with Dx > 0 (the four gradients sum to zero, at most two vanish).
  float *rec = sm.rec + tid * kSuRec;
  const float fb = (float)(bx.nb - 1), fc = (float)(bx.nc - 1);
  float dU = 0.f, dL = 0.f;
  int cu = 0, cl = 0;
  i64 zL0 = 0, zDy0 = 0, zDz0 = 0, zL1 = 0, zDy1 = 0, zDz1 = 0;
  int nz = 0;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const i64 Dx = Nx[m] << p.sh, Dy = Ny[m] << p.sh, Dz = Nz[m] << p.sh;
    if (Dx != 0) {
      float a, b, g, d;
      filter_slot(L[m], Dx, Dy, Dz, fb, fc, a, b, g, d);
      const int o = Dx < 0 ? 2 * cu++ : 2 * cl++ + 1;
      rec[kRecAl + o] = a;
      rec[kRecBe + o] = b;
      rec[kRecGa + o] = g;
      if (Dx < 0) dU = fmaxf(dU, d);
      else dL = fmaxf(dL, d);
    } else {
      if (nz == 0) {
        zL0 = L[m]; zDy0 = Dy; zDz0 = Dz;
      } else {
        zL1 = L[m]; zDy1 = Dy; zDz1 = Dz;
      }
      ++nz;
    }
  }
  const float INF = __int_as_float(0x7f800000);
  for (int q = cu; q < 3; ++q) {
    rec[kRecAl + 2 * q] = INF;
    rec[kRecBe + 2 * q] = 0.f;
    rec[kRecGa + 2 * q] = 0.f;
  }
  for (int q = cl; q < 3; ++q) {
    rec[kRecAl + 2 * q + 1] = INF;
    rec[kRecBe + 2 * q + 1] = 0.f;
    rec[kRecGa + 2 * q + 1] = 0.f;
  }
  rec[kRecDU] = dU;
  rec[kRecDL] = dL;
  rec[kRecHi] = (float)(bx.na - 1);
  rec[kRecI0] = __int_as_float(bx.i0);
  *reinterpret_cast<long long *>(rec + kRecBase) = ((long long)(bx.l0 - p.z0) * p.ry + bx.j0) * p.W;
  // Candidate rows of each slice: the cross-section's y-extent (a superset of the rows with
  // samples), narrowed exactly by the faces parallel to x.  Each unit is counted (no rank is
  // needed here, so the count does not wait on the shared-memory atomic).
  SuEdges EG;
  int kA = bx.nc, kB = bx.nc;
  if (CULL) {
    su_edges(V, EG);
    // slices k < kA lie below z1, k < kB at or below z2
    kA = min(max(((EG.z1 - s + (1 << p.sh) - 1) >> p.sh) - bx.l0, 0), bx.nc);
    kB = min(max(((EG.z2 - s) >> p.sh) + 1 - bx.l0, kA), bx.nc);
  }
  int units = 0;
  // one slice: its rows narrowed by the x-parallel faces, counted, recorded
  auto emit = [&](int k, int b_lo, int b_hi) {
    if (nz > 0) narrow_by_row_constraint<STRICT>(zL0 + zDz0 * (i64)k, zDy0, b_lo, b_hi);
    if (nz > 1) narrow_by_row_constraint<STRICT>(zL1 + zDz1 * (i64)k, zDy1, b_lo, b_hi);
    uint32_t e = kSuEmpty;
    if (b_hi >= b_lo) {
      const int n = b_hi - b_lo + 1;
      atomicAdd(&sm.hist[su_counter(n, warp)], 1u);
      e = (uint32_t)b_lo | ((uint32_t)(n - 1) << 10);
      ++units;
    }
    sm.slice[k][tid] = e;
  };
  if (CULL) {
    const int step = 1 << p.sh;
    int Z = s + (bx.l0 << p.sh);
    // the edges' first end points are vertices 0 (01 02 03), 1 (12 13) and 2 (23)
    const float zs0 = EG.zp[0], zs1 = EG.zp[3], zs2 = EG.zp[5], ys0 = EG.yp[0], ys1 = EG.yp[3], ys2 = EG.yp[5];
    const float k0 = EG.k[0], k1 = EG.k[1], k2 = EG.k[2], k3 = EG.k[3], k4 = EG.k[4], k5 = EG.k[5];
    for (int k = 0; k < bx.nc; ++k, Z += step) {
      // the slice's crossing points, edges chosen by selects (one straight-line body for all
      // slices): below z1 03 01 02; in [z1, z2] 03 02 12 13 and vertex 2 at z2; above 03 13 23
      const float Zf = (float)Z;
      const bool pa = k < kA, pb = !pa && k < kB, pc = !pa && !pb;
      const float d0 = Zf - zs0, d1 = Zf - zs1, d2 = Zf - zs2;
      const float y1 = __fmaf_rn(d0, k2, ys0);
      const float y2 = __fmaf_rn(pc ? d1 : d0, pa ? k0 : (pb ? k1 : k4), pc ? ys1 : ys0);
      const float y3 = __fmaf_rn(pa ? d0 : (pb ? d1 : d2), pa ? k1 : (pb ? k3 : k5), pa ? ys0 : (pb ? ys1 : ys2));
      const float y4 = pb ? __fmaf_rn(d1, k4, ys1) : y1;
      const float y5 = pb && Z == EG.z2 ? ys2 : y1;
      const float ymin = fminf(fminf(fminf(y1, y2), fminf(y3, y4)), y5);
      const float ymax = fmaxf(fmaxf(fmaxf(y1, y2), fmaxf(y3, y4)), y5);
      // the y-extent widened by 2 lattice units, in rows
      const int ylo = (int)floorf(ymin) - 2, yhi = (int)ceilf(ymax) + 2;
      const int b_lo = max(((ylo + s - 1) >> p.sh) - bx.j0, 0);
      const int b_hi = min(((yhi - s) >> p.sh) - bx.j0, bx.nb - 1);
      emit(k, b_lo, b_hi);
    }
  } else {
    for (int k = 0; k < bx.nc; ++k) emit(k, 0, bx.nb - 1);
  }
  return units ? bx.nc : 0;
}

// Block-wide exclusive prefix sum of one value per thread (all threads call it); `total`
// gets the sum.  Uses sm.warp_tot; ends with the block in step.
template <int SL>
__device__ __forceinline__ uint32_t su_block_scan(SuSmem<SL> &sm, uint32_t v, uint32_t &total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) sm.warp_tot[warp] = x;
  __syncthreads();
  uint32_t before = x - v;
  total = 0;
#pragma unroll
  for (int w = 0; w < kSuWarps; ++w) {
    const uint32_t t = sm.warp_tot[w];
    if (w < warp) before += t;
    total += t;
  }
  __syncthreads();
  return before;
}

// Filter data of one unit (a slice of one tet) for its rows.
struct SuUnit {
  float aU0, aL0, aU1, aL1, aU2, aL2;  // alpha + gamma c of each face slot
  float bU0, bL0, bU1, bL1, bU2, bL2;  // beta of each face slot
  float dU, dL, fhi0;
  int i0;
};

// One row at bf (the row index as a float): its interval, ORed into `row`.  Returns true if
// the filter could not certify the row (nothing is written then; the caller queues it).
template <bool STRICT, bool CLAMP>
__device__ __forceinline__ bool su_row(const SuUnit &u, float bf, uint32_t *row) {
  // tightest bound of each side; the bracket of the smallest of the faces' values is the
  // smallest of their brackets, so one certification per side suffices
  const float TU = fminf(__fmaf_rn(u.bU0, bf, u.aU0), fminf(__fmaf_rn(u.bU1, bf, u.aU1), __fmaf_rn(u.bU2, bf, u.aU2)));
  const float TL = fminf(__fmaf_rn(u.bL0, bf, u.aL0), fminf(__fmaf_rn(u.bL1, bf, u.aL1), __fmaf_rn(u.bL2, bf, u.aL2)));
  float thU = __fadd_ru(TU, u.dU), tlU = __fsub_rd(TU, u.dU);
  float thL = __fadd_ru(TL, u.dL), tlL = __fsub_rd(TL, u.dL);
  if (CLAMP) {  // only where the bound can change the row (as in the span kernel)
    tlU = fmaxf(tlU, STRICT ? 0.f : -1.f);
    thU = fminf(thU, STRICT ? u.fhi0 + 1.f : u.fhi0);
    tlL = fmaxf(tlL, STRICT ? -u.fhi0 : -u.fhi0 - 1.f);
    thL = fminf(thL, STRICT ? 1.f : 0.f);
  }
  float lo, hi;
  bool amb;
  if (STRICT) {  // a < T: a <= ceil(T) - 1; a > -T: a >= 1 - ceil(T)
    const float cU = ceilf(tlU), cL = ceilf(tlL);
    amb = (cU < thU) | (cL < thL);
    hi = fminf(u.fhi0, cU - 1.f);
    lo = fmaxf(0.f, 1.f - cL);
  } else {  // a <= T: a <= floor(T); a >= -T: a >= -floor(T)
    const float fU = floorf(thU), fL = floorf(thL);
    amb = (fU > tlU) | (fL > tlL);
    hi = fminf(u.fhi0, fU);
    lo = fmaxf(0.f, -fL);
  }
  const bool live = !amb && lo <= hi;
  // lo, hi are integral floats in [0, na - 1] when live; otherwise every access below is
  // predicated off
  const int x0 = u.i0 + small_float_to_int(lo);
  const int x1 = u.i0 + small_float_to_int(hi);
  or_span_lanes(row, x0, x1, live);
  return amb;
}

// Phase (3): rows b0 .. b0 + n - 1 of slice k of the tet in `slot` (tet index t).
template <bool STRICT, bool CLAMP, int SL>
__device__ __forceinline__ void su_walk(const Params &p, SuSmem<SL> &sm, int slot, long long t, int k, int b0, int n) {
  const float4 *R = reinterpret_cast<const float4 *>(sm.rec + slot * kSuRec);
  const float4 q0 = R[0], q1 = R[1], q2 = R[2], q3 = R[3], q4 = R[4], q5 = R[5];
  const float cf = (float)k;
  SuUnit u;
  u.aU0 = __fmaf_rn(q3.x, cf, q0.x);
  u.aL0 = __fmaf_rn(q3.y, cf, q0.y);
  u.aU1 = __fmaf_rn(q3.z, cf, q0.z);
  u.aL1 = __fmaf_rn(q3.w, cf, q0.w);
  u.aU2 = __fmaf_rn(q4.x, cf, q1.x);
  u.aL2 = __fmaf_rn(q4.y, cf, q1.y);
  u.bU0 = q1.z; u.bL0 = q1.w; u.bU1 = q2.x; u.bL1 = q2.y; u.bU2 = q2.z; u.bL2 = q2.w;
  u.dU = q4.z;
  u.dL = q4.w;
  u.fhi0 = q5.x;
  u.i0 = __float_as_int(q5.y);
  const long long base = (long long)(((unsigned long long)__float_as_uint(q5.w) << 32) | __float_as_uint(q5.z));
  const long long W = p.W;
  uint32_t *row = p.out + base + (long long)k * p.ry * W + (long long)b0 * W;
  float bf = (float)b0;
  // uncertain rows are collected as bits, 32 rows at a time, and queued after the rows, so
  // that the row loop has no call in it
  for (int r0 = 0; r0 < n; r0 += 32) {
    const int r1 = min(n, r0 + 32);
    uint32_t amb = 0;
    for (int r = r0; r < r1; ++r) {
      amb |= (uint32_t)su_row<STRICT, CLAMP>(u, bf, row) << (r - r0);
      bf += 1.f;
      row += W;
    }
    while (amb) {
      const int j = __ffs(amb) - 1;
      amb &= amb - 1u;
      queue_row_staged(p, sm.stage, t, b0 + r0 + j, k);
    }
  }
}

template <bool STRICT, bool CULL, bool CLAMP, bool STRIDED, int SL>
__global__ void __launch_bounds__(kSuBlock, SL == kSuSlicesSmall ? 7 : 5) k_slices(Params p) {
  chain_wait();  // vertices snapped, header zeroed
  chain_release();
  extern __shared__ __align__(16) unsigned char su_dyn_smem[];
  SuSmem<SL> &sm = *reinterpret_cast<SuSmem<SL> *>(su_dyn_smem);
  const int tid = threadIdx.x;
  TileCounters ctr;
  for (int i = tid; i < kSuCounters; i += kSuBlock) sm.hist[i] = 0u;
  if (tid == 0) sm.stage.n = 0;
  for (;;) {
    if (tid == 0) sm.tile = (long long)atomicAdd(&p.hdr->tile_counter, 1ull);
    __syncthreads();
    const long long tile = sm.tile;
    long long base, t;
    if (STRIDED) {  // slab launches: tile k holds tets k + j * tile_stride
      if (tile >= p.tile_stride) break;
      base = tile;
      t = base + (long long)tid * p.tile_stride;
    } else {
      base = tile * kSuBlock;
      if (base >= p.n_tets) break;
      t = base + tid;
    }
    if (t >= p.n_tets) t = -1;
    // (1) set up this thread's tet and its slices' row ranges; count units per counter
    const int nc = su_setup<STRICT, CULL, SL>(p, t, sm, ctr);
    __syncthreads();
    // (2) exclusive scan of the counters (two per thread) into cursors, then every unit to
    // its place (a cursor per counter: units of one counter come from one warp)
    {
      const uint32_t c0 = sm.hist[2 * tid], c1 = sm.hist[2 * tid + 1];
      uint32_t all = 0;
      const uint32_t before = su_block_scan(sm, c0 + c1, all);
      sm.cur[2 * tid] = before;
      sm.cur[2 * tid + 1] = before + c0;
      if (tid == kSuBlock - 1) sm.cur[kSuCounters] = all;
      sm.hist[2 * tid] = 0u;  // ready for the next tile (read no more in this one)
      sm.hist[2 * tid + 1] = 0u;
      __syncthreads();
    }
    const uint32_t total = sm.cur[kSuCounters];
#pragma unroll 4
    for (int k = 0; k < nc; ++k) {
      const uint32_t e = sm.slice[k][tid];
      if (e == kSuEmpty) continue;
      const int n = (int)(e >> 10) + 1;
      const uint32_t pos = atomicAdd(&sm.cur[su_counter(n, tid >> 5)], 1u);
      sm.unit[pos] = (uint16_t)(tid | (k << 7));
    }
    __syncthreads();
    if (tid == 0) ctr.spans += total;
    // (3) walk the units, longest first; a warp takes 32 neighbouring units of the order
    for (uint32_t i = tid; i < total; i += kSuBlock) {
      const uint32_t u = sm.unit[i];
      const int slot = (int)(u & 127u), k = (int)(u >> 7);
      const uint32_t e = sm.slice[k][slot];
      const int b0 = (int)(e & 1023u), n = (int)(e >> 10) + 1;
      const long long tt = STRIDED ? base + (long long)slot * p.tile_stride : base + slot;
      ctr.rows += (unsigned)n;
      su_walk<STRICT, CLAMP, SL>(p, sm, slot, tt, k, b0, n);
    }
    flush_stage(p, sm.stage);
  }
  flush_counters(p.hdr, ctr);
}

// ------------------------------------------------------------------ host side

typedef void (*SuKernel)(Params);

template <int SL>
static SuKernel su_kernel(int v) {
  switch (v) {
    case 0: return k_slices<false, false, false, false, SL>;
    case 1: return k_slices<false, false, true, false, SL>;
    case 2: return k_slices<false, true, false, false, SL>;
    case 3: return k_slices<false, true, true, false, SL>;
    case 4: return k_slices<true, false, false, false, SL>;
    case 5: return k_slices<true, false, true, false, SL>;
    case 6: return k_slices<true, true, false, false, SL>;
    case 7: return k_slices<true, true, true, false, SL>;
    case 8: return k_slices<false, false, false, true, SL>;
    case 9: return k_slices<false, false, true, true, SL>;
    case 10: return k_slices<false, true, false, true, SL>;
    case 11: return k_slices<false, true, true, true, SL>;
    case 12: return k_slices<true, false, false, true, SL>;
    case 13: return k_slices<true, false, true, true, SL>;
    case 14: return k_slices<true, true, false, true, SL>;
    default: return k_slices<true, true, true, true, SL>;
  }
}

constexpr int kSuMaxDevices = 64;
static int g_su_occ[kSuMaxDevices][2][16];  // resident blocks per SM per capacity and variant, 0 = not yet queried
static std::atomic<int> g_su_lock{0};

size_t slices_smem_bytes(int slices) {
  return slices <= kSuSlicesSmall ? sizeof(SuSmem<kSuSlicesSmall>) : sizeof(SuSmem<kSuSlices>);
}

int launch_slices(const Params &p_in, int variant, int slices, int sms, cudaStream_t stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kSuMaxDevices) return VOXTET_ERR_CUDA;
  const int c = slices <= kSuSlicesSmall ? 0 : 1;
  SuKernel kern = c == 0 ? su_kernel<kSuSlicesSmall>(variant & 15) : su_kernel<kSuSlices>(variant & 15);
  const size_t smem = slices_smem_bytes(slices);
  int occ = g_su_occ[dev][c][variant & 15];
  if (occ == 0) {
    while (g_su_lock.exchange(1)) {
    }
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(kern),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kSuBlock, smem);
    if (e == cudaSuccess && occ < 1) occ = 1;
    if (e == cudaSuccess) g_su_occ[dev][c][variant & 15] = occ;
    g_su_lock.store(0);
    if (e != cudaSuccess) return VOXTET_ERR_CUDA;
  }
  Params p = p_in;
  const bool strided = (variant & 8) != 0;
  long long grid = (long long)sms * occ;
  long long tiles = (p.n_tets + kSuBlock - 1) / kSuBlock;
  p.tile_stride = 0;
  if (strided) {  // at least one tile per resident block (see the span kernel's slab launches)
    long long stride = tiles;
    if (stride < grid) stride = p.n_tets < grid ? p.n_tets : grid;
    p.tile_stride = stride;
    tiles = stride;
  }
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  return launch_chained(kern, (unsigned)grid, kSuBlock, smem, stream, p) == cudaSuccess ? VOXTET_OK : VOXTET_ERR_CUDA;
}

}  // namespace voxtet
