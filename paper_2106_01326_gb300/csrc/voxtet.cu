// voxtet.cu -- sm_103a kernels and C ABI of the tetrahedral-mesh solid voxelizer.
//
// The operation is Section 3 ("Voxelization") of arXiv 2106.01326: visit the
// bounding box of every tetrahedron and mark the voxel-centre samples that pass
// the point-in-tetrahedron test of Section 4, Theorem 1 (closed reading by
// default).  The paper visits every sample of every box one by one; here the
// four affine orientation values of a tet are solved along each x-row of its
// box for the whole run of passing samples at once, so the per-sample test
// becomes a per-row interval.
//
// Kernels (one stream, in order):
//   k_prologue   zero the workspace header and redo bitmap, and (unless
//                accumulating) the grid
//   k_snap       float vertices -> lattice int4 (x, y, z, error bits); k_load_fixed
//                does the range check for vertices already on the lattice
//                (k_prep<FIXED> does the prologue and either in one launch for
//                calls with tets; k_exact then reports the vertices' errors)
//   k_slices     (voxtet_slices.cu) the same as k_voxelize with (tet, z-slice)
//                units sorted by exact row count; k_voxelize then takes the tets
//                it lists
//   k_voxelize   persistent; each block repeatedly claims a tile of tets and
//                (1) computes per tet the sample box, orientation and span
//                    count (whole z-slices, about span_rows rows per span),
//                (2) splits the tile into spans with a block-wide exclusive
//                    prefix sum,
//                (3) solves each row of each span for its sample interval with
//                    the single-precision filter, skipping rows outside each
//                    slice's cross-section, and
//                (4) ORs the interval into the bit grid: whole 32-bit words are
//                    stored, the two partial edge words use atomicOr since other
//                    tets may share them.
//                Faces parallel to x only restrict which rows of a slice can
//                hold samples; they are applied exactly when the slice table is
//                built.  Work the filter cannot certify is queued, not solved
//                here, so the hot loop carries no rarely used state: tets wider
//                than 2^20 lattice units go to the tet queue, uncertain rows to
//                the row queue (tets whose rows overflow it are flagged in the
//                redo bitmap).
//   k_exact_rows solves the queued rows with exact integers and ORs them in;
//   k_exact      the queued whole tets and the redo bitmap's (OR is idempotent,
//                so redoing a row is harmless).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

#include "voxtet.h"
#include "tet_math.cuh"
#include "voxtet_device.cuh"
#include "voxtet_slices.cuh"

namespace voxtet {

// ------------------------------------------------------------------ small kernels

__global__ void k_prologue(Header *hdr, uint32_t *redo, long long redo_words, uint32_t *out, long long n_words,
                           int clear) {
  chain_release();  // the snap kernel may be scheduled now; it waits for this one to complete
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (tid < 64) reinterpret_cast<uint32_t *>(hdr)[tid] = 0u;
  for (long long i = tid; i < redo_words; i += stride) redo[i] = 0u;
  if (!clear) return;
  if ((reinterpret_cast<uintptr_t>(out) & 15) == 0) {
    uint4 *o4 = reinterpret_cast<uint4 *>(out);
    const long long n4 = n_words >> 2;
    for (long long i = tid; i < n4; i += stride) o4[i] = make_uint4(0u, 0u, 0u, 0u);
    for (long long i = (n4 << 2) + tid; i < n_words; i += stride) out[i] = 0u;
  } else {
    for (long long i = tid; i < n_words; i += stride) out[i] = 0u;
  }
}

// X = round_half_even(((double)v - o) / h * 2^(20-k)), each double operation rounded to
// nearest.  When h is a power of two the quotient is exact and the host passes
// mul = 2^(20-k) / h instead (identical result, no double division).
// With a zero origin and mul = 2^m, m >= 0 (fast = 1), ((double)v - 0) * mul is exact in
// float as well (a power-of-two scale of a float, overflow aside, which the range check
// catches), and rintf rounds half to even like the double path: the same X on the FP32
// pipe instead of GB300's narrow FP64 unit.
struct SnapArgsK {  // the snap's scalars (see k_snap)
  double ox, oy, oz, h, scale, mul;
  int use_mul, fast;
};

// Vertex i snapped: the lattice point and, in w, its error bits (kErrNan, kErrRange; 0 if
// valid).  A vertex with w != 0 makes every tet naming it skip.
__device__ __forceinline__ int4 snap_one(const float *__restrict__ v, long long i, const SnapArgsK &a) {
  int X[3];
  int err = 0;
  const double o[3] = {a.ox, a.oy, a.oz};
#pragma unroll
  for (int q = 0; q < 3; ++q) {
    const float f = v[3 * i + q];
    X[q] = 0;
    if (!isfinite(f)) {
      err |= kErrNan;
      continue;
    }
    if (a.fast) {
      const float r = rintf(__fmul_rn(f, (float)a.mul));
      if (!(fabsf(r) <= (float)kCoordLimit)) {
        err |= kErrRange;
        continue;
      }
      X[q] = (int)r;
      continue;
    }
    const double d = __dsub_rn((double)f, o[q]);
    const double x = a.use_mul ? __dmul_rn(d, a.mul) : __dmul_rn(__ddiv_rn(d, a.h), a.scale);
    const long long r = __double2ll_rn(x);
    if (r < -kCoordLimit || r > kCoordLimit) {
      err |= kErrRange;
      continue;
    }
    X[q] = (int)r;
  }
  return make_int4(X[0], X[1], X[2], err);
}

// Lattice vertex i range-checked (w as in snap_one).
__device__ __forceinline__ int4 load_fixed_one(const int *__restrict__ xyz, long long i) {
  const int x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
  const bool bad = x < -kCoordLimit || x > kCoordLimit || y < -kCoordLimit || y > kCoordLimit ||
                   z < -kCoordLimit || z > kCoordLimit;
  return make_int4(bad ? 0 : x, bad ? 0 : y, bad ? 0 : z, bad ? kErrRange : 0);
}

__global__ void k_snap(const float *__restrict__ v, long long n, SnapArgsK a, int4 *__restrict__ out, Header *hdr) {
  chain_wait();  // the prologue has zeroed the header
  chain_release();
  const long long stride = (long long)gridDim.x * blockDim.x;
  int err = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int4 r = snap_one(v, i, a);
    out[i] = r;
    err |= r.w;
  }
  if (err) atomicOr(&hdr->status_bits, err);
}

__global__ void k_load_fixed(const int *__restrict__ xyz, long long n, int4 *__restrict__ out, Header *hdr) {
  chain_wait();  // the prologue has zeroed the header
  chain_release();
  const long long stride = (long long)gridDim.x * blockDim.x;
  int err = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int4 r = load_fixed_one(xyz, i);
    out[i] = r;
    err |= r.w;
  }
  if (err) atomicOr(&hdr->status_bits, err);
}

// The prologue and the snap (or the lattice load) of a call in one launch, the call's first.
// The vertices' error bits stay in their w fields; the call's last kernel (k_exact, with
// p.vflags set) folds them into the status, so nothing here orders against the header's
// zeroing.
template <bool FIXED>
__global__ void k_prep(Header *hdr, uint32_t *redo, long long redo_words, uint32_t *grid, long long n_words,
                       int clear, const void *__restrict__ src, long long n, SnapArgsK a, int4 *__restrict__ out) {
  chain_release();  // the next kernel may be scheduled now; it waits for this one to complete
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long stride = (long long)gridDim.x * blockDim.x;
  if (tid < 64) reinterpret_cast<uint32_t *>(hdr)[tid] = 0u;
  for (long long i = tid; i < redo_words; i += stride) redo[i] = 0u;
  if (clear) {
    if ((reinterpret_cast<uintptr_t>(grid) & 15) == 0) {
      uint4 *o4 = reinterpret_cast<uint4 *>(grid);
      const long long n4 = n_words >> 2;
      for (long long i = tid; i < n4; i += stride) o4[i] = make_uint4(0u, 0u, 0u, 0u);
      for (long long i = (n4 << 2) + tid; i < n_words; i += stride) grid[i] = 0u;
    } else {
      for (long long i = tid; i < n_words; i += stride) grid[i] = 0u;
    }
  }
  for (long long i = tid; i < n; i += stride)
    out[i] = FIXED ? load_fixed_one(static_cast<const int *>(src), i) : snap_one(static_cast<const float *>(src), i, a);
}

// Loads, orients (V6 > 0) and boxes a tet already known to be live; returns its extent.
__device__ __forceinline__ int oriented_tet(const Params &p, long long t, int3 V[4], Box &bx) {
  int dummy = 0;
  load_tet(p, t, V, dummy);
  const int E = tet_box(V, p.sh, p.rx, p.ry, p.z0, p.z1, bx);
  if (v6_sign(V, E) < 0) {
    const int3 tmp = V[2];
    V[2] = V[3];
    V[3] = tmp;
  }
  return E;
}

// z-slices per span: the tet's nc slices are split into equal spans of about
// span_rows bounding-box rows each, at most kMaxSlicesPerSpan (the size of each
// thread's slice table).  Equal spans keep the per-span work estimate meaningful.
__device__ __forceinline__ int slices_per_span(const Params &p, int nb, int nc) {
  int S = p.span_rows / nb;
  S = S < 1 ? 1 : (S > p.max_slices ? p.max_slices : S);
  const int n = (nc + S - 1) / S;
  return (nc + n - 1) / n;
}

// Phase (1): classify tet t and return its span count for the filter path (0 if it
// marks nothing or was queued for the exact kernel); `meta` gets the orientation flag and
// the slices per span, which the span phase reuses.
__device__ __forceinline__ uint32_t classify_tet(const Params &p, long long t, int &err, unsigned &n_degenerate,
                                                 unsigned &n_wide, float &work, uint32_t &meta) {
  int3 V[4];
  if (!load_tet(p, t, V, err)) return 0;
  Box bx;
  const int E = tet_box(V, p.sh, p.rx, p.ry, p.z0, p.z1, bx);
  const int sg = v6_sign(V, E);
  if (sg == 0) {
    ++n_degenerate;
    return 0;
  }
  if (bx.na <= 0 || bx.nb <= 0 || bx.nc <= 0) return 0;
  const bool wide = E > kNarrowExtent;
  n_wide += wide;
  // boxes taller than kMaxFilterRows rows (only in grids wider than 8192, sparse output)
  // exceed the slice table's 14-bit row fields and go to the exact kernel as well
  if (wide || p.exact_all || bx.nb > kMaxFilterRows) {
    const unsigned k = atomicAdd(&p.hdr->tetq_count, 1u);  // each tet is queued once: k < n_tets
    p.tetq[k] = (uint32_t)t;
    return 0;
  }
  const int S = slices_per_span(p, bx.nb, bx.nc);
  // Work estimate (x-rows the span loop will visit): the tet's shadow on the yz-plane
  // has area sum_m |n_m.x| / 4 (each shadow point is covered by two faces), which in
  // row units is that over (2s)^2, plus about one extra row per slice.
  {
    const float e1y = (float)(V[1].y - V[0].y), e1z = (float)(V[1].z - V[0].z);
    const float e2y = (float)(V[2].y - V[0].y), e2z = (float)(V[2].z - V[0].z);
    const float e3y = (float)(V[3].y - V[0].y), e3z = (float)(V[3].z - V[0].z);
    const float n1x = e2y * e3z - e2z * e3y, n2x = e3y * e1z - e3z * e1y, n3x = e1y * e2z - e1z * e2y;
    const float inv = __int_as_float((127 - 2 * p.sh) << 23);  // 1 / (2s)^2, an exact power of two
    work = (fabsf(n1x) + fabsf(n2x) + fabsf(n3x) + fabsf(n1x + n2x + n3x)) * 0.25f * inv + (float)bx.nc;
  }
  meta = (uint32_t)(sg < 0) | ((uint32_t)S << 1);
  return (uint32_t)((bx.nc + S - 1) / S);
}

// Slices per span: the slice table (one column per thread, in dynamic shared memory)
// has p.max_slices rows.  16 rows fit 512^3 grids, where a tet spans about 9 slices; from
// 1024^3 a tet spans 17 or more and 32 rows let one span hold it, so the spans sorted by
// the per-tet work estimate are even (measured on GB300: 1024^3 kernel 1.49 -> 1.18 ms;
// at 512^3 the larger table costs 1.5 %, the L1 it takes).
constexpr int kMaxSlicesPerSpan = 32;
constexpr size_t kSliceTableBytesMax = (size_t)kMaxSlicesPerSpan * kBlock * sizeof(uint32_t);
static size_t slice_table_bytes(int max_slices) { return (size_t)max_slices * kBlock * sizeof(uint32_t); }

// Phases (3)+(4): slices [c0, c1) (at most kMaxSlicesPerSpan) of a narrow tet, whose
// vertices V2 and V3 are swapped first when `flip` (the classification found V6 < 0).
// First the candidate rows of every slice are found and the non-empty slices written to
// this thread's column of `tab`, then one flat loop walks all candidate rows, so the
// lanes of a warp stay in step across slices.  Returns the rows visited.
template <bool STRICT, bool CULL, bool CLAMP>
__device__ __forceinline__ unsigned run_span(const Params &p, long long t, int3 V[4], const Box &bx, int c0, int c1,
                                             uint32_t (*tab)[kBlock], RowStage &stage, bool flip) {
  if (flip) {  // orient (classification found V6 < 0)
    const int3 tmp = V[2];
    V[2] = V[3];
    V[3] = tmp;
  }
  const int tid = threadIdx.x;
  const int ns = c1 - c0;
  // slice table: only slices with candidate rows, packed k | b_lo << 5 | (n - 1) << 19
  // (k < 32 slices, b_lo < 2^14, n <= 8192 rows).  Built before the face data so that the
  // edge lines and the face data are never live together.
  unsigned total = 0;
  int nt = 0;
  {
    EdgeLines EL;
    if (CULL) edge_lines(V, EL);
    const int s = 1 << (p.sh - 1);
    for (int k = 0; k < ns; ++k) {
      int b_lo = 0, b_hi = bx.nb - 1;
      if (CULL) slice_rows_sorted(EL, s + ((bx.l0 + c0 + k) << p.sh), s, p.sh, bx.j0, bx.nb, b_lo, b_hi);
      if (b_hi >= b_lo) {
        const int n = b_hi - b_lo + 1;
        tab[nt][tid] = (uint32_t)k | ((uint32_t)b_lo << 5) | ((uint32_t)(n - 1) << 19);
        ++nt;
        total += (unsigned)n;
      }
    }
  }
  if (total == 0) return 0;
  // Filter data per face, built one face at a time; faces parallel to x (at most
  // two) become neutral upper bounds here and exact row conditions below.
  float al[4], be[4], ga[4], de[4];
  bool up[4];
  i64 zL0 = 0, zDy0 = 0, zDz0 = 0, zL1 = 0, zDy1 = 0, zDz1 = 0;
  int nz = 0;
  {
    const float fb = (float)(bx.nb - 1), fc = (float)(bx.nc - 1);
#define VOXTET_SLOT(M)                                                                   \
  {                                                                                      \
    i64 L, Dx, Dy, Dz;                                                                   \
    slot_exact<M>(V, bx, p.sh, L, Dx, Dy, Dz);                                           \
    if (Dx != 0) {                                                                       \
      up[M] = Dx < 0;                                                                    \
      filter_slot(L, Dx, Dy, Dz, fb, fc, al[M], be[M], ga[M], de[M]);                    \
    } else {                                                                             \
      up[M] = true;                                                                      \
      al[M] = 1.0e30f;                                                                   \
      be[M] = ga[M] = de[M] = 0.f;                                                       \
      if (nz == 0) {                                                                     \
        zL0 = L; zDy0 = Dy; zDz0 = Dz;                                                   \
      } else {                                                                           \
        zL1 = L; zDy1 = Dy; zDz1 = Dz;                                                   \
      }                                                                                  \
      ++nz;                                                                              \
    }                                                                                    \
  }
    VOXTET_SLOT(0)
    VOXTET_SLOT(1)
    VOXTET_SLOT(2)
    VOXTET_SLOT(3)
#undef VOXTET_SLOT
  }
  if (nz > 0) {  // faces parallel to x: exact row conditions narrow the table's entries
    int nt2 = 0;
    total = 0;
    for (int m = 0; m < nt; ++m) {
      const uint32_t e = tab[m][tid];
      const int k = (int)(e & 31u);
      int b_lo = (int)((e >> 5) & 0x3FFFu);
      int b_hi = b_lo + (int)(e >> 19);
      narrow_by_row_constraint<STRICT>(zL0 + zDz0 * (i64)(c0 + k), zDy0, b_lo, b_hi);
      if (nz > 1) narrow_by_row_constraint<STRICT>(zL1 + zDz1 * (i64)(c0 + k), zDy1, b_lo, b_hi);
      if (b_hi >= b_lo) {
        const int n = b_hi - b_lo + 1;
        tab[nt2][tid] = (uint32_t)k | ((uint32_t)b_lo << 5) | ((uint32_t)(n - 1) << 19);
        ++nt2;
        total += (unsigned)n;
      }
    }
    nt = nt2;
    if (total == 0) return 0;
  }
  // Order the faces upper bounds first.  Every live tet has at least one face with
  // Dx < 0 and one with Dx > 0 (the four gradients sum to zero and at most two are
  // zero), so slot 0 is always an upper bound and slot 3 a lower bound; only slots 1
  // and 2 need a flag.
  bool up1, up2;
  {
    const int nup = (int)up[0] + (int)up[1] + (int)up[2] + (int)up[3];
    int pos[4], cu = 0, cl = nup;
#pragma unroll
    for (int m = 0; m < 4; ++m) pos[m] = up[m] ? cu++ : cl++;
    float a2[4], b2[4], g2[4], d2[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      a2[q] = al[0]; b2[q] = be[0]; g2[q] = ga[0]; d2[q] = de[0];
#pragma unroll
      for (int m = 1; m < 4; ++m)
        if (pos[m] == q) {
          a2[q] = al[m]; b2[q] = be[m]; g2[q] = ga[m]; d2[q] = de[m];
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      al[q] = a2[q]; be[q] = b2[q]; ga[q] = g2[q]; de[q] = d2[q];
    }
    up1 = nup >= 2;
    up2 = nup >= 3;
  }

  // walk the candidate rows slice by slice; moving to the next table entry is a short
  // straight-line step (no empty slices in the table)
  int m_tab = 0, b = 0, b_end = 0;
  uint32_t e_next = tab[0][tid];  // the next table entry, loaded one slice ahead
  float bf = 0.f, ac[4];
  uint32_t *row = p.out;
  const float fhi0 = (float)(bx.na - 1);
  // row (b, k) of the span is row00 + k * slice_words + b * W; with k < 32 and b < ry the
  // offset is below 32 * ry * W <= 32 * 65536 * 2048 = 2^32 words for every accepted grid
  uint32_t *const row00 = p.out + ((size_t)(bx.l0 - p.z0 + c0) * p.ry + bx.j0) * p.W;
  const unsigned slice_words = (unsigned)p.ry * (unsigned)p.W;
  for (unsigned r = 0; r < total; ++r) {
    if (b == b_end) {
      const uint32_t e = e_next;
      ++m_tab;
      e_next = tab[m_tab < nt ? m_tab : nt - 1][tid];
      const int k = (int)(e & 31u);
      b = (int)((e >> 5) & 0x3FFFu);
      b_end = b + 1 + (int)(e >> 19);
      bf = (float)b;
      const float cf = (float)(c0 + k);
#pragma unroll
      for (int m = 0; m < 4; ++m) ac[m] = __fmaf_rn(ga[m], cf, al[m]);
      row = row00 + ((unsigned)k * slice_words + (unsigned)b * (unsigned)p.W);
    }
    float lo = 0.f, hi = fhi0;
    bool amb = false;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const float tt = __fmaf_rn(be[m], bf, ac[m]);
      const bool upm = m == 0 || (m == 1 && up1) || (m == 2 && up2);
      float tl = __fsub_rd(tt, de[m]);
      float th = __fadd_ru(tt, de[m]);
      if (CLAMP) {
        // only the part of the bracket where this face's bound can change the row counts:
        // beyond it the bound is cut by the box or the row is empty whatever t is, so an
        // integer there is no reason to queue the row (wide boxes of fine grids have large
        // brackets on steep faces)
        tl = fmaxf(tl, STRICT ? (upm ? 0.f : -fhi0) : (upm ? -1.f : -fhi0 - 1.f));
        th = fminf(th, STRICT ? (upm ? fhi0 + 1.f : 1.f) : (upm ? fhi0 : 0.f));
      }
      float v;
      if (STRICT) {
        const float cc = ceilf(tl);
        amb |= cc < th;
        v = cc - 1.f;
      } else {
        const float f = floorf(th);
        amb |= f > tl;
        v = f;
      }
      if (upm) hi = fminf(hi, v);
      else lo = fmaxf(lo, -v);
    }
    const bool live = !amb && lo <= hi;
    // lo, hi are integral floats in [0, na - 1] when live; when not, the word indices
    // below are meaningless but every access through them is predicated off
    const int x0 = bx.i0 + small_float_to_int(lo);
    const int x1 = bx.i0 + small_float_to_int(hi);
    or_span_lanes(row, x0, x1, live);
    if (amb) queue_row_staged(p, stage, t, b, c0 + (int)(tab[m_tab - 1][tid] & 31u));
    ++b;
    bf += 1.f;
    row += p.W;
  }
  return total;
}

// ------------------------------------------------------------------ the fused kernel

constexpr int kTile = 512;      // tets per tile
constexpr int kSmallTile = 128;  // tets per tile at the end of a single-mesh launch
constexpr int kPerThread = kTile / kBlock;

constexpr int kSortedSpans = 2048;  // tiles with more spans run in their natural order
constexpr int kBuckets = 32;

struct TileSmem {
  uint32_t off[kTile + 1];
  uint32_t warp_tot[kBlock / 32];
  uint32_t order[kSortedSpans];  // spans by estimated work: tet slot << 16 | span within the tet
  uint8_t meta[kTile];           // per tet slot: 1 if V6 < 0 (swap V2, V3) | slices per span << 1
  uint32_t bucket[kBuckets];
  float wmin, wmax;
  RowStage stage;
};

// Phases (1)-(4) for tets [base, base + kTile) of one mesh.  All threads of the block
// call it; it begins and ends with the block in step.
// Tet in slot i of the tile that starts at `base`: base + i, or, in a slab launch
// (STRIDED, base = the tile's number), base + i * tile_stride, so that the tets of the
// slab -- one contiguous run in a mesh numbered along z -- spread over every tile.
// In list mode (the tets the slice-unit kernel left over), slot i of the tile starting at
// list position `base` holds tetq[n_tets - 1 - (base + i)].  Returns -1 past `end`.
template <bool STRIDED>
__device__ __forceinline__ long long tile_tet(const Params &p, long long base, long long i, long long end) {
  if (STRIDED) {
    const long long t = base + i * p.tile_stride;
    return t < end ? t : -1;
  }
  const long long k = base + i;
  if (k >= end) return -1;
  return p.list_mode ? (long long)p.tetq[p.n_tets - 1 - k] : k;
}

// Slots whose tet is at or past `end` are empty.
template <bool STRICT, bool CULL, bool CLAMP, bool STRIDED>
__device__ __forceinline__ void process_tile(const Params &p, long long base, long long end, TileSmem &sm,
                                             uint32_t (*slice_tab)[kBlock], TileCounters &ctr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // (1) classification and span counts of this thread's kPerThread consecutive tets
  uint32_t cnt[kPerThread];
  float work[kPerThread];
  uint32_t mine = 0;
  float wlo = 3.0e38f, whi = 0.f;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    const long long t = tile_tet<STRIDED>(p, base, (long long)tid * kPerThread + k, end);
    work[k] = 0.f;
    uint32_t mt = 0;
    cnt[k] = t >= 0 ? classify_tet(p, t, ctr.err, ctr.degenerate, ctr.wide, work[k], mt) : 0u;
    sm.meta[tid * kPerThread + k] = (uint8_t)mt;
    if (cnt[k]) {
      work[k] /= (float)cnt[k];  // per span
      wlo = fminf(wlo, work[k]);
      whi = fmaxf(whi, work[k]);
    }
    mine += cnt[k];
  }

  // (2) block-wide exclusive prefix sum of span counts
  uint32_t x = mine;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, d);
    if (lane >= d) x += y;
  }
  if (lane == 31) sm.warp_tot[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kBlock / 32 ? sm.warp_tot[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, w, d);
      if (lane >= d) w += y;
    }
    if (lane < kBlock / 32) sm.warp_tot[lane] = w;
  }
  __syncthreads();
  uint32_t run = (warp ? sm.warp_tot[warp - 1] : 0u) + x - mine;
#pragma unroll
  for (int k = 0; k < kPerThread; ++k) {
    sm.off[tid * kPerThread + k] = run;
    run += cnt[k];
  }
  if (tid == kBlock - 1) sm.off[kTile] = run;
  // range of the per-span work estimates over the tile
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    wlo = fminf(wlo, __shfl_xor_sync(0xFFFFFFFFu, wlo, d));
    whi = fmaxf(whi, __shfl_xor_sync(0xFFFFFFFFu, whi, d));
  }
  if (tid < kBuckets) sm.bucket[tid] = 0u;
  if (tid == 0) {
    sm.wmin = 3.0e38f;
    sm.wmax = 0.f;
  }
  __syncthreads();
  if (lane == 0) {
    atomicMin(reinterpret_cast<int *>(&sm.wmin), __float_as_int(wlo));  // non-negative floats order as ints
    atomicMax(reinterpret_cast<int *>(&sm.wmax), __float_as_int(whi));
  }
  __syncthreads();
  const uint32_t total = sm.off[kTile];
  if (tid == 0) ctr.spans += total;

  // (2b) counting sort of the spans by estimated work (32 buckets over the tile's
  // range), so that the lanes of a warp get spans of similar length
  const bool sorted = total <= (uint32_t)kSortedSpans;
  if (sorted) {
    const float w0 = sm.wmin, scale = (float)kBuckets / fmaxf(sm.wmax - sm.wmin, 1e-6f);
    int bk[kPerThread];
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      bk[k] = min(kBuckets - 1, max(0, (int)((work[k] - w0) * scale)));
      if (cnt[k]) atomicAdd(&sm.bucket[bk[k]], cnt[k]);
    }
    __syncthreads();
    if (warp == 0) {  // exclusive prefix over the buckets
      const uint32_t v = sm.bucket[lane];
      uint32_t incl = v;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, d);
        if (lane >= d) incl += y;
      }
      sm.bucket[lane] = incl - v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kPerThread; ++k) {
      if (cnt[k]) {
        const uint32_t pos = atomicAdd(&sm.bucket[bk[k]], cnt[k]);
        // span q of the tet in slot u is stored as u << 16 | q (q < 2^16: a tet spans at most 65536 slices)
        for (uint32_t q = 0; q < cnt[k]; ++q) sm.order[pos + q] = ((uint32_t)(tid * kPerThread + k) << 16) | q;
      }
    }
    __syncthreads();
  }

  // (3)+(4) spans, by estimated work when sorted (the sort recorded each span's tet slot
  // and its index within the tet); unsorted, span i belongs to the largest slot u with
  // off[u] <= i
  // Rounds of kBlock spans, dealt forwards and backwards in turn: each warp still gets 32
  // neighbouring spans of the work order, and no thread takes the largest of every round
  // (the block waits at the tile's end for its slowest thread).
  for (uint32_t r0 = 0; r0 < total; r0 += kBlock) {
    const uint32_t i = r0 + (((r0 / kBlock) & 1u) ? (uint32_t)(kBlock - 1 - tid) : (uint32_t)tid);
    if (i >= total) continue;
    int a = 0;
    uint32_t q = 0;
    if (sorted) {
      const uint32_t o = sm.order[i];
      a = (int)(o >> 16);
      q = o & 0xFFFFu;
    } else {
      int bnd = kTile - 1;
      while (a < bnd) {
        const int mid = (a + bnd + 1) >> 1;
        if (sm.off[mid] <= i) a = mid;
        else bnd = mid - 1;
      }
      q = i - sm.off[a];
    }
    const long long t = tile_tet<STRIDED>(p, base, a, end);
    int3 V[4];
    Box bx;
    int dummy = 0;
    load_tet(p, t, V, dummy);
    tet_box(V, p.sh, p.rx, p.ry, p.z0, p.z1, bx);
    const uint32_t mt = sm.meta[a];
    const int S = (int)(mt >> 1);
    const int c0 = (int)q * S;
    ctr.rows += run_span<STRICT, CULL, CLAMP>(p, t, V, bx, c0, min(c0 + S, bx.nc), slice_tab, sm.stage, (mt & 1u) != 0);
  }
  flush_stage(p, sm.stage);
}

// The slice table lives in dynamic shared memory: p.max_slices rows of kBlock words.
__device__ __forceinline__ uint32_t (*dynamic_slice_table())[kBlock] {
  extern __shared__ uint32_t voxtet_dyn_smem[];
  return reinterpret_cast<uint32_t (*)[kBlock]>(voxtet_dyn_smem);
}

template <bool STRICT, bool CULL, bool CLAMP, bool STRIDED>
__global__ void __launch_bounds__(kBlock, VOXTET_MIN_BLOCKS) k_voxelize(Params p) {
  chain_wait();  // vertices snapped, header zeroed; in list mode the slice-unit kernel has listed its tets
  chain_release();
  __shared__ TileSmem sm;
  uint32_t (*const slice_tab)[kBlock] = dynamic_slice_table();
  __shared__ unsigned long long tile_s;
  TileCounters ctr;
  if (threadIdx.x == 0) sm.stage.n = 0;
  // Guided tiles: full tiles first, then quarter tiles for the last stretch (about two
  // per block), so that blocks finish close together at the end of the kernel.  In list
  // mode the tets are the ones the slice-unit kernel listed (stream-ordered before this launch).
  const long long big = p.big_tiles;
  const long long n_tets = p.list_mode ? min((long long)p.hdr->listq_count, p.n_tets) : p.n_tets;
  if (n_tets == 0) return;  // list mode with nothing listed (the block is still in step: no barrier yet)
  for (;;) {
    if (threadIdx.x == 0) tile_s = atomicAdd(p.list_mode ? &p.hdr->list_tile_counter : &p.hdr->tile_counter, 1ull);
    __syncthreads();
    const long long tile = (long long)tile_s;
    if (STRIDED) {
      if (tile >= p.tile_stride) break;
      process_tile<STRICT, CULL, CLAMP, true>(p, tile, p.n_tets, sm, slice_tab, ctr);
      continue;
    }
    const long long base = tile < big ? tile * kTile : big * kTile + (tile - big) * kSmallTile;
    if (base >= n_tets) break;
    const long long end = min(n_tets, base + (tile < big ? kTile : kSmallTile));
    process_tile<STRICT, CULL, CLAMP, false>(p, base, end, sm, slice_tab, ctr);
  }
  flush_counters(p.hdr, ctr);
}

// ------------------------------------------------------------------ the exact kernel

// Every bounding-box row of tet t, solved with exact integers of type T by the
// threads of one block (threads stride over the rows).
template <bool STRICT, typename T>
__device__ __forceinline__ void exact_tet_rows(const Params &p, const int3 V[4], const Box &bx) {
  Exact<T> X;
  exact_setup<T>(V, bx, p.sh, X);
  int slot[4], nup = 0, nlo = 0;
  slot_order<T>(X, slot, nup, nlo);
  permute_slots<T>(X, slot);
  const unsigned long long rows = (unsigned long long)bx.nb * (unsigned long long)bx.nc;
  for (unsigned long long r = threadIdx.x; r < rows; r += blockDim.x) {
    const int c = (int)(r / (unsigned long long)bx.nb), b = (int)(r - (unsigned long long)c * bx.nb);
    int lo, hi;
    if (exact_row<STRICT, T>(X, nup, nlo, bx.na, b, c, lo, hi)) {
      uint32_t *row = p.out + ((size_t)(bx.l0 - p.z0 + c) * p.ry + (bx.j0 + b)) * p.W;
      or_span(row, bx.i0 + lo, bx.i0 + hi);
    }
  }
}

template <bool STRICT>
__device__ __forceinline__ void exact_tet(const Params &p, long long t) {
  int3 V[4];
  Box bx;
  const int E = oriented_tet(p, t, V, bx);
  if (E <= kNarrowExtent) exact_tet_rows<STRICT, i64>(p, V, bx);
  else exact_tet_rows<STRICT, i128>(p, V, bx);
}

// The queued rows of one mesh (a thread each), by blocks bi of bn.
template <bool STRICT>
__device__ __forceinline__ void exact_rows_job(const Params &p, unsigned bi, unsigned bn) {
  const unsigned n_rq = min(p.hdr->rowq_count, p.q_cap);
  const unsigned gtid = bi * blockDim.x + threadIdx.x, gsz = bn * blockDim.x;
  for (unsigned i = gtid; i < n_rq; i += gsz) {
    const RowItem it = p.rowq[i];
    int3 V[4];
    Box bx;
    oriented_tet(p, it.tet, V, bx);
    Exact<i64> X;
    exact_setup<i64>(V, bx, p.sh, X);
    int lo, hi;
    if (exact_row_probe<STRICT>(X, bx.na, it.b, it.c, lo, hi)) {
      uint32_t *row = p.out + ((size_t)(bx.l0 - p.z0 + it.c) * p.ry + (bx.j0 + it.b)) * p.W;
      or_span(row, bx.i0 + lo, bx.i0 + hi);
    }
  }
}

// The rest of the exact work of one mesh: its queued tets (a block each) and, after a
// row-queue overflow, the tets flagged in its redo bitmap; by blocks bi of bn.
template <bool STRICT>
__device__ __forceinline__ void exact_tets_job(const Params &p, unsigned bi, unsigned bn) {
  const unsigned n_tq = min((unsigned long long)p.hdr->tetq_count, (unsigned long long)p.n_tets);
  for (unsigned q = bi; q < n_tq; q += bn) exact_tet<STRICT>(p, p.tetq[q]);
  if (p.hdr->rowq_count > p.q_cap) {
    for (long long t = bi; t < p.n_tets; t += bn)
      if ((p.redo[t >> 5] >> (t & 31)) & 1u) exact_tet<STRICT>(p, t);
  }
}

template <bool STRICT>
__device__ __forceinline__ void exact_job(const Params &p, unsigned bi, unsigned bn) {
  exact_tets_job<STRICT>(p, bi, bn);
  exact_rows_job<STRICT>(p, bi, bn);
}

// The queued rows, in a kernel of their own: the 64-bit row solve needs far fewer registers
// than the tet path's 128-bit one, so many more threads are resident.
template <bool STRICT>
__global__ void __launch_bounds__(128) k_exact_rows(Params p) {
  chain_wait();  // every row is queued
  chain_release();
  exact_rows_job<STRICT>(p, blockIdx.x, gridDim.x);
}

template <bool STRICT>
__global__ void __launch_bounds__(128) k_exact(Params p) {
  chain_wait();  // every tet is queued
  if (p.vflags) {  // the vertices' error bits, left in verts4[i].w by the fused prologue and snap
    int err = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < p.n_verts; i += stride)
      err |= p.verts4[i].w;
    err = __reduce_or_sync(0xFFFFFFFFu, err);
    if ((threadIdx.x & 31) == 0 && err) atomicOr(&p.hdr->status_bits, err);
  }
  exact_tets_job<STRICT>(p, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ batched kernels
//
// A batch is a device table of jobs, each a complete single-mesh problem (its own
// Params, snap arguments and workspace slice with the single-mesh layout).  One
// persistent launch per kernel type covers all jobs: the voxelize kernel claims
// tiles from one counter across the batch and finds a tile's job by bisection
// over the per-job tile offsets.

struct SnapArgs {
  const float *verts;
  double ox, oy, oz, h, scale, mul;
  int use_mul;
  int fixed;  // 1: vertices are int32 lattice coordinates (range check only)
  int fast;   // 1: zero origin and mul = 2^m, m >= 0: the snap in float (as in k_snap)
};

struct ZeroArgs {
  long long grid_words;
  int clear;
};

struct JobDesc {
  Params p;
  SnapArgs s;
  ZeroArgs z;
  long long pad;
};

struct BatchHeader {
  int n_jobs;
  int pad0;
  unsigned long long total_tiles;
  unsigned long long total_verts;
  unsigned long long tile_counter;
  unsigned long long reserved[28];
};
static_assert(sizeof(BatchHeader) == 256, "batch header is 256 bytes");

// Largest j in [0, n) with base[j] <= x (base ascending, base[0] = 0).
__device__ __forceinline__ int find_job(const unsigned long long *base, int n, unsigned long long x) {
  int a = 0, b = n - 1;
  while (a < b) {
    const int mid = (a + b + 1) >> 1;
    if (base[mid] <= x) a = mid;
    else b = mid - 1;
  }
  return a;
}

// Every job's header (64 words), redo bitmap and, unless accumulating, grid, zeroed in one
// pass: word g of the batch's zeroing belongs to the job j with zero_base[j] <= g <
// zero_base[j + 1] (host-built prefix), so consecutive threads store consecutive words
// whatever the jobs' sizes, instead of every thread visiting every job in turn.
__global__ void k_prologue_batched(const BatchHeader *bh, const JobDesc *jobs, const unsigned long long *zero_base) {
  const int n = bh->n_jobs;
  if (n <= 0) return;
  const unsigned long long total = zero_base[n];
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int j = find_job(zero_base, n, g);
  for (; g < total; g += stride) {
    while (g >= zero_base[j + 1]) ++j;  // zero_base[n] = total > g, so j stays below n
    const Params &p = jobs[j].p;
    const long long i = (long long)(g - zero_base[j]);
    const long long redo_words = (p.n_tets + 31) / 32;
    if (i < 64) reinterpret_cast<uint32_t *>(p.hdr)[i] = 0u;
    else if (i < 64 + redo_words) p.redo[i - 64] = 0u;
    else p.out[i - 64 - redo_words] = 0u;  // counted only when the job clears its grid
  }
}

__global__ void k_snap_batched(const BatchHeader *bh, const JobDesc *jobs, const unsigned long long *vert_base) {
  const int n = bh->n_jobs;
  const unsigned long long total = bh->total_verts;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long g = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += stride) {
    const int j = find_job(vert_base, n, g);
    const JobDesc &d = jobs[j];
    const long long i = (long long)(g - vert_base[j]);
    int X[3] = {0, 0, 0};
    int flag = 0, err = 0;
    if (d.s.fixed) {
      const int *xyz = reinterpret_cast<const int *>(d.s.verts);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int x = xyz[3 * i + q];
        if (x < -kCoordLimit || x > kCoordLimit) {
          flag = 1;
          err |= kErrRange;
        } else {
          X[q] = x;
        }
      }
    } else {
      const double o[3] = {d.s.ox, d.s.oy, d.s.oz};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float f = d.s.verts[3 * i + q];
        if (!isfinite(f)) {
          flag = 1;
          err |= kErrNan;
          continue;
        }
        if (d.s.fast) {
          const float rf = rintf(__fmul_rn(f, (float)d.s.mul));
          if (!(fabsf(rf) <= (float)kCoordLimit)) {
            flag = 1;
            err |= kErrRange;
            continue;
          }
          X[q] = (int)rf;
          continue;
        }
        const double dd = __dsub_rn((double)f, o[q]);
        const double x = d.s.use_mul ? __dmul_rn(dd, d.s.mul) : __dmul_rn(__ddiv_rn(dd, d.s.h), d.s.scale);
        const long long r = __double2ll_rn(x);
        if (r < -kCoordLimit || r > kCoordLimit) {
          flag = 1;
          err |= kErrRange;
          continue;
        }
        X[q] = (int)r;
      }
    }
    const_cast<int4 *>(d.p.verts4)[i] = make_int4(X[0], X[1], X[2], flag);
    if (err) atomicOr(&d.p.hdr->status_bits, err);
  }
}

// Row culling is one choice for a whole batch (opts->row_cull; the automatic choice culls at
// every grid side), so the kernel is compiled per choice with only that tile path in it (the
// kernel holding both spilled 328 B per thread at 80 registers against 92 B; measured on
// GB300, 256 jobs at 32^3-128^3: a replay 1.00 -> 0.94 ms).
static_assert(kCullMinRes <= 1, "the jobs of a batch share one culling choice");

template <bool STRICT, bool CULL>
__global__ void __launch_bounds__(kBlock, VOXTET_MIN_BLOCKS)
    k_voxelize_batched(BatchHeader *bh, const JobDesc *jobs, const unsigned long long *tile_base) {
  __shared__ TileSmem sm;
  uint32_t (*const slice_tab)[kBlock] = dynamic_slice_table();
  __shared__ Params sp;
  __shared__ unsigned long long tile_s;
  __shared__ int job_s;
  TileCounters ctr;
  const int n = bh->n_jobs;
  const unsigned long long total = bh->total_tiles;
  int cur = -1;
  if (threadIdx.x == 0) sm.stage.n = 0;
  for (;;) {
    if (threadIdx.x == 0) {
      tile_s = atomicAdd(&bh->tile_counter, 1ull);
      job_s = tile_s < total ? find_job(tile_base, n, tile_s) : -1;
    }
    __syncthreads();
    const int j = job_s;
    if (j < 0) break;
    if (j != cur) {  // a new job: flush the previous job's counters, load its Params
      if (cur >= 0) flush_counters(sp.hdr, ctr);
      __syncthreads();
      if (threadIdx.x < sizeof(Params) / sizeof(uint32_t))
        reinterpret_cast<uint32_t *>(&sp)[threadIdx.x] = reinterpret_cast<const uint32_t *>(&jobs[j].p)[threadIdx.x];
      __syncthreads();
      cur = j;
    }
    const long long base = (long long)(tile_s - tile_base[j]) * kTile;
    const long long end = min(sp.n_tets, base + kTile);
    process_tile<STRICT, CULL, false, false>(sp, base, end, sm, slice_tab, ctr);
  }
  if (cur >= 0) flush_counters(sp.hdr, ctr);
}

// The exact work of every job at once: job j owns blocks block_base[j] .. block_base[j + 1] - 1
// (a host-built share of the grid, at least one block, more for jobs with more tets), so no
// block visits the jobs one after another.
template <bool STRICT>
__global__ void __launch_bounds__(128) k_exact_batched(const BatchHeader *bh, const JobDesc *jobs,
                                                       const unsigned long long *block_base) {
  const int n = bh->n_jobs;
  if (n <= 0 || blockIdx.x >= block_base[n]) return;
  const int j = find_job(block_base, n, blockIdx.x);
  const unsigned bi = blockIdx.x - (unsigned)block_base[j];
  const unsigned bn = (unsigned)(block_base[j + 1] - block_base[j]);
  exact_job<STRICT>(jobs[j].p, bi, bn);
}

// Copies each job's device-detected error bits into a dense array for one readback.
__global__ void k_gather_status(const BatchHeader *bh, const JobDesc *jobs, int *status) {
  const int n = bh->n_jobs;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
    status[j] = jobs[j].p.hdr->status_bits;
}

// ------------------------------------------------------------------ host side

static std::atomic<unsigned long long> g_launches{0};

constexpr int kMaxDevices = 64;
constexpr int kExactBlock = 128;
typedef void (*VoxKernel)(Params);
// k_voxelize variants indexed by (strided << 3) | (strict << 2) | (cull << 1) | clamp
constexpr int kVariants = 16;
template <bool STRIDED>
static VoxKernel voxelize_kernel_s(int idx) {
  switch (idx) {
    case 0: return k_voxelize<false, false, false, STRIDED>;
    case 1: return k_voxelize<false, false, true, STRIDED>;
    case 2: return k_voxelize<false, true, false, STRIDED>;
    case 3: return k_voxelize<false, true, true, STRIDED>;
    case 4: return k_voxelize<true, false, false, STRIDED>;
    case 5: return k_voxelize<true, false, true, STRIDED>;
    case 6: return k_voxelize<true, true, false, STRIDED>;
    default: return k_voxelize<true, true, true, STRIDED>;
  }
}
static VoxKernel voxelize_kernel(int idx) {
  return idx & 8 ? voxelize_kernel_s<true>(idx & 7) : voxelize_kernel_s<false>(idx & 7);
}

struct DeviceInfo {
  int sms = 0;
  int occ[kVariants] = {};  // resident blocks per SM of each k_voxelize variant
  int occ_exact = 0;        // resident blocks per SM of the exact kernels (tets, rows)
  int occ_rows = 0;
  bool ready = false;
};
static DeviceInfo g_dev[kMaxDevices];
static std::atomic<int> g_dev_lock{0};

// Events of the last profiled call, per host thread (the elapsed time is read back
// by voxtet_read_stats on the same thread).
struct ProfileEvents {
  cudaEvent_t start = nullptr, stop = nullptr;
  int device = -1;
  bool pending = false;
};
static thread_local ProfileEvents t_prof;

static cudaError_t profile_begin(cudaStream_t stream) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (t_prof.device != dev || !t_prof.start) {
    if (t_prof.start) {
      cudaEventDestroy(t_prof.start);
      cudaEventDestroy(t_prof.stop);
    }
    e = cudaEventCreate(&t_prof.start);
    if (e == cudaSuccess) e = cudaEventCreate(&t_prof.stop);
    if (e != cudaSuccess) return e;
    t_prof.device = dev;
  }
  t_prof.pending = false;
  return cudaEventRecord(t_prof.start, stream);
}

static cudaError_t device_info(DeviceInfo *&out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  DeviceInfo &d = g_dev[dev];
  if (!d.ready) {
    while (g_dev_lock.exchange(1)) {
    }
    if (!d.ready) {
      e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
      for (int v = 0; v < kVariants && e == cudaSuccess; ++v) {
        e = cudaFuncSetAttribute(reinterpret_cast<const void *>(voxelize_kernel(v)),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSliceTableBytesMax);
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ[v], voxelize_kernel(v), kBlock,
                                                            kSliceTableBytesMax);
      }
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ_exact, k_exact<false>, kExactBlock, 0);
      if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d.occ_rows, k_exact_rows<false>, kExactBlock, 0);
      if (e == cudaSuccess && d.occ_exact < 1) d.occ_exact = 1;
      if (e == cudaSuccess && d.occ_rows < 1) d.occ_rows = 1;
      if (e == cudaSuccess) d.ready = true;
    }
    g_dev_lock.store(0);
    if (e != cudaSuccess) return e;
  }
  out = &d;
  return cudaSuccess;
}

static int log2_res(int res) {
  if (res < 1 || res > VOXTET_MAX_RES || (res & (res - 1))) return -1;
  int k = 0;
  while ((1 << k) != res) ++k;
  return k;
}

// The grid of one call: rx x ry x rz voxels, slices z0 <= l < z1 produced, lattice
// exponent K (the lattice step is 2^(20-K) per voxel, K = ceil(log2 of the longest side)).
struct GridDims {
  int rx, ry, rz, z0, z1, K;
  int longest() const { return rx > ry ? (rx > rz ? rx : rz) : (ry > rz ? ry : rz); }
  long long out_words() const { return (long long)(z1 - z0) * ry * ((rx + 31) / 32); }
};

static GridDims cubic_dims(int res, int k) { return GridDims{res, res, res, 0, res, k}; }

// General grid from the caller's sides and slab; VOXTET_ERR_RES for a side outside
// [1, VOXTET_MAX_RES], VOXTET_ERR_ARG for a slab outside [0, rz].
static int general_dims(const int32_t res[3], int32_t z_begin, int32_t z_end, GridDims &g) {
  for (int q = 0; q < 3; ++q)
    if (res[q] < 1 || res[q] > VOXTET_MAX_RES) return VOXTET_ERR_RES;
  g.rx = res[0];
  g.ry = res[1];
  g.rz = res[2];
  if (z_begin < 0 || z_end > g.rz || z_begin > z_end) return VOXTET_ERR_ARG;
  g.z0 = z_begin;
  g.z1 = z_end;
  g.K = 0;
  while ((1 << g.K) < g.longest()) ++g.K;
  return VOXTET_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carved workspace: header, snapped vertices, tet queue, row queue, redo bitmap.
struct Workspace {
  Header *hdr;
  int4 *verts4;
  uint32_t *tetq;
  RowItem *rowq;
  uint32_t *redo;
  unsigned q_cap;
  long long redo_words;
};

// Layout: header, snapped vertices, tet queue, redo bitmap, row queue.  The row queue
// comes last and takes whatever the caller's workspace holds beyond the minimum
// (ws_bytes; 0 = the minimum), so a larger workspace means fewer whole-tet redos.
static size_t workspace_bytes(long long n_tets, long long n_verts, Workspace *w, void *base, size_t ws_bytes = 0) {
  unsigned long long q = row_queue_capacity(n_tets);
  const long long redo_words = (n_tets + 31) / 32;
  size_t o = sizeof(Header);
  const size_t o_v = o;
  o += align256((size_t)n_verts * sizeof(int4));
  const size_t o_t = o;
  o += align256((size_t)n_tets * sizeof(uint32_t));
  const size_t o_b = o;
  o += align256((size_t)redo_words * sizeof(uint32_t));
  const size_t o_r = o;
  o += align256((size_t)q * sizeof(RowItem));
  if (ws_bytes > o) {
    unsigned long long more = (ws_bytes - o_r) / sizeof(RowItem);
    if (more > 0xFFFFFFFFull) more = 0xFFFFFFFFull;
    if (more > q) q = more;
  }
  if (w) {
    char *c = reinterpret_cast<char *>(base);
    w->hdr = reinterpret_cast<Header *>(c);
    w->verts4 = reinterpret_cast<int4 *>(c + o_v);
    w->tetq = reinterpret_cast<uint32_t *>(c + o_t);
    w->rowq = reinterpret_cast<RowItem *>(c + o_r);
    w->redo = reinterpret_cast<uint32_t *>(c + o_b);
    w->q_cap = (unsigned)q;
    w->redo_words = redo_words;
  }
  return o;
}

static int map_status_bits(int bits) {
  if (bits & kErrNan) return VOXTET_ERR_NAN;
  if (bits & kErrRange) return VOXTET_ERR_RANGE;
  if (bits & kErrIndex) return VOXTET_ERR_INDEX;
  return VOXTET_OK;
}

static void resolve_opts(const voxtet_opts *in, voxtet_opts &o) {
  voxtet_default_opts(&o);
  if (in) o = *in;
}

static int check_opts(const voxtet_opts &o) {
  if (o.mode != 0 && o.mode != 1) return VOXTET_ERR_ARG;
  if (o.accumulate != 0 && o.accumulate != 1) return VOXTET_ERR_ARG;
  if (o.use_filter != 0 && o.use_filter != 1) return VOXTET_ERR_ARG;
  if (o.sync != 0 && o.sync != 1) return VOXTET_ERR_ARG;
  if (o.span_rows < 0 || o.span_rows > (1 << 20)) return VOXTET_ERR_ARG;
  if (o.block != 0 && o.block != kBlock) return VOXTET_ERR_ARG;
  if (o.profile != 0 && o.profile != 1) return VOXTET_ERR_ARG;
  if (o.row_cull < 0 || o.row_cull > 2) return VOXTET_ERR_ARG;
  if (o.kernel < 0 || o.kernel > 2) return VOXTET_ERR_ARG;
  return VOXTET_OK;
}

// Which distribution of the scanline work a call uses (both give the same grid).
// Automatic: slice units where they measured faster on GB300 (sliver mesh, 1.3M tets:
// 512^3 kernel 332 -> 309 us, 1024^3 1075 -> 1038 us), spans elsewhere.
static bool use_slice_units(const voxtet_opts &o, const GridDims &g) {
  if (o.kernel == 2) return true;
  if (o.kernel == 1) return false;
  // slice units up to 1024 per side (measured on GB300 with culling on: 64^3 grid of the 8^3
  // lattice 45.1 -> 39.9 us, 256^3 torus 24.6 -> 19.5 us, 512^3 sliver mesh 330 -> 279 us);
  // from 2048 a tet spans more slices than a tile holds
  return g.longest() <= 1024;
}

// Shared tail of both entry points: vertices are already in the workspace.
static int run_voxelize(const Workspace &w, long long n_verts, const int32_t *tets, long long n_tets,
                        const GridDims &g, uint32_t *out, const voxtet_opts &o, cudaStream_t stream,
                        bool vflags = false) {
  DeviceInfo *dev = nullptr;
  if (device_info(dev) != cudaSuccess) return VOXTET_ERR_CUDA;
  if (n_tets > 0) {
    Params p{};  // every field zero unless set below (list_mode = 0)
    p.vflags = vflags ? 1 : 0;
    p.verts4 = w.verts4;
    p.tets = reinterpret_cast<const int4 *>(tets);
    p.n_tets = n_tets;
    p.n_verts = n_verts;
    p.out = out;
    p.hdr = w.hdr;
    p.tetq = w.tetq;
    p.rowq = w.rowq;
    p.redo = w.redo;
    p.q_cap = w.q_cap;
    p.rx = g.rx;
    p.ry = g.ry;
    p.z0 = g.z0;
    p.z1 = g.z1;
    p.W = (g.rx + 31) / 32;
    p.sh = kLatticeBits - g.K;
    p.span_rows = o.span_rows > 0 ? o.span_rows : default_span_rows(g.longest());
    p.max_slices = g.longest() >= 1024 ? 32 : 16;
    p.exact_all = o.use_filter ? 0 : 1;
    const bool cull = o.row_cull == 1 || (o.row_cull == 0 && g.longest() >= kCullMinRes);
    const bool clamp = g.longest() >= kClampMinRes;
    // Slabs thinner than an eighth of the grid take strided tiles (their tets are a thin band
    // of a mesh numbered along z, which contiguous tiles would hand to a few blocks); thicker
    // slabs keep contiguous tiles, whose spatially coherent ORs use L2 better (measured on
    // GB300, brick-sparse torus: 4096^3 in quarter slabs 17.7 ms strided, 11.5 contiguous;
    // 8192^3 in 1/32 slabs 100 ms strided, 111 contiguous).
    const bool strided = (long long)(g.z1 - g.z0) * 8 < g.rz;
    const int variant = (strided ? 8 : 0) | (o.mode == 1 ? 4 : 0) | (cull ? 2 : 0) | (clamp ? 1 : 0);
    long long grid = (long long)dev->sms * (dev->occ[variant] > 0 ? dev->occ[variant] : 1);
    const long long tail = 2 * grid * kSmallTile;
    p.big_tiles = n_tets > tail ? (n_tets - tail) / kTile : 0;
    long long tiles = p.big_tiles + (n_tets - p.big_tiles * kTile + kSmallTile - 1) / kSmallTile;
    // a thin slab of the grid: strided tiles, so the slab's tets (often one contiguous run of
    // a mesh numbered by z) are shared by every block (measured on GB300: an 8192^3 grid in
    // slabs of 256 slices ran at half the speed of the whole grid with contiguous tiles)
    p.tile_stride = 0;
    if (strided) {
      // at least one tile per resident block: a slab's share of a mesh is often small, and
      // fewer, fuller tiles would leave blocks idle (tile slots past the mesh stay empty)
      long long stride = (n_tets + kTile - 1) / kTile;
      if (stride < grid) stride = n_tets < grid ? n_tets : grid;
      p.tile_stride = stride;
      tiles = stride;
    }
    if (grid > tiles) grid = tiles;
    if (o.profile && profile_begin(stream) != cudaSuccess) return VOXTET_ERR_CUDA;
    if (use_slice_units(o, g)) {
      // slice units for the tets that fit them, then the span kernel over the tets it listed
      // 16 slices per tet (7 blocks per SM) up to 512 voxels per side, where a tet of a mesh
      // fine enough for the grid spans a few slices (sliver mesh: at most 13), 32 above
      // (measured on GB300, sliver mesh 512^3: 308 -> 285 us with 16); a tet spanning more
      // goes to the list pass either way
      const int cap = g.longest() <= 512 ? kSuSlicesSmall : kSuSlices;
      if (launch_slices(p, variant, cap, dev->sms, stream) != VOXTET_OK) return VOXTET_ERR_CUDA;
      g_launches.fetch_add(1);
      Params q = p;
      q.list_mode = 1;
      q.tile_stride = 0;
      q.big_tiles = (n_tets + kTile - 1) / kTile + 1;  // whole tiles only
      // one block per SM: the list is usually empty or short (tets spanning more than 32
      // slices or 1024 rows per slice), and an empty list then costs one short wave
      const int lv = variant & 7;
      if (launch_chained(voxelize_kernel(lv), (unsigned)dev->sms, kBlock, slice_table_bytes(q.max_slices), stream,
                         q) != cudaSuccess)
        return VOXTET_ERR_CUDA;
    } else {
      if (launch_chained(voxelize_kernel(variant), (unsigned)grid, kBlock, slice_table_bytes(p.max_slices), stream,
                         p) != cudaSuccess)
        return VOXTET_ERR_CUDA;
    }
    g_launches.fetch_add(1);
    if (cudaGetLastError() != cudaSuccess) return VOXTET_ERR_CUDA;
    if (o.profile) {
      if (cudaEventRecord(t_prof.stop, stream) != cudaSuccess) return VOXTET_ERR_CUDA;
      t_prof.pending = true;
    }
    // one wave of resident blocks each: the queued rows are spread evenly over the threads
    const unsigned rg = (unsigned)dev->sms * (unsigned)dev->occ_rows;
    if (launch_chained(o.mode == 1 ? k_exact_rows<true> : k_exact_rows<false>, rg, kExactBlock, 0, stream, p) !=
        cudaSuccess)
      return VOXTET_ERR_CUDA;
    g_launches.fetch_add(1);
    const unsigned eg = (unsigned)dev->sms * (unsigned)dev->occ_exact;
    if (launch_chained(o.mode == 1 ? k_exact<true> : k_exact<false>, eg, kExactBlock, 0, stream, p) != cudaSuccess)
      return VOXTET_ERR_CUDA;
    g_launches.fetch_add(1);
    if (cudaGetLastError() != cudaSuccess) return VOXTET_ERR_CUDA;
  }
  if (o.sync) {
    if (cudaStreamSynchronize(stream) != cudaSuccess) return VOXTET_ERR_CUDA;
    int bits = 0;
    if (cudaMemcpy(&bits, &w.hdr->status_bits, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      return VOXTET_ERR_CUDA;
    return map_status_bits(bits);
  }
  return VOXTET_OK;
}

static int launch_prologue(const Workspace &w, uint32_t *out, long long n_words, int clear, cudaStream_t stream) {
  DeviceInfo *dev = nullptr;
  if (device_info(dev) != cudaSuccess) return VOXTET_ERR_CUDA;
  long long blocks = clear ? (n_words / 4 + 255) / 256 : (w.redo_words + 255) / 256;
  const long long cap = (long long)dev->sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_prologue<<<(unsigned)blocks, 256, 0, stream>>>(w.hdr, w.redo, w.redo_words, out, n_words, clear);
  g_launches.fetch_add(1);
  return cudaGetLastError() == cudaSuccess ? VOXTET_OK : VOXTET_ERR_CUDA;
}

static int grid_blocks(long long n, int per_block, int sms) {
  long long b = (n + per_block - 1) / per_block;
  const long long cap = (long long)sms * 16;
  if (b > cap) b = cap;
  return (int)(b < 1 ? 1 : b);
}

// Sizes, alignment and workspace capacity shared by every single-mesh entry point.
static int buffer_checks(long long n_verts, const void *tets, long long n_tets, const uint32_t *out, void *ws,
                         size_t ws_bytes, bool out_may_be_null = false) {
  if (n_verts < 0 || n_tets < 0 || n_verts > 0x7FFFFFFFLL || n_tets > 0xFFFFFFFFLL) return VOXTET_ERR_ARG;
  if (!out && !out_may_be_null) return VOXTET_ERR_ARG;
  if (n_tets > 0 && (!tets || (reinterpret_cast<uintptr_t>(tets) & 15))) return VOXTET_ERR_ARG;
  if (reinterpret_cast<uintptr_t>(out) & 3) return VOXTET_ERR_ARG;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255)) return VOXTET_ERR_WORKSPACE;
  if (ws_bytes < workspace_bytes(n_tets, n_verts, nullptr, nullptr)) return VOXTET_ERR_WORKSPACE;
  return VOXTET_OK;
}

static int common_checks(long long n_verts, const void *tets, long long n_tets, int res, const uint32_t *out,
                         void *ws, size_t ws_bytes, const voxtet_opts &o, int &k) {
  int st = check_opts(o);
  if (st != VOXTET_OK) return st;
  k = log2_res(res);
  if (k < 0) return VOXTET_ERR_RES;
  return buffer_checks(n_verts, tets, n_tets, out, ws, ws_bytes);
}

// The snap's scalars: X = round_half_even(((double)v - o) / h * 2^(20-K)).
static SnapArgsK snap_args(const float grid_origin[3], float voxel_size, int K) {
  SnapArgsK a;
  a.ox = (double)grid_origin[0];
  a.oy = (double)grid_origin[1];
  a.oz = (double)grid_origin[2];
  a.h = (double)voxel_size;
  a.scale = std::ldexp(1.0, kLatticeBits - K);
  int e2 = 0;
  const double mant = std::frexp(a.h, &e2);
  a.use_mul = mant == 0.5 ? 1 : 0;
  a.mul = a.use_mul ? std::ldexp(1.0, kLatticeBits - K - (e2 - 1)) : 0.0;
  a.fast = a.use_mul && a.mul >= 1.0 && a.mul <= 0x1p100 && grid_origin[0] == 0.0f && grid_origin[1] == 0.0f &&
           grid_origin[2] == 0.0f;
  return a;
}

// Snap kernel launch (after a separate prologue; errors go to the header at once).
static int launch_snap(const Workspace &w, const float *d_verts, long long n_verts, const float grid_origin[3],
                       float voxel_size, int K, cudaStream_t stream) {
  DeviceInfo *dev = nullptr;
  if (device_info(dev) != cudaSuccess) return VOXTET_ERR_CUDA;
  if (n_verts <= 0) return VOXTET_OK;
  if (launch_chained(k_snap, (unsigned)grid_blocks(n_verts, 256, dev->sms), 256, 0, stream, d_verts, n_verts,
                     snap_args(grid_origin, voxel_size, K), w.verts4, w.hdr) != cudaSuccess)
    return VOXTET_ERR_CUDA;
  g_launches.fetch_add(1);
  return cudaGetLastError() == cudaSuccess ? VOXTET_OK : VOXTET_ERR_CUDA;
}

// The prologue and the vertex snap (FIXED: the lattice load) in one launch.  Only for calls
// with tets: their k_exact folds the vertices' error bits into the status (p.vflags).
template <bool FIXED>
static int launch_prep(const Workspace &w, uint32_t *out, long long n_words, int clear, const void *src,
                       long long n_verts, const SnapArgsK &a, cudaStream_t stream) {
  DeviceInfo *dev = nullptr;
  if (device_info(dev) != cudaSuccess) return VOXTET_ERR_CUDA;
  long long work = n_verts;
  if (clear && n_words / 4 > work) work = n_words / 4;
  if (w.redo_words > work) work = w.redo_words;
  long long blocks = (work + 255) / 256;
  const long long cap = (long long)dev->sms * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  k_prep<FIXED><<<(unsigned)blocks, 256, 0, stream>>>(w.hdr, w.redo, w.redo_words, out, n_words, clear, src, n_verts,
                                                      a, w.verts4);
  g_launches.fetch_add(1);
  return cudaGetLastError() == cudaSuccess ? VOXTET_OK : VOXTET_ERR_CUDA;
}

// The front of a dense call: one fused launch when the call has tets (vflags = true: the exact
// kernel reports the vertices' errors), else the prologue and a snap that reports them itself.
static int launch_front(const Workspace &w, uint32_t *out, long long n_words, int clear, const void *src,
                        long long n_verts, long long n_tets, const SnapArgsK &a, bool fixed, cudaStream_t stream,
                        bool &vflags) {
  vflags = n_tets > 0 && n_verts > 0;
  if (vflags)
    return fixed ? launch_prep<true>(w, out, n_words, clear, src, n_verts, a, stream)
                 : launch_prep<false>(w, out, n_words, clear, src, n_verts, a, stream);
  int st = launch_prologue(w, out, n_words, clear, stream);
  if (st != VOXTET_OK || n_verts <= 0) return st;
  DeviceInfo *dev = nullptr;
  if (device_info(dev) != cudaSuccess) return VOXTET_ERR_CUDA;
  const unsigned blocks = (unsigned)grid_blocks(n_verts, 256, dev->sms);
  const cudaError_t e =
      fixed ? launch_chained(k_load_fixed, blocks, 256, 0, stream, static_cast<const int *>(src), n_verts, w.verts4,
                             w.hdr)
            : launch_chained(k_snap, blocks, 256, 0, stream, static_cast<const float *>(src), n_verts, a, w.verts4,
                             w.hdr);
  if (e != cudaSuccess) return VOXTET_ERR_CUDA;
  g_launches.fetch_add(1);
  return VOXTET_OK;
}

static int float_input_checks(const float *d_verts, long long n_verts, const float grid_origin[3],
                              float voxel_size) {
  if (!grid_origin) return VOXTET_ERR_ARG;
  if (n_verts > 0 && (!d_verts || (reinterpret_cast<uintptr_t>(d_verts) & 3))) return VOXTET_ERR_ARG;
  if (!(voxel_size > 0.0f) || !std::isfinite(voxel_size)) return VOXTET_ERR_ARG;
  for (int q = 0; q < 3; ++q)
    if (!std::isfinite(grid_origin[q])) return VOXTET_ERR_ARG;
  return VOXTET_OK;
}

}  // namespace voxtet

using namespace voxtet;

extern "C" {

void voxtet_default_opts(voxtet_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mode = 0;
  o->accumulate = 0;
  o->use_filter = 1;
  o->sync = 1;
  o->span_rows = 0;
  o->block = 0;
  o->profile = 0;
  o->row_cull = 0;
  o->kernel = 0;
}

size_t voxtet_workspace_size(int64_t n_tets, int64_t n_verts, int32_t res) {
  if (n_tets < 0 || n_verts < 0) return 0;
  const size_t minimum = workspace_bytes(n_tets, n_verts, nullptr, nullptr);
  // Uncertain rows grow with the rows a tet spans, about (res / 512)^2 for a given mesh:
  // from 1024 up the row queue gets n_tets * (res / 512)^2 / 8 entries (measured on the
  // sliver and torus workloads: 0.4-0.9 uncertain rows per tet at 1024^3-8192^3 with the
  // clamped filter), so that a queue overflow and whole-tet redos stay rare.
  if (res <= 512) return minimum;
  const double scale = (double)res / 512.0;
  const double want = (double)n_tets * scale * scale / 8.0;
  const unsigned long long q = want > 4.0e9 ? 4000000000ull : (unsigned long long)want;
  if (q <= row_queue_capacity(n_tets)) return minimum;
  return minimum + align256((size_t)(q - row_queue_capacity(n_tets)) * sizeof(RowItem));
}

int voxelize_tets(const float *d_verts, int64_t n_verts, const int32_t *d_tets, int64_t n_tets,
                  const float grid_origin[3], float voxel_size, int32_t res, uint32_t *d_out_bits, void *d_workspace,
                  size_t ws_bytes, const voxtet_opts *opts, void *stream_) {
  voxtet_opts o;
  resolve_opts(opts, o);
  int k = 0;
  int st = common_checks(n_verts, d_tets, n_tets, res, d_out_bits, d_workspace, ws_bytes, o, k);
  if (st != VOXTET_OK) return st;
  st = float_input_checks(d_verts, n_verts, grid_origin, voxel_size);
  if (st != VOXTET_OK) return st;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  Workspace w;
  workspace_bytes(n_tets, n_verts, &w, d_workspace, ws_bytes);
  const GridDims g = cubic_dims(res, k);
  bool vflags = false;
  st = launch_front(w, d_out_bits, g.out_words(), o.accumulate ? 0 : 1, d_verts, n_verts, n_tets,
                    snap_args(grid_origin, voxel_size, g.K), false, stream, vflags);
  if (st != VOXTET_OK) return st;
  return run_voxelize(w, n_verts, d_tets, n_tets, g, d_out_bits, o, stream, vflags);
}

int voxelize_tets_grid(const float *d_verts, int64_t n_verts, const int32_t *d_tets, int64_t n_tets,
                       const float grid_origin[3], float voxel_size, const int32_t res[3], int32_t z_begin,
                       int32_t z_end, uint32_t *d_out_bits, void *d_workspace, size_t ws_bytes,
                       const voxtet_opts *opts, void *stream_) {
  voxtet_opts o;
  resolve_opts(opts, o);
  int st = check_opts(o);
  if (st != VOXTET_OK) return st;
  if (!res) return VOXTET_ERR_ARG;
  GridDims g;
  st = general_dims(res, z_begin, z_end, g);
  if (st != VOXTET_OK) return st;
  // an empty slab writes nothing, so its output pointer may be NULL
  st = buffer_checks(n_verts, d_tets, n_tets, d_out_bits, d_workspace, ws_bytes, g.out_words() == 0);
  if (st != VOXTET_OK) return st;
  st = float_input_checks(d_verts, n_verts, grid_origin, voxel_size);
  if (st != VOXTET_OK) return st;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  Workspace w;
  workspace_bytes(n_tets, n_verts, &w, d_workspace, ws_bytes);
  bool vflags = false;
  st = launch_front(w, d_out_bits, g.out_words(), o.accumulate ? 0 : 1, d_verts, n_verts, n_tets,
                    snap_args(grid_origin, voxel_size, g.K), false, stream, vflags);
  if (st != VOXTET_OK) return st;
  return run_voxelize(w, n_verts, d_tets, n_tets, g, d_out_bits, o, stream, vflags);
}

int voxelize_tets_fixed(const int32_t *d_xyz, int64_t n_verts, const int32_t *d_tets, int64_t n_tets, int32_t res,
                        uint32_t *d_out_bits, void *d_workspace, size_t ws_bytes, const voxtet_opts *opts,
                        void *stream_) {
  voxtet_opts o;
  resolve_opts(opts, o);
  int k = 0;
  int st = common_checks(n_verts, d_tets, n_tets, res, d_out_bits, d_workspace, ws_bytes, o, k);
  if (st != VOXTET_OK) return st;
  if (n_verts > 0 && (!d_xyz || (reinterpret_cast<uintptr_t>(d_xyz) & 3))) return VOXTET_ERR_ARG;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  Workspace w;
  workspace_bytes(n_tets, n_verts, &w, d_workspace, ws_bytes);
  const GridDims g = cubic_dims(res, k);
  bool vflags = false;
  st = launch_front(w, d_out_bits, g.out_words(), o.accumulate ? 0 : 1, d_xyz, n_verts, n_tets, SnapArgsK{}, true,
                    stream, vflags);
  if (st != VOXTET_OK) return st;
  return run_voxelize(w, n_verts, d_tets, n_tets, g, d_out_bits, o, stream, vflags);
}

int voxtet_last_status(const void *d_workspace, void *stream_) {
  if (!d_workspace) return VOXTET_ERR_WORKSPACE;
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream_)) != cudaSuccess) return VOXTET_ERR_CUDA;
  int bits = 0;
  if (cudaMemcpy(&bits, &reinterpret_cast<const Header *>(d_workspace)->status_bits, sizeof(int),
                 cudaMemcpyDeviceToHost) != cudaSuccess)
    return VOXTET_ERR_CUDA;
  return map_status_bits(bits);
}

int voxtet_status_async(const void *d_workspace, int32_t *status_word, void *stream_) {
  if (!d_workspace || !status_word) return VOXTET_ERR_ARG;
  const cudaError_t e = cudaMemcpyAsync(status_word, &reinterpret_cast<const Header *>(d_workspace)->status_bits,
                                        sizeof(int32_t), cudaMemcpyDefault, reinterpret_cast<cudaStream_t>(stream_));
  return e == cudaSuccess ? VOXTET_OK : VOXTET_ERR_CUDA;
}

int voxtet_status_of_word(int32_t status_word) { return map_status_bits(status_word); }

int voxtet_read_stats(const void *d_workspace, voxtet_stats *out, void *stream_) {
  if (!d_workspace || !out) return VOXTET_ERR_ARG;
  if (cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream_)) != cudaSuccess) return VOXTET_ERR_CUDA;
  Header h;
  if (cudaMemcpy(&h, d_workspace, sizeof(Header), cudaMemcpyDeviceToHost) != cudaSuccess) return VOXTET_ERR_CUDA;
  std::memset(out, 0, sizeof(*out));
  out->spans = h.spans;
  out->rows = h.rows;
  out->fallback_rows = h.rowq_count;
  out->degenerate_tets = h.degenerate;
  out->wide_tets = h.wide;
  out->exact_tets = h.tetq_count;
  if (t_prof.pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(t_prof.stop) != cudaSuccess ||
        cudaEventElapsedTime(&ms, t_prof.start, t_prof.stop) != cudaSuccess)
      return VOXTET_ERR_CUDA;
    out->kernel_ns = (uint64_t)((double)ms * 1.0e6);
  }
  return VOXTET_OK;
}

const char *voxtet_strerror(int s) {
  switch (s) {
    case VOXTET_OK: return "ok";
    case VOXTET_ERR_ARG: return "invalid argument";
    case VOXTET_ERR_RES: return "resolution must be a power of two in [1, VOXTET_MAX_RES] (grid sides: in [1, VOXTET_MAX_RES])";
    case VOXTET_ERR_INDEX: return "tetrahedron vertex index out of range";
    case VOXTET_ERR_RANGE: return "snapped vertex coordinate beyond 2^21 lattice units";
    case VOXTET_ERR_NAN: return "non-finite vertex coordinate";
    case VOXTET_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case VOXTET_ERR_CUDA: return "CUDA runtime error";
    case VOXTET_ERR_TIMEOUT: return "device-side wait timed out";
    case VOXTET_ERR_NOMEM: return "arena too small";
    default: return "unknown status";
  }
}

uint64_t voxtet_launch_count(void) { return g_launches.load(); }

}  // extern "C"

// ------------------------------------------------------------------ batches (host side)

namespace voxtet {

// Layout of a batch workspace: BatchHeader, JobDesc[cap], tile_base[cap + 1],
// vert_base[cap + 1], zero_base[cap + 1], block_base[cap + 1], status[cap] (each 256-byte
// aligned), then one single-mesh workspace slice per job.  The leading part (up to the
// first slice) is built on the host and uploaded with one copy per run.
struct BatchLayout {
  size_t o_table, o_tiles, o_verts, o_zero, o_blocks, o_status, o_slices;
};

static BatchLayout batch_layout(int cap) {
  BatchLayout L;
  size_t o = sizeof(BatchHeader);
  L.o_table = o;
  o += align256((size_t)cap * sizeof(JobDesc));
  L.o_tiles = o;
  o += align256((size_t)(cap + 1) * sizeof(unsigned long long));
  L.o_verts = o;
  o += align256((size_t)(cap + 1) * sizeof(unsigned long long));
  L.o_zero = o;
  o += align256((size_t)(cap + 1) * sizeof(unsigned long long));
  L.o_blocks = o;
  o += align256((size_t)(cap + 1) * sizeof(unsigned long long));
  L.o_status = o;
  o += align256((size_t)cap * sizeof(int));
  L.o_slices = o;
  return L;
}

static int check_job(const voxtet_job &j, int &k) {
  k = log2_res(j.res);
  if (k < 0) return VOXTET_ERR_RES;
  if (j.n_verts < 0 || j.n_tets < 0 || j.n_verts > 0x7FFFFFFFLL || j.n_tets > 0xFFFFFFFFLL) return VOXTET_ERR_ARG;
  if (!j.d_out_bits || (reinterpret_cast<uintptr_t>(j.d_out_bits) & 3)) return VOXTET_ERR_ARG;
  if (j.n_tets > 0 && (!j.d_tets || (reinterpret_cast<uintptr_t>(j.d_tets) & 15))) return VOXTET_ERR_ARG;
  if (j.n_verts > 0 && (!j.d_verts || (reinterpret_cast<uintptr_t>(j.d_verts) & 3))) return VOXTET_ERR_ARG;
  if (j.span_rows < 0 || j.span_rows > (1 << 20)) return VOXTET_ERR_ARG;
  if (!j.fixed_point) {
    if (!(j.voxel_size > 0.0f) || !std::isfinite(j.voxel_size)) return VOXTET_ERR_ARG;
    for (int q = 0; q < 3; ++q)
      if (!std::isfinite(j.origin[q])) return VOXTET_ERR_ARG;
  }
  return VOXTET_OK;
}

static size_t job_slice_bytes(const voxtet_job &j, bool valid) {
  return valid ? align256(voxtet_workspace_size(j.n_tets, j.n_verts, j.res)) : align256(sizeof(Header));
}

// Blocks of the batched exact kernel: fixed per capacity (a plan's graph keeps its launch
// shape while its jobs change), at least one per job.
static long long exact_batch_blocks(int cap) {
  DeviceInfo *dev = nullptr;
  const long long sms = device_info(dev) == cudaSuccess ? dev->sms : 152;
  return cap > sms * 4 ? (long long)cap : sms * 4;
}

// Builds the host image of the table part of a batch workspace.  Returns the bytes
// of workspace the batch needs (0 on a batch-level argument error).
static size_t build_batch_image(const voxtet_job *jobs, int n, int cap, const voxtet_opts &o, char *ws_dev,
                                std::vector<char> *image, int *host_status) {
  const BatchLayout L = batch_layout(cap);
  size_t need = L.o_slices;
  std::vector<int> ok(n);
  std::vector<int> kk(n);
  for (int j = 0; j < n; ++j) {
    const int st = check_job(jobs[j], kk[j]);
    ok[j] = st == VOXTET_OK;
    if (host_status) host_status[j] = st;
    need += job_slice_bytes(jobs[j], ok[j]);
  }
  if (!image) return need;
  image->assign(L.o_slices, 0);
  char *img = image->data();
  BatchHeader *bh = reinterpret_cast<BatchHeader *>(img);
  JobDesc *tab = reinterpret_cast<JobDesc *>(img + L.o_table);
  unsigned long long *tiles = reinterpret_cast<unsigned long long *>(img + L.o_tiles);
  unsigned long long *vbase = reinterpret_cast<unsigned long long *>(img + L.o_verts);
  unsigned long long *zbase = reinterpret_cast<unsigned long long *>(img + L.o_zero);
  unsigned long long *bbase = reinterpret_cast<unsigned long long *>(img + L.o_blocks);
  size_t off = L.o_slices;
  unsigned long long tsum = 0, vsum = 0, zsum = 0;
  long long all_tets = 0;
  for (int j = 0; j < n; ++j) all_tets += ok[j] ? jobs[j].n_tets : 0;
  const long long spare = exact_batch_blocks(cap) - n;  // blocks beyond one per job, shared by tets
  unsigned long long bsum = 0;
  for (int j = 0; j < n; ++j) {
    const voxtet_job &J = jobs[j];
    const long long nt = ok[j] ? J.n_tets : 0, nv = ok[j] ? J.n_verts : 0;
    Workspace w;
    workspace_bytes(nt, nv, &w, ws_dev + off, ok[j] ? job_slice_bytes(J, true) : 0);
    off += job_slice_bytes(J, ok[j]);
    JobDesc &d = tab[j];
    std::memset(&d, 0, sizeof(d));
    const int res = ok[j] ? J.res : 1;
    const int k = ok[j] ? kk[j] : 0;
    d.p.verts4 = w.verts4;
    d.p.tets = reinterpret_cast<const int4 *>(J.d_tets);
    d.p.n_tets = nt;
    d.p.n_verts = nv;
    d.p.out = J.d_out_bits;
    d.p.hdr = w.hdr;
    d.p.tetq = w.tetq;
    d.p.rowq = w.rowq;
    d.p.redo = w.redo;
    d.p.q_cap = w.q_cap;
    d.p.max_slices = 16;  // batch jobs are small grids (see kMaxSlicesPerSpan)
    d.p.rx = res;
    d.p.ry = res;
    d.p.z0 = 0;
    d.p.z1 = res;
    d.p.W = (res + 31) / 32;
    d.p.sh = kLatticeBits - k;
    d.p.span_rows = J.span_rows > 0 ? J.span_rows : (o.span_rows > 0 ? o.span_rows : default_span_rows(res));
    d.p.exact_all = o.use_filter ? 0 : 1;
    d.p.cull = (o.row_cull == 1 || (o.row_cull == 0 && res >= kCullMinRes)) ? 1 : 0;
    d.s.verts = reinterpret_cast<const float *>(J.d_verts);
    d.s.fixed = J.fixed_point ? 1 : 0;
    if (ok[j] && !J.fixed_point) {
      d.s.ox = J.origin[0];
      d.s.oy = J.origin[1];
      d.s.oz = J.origin[2];
      d.s.h = (double)J.voxel_size;
      d.s.scale = std::ldexp(1.0, kLatticeBits - k);
      int e2 = 0;
      const double mant = std::frexp(d.s.h, &e2);
      d.s.use_mul = mant == 0.5 ? 1 : 0;
      d.s.mul = d.s.use_mul ? std::ldexp(1.0, kLatticeBits - k - (e2 - 1)) : 0.0;
      d.s.fast = d.s.use_mul && d.s.mul >= 1.0 && d.s.mul <= 0x1p100 && J.origin[0] == 0.0f && J.origin[1] == 0.0f &&
                 J.origin[2] == 0.0f;
    }
    d.z.grid_words = ok[j] ? (long long)res * res * d.p.W : 0;
    d.z.clear = (ok[j] && !o.accumulate) ? 1 : 0;
    tiles[j] = tsum;
    vbase[j] = vsum;
    zbase[j] = zsum;
    bbase[j] = bsum;
    tsum += (unsigned long long)((nt + kTile - 1) / kTile);
    vsum += (unsigned long long)nv;
    // header words, redo bitmap words, grid words (k_prologue_batched's order)
    zsum += 64ull + (unsigned long long)((nt + 31) / 32) + (d.z.clear ? (unsigned long long)d.z.grid_words : 0ull);
    bsum += 1ull + (all_tets > 0 && spare > 0 ? (unsigned long long)((double)spare * (double)nt / (double)all_tets) : 0ull);
  }
  tiles[n] = tsum;
  vbase[n] = vsum;
  zbase[n] = zsum;
  bbase[n] = bsum;

  bh->n_jobs = n;
  bh->total_tiles = tsum;
  bh->total_verts = vsum;
  bh->tile_counter = 0;
  return need;
}

typedef void (*BatchVoxKernel)(BatchHeader *, const JobDesc *, const unsigned long long *);

static BatchVoxKernel batch_vox_kernel(bool strict, bool cull) {
  if (strict) return cull ? k_voxelize_batched<true, true> : k_voxelize_batched<true, false>;
  return cull ? k_voxelize_batched<false, true> : k_voxelize_batched<false, false>;
}

// Enqueues the batch kernels on `stream` (the table must already be uploaded); `cull`: the
// batch's jobs skip rows outside each slice's cross-section (opts->row_cull != 2).
static int launch_batch(char *ws, int cap, int strict, bool cull, cudaStream_t stream) {
  DeviceInfo *dev = nullptr;
  if (device_info(dev) != cudaSuccess) return VOXTET_ERR_CUDA;
  const BatchLayout L = batch_layout(cap);
  BatchHeader *bh = reinterpret_cast<BatchHeader *>(ws);
  JobDesc *tab = reinterpret_cast<JobDesc *>(ws + L.o_table);
  const unsigned long long *tiles = reinterpret_cast<const unsigned long long *>(ws + L.o_tiles);
  const unsigned long long *vbase = reinterpret_cast<const unsigned long long *>(ws + L.o_verts);
  const unsigned long long *zbase = reinterpret_cast<const unsigned long long *>(ws + L.o_zero);
  const unsigned long long *bbase = reinterpret_cast<const unsigned long long *>(ws + L.o_blocks);
  int *status = reinterpret_cast<int *>(ws + L.o_status);
  const unsigned g8 = (unsigned)dev->sms * 8;
  const unsigned eb = (unsigned)exact_batch_blocks(cap);
  k_prologue_batched<<<g8, 256, 0, stream>>>(bh, tab, zbase);
  k_snap_batched<<<g8, 256, 0, stream>>>(bh, tab, vbase);
  int occ = 0;
  const BatchVoxKernel vk = batch_vox_kernel(strict != 0, cull);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, vk, kBlock, slice_table_bytes(16));
  vk<<<(unsigned)dev->sms * (occ > 0 ? occ : 1), kBlock, slice_table_bytes(16), stream>>>(bh, tab, tiles);
  if (strict) k_exact_batched<true><<<eb, kExactBlock, 0, stream>>>(bh, tab, bbase);
  else k_exact_batched<false><<<eb, kExactBlock, 0, stream>>>(bh, tab, bbase);
  k_gather_status<<<(cap + 255) / 256 > 0 ? (cap + 255) / 256 : 1, 256, 0, stream>>>(bh, tab, status);
  g_launches.fetch_add(5);
  return cudaGetLastError() == cudaSuccess ? VOXTET_OK : VOXTET_ERR_CUDA;
}

static int read_job_status(char *ws, int cap, int n, int *host_status, cudaStream_t stream) {
  if (cudaStreamSynchronize(stream) != cudaSuccess) return VOXTET_ERR_CUDA;
  if (!host_status || n == 0) return VOXTET_OK;
  const BatchLayout L = batch_layout(cap);
  std::vector<int> bits(n);
  if (cudaMemcpy(bits.data(), ws + L.o_status, (size_t)n * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return VOXTET_ERR_CUDA;
  for (int j = 0; j < n; ++j)
    if (host_status[j] == VOXTET_OK) host_status[j] = map_status_bits(bits[j]);
  return VOXTET_OK;
}

}  // namespace voxtet

struct voxtet_plan {
  char *ws = nullptr;
  size_t ws_bytes = 0;
  int cap = 0;
  voxtet_opts opts;
  int device = -1;
  char *pinned = nullptr;  // host image of the table part, uploaded by the graph
  size_t image_bytes = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t done = nullptr;
  bool in_flight = false;
  int n_jobs = 0;
  std::vector<int> host_status;
};

extern "C" {

size_t voxtet_batch_workspace_size(const voxtet_job *jobs, int32_t n_jobs, int32_t max_jobs) {
  if (n_jobs < 0 || max_jobs < n_jobs || (n_jobs > 0 && !jobs)) return 0;
  voxtet_opts o;
  voxtet_default_opts(&o);
  std::vector<int> st((size_t)(n_jobs > 0 ? n_jobs : 1));
  return build_batch_image(jobs, n_jobs, max_jobs > 0 ? max_jobs : 1, o, nullptr, nullptr, st.data());
}

int voxelize_tets_batched(const voxtet_job *jobs, int32_t n_jobs, void *d_ws, size_t ws_bytes,
                          const voxtet_opts *opts, void *stream_, int32_t *job_status) {
  voxtet_opts o;
  resolve_opts(opts, o);
  int st = check_opts(o);
  if (st != VOXTET_OK) return st;
  if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return VOXTET_ERR_ARG;
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return VOXTET_ERR_WORKSPACE;
  const int cap = n_jobs > 0 ? n_jobs : 1;
  std::vector<int> hs((size_t)cap, VOXTET_OK);
  std::vector<char> image;
  const size_t need = build_batch_image(jobs, n_jobs, cap, o, reinterpret_cast<char *>(d_ws), &image, hs.data());
  if (need > ws_bytes) return VOXTET_ERR_WORKSPACE;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (cudaMemcpyAsync(d_ws, image.data(), image.size(), cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return VOXTET_ERR_CUDA;
  st = launch_batch(reinterpret_cast<char *>(d_ws), cap, o.mode == 1, o.row_cull != 2, stream);
  if (st != VOXTET_OK) return st;
  if (o.sync) {
    st = read_job_status(reinterpret_cast<char *>(d_ws), cap, n_jobs, hs.data(), stream);
    if (st != VOXTET_OK) return st;
    if (job_status)
      for (int j = 0; j < n_jobs; ++j) job_status[j] = hs[j];
  } else if (job_status) {
    for (int j = 0; j < n_jobs; ++j) job_status[j] = hs[j];
  }
  return VOXTET_OK;
}

int voxtet_plan_create(void *d_ws, size_t ws_bytes, int32_t max_jobs, const voxtet_opts *opts, voxtet_plan **out) {
  if (!out || max_jobs < 1) return VOXTET_ERR_ARG;
  *out = nullptr;
  if (!d_ws || (reinterpret_cast<uintptr_t>(d_ws) & 255)) return VOXTET_ERR_WORKSPACE;
  voxtet_opts o;
  resolve_opts(opts, o);
  const int st = check_opts(o);
  if (st != VOXTET_OK) return st;
  voxtet_plan *p = new voxtet_plan();
  p->ws = reinterpret_cast<char *>(d_ws);
  p->ws_bytes = ws_bytes;
  p->cap = max_jobs;
  p->opts = o;
  p->image_bytes = batch_layout(max_jobs).o_slices;
  if (cudaGetDevice(&p->device) != cudaSuccess ||
      cudaHostAlloc(reinterpret_cast<void **>(&p->pinned), p->image_bytes, cudaHostAllocDefault) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->done, cudaEventDisableTiming) != cudaSuccess) {
    voxtet_plan_destroy(p);
    return VOXTET_ERR_CUDA;
  }
  *out = p;
  return VOXTET_OK;
}

int voxtet_plan_run(voxtet_plan *p, const voxtet_job *jobs, int32_t n_jobs, void *stream_) {
  if (!p || n_jobs < 0 || n_jobs > p->cap || (n_jobs > 0 && !jobs)) return VOXTET_ERR_ARG;
  if (p->in_flight && cudaEventSynchronize(p->done) != cudaSuccess) return VOXTET_ERR_CUDA;
  p->in_flight = false;
  p->host_status.assign((size_t)(n_jobs > 0 ? n_jobs : 1), VOXTET_OK);
  std::vector<char> image;
  const size_t need = build_batch_image(jobs, n_jobs, p->cap, p->opts, p->ws, &image, p->host_status.data());
  if (need > p->ws_bytes) return VOXTET_ERR_NOMEM;
  std::memcpy(p->pinned, image.data(), p->image_bytes);
  cudaGraphExec_t &exec = p->exec;
  if (!exec) {  // capture the upload and the kernels once; later runs replay them
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return VOXTET_ERR_CUDA;
    cudaMemcpyAsync(p->ws, p->pinned, p->image_bytes, cudaMemcpyHostToDevice, p->cap_stream);
    const unsigned long long before = g_launches.load();
    const int st = launch_batch(p->ws, p->cap, p->opts.mode == 1, p->opts.row_cull != 2, p->cap_stream);
    g_launches.store(before);  // captured, not launched
    if (cudaStreamEndCapture(p->cap_stream, &g) != cudaSuccess || st != VOXTET_OK) {
      if (g) cudaGraphDestroy(g);
      return VOXTET_ERR_CUDA;
    }
    const cudaError_t e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      exec = nullptr;
      return VOXTET_ERR_CUDA;
    }
  }
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  if (cudaGraphLaunch(exec, stream) != cudaSuccess) return VOXTET_ERR_CUDA;
  g_launches.fetch_add(5);
  if (cudaEventRecord(p->done, stream) != cudaSuccess) return VOXTET_ERR_CUDA;
  p->in_flight = true;
  p->n_jobs = n_jobs;
  return VOXTET_OK;
}

int voxtet_plan_wait(voxtet_plan *p, int32_t *job_status) {
  if (!p) return VOXTET_ERR_ARG;
  if (p->in_flight && cudaEventSynchronize(p->done) != cudaSuccess) return VOXTET_ERR_CUDA;
  p->in_flight = false;
  if (!job_status || p->n_jobs == 0) return VOXTET_OK;
  const int st = read_job_status(p->ws, p->cap, p->n_jobs, p->host_status.data(), nullptr);
  if (st != VOXTET_OK) return st;
  for (int j = 0; j < p->n_jobs; ++j) job_status[j] = p->host_status[j];
  return VOXTET_OK;
}

int voxtet_plan_query(voxtet_plan *p) {
  if (!p) return VOXTET_ERR_ARG;
  if (!p->in_flight) return 1;
  const cudaError_t e = cudaEventQuery(p->done);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  return VOXTET_ERR_CUDA;
}

void voxtet_plan_destroy(voxtet_plan *p) {
  if (!p) return;
  if (p->in_flight && p->done) cudaEventSynchronize(p->done);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->done) cudaEventDestroy(p->done);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->pinned) cudaFreeHost(p->pinned);
  delete p;
}

}  // extern "C"

// ------------------------------------------------------------------ entry point without allocation
//
// voxelize_tets_noalloc runs the same kernels as voxelize_tets, but its workspace is
// the fixed array below instead of a caller-provided buffer, for callers that cannot
// allocate device memory at call time.  The array is part of this library's device
// image, so every GPU that loads the library holds VOXTET_NOALLOC_SCRATCH_BYTES of it
// until the process exits.  All calls share it and it keeps the last call's contents;
// the kernels clear what must start at zero (header, redo bitmap) on every call.

namespace voxtet {

static __device__ __align__(256) unsigned char g_noalloc_scratch[VOXTET_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch, looked up once per device (the host-side name
// of a __device__ array is only a stand-in and must not be handed to a kernel).
static void *g_noalloc_addr[kMaxDevices];
static std::atomic<int> g_noalloc_lock{0};

static int noalloc_scratch(void *&addr) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return VOXTET_ERR_CUDA;
  while (g_noalloc_lock.exchange(1)) {
  }
  int st = VOXTET_OK;
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) st = VOXTET_ERR_CUDA;
    else g_noalloc_addr[dev] = p;
  }
  addr = g_noalloc_addr[dev];
  g_noalloc_lock.store(0);
  return st;
}

}  // namespace voxtet

extern "C" int voxelize_tets_noalloc(const float *d_verts, int64_t n_verts, const int32_t *d_tets, int64_t n_tets,
                                     const float grid_origin[3], float voxel_size, int32_t res,
                                     uint32_t *d_out_bits, const voxtet_opts *opts, void *stream) {
  if (n_tets < 0 || n_verts < 0) return VOXTET_ERR_ARG;
  // the minimum workspace must fit; the row queue then takes the rest of the scratch
  if (voxtet_workspace_size(n_tets, n_verts, 1) > (size_t)VOXTET_NOALLOC_SCRATCH_BYTES) return VOXTET_ERR_NOMEM;
  voxtet_opts o;
  resolve_opts(opts, o);
  o.profile = 0;  // profiling would create CUDA events
  void *ws = nullptr;
  const int st = noalloc_scratch(ws);
  if (st != VOXTET_OK) return st;
  return voxelize_tets(d_verts, n_verts, d_tets, n_tets, grid_origin, voxel_size, res, d_out_bits, ws,
                       (size_t)VOXTET_NOALLOC_SCRATCH_BYTES, &o, stream);
}

// The status word sits at the start of the fixed array (its workspace header).
extern "C" int voxtet_noalloc_status_async(int32_t *status_word, void *stream) {
  if (!status_word) return VOXTET_ERR_ARG;
  void *ws = nullptr;
  const int st = noalloc_scratch(ws);
  if (st != VOXTET_OK) return st;
  return voxtet_status_async(ws, status_word, stream);
}

// ------------------------------------------------------------------ brick-sparse output
//
// Section 5 ("Octrees") notes that voxel data is usually stored sparsely.  Here a grid
// is produced one z-slab at a time into a dense slab buffer (the fused kernels
// unchanged, on the slab's slices), and the slab is then compacted into bricks of
// 32 x 8 x 8 voxels: the brick's 64 row-words of the dense layout, word dz * 8 + dy.
// Three bandwidth-bound kernels per slab: count the non-empty bricks of each block of
// bricks, scan the block counts (one block, which also advances the running total),
// and write keys and words of the non-empty bricks in slab order, so the output is
// sorted by (bz, by, bx).

namespace voxtet {

constexpr int kBrickRows = 8;                        // y rows per brick
constexpr int kBrickSlices = 8;                      // z slices per brick
constexpr int kBrickWords = kBrickRows * kBrickSlices;
constexpr int kCompactBlock = 128;

constexpr int kSparseSpanRows = 64;  // default span size of the slab launches of the sparse path

struct SparseHeader {
  unsigned long long total;  // non-empty bricks of all slabs so far (may exceed the capacity)
  int sticky_bits;           // device-detected status bits of every slab
  int pad;
  unsigned long long reserved[30];
};
static_assert(sizeof(SparseHeader) == 256, "sparse header is 256 bytes");

struct SlabBricks {
  uint32_t *dense;        // [nz][ry][W] words of the slab
  int W, ry, nz;          // words per row, rows per slice, slices in the slab
  int nby, nbz;           // bricks along y and z in the slab
  int bz0;                // global brick z of the slab's first slice
  long long n;            // W * nby * nbz bricks, bx fastest
};

__device__ __forceinline__ uint32_t *brick_origin(const SlabBricks &s, long long b, int &bx, int &by, int &bz,
                                                  int &ny, int &nz) {
  bx = (int)(b % s.W);
  const long long t = b / s.W;
  by = (int)(t % s.nby);
  bz = (int)(t / s.nby);
  ny = min(kBrickRows, s.ry - by * kBrickRows);
  nz = min(kBrickSlices, s.nz - bz * kBrickSlices);
  return s.dense + ((size_t)bz * kBrickSlices * s.ry + (size_t)by * kBrickRows) * s.W + bx;
}

// OR of a brick's row-words (rows past the slab's edges are absent).  Consecutive
// threads take consecutive bx, so every load of a warp is one contiguous run of words.
__device__ __forceinline__ bool brick_nonempty(const SlabBricks &s, long long b) {
  int bx, by, bz, ny, nz;
  const uint32_t *o = brick_origin(s, b, bx, by, bz, ny, nz);
  uint32_t acc = 0;
  if (ny == kBrickRows && nz == kBrickSlices) {  // whole brick: 64 independent loads in flight
#pragma unroll
    for (int r = 0; r < kBrickWords; ++r) acc |= o[((size_t)(r >> 3) * s.ry + (r & 7)) * s.W];
  } else {
    for (int dz = 0; dz < nz; ++dz)
      for (int dy = 0; dy < ny; ++dy) acc |= o[((size_t)dz * s.ry + dy) * s.W];
  }
  return acc != 0;
}

__global__ void __launch_bounds__(kCompactBlock) k_brick_count(SlabBricks s, unsigned long long *block_counts) {
  const long long b = (long long)blockIdx.x * kCompactBlock + threadIdx.x;
  const bool ne = b < s.n && brick_nonempty(s, b);
  const int c = __syncthreads_count(ne);
  if (threadIdx.x == 0) block_counts[blockIdx.x] = (unsigned long long)c;
}

// The same counts when rows hold a multiple of 4 words: a thread takes 4 neighbouring
// bricks (one 16-byte load per row), so a warp covers the 128 bricks of one write block
// and a warp-wide load reads 512 contiguous bytes.
__global__ void __launch_bounds__(kCompactBlock) k_brick_count4(SlabBricks s, unsigned long long *block_counts,
                                                                long long n_blocks) {
  const long long gt = (long long)blockIdx.x * kCompactBlock + threadIdx.x;
  const long long b0 = gt * 4;
  unsigned c = 0;
  if (b0 < s.n) {
    int bx, by, bz, ny, nz;
    const uint32_t *o = brick_origin(s, b0, bx, by, bz, ny, nz);
    uint32_t a0 = 0, a1 = 0, a2 = 0, a3 = 0;
    if (ny == kBrickRows && nz == kBrickSlices) {
#pragma unroll
      for (int r = 0; r < kBrickWords; ++r) {
        const uint4 v = *reinterpret_cast<const uint4 *>(o + ((size_t)(r >> 3) * s.ry + (r & 7)) * s.W);
        a0 |= v.x;
        a1 |= v.y;
        a2 |= v.z;
        a3 |= v.w;
      }
    } else {
      for (int dz = 0; dz < nz; ++dz)
        for (int dy = 0; dy < ny; ++dy) {
          const uint4 v = *reinterpret_cast<const uint4 *>(o + ((size_t)dz * s.ry + dy) * s.W);
          a0 |= v.x;
          a1 |= v.y;
          a2 |= v.z;
          a3 |= v.w;
        }
    }
    c = (a0 != 0) + (a1 != 0) + (a2 != 0) + (a3 != 0);
  }
  c = __reduce_add_sync(0xFFFFFFFFu, c);
  const long long wb = gt >> 5;  // this warp's write block
  if ((threadIdx.x & 31) == 0 && wb < n_blocks) block_counts[wb] = (unsigned long long)c;
}

// One block: exclusive scan of the block counts in place, offset by the running total,
// which then advances; the slab's device-detected status bits join the sticky bits.
__global__ void __launch_bounds__(1024) k_brick_scan(unsigned long long *counts, long long n_blocks,
                                                     SparseHeader *sh, const Header *slab_hdr) {
  __shared__ unsigned long long warp_sums[32];
  __shared__ unsigned long long carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    carry = sh->total;
    sh->sticky_bits |= slab_hdr->status_bits;
  }
  __syncthreads();
  for (long long base = 0; base < n_blocks; base += 1024) {
    const long long i = base + tid;
    const unsigned long long v = i < n_blocks ? counts[i] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
      unsigned long long w = warp_sums[lane];
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, w, d);
        if (lane >= d) w += y;
      }
      warp_sums[lane] = w;  // inclusive
    }
    __syncthreads();
    const unsigned long long before = carry + (warp ? warp_sums[warp - 1] : 0ull) + x - v;
    if (i < n_blocks) counts[i] = before;
    __syncthreads();
    if (tid == 0) carry += warp_sums[31];
    __syncthreads();
  }
  if (tid == 0) sh->total = carry;
}

// Each warp stages its 32 consecutive bricks' row-words in shared memory (lane l loads
// word r of brick l: a warp-wide load of row r is one contiguous run), then writes
// every non-empty brick with two 128-byte stores.
__global__ void __launch_bounds__(kCompactBlock) k_brick_write(SlabBricks s, const unsigned long long *block_offsets,
                                                               uint64_t *keys, uint32_t *words, long long cap) {
  __shared__ uint32_t stage[kCompactBlock / 32][kBrickWords][33];
  __shared__ unsigned warp_base[kCompactBlock / 32];
  const long long b = (long long)blockIdx.x * kCompactBlock + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t acc = 0;
  int bx = 0, by = 0, bz = 0;
  if (b < s.n) {
    int ny, nz;
    const uint32_t *o = brick_origin(s, b, bx, by, bz, ny, nz);
    if (ny == kBrickRows && nz == kBrickSlices) {
#pragma unroll
      for (int r = 0; r < kBrickWords; ++r) {
        const uint32_t v = o[((size_t)(r >> 3) * s.ry + (r & 7)) * s.W];
        stage[warp][r][lane] = v;
        acc |= v;
      }
    } else {
      for (int dz = 0; dz < kBrickSlices; ++dz)
        for (int dy = 0; dy < kBrickRows; ++dy) {
          const uint32_t v = (dz < nz && dy < ny) ? o[((size_t)dz * s.ry + dy) * s.W] : 0u;
          stage[warp][dz * kBrickRows + dy][lane] = v;
          acc |= v;
        }
    }
  }
  const bool ne = acc != 0;
  if (ne) {  // clear what was staged: the slab is left all zero for the next one
    int ny, nz;
    uint32_t *o = brick_origin(s, b, bx, by, bz, ny, nz);
    if (ny == kBrickRows && nz == kBrickSlices) {
#pragma unroll
      for (int r = 0; r < kBrickWords; ++r) o[((size_t)(r >> 3) * s.ry + (r & 7)) * s.W] = 0u;
    } else {
      for (int dz = 0; dz < nz; ++dz)
        for (int dy = 0; dy < ny; ++dy) o[((size_t)dz * s.ry + dy) * s.W] = 0u;
    }
  }
  const unsigned m = __ballot_sync(0xFFFFFFFFu, ne);
  if (lane == 0) warp_base[warp] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned run = 0;
    for (int w = 0; w < kCompactBlock / 32; ++w) {
      const unsigned c = warp_base[w];
      warp_base[w] = run;
      run += c;
    }
  }
  __syncthreads();
  const unsigned long long first = block_offsets[blockIdx.x] + warp_base[warp];
  if (ne) {
    const unsigned long long slot = first + (unsigned long long)__popc(m & ((1u << lane) - 1u));
    if (slot < (unsigned long long)cap)
      keys[slot] = (uint64_t)bx | ((uint64_t)by << 16) | ((uint64_t)(s.bz0 + bz) << 32);
  }
  unsigned mm = m;
  for (unsigned long long slot = first; mm; ++slot) {
    const int j = __ffs(mm) - 1;
    mm &= mm - 1;
    if (slot >= (unsigned long long)cap) break;
    uint32_t *dst = words + slot * kBrickWords;
    dst[lane] = stage[warp][lane][j];
    dst[32 + lane] = stage[warp][32 + lane][j];
  }
}

// Marks slab z / depth for every slice z that the samples of some tet reach (the same
// z-range as tet_box), so that slabs no tet reaches are skipped: they hold no brick.  Tets
// with an index out of range or a vertex that failed its snap mark nothing; slab 0 is
// always voxelized, and its launch and the snap report those errors.
__global__ void k_slab_marks(const int4 *__restrict__ tets, long long n_tets, const int4 *__restrict__ verts4,
                             long long n_verts, int sh, int rz, int depth, uint32_t *marks) {
  const unsigned long long nv = (unsigned long long)n_verts;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n_tets;
       t += (long long)gridDim.x * blockDim.x) {
    const int4 q = tets[t];
    if (q.x < 0 || q.y < 0 || q.z < 0 || q.w < 0 || (unsigned long long)q.x >= nv ||
        (unsigned long long)q.y >= nv || (unsigned long long)q.z >= nv || (unsigned long long)q.w >= nv)
      continue;
    const int4 A = verts4[q.x], B = verts4[q.y], C = verts4[q.z], D = verts4[q.w];
    if ((A.w | B.w | C.w | D.w) != 0) continue;
    int lo = 0, n = 0;
    axis_box(imin4(A.z, B.z, C.z, D.z), imax4(A.z, B.z, C.z, D.z), sh, 0, rz - 1, lo, n);
    if (n <= 0) continue;
    for (int sl = lo / depth; sl <= (lo + n - 1) / depth; ++sl) {
      const uint32_t bit = 1u << (sl & 31);
      if (!(marks[sl >> 5] & bit)) atomicOr(marks + (sl >> 5), bit);
    }
  }
}

// Scratch: header, one dense slab, the per-block counts of a slab's bricks, one bit per
// slab for the slabs some tet reaches.
static size_t sparse_scratch_bytes(const GridDims &g, int depth, long long *n_blocks_out) {
  const long long W = (g.rx + 31) / 32;
  const long long nby = (g.ry + kBrickRows - 1) / kBrickRows;
  const long long nbz = (depth + kBrickSlices - 1) / kBrickSlices;
  const long long n_blocks = (W * nby * nbz + kCompactBlock - 1) / kCompactBlock;
  if (n_blocks_out) *n_blocks_out = n_blocks;
  const long long n_slabs = (g.rz + depth - 1) / depth;
  return align256(sizeof(SparseHeader)) + align256((size_t)depth * g.ry * W * 4) +
         align256((size_t)(n_blocks > 0 ? n_blocks : 1) * 8) + align256((size_t)((n_slabs + 31) / 32) * 4);
}

static int sparse_dims(const int32_t res[3], int32_t depth, GridDims &g) {
  if (!res) return VOXTET_ERR_ARG;
  for (int q = 0; q < 3; ++q)
    if (res[q] < 1 || res[q] > VOXTET_SPARSE_MAX_SIDE) return VOXTET_ERR_RES;
  if (depth < kBrickSlices || depth % kBrickSlices != 0) return VOXTET_ERR_ARG;
  g.rx = res[0];
  g.ry = res[1];
  g.rz = res[2];
  g.z0 = 0;
  g.z1 = res[2];
  g.K = 0;
  while ((1 << g.K) < g.longest()) ++g.K;
  return VOXTET_OK;
}

}  // namespace voxtet

extern "C" {

size_t voxtet_sparse_scratch_size(const int32_t res[3], int32_t slab_depth) {
  GridDims g;
  if (sparse_dims(res, slab_depth, g) != VOXTET_OK) return 0;
  return sparse_scratch_bytes(g, slab_depth, nullptr);
}

int voxelize_tets_sparse(const float *d_verts, int64_t n_verts, const int32_t *d_tets, int64_t n_tets,
                         const float grid_origin[3], float voxel_size, const int32_t res[3], int32_t slab_depth,
                         uint64_t *d_brick_keys, uint32_t *d_brick_words, int64_t max_bricks, int64_t *n_bricks,
                         void *d_scratch, size_t scratch_bytes, void *d_workspace, size_t ws_bytes,
                         const voxtet_opts *opts, void *stream_) {
  voxtet_opts o;
  resolve_opts(opts, o);
  int st = check_opts(o);
  if (st != VOXTET_OK) return st;
  if (o.accumulate) return VOXTET_ERR_ARG;
  GridDims g;
  st = sparse_dims(res, slab_depth, g);
  if (st != VOXTET_OK) return st;
  if (!n_bricks || max_bricks < 0) return VOXTET_ERR_ARG;
  if (max_bricks > 0 && (!d_brick_keys || !d_brick_words || (reinterpret_cast<uintptr_t>(d_brick_keys) & 7) ||
                         (reinterpret_cast<uintptr_t>(d_brick_words) & 3)))
    return VOXTET_ERR_ARG;
  long long n_blocks = 0;
  if (!d_scratch || (reinterpret_cast<uintptr_t>(d_scratch) & 255) ||
      scratch_bytes < sparse_scratch_bytes(g, slab_depth, &n_blocks))
    return VOXTET_ERR_WORKSPACE;
  // the dense slab inside the scratch stands in for the output buffer in the shared checks
  uint32_t *dense = reinterpret_cast<uint32_t *>(static_cast<char *>(d_scratch) + align256(sizeof(SparseHeader)));
  unsigned long long *block_counts = reinterpret_cast<unsigned long long *>(
      reinterpret_cast<char *>(dense) + align256((size_t)slab_depth * g.ry * ((g.rx + 31) / 32) * 4));
  uint32_t *slab_marks = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(block_counts) +
                                                      align256((size_t)(n_blocks > 0 ? n_blocks : 1) * 8));
  const int n_slabs = (g.rz + slab_depth - 1) / slab_depth;
  const int mark_words = (n_slabs + 31) / 32;
  SparseHeader *sh = static_cast<SparseHeader *>(d_scratch);
  st = buffer_checks(n_verts, d_tets, n_tets, dense, d_workspace, ws_bytes);
  if (st != VOXTET_OK) return st;
  st = float_input_checks(d_verts, n_verts, grid_origin, voxel_size);
  if (st != VOXTET_OK) return st;
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(stream_);
  Workspace w;
  workspace_bytes(n_tets, n_verts, &w, d_workspace, ws_bytes);
  if (cudaMemsetAsync(sh, 0, sizeof(SparseHeader), stream) != cudaSuccess) return VOXTET_ERR_CUDA;
  voxtet_opts inner = o;
  inner.sync = 0;
  inner.profile = 0;
  // A slab launch holds only the tets that reach the slab, so it has far fewer spans than a
  // whole-grid launch; spans of one slice (about 64 rows) keep the threads evenly busy
  // (measured on GB300, torus_73 with 128 MiB slabs: 4096^3 6.6 -> 6.0 ms, 8192^3 38 -> 34 ms).
  if (inner.span_rows == 0) inner.span_rows = kSparseSpanRows;
  const int W = (g.rx + 31) / 32;
  // slab 0's prologue, the snap, and the marks of the slabs some tet reaches
  std::vector<uint32_t> marks((size_t)mark_words, 0u);
  {
    GridDims g0 = g;
    g0.z1 = slab_depth < g.rz ? slab_depth : g.rz;
    st = launch_prologue(w, dense, g0.out_words(), 1, stream);
    if (st != VOXTET_OK) return st;
    st = launch_snap(w, d_verts, n_verts, grid_origin, voxel_size, g.K, stream);
    if (st != VOXTET_OK) return st;
    if (cudaMemsetAsync(slab_marks, 0, (size_t)mark_words * 4, stream) != cudaSuccess) return VOXTET_ERR_CUDA;
    if (n_tets > 0 && n_verts > 0) {
      DeviceInfo *dev = nullptr;
      if (device_info(dev) != cudaSuccess) return VOXTET_ERR_CUDA;
      k_slab_marks<<<grid_blocks(n_tets, 256, dev->sms), 256, 0, stream>>>(
          reinterpret_cast<const int4 *>(d_tets), n_tets, w.verts4, n_verts, kLatticeBits - g.K, g.rz, slab_depth,
          slab_marks);
      g_launches.fetch_add(1);
    }
    if (cudaMemcpyAsync(marks.data(), slab_marks, (size_t)mark_words * 4, cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(stream) != cudaSuccess)
      return VOXTET_ERR_CUDA;
  }
  for (int z0 = 0, si = 0; z0 < g.rz; z0 += slab_depth, ++si) {
    if (si > 0 && !((marks[(size_t)si >> 5] >> (si & 31)) & 1u)) continue;  // no tet reaches it: no bricks
    GridDims gs = g;
    gs.z0 = z0;
    gs.z1 = z0 + slab_depth < g.rz ? z0 + slab_depth : g.rz;
    if (si > 0) {  // the slab is zero: the previous slab's k_brick_write cleared every brick it held
      st = launch_prologue(w, dense, gs.out_words(), 0, stream);
      if (st != VOXTET_OK) return st;
    }
    st = run_voxelize(w, n_verts, d_tets, n_tets, gs, dense, inner, stream);
    if (st != VOXTET_OK) return st;
    SlabBricks s;
    s.dense = dense;
    s.W = W;
    s.ry = g.ry;
    s.nz = gs.z1 - gs.z0;
    s.nby = (g.ry + kBrickRows - 1) / kBrickRows;
    s.nbz = (s.nz + kBrickSlices - 1) / kBrickSlices;
    s.bz0 = z0 / kBrickSlices;
    s.n = (long long)s.W * s.nby * s.nbz;
    const long long nb = (s.n + kCompactBlock - 1) / kCompactBlock;
    if (s.W % 4 == 0) {
      const long long threads = s.n / 4;
      k_brick_count4<<<(unsigned)((threads + kCompactBlock - 1) / kCompactBlock), kCompactBlock, 0, stream>>>(
          s, block_counts, nb);
    } else {
      k_brick_count<<<(unsigned)nb, kCompactBlock, 0, stream>>>(s, block_counts);
    }
    k_brick_scan<<<1, 1024, 0, stream>>>(block_counts, nb, sh, w.hdr);
    k_brick_write<<<(unsigned)nb, kCompactBlock, 0, stream>>>(s, block_counts, d_brick_keys, d_brick_words,
                                                               (long long)max_bricks);
    g_launches.fetch_add(3);
    if (cudaGetLastError() != cudaSuccess) return VOXTET_ERR_CUDA;
  }
  if (cudaStreamSynchronize(stream) != cudaSuccess) return VOXTET_ERR_CUDA;
  SparseHeader h;
  if (cudaMemcpy(&h, sh, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return VOXTET_ERR_CUDA;
  *n_bricks = (int64_t)h.total;
  st = map_status_bits(h.sticky_bits);
  if (st != VOXTET_OK) return st;
  return h.total > (unsigned long long)max_bricks ? VOXTET_ERR_NOMEM : VOXTET_OK;
}

}  // extern "C"
