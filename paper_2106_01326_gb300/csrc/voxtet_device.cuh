// voxtet_device.cuh -- device-side types and helpers shared by the voxelizer's kernels.
//
// The workspace header, the per-launch parameters, the OR writes into the bit grid,
// the checked tet load, the per-slice candidate-row range (edge lines of the tet's
// cross-section), the exact row narrowing of faces parallel to x, the block-staged
// queue of rows the filter could not certify and the per-block counters.  Both the
// span kernel (voxtet.cu) and the slice-unit kernel (voxtet_slices.cu) use them, so
// their grids and queues agree by construction.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tet_math.cuh"

namespace voxtet {

#ifndef VOXTET_MIN_BLOCKS
#define VOXTET_MIN_BLOCKS 6  // resident blocks per SM the register budget is sized for
#endif

// Threads per block.  128-thread blocks of 512-tet tiles, 6 per SM, wait less at the tile
// barriers than 256-thread blocks of 1024-tet tiles, 3 per SM (measured on GB300: sliver
// mesh 512^3 kernel 336 -> 330 us, 1024^3 1117 -> 1088 us; torus 48^3 at 256^3 26.2 -> 24.1 us).
constexpr int kBlock = 128;
// Bounding-box rows per span (whole z-slices) when the caller does not choose (the
// autotuner picks per mesh).  Measured on GB300 with the sliver and torus meshes: 256 is
// best or within 13 % of it at every size except 1024^3, where 1024 (with 32-slice
// spans) keeps a typical tet in one span, whose work estimate then sorts the lanes
// evenly (sliver mesh 1.49 -> 1.15 ms); from 2048^3 spans that long can take twice as long.
static __host__ __device__ int default_span_rows(int res) { return res >= 1024 && res < 2048 ? 1024 : 256; }
// Automatic row culling from this grid side up, i.e. always: measured on GB300, a 64^3 grid of
// the 8^3 lattice 71.7 -> 47.1 us with culling, the 256-job batch at 32^3-128^3 940 -> 861 us
// (culling every job, so one tile path compiled in)
constexpr int kCullMinRes = 1;
constexpr int kMaxFilterRows = 8192;    // box rows per slice the fused kernel's slice table can hold
// From this grid side up the filter clamps each face's bracket to the range where the
// face can change a row (measured on GB300: 4% slower per row up to 1024^3 grids, where
// few rows are uncertain; from 2048^3 it queues about 10x fewer rows and is faster)
constexpr int kClampMinRes = 2048;

// Workspace header (first 256 bytes of the workspace).
struct Header {
  int status_bits;
  unsigned tetq_count;  // tets queued for the exact kernel
  unsigned rowq_count;  // rows queued for the exact kernel (may exceed the capacity)
  unsigned listq_count;  // tets the slice-unit kernel left to the span kernel (kept at the back of tetq)
  unsigned long long tile_counter;
  unsigned long long spans;
  unsigned long long rows;
  unsigned long long degenerate;
  unsigned long long wide;
  unsigned long long list_tile_counter;  // tiles claimed by the span kernel in list mode
  unsigned long long reserved[24];
};
static_assert(sizeof(Header) == 256, "header is 256 bytes");

// A row the filter could not certify: tet index and (b, c) within its sample box.
struct RowItem {
  uint32_t tet;
  uint16_t b, c;
};

struct Params {
  const int4 *verts4;
  const int4 *tets;
  long long n_tets;
  long long n_verts;
  uint32_t *out;
  Header *hdr;
  uint32_t *tetq;   // [n_tets]
  RowItem *rowq;    // [q_cap]
  uint32_t *redo;   // [ceil(n_tets / 32)] bitmap
  unsigned q_cap;
  int rx, ry;       // samples per row and rows per slice
  int z0, z1;       // slices z0 <= l < z1 are produced; out holds (z1 - z0) * ry * W words
  int W;            // words per row, ceil(rx / 32)
  int sh;           // log2 of the lattice step per voxel, 20 - ceil(log2(longest side))
  int span_rows;    // target bounding-box rows per span
  int exact_all;    // 1: every tet goes to the exact kernel
  int max_slices;   // slices a span may hold (16 or 32): the slice table's rows in dynamic shared memory
  int cull;         // 1: skip rows outside each slice's cross-section (batched kernel)
  long long big_tiles;  // single-mesh launch: tiles of kTile tets before the kSmallTile tail
  long long tile_stride;  // > 0: tile k holds tets k + j * tile_stride (slab launches), else contiguous tiles
  int list_mode;    // span kernel: 1 = its tets are the hdr->listq_count ones listed at the back of tetq
  int vflags;       // exact kernel: 1 = fold the vertices' error bits (verts4[i].w) into the status
};

// Row-queue capacity for a mesh of n_tets tets.
static unsigned long long row_queue_capacity(long long n_tets) {
  return (unsigned long long)(n_tets < 65536 ? 65536 : n_tets);
}


// ------------------------------------------------------------------ chained launches
//
// The kernels of one call run back to back on one stream.  Each after the first is launched
// as a programmatic dependent of the one before it (launch_chained), so that its blocks are
// scheduled while the previous kernel drains instead of after it; every such kernel calls
// chain_wait() before it touches memory, which returns once the previous kernel has completed
// and its writes are visible (at once for a kernel launched the ordinary way).  chain_release()
// lets the next kernel's launch begin; it orders nothing, the next kernel's chain_wait() does.

__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void chain_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... Args, typename... Actual>
static cudaError_t launch_chained(void (*kernel)(Args...), unsigned grid, unsigned block, size_t smem,
                                  cudaStream_t stream, Actual &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<Actual &&>(args)...);
}

// ------------------------------------------------------------------ OR writes

// OR the samples x0..x1 (inclusive, absolute x indices) into one row of words.
// Used by the exact kernel; any word may be shared with other tets.
__device__ __forceinline__ void or_span(uint32_t *__restrict__ row, int x0, int x1) {
  const int w0 = x0 >> 5, w1 = x1 >> 5;
  const uint32_t m0 = 0xFFFFFFFFu << (x0 & 31);
  const uint32_t m1 = 0xFFFFFFFFu >> (31 - (x1 & 31));
  if (w0 == w1) {
    atomicOr(row + w0, m0 & m1);
    return;
  }
  atomicOr(row + w0, m0);
  for (int w = w0 + 1; w < w1; ++w) row[w] = 0xFFFFFFFFu;  // whole words: a plain store is an OR
  atomicOr(row + w1, m1);
}

// The same for the hot loop, shaped to keep the lanes of a warp together: the first
// word is always ORed (a zero mask when `live` is false), the second word only under
// a predicate, and the rarely needed run of whole middle words behind a branch.
__device__ __forceinline__ void or_span_lanes(uint32_t *__restrict__ row, int x0, int x1, bool live) {
  const int w0 = x0 >> 5, w1 = x1 >> 5;
  const uint32_t m1 = 0xFFFFFFFFu >> (31 - (x1 & 31));
  uint32_t m0 = 0xFFFFFFFFu << (x0 & 31);
  m0 = w0 == w1 ? (m0 & m1) : m0;
  if (live) atomicOr(row + w0, m0);
  if (live && w1 != w0) atomicOr(row + w1, m1);
  if (live && w1 > w0 + 1) {
    for (int w = w0 + 1; w < w1; ++w) row[w] = 0xFFFFFFFFu;
  }
}

// ------------------------------------------------------------------ per-tet helpers

// Loads tet t; false if an index is out of range (recorded) or a vertex failed its snap
// (already recorded by the snap kernel).
__device__ __forceinline__ bool load_tet(const Params &p, long long t, int3 V[4], int &err) {
  const int4 q = p.tets[t];
  const unsigned long long nv = (unsigned long long)p.n_verts;
  if (q.x < 0 || q.y < 0 || q.z < 0 || q.w < 0 || (unsigned long long)q.x >= nv || (unsigned long long)q.y >= nv ||
      (unsigned long long)q.z >= nv || (unsigned long long)q.w >= nv) {
    err |= kErrIndex;
    return false;
  }
  const int4 A = p.verts4[q.x], B = p.verts4[q.y], C = p.verts4[q.z], D = p.verts4[q.w];
  V[0] = make_int3(A.x, A.y, A.z);
  V[1] = make_int3(B.x, B.y, B.z);
  V[2] = make_int3(C.x, C.y, C.z);
  V[3] = make_int3(D.x, D.y, D.z);
  return (A.w | B.w | C.w | D.w) == 0;
}


// Edge lines of a tet for the per-slice row range, with the vertices sorted by z
// (z0 <= z1 <= z2 <= z3).  Edge (p, q) crosses the plane at height Z at
// y = y_p + (Z - z_p) k with k = (y_q - y_p) / (z_q - z_p) (k = 0 for horizontal edges,
// whose end points the other edges also reach).  Z - z_p is exact in float
// (|Z|, |z_p| <= 2^21) and k carries one rounding, so each crossing point is within
// u 2^22 + u 2^21 < 0.4 lattice units of the true one.  Edge order: 01 02 03 12 13 23.
struct EdgeLines {
  float zp[6], yp[6], k[6];
  int z1, z2;
};

__device__ __forceinline__ void edge_lines(const int3 V[4], EdgeLines &E) {
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
    E.k[e] = dz != 0 ? __fdiv_rn((float)(y[qi] - y[pi]), (float)dz) : 0.f;
  }
  E.z1 = z[1];
  E.z2 = z[2];
}

// Candidate rows [b_lo, b_hi] of the slice at height Z (inside the tet's z-range):
// the cross-section's y-extent, widened by 2 lattice units, in row indices.
__device__ __forceinline__ void slice_rows_sorted(const EdgeLines &E, int Z, int s, int sh, int j0, int nb,
                                                  int &b_lo, int &b_hi) {
  const float Zf = (float)Z;
  const bool le1 = Z <= E.z1, le2 = Z <= E.z2, ge1 = Z >= E.z1, ge2 = Z >= E.z2;
  const bool valid[6] = {le1, le2, true, ge1 && le2, ge1, ge2};
  float ymin = 3.0e38f, ymax = -3.0e38f;
#pragma unroll
  for (int e = 0; e < 6; ++e) {
    const float y = __fmaf_rn(Zf - E.zp[e], E.k[e], E.yp[e]);
    if (valid[e]) {
      ymin = fminf(ymin, y);
      ymax = fmaxf(ymax, y);
    }
  }
  const int ylo = (int)floorf(ymin) - 2, yhi = (int)ceilf(ymax) + 2;
  b_lo = max(((ylo + s - 1) >> sh) - j0, 0);
  b_hi = min(((yhi - s) >> sh) - j0, nb - 1);
}

// Queue row (b, c) of tet t for the exact kernel; if the row queue is full, flag the
// whole tet for an exact redo instead.
__device__ __forceinline__ void queue_row(const Params &p, long long t, int b, int c) {
  const unsigned k = atomicAdd(&p.hdr->rowq_count, 1u);
  if (k < p.q_cap) {
    RowItem it;
    it.tet = (uint32_t)t;
    it.b = (uint16_t)b;
    it.c = (uint16_t)c;
    p.rowq[k] = it;
  } else {
    atomicOr(&p.redo[t >> 5], 1u << (t & 31));
  }
}

// Rows allowed by a constraint that does not depend on x (a face parallel to the x
// axis): lam = H0 + Dy b along the slice, exact.  Narrows [b_lo, b_hi] by bisection
// on the monotone lam(b), probing only rows inside the box.
template <bool STRICT>
__device__ __forceinline__ void narrow_by_row_constraint(i64 H0, i64 Dy, int &b_lo, int &b_hi) {
  if (b_lo > b_hi) return;
  if (Dy == 0) {
    if (!lam_ok<STRICT, i64>(H0)) b_hi = b_lo - 1;
    return;
  }
  if (Dy > 0) {  // increasing: smallest b in [b_lo, b_hi + 1] that is ok
    int x = b_lo, y = b_hi + 1;
    while (x < y) {
      const int mid = (x + y) >> 1;
      if (lam_ok<STRICT, i64>(H0 + Dy * (i64)mid)) y = mid;
      else x = mid + 1;
    }
    b_lo = x;
  } else {  // decreasing: largest b in [b_lo - 1, b_hi] that is ok
    int x = b_lo - 1, y = b_hi;
    while (x < y) {
      const int mid = (x + y + 1) >> 1;
      if (lam_ok<STRICT, i64>(H0 + Dy * (i64)mid)) x = mid;
      else y = mid - 1;
    }
    b_hi = x;
  }
}

// Uncertain rows are first collected in a per-block shared-memory buffer and moved
// to the global row queue with one atomic per tile, so that thousands of threads do
// not contend on the queue counter.
constexpr int kStage = 512;
template <int N>
struct RowStageN {
  RowItem items[N];
  uint32_t n;
  uint32_t base;
};
typedef RowStageN<kStage> RowStage;

template <int N>
__device__ __forceinline__ void queue_row_staged(const Params &p, RowStageN<N> &st, long long t, int b, int c) {
  const uint32_t k = atomicAdd(&st.n, 1u);
  if (k < (uint32_t)N) {
    RowItem it;
    it.tet = (uint32_t)t;
    it.b = (uint16_t)b;
    it.c = (uint16_t)c;
    st.items[k] = it;
  } else {
    queue_row(p, t, b, c);
  }
}

// Moves a block's staged rows to the global queue (all threads of the block call it).
template <int N>
__device__ __forceinline__ void flush_stage(const Params &p, RowStageN<N> &st) {
  __syncthreads();
  const uint32_t n = min(st.n, (uint32_t)N);
  if (n) {
    if (threadIdx.x == 0) st.base = atomicAdd(&p.hdr->rowq_count, n);
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
      const unsigned k = st.base + i;
      const RowItem it = st.items[i];
      if (k < p.q_cap) p.rowq[k] = it;
      else atomicOr(&p.redo[it.tet >> 5], 1u << (it.tet & 31));
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) st.n = 0;
}

// Exact conversion of an integral float in [0, 2^22) to int without the conversion
// unit: adding 2^23 puts the integer in the low mantissa bits.
__device__ __forceinline__ int small_float_to_int(float f) {
  return __float_as_int(__fadd_rn(f, 8388608.0f)) - 0x4B000000;
}


struct TileCounters {
  int err = 0;
  unsigned degenerate = 0, wide = 0, rows = 0;
  unsigned long long spans = 0;
};


// Adds a block's counters to a mesh's header: one atomic per warp and counter.
__device__ __forceinline__ void flush_counters(Header *hdr, TileCounters &ctr) {
  const int lane = threadIdx.x & 31;
  unsigned long long rows_w = ctr.rows, deg_w = ctr.degenerate, wide_w = ctr.wide;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    rows_w += __shfl_down_sync(0xFFFFFFFFu, rows_w, d);
    deg_w += __shfl_down_sync(0xFFFFFFFFu, deg_w, d);
    wide_w += __shfl_down_sync(0xFFFFFFFFu, wide_w, d);
  }
  const int err = __reduce_or_sync(0xFFFFFFFFu, ctr.err);
  if (lane == 0) {
    if (rows_w) atomicAdd(&hdr->rows, rows_w);
    if (deg_w) atomicAdd(&hdr->degenerate, deg_w);
    if (wide_w) atomicAdd(&hdr->wide, wide_w);
    if (err) atomicOr(&hdr->status_bits, err);
  }
  if (threadIdx.x == 0 && ctr.spans) atomicAdd(&hdr->spans, ctr.spans);
  ctr = TileCounters();
}


}  // namespace voxtet
