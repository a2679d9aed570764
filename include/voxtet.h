/*
 * voxtet.h -- C ABI of the GB300 (sm_103a) solid voxelizer for tetrahedral meshes.
 *
 * The operation is the voxelization step of arXiv 2106.01326 (Section 3,
 * "Voxelization"): every voxel-centre sample that lies in some tetrahedron of
 * the mesh is marked in a dense binary grid, using the point-in-tetrahedron
 * test of Section 4, Theorem 1.  This library computes that grid exactly:
 *
 *   - Vertices are snapped to a fixed-point lattice on which the grid spans
 *     [0, 2^20] per axis: X = round_half_even(((double)v - origin) / voxel_size
 *     * 2^(20-k)) for res = 2^k, each double operation rounded to nearest.
 *     |X| <= 2^21 is required (vertices may lie up to one grid extent outside).
 *   - Voxel (i, j, l) is sampled at its centre ((2i+1)s, (2j+1)s, (2l+1)s),
 *     s = 2^(19-k) lattice units.
 *   - A sample is set iff it lies in the CLOSED tetrahedron (mode 0; Theorem 1
 *     with non-strict comparisons) or its interior (mode 1; Theorem 1 as
 *     stated) of at least one tetrahedron with non-zero signed volume
 *     (Lemma 1.1's det(AB, AC, AD)).  Tetrahedra of either orientation are
 *     accepted; zero-volume ones mark nothing.  The grid is a union, so it does
 *     not depend on tetrahedron order, duplicates or overlaps.
 *   - Every decision is exact: a single-precision filter with a proven error
 *     bound answers the easy cases and exact 64/128-bit integer arithmetic the
 *     rest, so results are bit-identical to an exact reference.
 *
 * Grid layout (out_bits): uint32 words, W = ceil(res / 32) words per x-row;
 * bit (i, j, l) is word (l * res + j) * W + (i >> 5), bit (i & 31) (least
 * significant bit = lowest x).  z is slowest, x fastest.  Padding bits of the
 * last word of a row are zero whenever a call returns VOXTET_OK.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* / documented as DEVICE are CUDA device pointers; the
 *     caller owns and allocates every buffer (mesh, grid, workspace).  The
 *     library allocates no device memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; with opts->sync = 1 the call synchronizes it and
 *     returns device-detected errors, otherwise they are read later with
 *     voxtet_last_status().
 *   - Arguments are validated on the host before anything is launched; a
 *     rejected call returns a negative status and touches nothing.
 *   - Calls on different streams with disjoint workspaces and grids are
 *     independent.  Two in-flight calls sharing a workspace race.
 *   - A call's first kernel is an ordinary launch, so everything enqueued on
 *     `stream` before the call has completed when it starts; the call's later
 *     kernels are programmatic dependents of the kernel before them and wait
 *     for it on the device.  With opts->sync = 0 (and the workspace and grid
 *     allocated beforehand) voxelize_tets, voxelize_tets_fixed and
 *     voxelize_tets_grid take no host-side action between launches, so a
 *     stream capture of such a call replays as the call, device-detected
 *     errors included (read them from the workspace); make the first call on
 *     a device outside any capture (it sets kernel attributes once).
 */
#ifndef VOXTET_H
#define VOXTET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    VOXTET_OK = 0,
    VOXTET_ERR_ARG = -1,       /* null pointer, negative size, bad option, non-positive voxel_size */
    VOXTET_ERR_RES = -2,       /* res not a power of two in [1, VOXTET_MAX_RES] (general grids: a side
                                  outside [1, VOXTET_MAX_RES]) */
    VOXTET_ERR_INDEX = -3,     /* a tetrahedron names a vertex outside [0, n_verts) (device-detected) */
    VOXTET_ERR_RANGE = -4,     /* a snapped coordinate exceeds 2^21 in magnitude (device-detected) */
    VOXTET_ERR_NAN = -5,       /* a vertex coordinate is NaN or infinite (device-detected) */
    VOXTET_ERR_WORKSPACE = -6, /* workspace missing, misaligned or smaller than voxtet_workspace_size() */
    VOXTET_ERR_CUDA = -7,      /* a CUDA runtime call or launch failed */
    VOXTET_ERR_TIMEOUT = -8,   /* a bounded device-side wait gave up (batched/served paths) */
    VOXTET_ERR_NOMEM = -9      /* a caller-provided arena is too small for the requested jobs */
} voxtet_status;

/* Largest grid resolution accepted by the GPU entry points (a 16384^3 grid of
 * bits is 512 GiB, beyond any single device). */
#define VOXTET_MAX_RES 8192

typedef struct {
    int32_t mode;       /* 0 = closed tetrahedra (default), 1 = open interiors (Theorem 1 as stated) */
    int32_t accumulate; /* 0 = clear out_bits first (default), 1 = OR into its current contents */
    int32_t use_filter; /* 1 = single-precision filter + exact fallback (default), 0 = exact integer only */
    int32_t sync;       /* 1 = synchronize the stream and return device-detected status (default 1) */
    int32_t span_rows;  /* bounding-box x-rows per work item (whole z-slices, at most 16 of them, 32 when the
                           grid's longest side is 1024 or more); 0 = automatic (256, 1024 for grids whose
                           longest side is in [1024, 2048), 64 for the slabs of voxelize_tets_sparse) */
    int32_t block;      /* threads per block of the scanline kernel; 0 = automatic (only 128 is accepted) */
    int32_t profile;    /* 1 = record CUDA events around the main kernel on `stream` (see voxtet_stats) */
    int32_t row_cull;   /* skip x-rows outside each z-slice's cross-section: 0 = automatic (on: it measured
                           faster at every grid size), 1 = on, 2 = off */
    int32_t kernel;     /* work distribution of the scanline step: 0 = automatic (slice units when the grid's
                           longest side is at most 1024, else spans), 1 = spans (runs of whole z-slices of
                           one tet per thread, sorted by estimated work), 2 = slice units (one (tet, z-slice)
                           per thread, sorted by exact row count; tets spanning more than 32 slices or 1024
                           rows per slice still go to spans).  Same grid either way; batches use spans. */
} voxtet_opts;

/* Counters the last call on a workspace left in it (read with voxtet_read_stats). */
typedef struct {
    uint64_t spans;           /* work items distributed to threads: (tet, run of z-slices) spans, or
                                 (tet, z-slice) units with the slice-unit distribution */
    uint64_t rows;            /* candidate x-rows solved by the single-precision filter */
    uint64_t fallback_rows;   /* rows the filter could not certify (re-solved with exact integers) */
    uint64_t degenerate_tets; /* tetrahedra with zero signed volume (skipped) */
    uint64_t wide_tets;       /* tetrahedra wider than 2^20 lattice units (128-bit exact path) */
    uint64_t kernel_ns;       /* device time of the main kernel of the last profiled call on this thread, else 0 */
    uint64_t exact_tets;      /* tetrahedra solved entirely with exact integers (wider than 2^20 lattice
                                 units, boxes taller than 8192 rows, or use_filter = 0) */
    uint64_t reserved;
} voxtet_stats;

/* Fill *opts with the defaults listed above. */
void voxtet_default_opts(voxtet_opts *opts);

/* Bytes of device workspace recommended for a call with these sizes (the workspace
 * must be 256-byte aligned).  It holds a 256-byte status/counter header, the
 * snapped vertices (16 B per vertex), a queue of tetrahedra for the exact solver
 * (4 B per tetrahedron), a redo bitmap (1 bit per tetrahedron) and, last, a queue
 * of rows the filter could not certify (8 B per entry): max(65536, n_tets)
 * entries, or n_tets * (res / 512)^2 / 8 when res > 512 and that is more (fine
 * grids leave more rows uncertain).  Calls accept any workspace of at least the
 * res <= 512 size and give the row queue everything beyond it; when the queue
 * overflows, the affected tetrahedra are re-solved whole with exact integers
 * (correct, slower).  For general or sparse grids pass the longest side as res.
 * Returns 0 for negative sizes. */
size_t voxtet_workspace_size(int64_t n_tets, int64_t n_verts, int32_t res);

/* Voxelize a mesh given in world coordinates (Section 3, "Voxelization";
 * point test of Section 4, Theorem 1).
 *   d_verts      DEVICE float32 [n_verts][3] (x, y, z), any alignment of 4 bytes
 *   d_tets       DEVICE int32 [n_tets][4] vertex indices, 16-byte aligned
 *   grid_origin  HOST float[3]: world position of the grid's lower corner
 *   voxel_size   HOST: edge length of a (cubic) voxel, > 0 and finite
 *   res          voxels per axis: a power of two in [1, VOXTET_MAX_RES]
 *   d_out_bits   DEVICE uint32 [res * res * W] (layout above), 4-byte aligned
 *   d_workspace  DEVICE scratch of voxtet_workspace_size() bytes, 256-byte aligned
 *   opts         HOST, may be NULL for defaults
 * Returns VOXTET_OK or a negative voxtet_status.  n_tets = 0 yields an empty
 * grid.  On a device-detected error the grid contents are unspecified. */
int voxelize_tets(const float *d_verts, int64_t n_verts, const int32_t *d_tets, int64_t n_tets,
                  const float grid_origin[3], float voxel_size, int32_t res, uint32_t *d_out_bits,
                  void *d_workspace, size_t ws_bytes, const voxtet_opts *opts, void *stream);

/* Same operation on vertices already on the 2^20-per-grid lattice
 * (d_xyz: DEVICE int32 [n_verts][3], |X| <= 2^21), skipping the snap. */
int voxelize_tets_fixed(const int32_t *d_xyz, int64_t n_verts, const int32_t *d_tets, int64_t n_tets,
                        int32_t res, uint32_t *d_out_bits, void *d_workspace, size_t ws_bytes,
                        const voxtet_opts *opts, void *stream);

/* The same operation on a general grid, or on a z-slab of one (the paper fixes
 * no grid; its voxelization loop of Section 3 is unchanged by the grid's shape).
 *   res          HOST int32[3]: voxels along x, y, z, each in [1, VOXTET_MAX_RES],
 *                any values (not only powers of two, not necessarily equal)
 *   z_begin, z_end  the slices z_begin <= l < z_end are produced,
 *                0 <= z_begin <= z_end <= res[2]; (0, res[2]) is the whole grid
 *   d_out_bits   DEVICE uint32 [(z_end - z_begin) * res[1] * W], W = ceil(res[0] / 32):
 *                bit (i, j, l) is word ((l - z_begin) * res[1] + j) * W + (i >> 5),
 *                bit i & 31; padding bits are zero.  May be NULL only when the
 *                slab is empty (z_begin == z_end), which writes nothing.
 * The lattice keeps voxel centres on lattice points: with K = ceil(log2(max side))
 * a voxel spans 2^(20-K) lattice units (so the longest side spans at most 2^20),
 * X = round_half_even(((double)v - o) / h * 2^(20-K)) and |X| <= 2^21 is required.
 * A cubic 2^k grid gives exactly voxelize_tets's grid; a grid whose longest side
 * lies in (2^(k-1), 2^k] is the [0:rz, 0:ry, 0:rx] block of the 2^k grid with the
 * same origin and voxel size, and slabs of one grid concatenate to the whole grid,
 * so ranks that each produce one slab need no exchange.  Other arguments and the
 * workspace are as for voxelize_tets (voxtet_workspace_size with any valid res).
 * Returns VOXTET_ERR_RES for a side outside [1, VOXTET_MAX_RES] and VOXTET_ERR_ARG
 * for a slab outside [0, res[2]] or res == NULL. */
int voxelize_tets_grid(const float *d_verts, int64_t n_verts, const int32_t *d_tets, int64_t n_tets,
                       const float grid_origin[3], float voxel_size, const int32_t res[3], int32_t z_begin,
                       int32_t z_end, uint32_t *d_out_bits, void *d_workspace, size_t ws_bytes,
                       const voxtet_opts *opts, void *stream);

/* ------------------------------------------------------------------ sparse output
 *
 * Brick-sparse grids (Section 5, "Octrees", notes that voxel data is usually
 * stored sparsely).  The grid is a general grid as in voxelize_tets_grid (same
 * lattice, same samples, same bits) with sides up to VOXTET_SPARSE_MAX_SIDE, cut
 * into bricks of 32 x 8 x 8 voxels (x, y, z).  Only bricks holding a set voxel are
 * returned: brick (bx, by, bz) covers voxels 32bx <= i < 32bx + 32, 8by <= j <
 * 8by + 8, 8bz <= l < 8bz + 8; its VOXTET_BRICK_WORDS words are word dz * 8 + dy
 * = bits of voxels (32bx + bit, 8by + dy, 8bz + dz); its key is
 * bx | by << 16 | bz << 32.  Keys come out in increasing order.  Voxels outside
 * the grid (a partial last brick) are zero. */
#define VOXTET_SPARSE_MAX_SIDE 65536
#define VOXTET_BRICK_WORDS 64

/* Bytes of device scratch voxelize_tets_sparse needs for this grid and slab depth
 * (256-byte aligned): a dense slab of slab_depth slices, compaction counters and one
 * bit per slab.  0 if the arguments are invalid. */
size_t voxtet_sparse_scratch_size(const int32_t res[3], int32_t slab_depth);

/* Voxelize into bricks.  The grid is built slab_depth slices at a time (a multiple
 * of 8, >= 8) in d_scratch and each slab is compacted; slabs that no tetrahedron
 * reaches are skipped.  Larger slabs mean fewer passes over the tetrahedra; slabs
 * of about the size of the GPU's L2 cache (128 MiB on GB300) are fastest.
 *   res            HOST int32[3], sides in [1, VOXTET_SPARSE_MAX_SIDE]
 *   d_brick_keys   DEVICE uint64 [max_bricks], 8-byte aligned
 *   d_brick_words  DEVICE uint32 [max_bricks][VOXTET_BRICK_WORDS], 4-byte aligned
 *   n_bricks       HOST out: the number of non-empty bricks, also when it exceeds
 *                  max_bricks (then VOXTET_ERR_NOMEM is returned and only the first
 *                  max_bricks bricks are written)
 *   d_scratch      DEVICE, voxtet_sparse_scratch_size(res, slab_depth) bytes, 256-byte aligned
 * Other arguments as voxelize_tets; opts->accumulate must be 0.  The call always
 * synchronizes `stream` (it returns the brick count). */
int voxelize_tets_sparse(const float *d_verts, int64_t n_verts, const int32_t *d_tets, int64_t n_tets,
                         const float grid_origin[3], float voxel_size, const int32_t res[3], int32_t slab_depth,
                         uint64_t *d_brick_keys, uint32_t *d_brick_words, int64_t max_bricks, int64_t *n_bricks,
                         void *d_scratch, size_t scratch_bytes, void *d_workspace, size_t ws_bytes,
                         const voxtet_opts *opts, void *stream);

/* Synchronize `stream` and return the device-detected status the last call on
 * this workspace recorded (VOXTET_OK if none). */
int voxtet_last_status(const void *d_workspace, void *stream);

/* Without synchronizing: enqueue on `stream` a copy of the device-detected status
 * word the last call on this workspace left (4 bytes) into *status_word, which may
 * be pinned host or device memory; once the stream has passed that point,
 * voxtet_status_of_word(*status_word) is that call's device-detected status.  For
 * callers that keep many calls in flight (a pipeline of host meshes). */
int voxtet_status_async(const void *d_workspace, int32_t *status_word, void *stream);
int voxtet_status_of_word(int32_t status_word);

/* Synchronize `stream` and copy the last call's counters to *out (HOST). */
int voxtet_read_stats(const void *d_workspace, voxtet_stats *out, void *stream);

/* Static English text for a status code. */
const char *voxtet_strerror(int status);

/* Number of CUDA kernels this library has launched since it was loaded. */
uint64_t voxtet_launch_count(void);

/* ------------------------------------------------------------------ batches
 *
 * Many meshes of uneven size and resolution voxelized together: one persistent
 * launch per kernel type covers every job (the paper voxelizes one mesh per
 * CPU/GPU run, Section 3 "Parallelization"; Table 1 shows small meshes gain little
 * from the GPU because of per-mesh transfer and launch overheads, which batching
 * amortizes).  Each job has the semantics of voxelize_tets. */
typedef struct {
    const void *d_verts;   /* DEVICE float32 [n_verts][3], or int32 lattice coordinates if fixed_point */
    int64_t n_verts;
    const int32_t *d_tets; /* DEVICE int32 [n_tets][4], 16-byte aligned */
    int64_t n_tets;
    float origin[3];       /* grid corner (ignored if fixed_point) */
    float voxel_size;      /* > 0 (ignored if fixed_point) */
    int32_t res;           /* power of two in [1, VOXTET_MAX_RES] */
    int32_t span_rows;     /* bounding-box rows per work item; 0 = opts->span_rows or automatic */
    int32_t fixed_point;   /* 1: d_verts holds lattice coordinates as in voxelize_tets_fixed */
    int32_t reserved;
    uint32_t *d_out_bits;  /* DEVICE grid of this job, layout as for voxelize_tets */
} voxtet_job;

/* Bytes of device workspace (256-byte aligned) a batch of these jobs needs when
 * the batch table is sized for max_jobs >= n_jobs jobs: a table part that grows
 * with max_jobs plus one voxtet_workspace_size() slice per job.  0 on bad input. */
size_t voxtet_batch_workspace_size(const voxtet_job *jobs, int32_t n_jobs, int32_t max_jobs);

/* Voxelize a batch (jobs: HOST array).  Per-job argument errors are reported in
 * job_status (HOST int32[n_jobs], may be NULL) and such jobs touch nothing; with
 * opts->sync = 1 job_status also receives each job's device-detected status.
 * Returns VOXTET_OK unless the batch as a whole is invalid (bad options,
 * workspace too small: VOXTET_ERR_WORKSPACE) or CUDA fails. */
int voxelize_tets_batched(const voxtet_job *jobs, int32_t n_jobs, void *d_workspace, size_t ws_bytes,
                          const voxtet_opts *opts, void *stream, int32_t *job_status);

/* A reusable batch plan: the first run captures the table upload and the batch
 * kernels into a CUDA graph; later runs rewrite the table (a pinned host buffer the
 * plan owns) and replay the graph on the caller's stream, whatever the jobs, as
 * long as there are at most max_jobs of them and they fit the workspace.  A plan
 * runs one batch at a time: voxtet_plan_run waits for the plan's previous run
 * before reusing its buffer.  Use several plans (each with its own workspace) to
 * keep several batches in flight. */
typedef struct voxtet_plan voxtet_plan;

int voxtet_plan_create(void *d_workspace, size_t ws_bytes, int32_t max_jobs, const voxtet_opts *opts,
                       voxtet_plan **plan);
/* Enqueue a batch on `stream`; VOXTET_ERR_NOMEM if it does not fit the workspace. */
int voxtet_plan_run(voxtet_plan *plan, const voxtet_job *jobs, int32_t n_jobs, void *stream);
/* 1 if the plan's last run has finished, 0 if not, negative on error (does not block). */
int voxtet_plan_query(voxtet_plan *plan);
/* Wait for the last run; fill job_status (HOST int32[n_jobs], may be NULL). */
int voxtet_plan_wait(voxtet_plan *plan, int32_t *job_status);
void voxtet_plan_destroy(voxtet_plan *plan);

/* Size of the fixed device scratch behind voxelize_tets_noalloc (16 MiB). */
#define VOXTET_NOALLOC_SCRATCH_BYTES (16u << 20)

/* voxelize_tets without a workspace argument, for callers that cannot allocate
 * device memory when they call: a plugin or library running inside a host
 * application that owns the whole device-memory budget (a renderer or simulation
 * that reserves the device's memory up front and hands out only its own buffers),
 * or a latency-critical loop that must not enter cudaMalloc, which can synchronize
 * the device and take milliseconds.  (The paper has no counterpart; this is an
 * interface convenience.)
 *
 * The workspace is a fixed array of VOXTET_NOALLOC_SCRATCH_BYTES compiled into
 * the library: every GPU that loads the library holds it until the process exits.
 * The minimum (grid-independent) workspace, voxtet_workspace_size(n_tets, n_verts,
 * res) with any res <= 512, must fit in it, else the call returns VOXTET_ERR_NOMEM
 * before anything is launched (about 1M tetrahedra with 200k vertices fit); the
 * queue of rows the filter could not certify then takes the rest of the array.  The
 * function itself calls no allocator; opts->profile is ignored.  The first call on
 * each device (this one or voxtet_noalloc_status_async) looks up the array's device
 * address with cudaGetSymbolAddress, with that device current, so make that first
 * call before any stream capture.
 *
 * With opts->sync = 1 the call synchronizes `stream` and returns the device-detected
 * status, as voxelize_tets does.  With opts->sync = 0 it returns once the work is
 * enqueued; read the device-detected status with voxtet_noalloc_status_async.
 *
 * All calls share the one array and it keeps the last call's contents; what must
 * start at zero (status header, redo bitmap) is cleared by every call.  Calls that
 * overlap on the GPU (on different streams or host threads without ordering) race on
 * it and give undefined results.  Other arguments, ownership and status codes are
 * those of voxelize_tets. */
int voxelize_tets_noalloc(const float *d_verts, int64_t n_verts, const int32_t *d_tets, int64_t n_tets,
                          const float grid_origin[3], float voxel_size, int32_t res, uint32_t *d_out_bits,
                          const voxtet_opts *opts, void *stream);

/* voxtet_status_async for the fixed array behind voxelize_tets_noalloc: enqueue on
 * `stream` a copy of the status word the last voxelize_tets_noalloc call left
 * (4 bytes) into *status_word (pinned host or device memory), without
 * synchronizing; once the stream has passed that point,
 * voxtet_status_of_word(*status_word) is that call's device-detected status.
 * Allocates nothing.  VOXTET_ERR_ARG if status_word is NULL. */
int voxtet_noalloc_status_async(int32_t *status_word, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VOXTET_H */
