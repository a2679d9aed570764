/*
 * voxtet_oracle.c -- CPU oracle for solid voxelization of tetrahedral meshes.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously correct
 * reference that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * What it computes (arXiv 2106.01326, Section 3 "Voxelization" and Section 4,
 * Theorem 1), with the readings this project fixes where the paper is silent:
 *
 *   - Vertices are snapped to a fixed-point lattice: the grid's extent maps to
 *     [0, 2^20] per axis, X = round_half_even(((double)v - o) / h * 2^(20-k))
 *     for a grid of res = 2^k voxels per axis (each double operation rounded
 *     to nearest).  |X| <= 2^21 is required.
 *   - Voxel (i, j, l) is sampled at its centre P = ((2i+1)s, (2j+1)s, (2l+1)s)
 *     in lattice units, s = 2^(19-k).
 *   - The paper iterates over the bounding box of every tetrahedron and applies
 *     the point-in-tetrahedron test of Theorem 1 to each sample in it.  With
 *     a = PA, b = PB, c = PC, d = PD and D_a = det(b,c,d), D_b = det(a,c,d),
 *     D_c = det(a,b,d), D_d = det(a,b,c), Theorem 1 puts P strictly inside iff
 *     (D_a>0, D_b<0, D_c>0, D_d<0) or the reverse pattern.
 *   - Reading "closed": the grid marks samples of the CLOSED tetrahedron, so
 *     the four strict comparisons become non-strict (a sample on a face shared
 *     by two tets is then inside both, and no holes open along shared faces).
 *     mode = 1 keeps the paper's strict test.
 *   - Reading "degenerate": a tetrahedron whose signed volume
 *     det(AB, AC, AD) (Lemma 1.1's proof) is zero marks nothing.
 *   - The grid is the union over tetrahedra; it does not depend on their order.
 *
 * Determinants are evaluated exactly in 128-bit integers: differences of
 * lattice coordinates are below 2^23 in magnitude, so each of the six triple
 * products is below 2^69.
 *
 * Output layout: bit (i, j, l) is word (l*res + j)*W + (i >> 5), bit (i & 31),
 * W = ceil(res / 32); padding bits are zero.
 *
 * General grids (the *_grid functions): res = (rx, ry, rz) voxels of the same
 * edge h, any sizes in [1, 2^19].  The lattice keeps voxel centres on lattice
 * points: K = ceil(log2(max(rx, ry, rz))), the lattice step is 2^(20-K) per
 * voxel (so the grid's longest side spans at most 2^20 lattice units) and
 * X = round_half_even(((double)v - o) / h * 2^(20-K)); samples sit at
 * (2i+1)s with s = 2^(19-K).  For rx = ry = rz = 2^k this is the cubic grid
 * above.  Bit (i, j, l) is word ((l - z0)*ry + j)*W + (i >> 5) with
 * W = ceil(rx / 32), for the slab of slices z0 <= l < z1 that a call produces.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef __int128 i128;

/* Threads of one parallel region: n_threads > 0 asks for that many, 0 for the
 * OpenMP default.  It is given to each region as a num_threads clause, so one
 * call never changes the thread count of later calls.  The team size the last
 * region actually ran with is kept for voxtet_oracle_last_threads(). */
static int team_size(int32_t n_threads) {
#ifdef _OPENMP
    return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

int voxtet_oracle_last_team = 0;  /* shared with paper_cpu.c (same library) */

static void note_team(void) {
#ifdef _OPENMP
    voxtet_oracle_last_team = omp_get_num_threads();
#else
    voxtet_oracle_last_team = 1;
#endif
}

/* status codes (numeric values are part of the documented interface) */
#define OR_OK 0
#define OR_ERR_ARG (-1)
#define OR_ERR_RES (-2)
#define OR_ERR_INDEX (-3)
#define OR_ERR_RANGE (-4)
#define OR_ERR_NAN (-5)

#define LATTICE_BITS 20
#define COORD_LIMIT (1 << 21)

static int log2_res(int32_t res) {
    if (res < 1 || res > (1 << 19)) return -1;
    if (res & (res - 1)) return -1;
    int k = 0;
    while ((1 << k) != res) ++k;
    return k;
}

/* K = ceil(log2(max(res))) of a general grid, or -1 if a side is outside [1, 2^19]. */
static int grid_exponent(const int32_t res[3]) {
    int32_t mx = 0;
    for (int q = 0; q < 3; ++q) {
        if (res[q] < 1 || res[q] > (1 << 19)) return -1;
        if (res[q] > mx) mx = res[q];
    }
    int K = 0;
    while (((int32_t)1 << K) < mx) ++K;
    return K;
}

/* floor(a / b) for b > 0, without relying on the sign convention of '/'. */
static int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

static int64_t ceil_div(int64_t a, int64_t b) { return -floor_div(-a, b); }

/* determinant of the 3x3 matrix whose ROWS are r0, r1, r2 */
static i128 det3(const int64_t r0[3], const int64_t r1[3], const int64_t r2[3]) {
    i128 m0 = (i128)r1[1] * r2[2] - (i128)r1[2] * r2[1];
    i128 m1 = (i128)r1[0] * r2[2] - (i128)r1[2] * r2[0];
    i128 m2 = (i128)r1[0] * r2[1] - (i128)r1[1] * r2[0];
    return (i128)r0[0] * m0 - (i128)r0[1] * m1 + (i128)r0[2] * m2;
}

/* Signed volume times 6: det(AB, AC, AD) (Lemma 1.1's proof). */
static i128 signed_volume6(const int64_t A[3], const int64_t B[3], const int64_t C[3], const int64_t D[3]) {
    int64_t ab[3], ac[3], ad[3];
    for (int q = 0; q < 3; ++q) {
        ab[q] = B[q] - A[q];
        ac[q] = C[q] - A[q];
        ad[q] = D[q] - A[q];
    }
    return det3(ab, ac, ad);
}

/* Theorem 1's test for sample P against tetrahedron ABCD.  strict = 1 is the
 * paper's statement; strict = 0 is the closed reading. */
static int theorem1_inside(const int64_t A[3], const int64_t B[3], const int64_t C[3], const int64_t D[3],
                           const int64_t P[3], int strict) {
    int64_t a[3], b[3], c[3], d[3];
    for (int q = 0; q < 3; ++q) {
        a[q] = A[q] - P[q];
        b[q] = B[q] - P[q];
        c[q] = C[q] - P[q];
        d[q] = D[q] - P[q];
    }
    i128 Da = det3(b, c, d);
    i128 Db = det3(a, c, d);
    i128 Dc = det3(a, b, d);
    i128 Dd = det3(a, b, c);
    if (strict)
        return (Da > 0 && Db < 0 && Dc > 0 && Dd < 0) || (Da < 0 && Db > 0 && Dc < 0 && Dd > 0);
    return (Da >= 0 && Db <= 0 && Dc >= 0 && Dd <= 0) || (Da <= 0 && Db >= 0 && Dc <= 0 && Dd >= 0);
}

/* ------------------------------------------------------------------ snap */

static int snap_k(const float *verts, int64_t n_verts, const float origin[3], float voxel_size, int k,
                  int32_t *xyz) {
    if (n_verts < 0 || !(voxel_size > 0.0f) || !isfinite(voxel_size)) return OR_ERR_ARG;
    for (int q = 0; q < 3; ++q)
        if (!isfinite(origin[q])) return OR_ERR_ARG;
    const double scale = ldexp(1.0, LATTICE_BITS - k); /* exact power of two */
    const double h = (double)voxel_size;
    int status = OR_OK;
    for (int64_t v = 0; v < n_verts; ++v) {
        for (int q = 0; q < 3; ++q) {
            float f = verts[3 * v + q];
            if (!isfinite(f)) {
                status = OR_ERR_NAN;
                xyz[3 * v + q] = 0;
                continue;
            }
            volatile double diff = (double)f - (double)origin[q]; /* rounded to nearest */
            volatile double quot = diff / h;                      /* rounded to nearest */
            double x = quot * scale;                              /* exact */
            double r = nearbyint(x);                              /* ties to even (default mode) */
            if (!(fabs(r) <= (double)COORD_LIMIT)) {
                if (status == OR_OK) status = OR_ERR_RANGE;
                xyz[3 * v + q] = 0;
                continue;
            }
            xyz[3 * v + q] = (int32_t)r;
        }
    }
    return status;
}

int voxtet_oracle_snap(const float *verts, int64_t n_verts, const float origin[3], float voxel_size,
                       int32_t res, int32_t *xyz) {
    int k = log2_res(res);
    if (k < 0) return OR_ERR_RES;
    return snap_k(verts, n_verts, origin, voxel_size, k, xyz);
}

int voxtet_oracle_snap_grid(const float *verts, int64_t n_verts, const float origin[3], float voxel_size,
                            const int32_t res[3], int32_t *xyz) {
    int K = grid_exponent(res);
    if (K < 0) return OR_ERR_RES;
    return snap_k(verts, n_verts, origin, voxel_size, K, xyz);
}

/* ------------------------------------------------------------------ voxelize */

typedef struct {
    int32_t lo[3], hi[3]; /* inclusive sample-index box, clamped; empty if lo > hi */
    int32_t live;         /* non-degenerate and non-empty box */
} tet_box;

static int validate(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets) {
    for (int64_t v = 0; v < 3 * n_verts; ++v)
        if (xyz[v] < -COORD_LIMIT || xyz[v] > COORD_LIMIT) return OR_ERR_RANGE;
    for (int64_t t = 0; t < 4 * n_tets; ++t)
        if (tets[t] < 0 || (int64_t)tets[t] >= n_verts) return OR_ERR_INDEX;
    return OR_OK;
}

static void load_vertex(const int32_t *xyz, int32_t idx, int64_t out[3]) {
    out[0] = xyz[3 * (int64_t)idx + 0];
    out[1] = xyz[3 * (int64_t)idx + 1];
    out[2] = xyz[3 * (int64_t)idx + 2];
}

/* Bounding box of a tet in sample indices: samples (2i+1)s with min <= (2i+1)s <= max. */
static void sample_box(const int64_t V[4][3], int64_t s, const int32_t res[3], tet_box *b) {
    for (int q = 0; q < 3; ++q) {
        int64_t mn = V[0][q], mx = V[0][q];
        for (int m = 1; m < 4; ++m) {
            if (V[m][q] < mn) mn = V[m][q];
            if (V[m][q] > mx) mx = V[m][q];
        }
        int64_t lo = ceil_div(mn - s, 2 * s);
        int64_t hi = floor_div(mx - s, 2 * s);
        if (lo < 0) lo = 0;
        if (hi > res[q] - 1) hi = res[q] - 1;
        b->lo[q] = (int32_t)lo;
        b->hi[q] = (int32_t)hi;
    }
}

static void prepare(const int32_t *xyz, const int32_t *tets, int64_t n_tets, const int32_t res[3], int64_t s,
                    int mode, int32_t n_threads, tet_box *boxes, int64_t *n_degenerate) {
    int64_t degenerate = 0;
#pragma omp parallel for schedule(static) reduction(+ : degenerate) num_threads(team_size(n_threads))
    for (int64_t t = 0; t < n_tets; ++t) {
        int64_t V[4][3];
        for (int m = 0; m < 4; ++m) load_vertex(xyz, tets[4 * t + m], V[m]);
        i128 v6 = signed_volume6(V[0], V[1], V[2], V[3]);
        sample_box(V, s, res, &boxes[t]);
        int empty = 0;
        for (int q = 0; q < 3; ++q)
            if (boxes[t].lo[q] > boxes[t].hi[q]) empty = 1;
        if (v6 == 0) degenerate += 1;
        /* strict mode needs no degeneracy rule: Theorem 1's strict patterns
         * cannot hold when the four determinants sum to zero. */
        boxes[t].live = !empty && (mode == 1 || v6 != 0);
    }
    *n_degenerate = degenerate;
}

/* Samples are visited per tet over its bounding box (the paper's loop order),
 * with the grid split into z-chunks so that each thread owns whole words.
 * Only slices z0 <= l < z1 are produced; out_bits holds (z1 - z0)*ry*W words
 * (slice z0 first).  k is the lattice exponent (sample step 2^(20-k)). */
static int voxelize_core(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                         const int32_t res[3], int k, int32_t mode, int32_t n_threads, int32_t z0, int32_t z1,
                         uint32_t *out_bits, int64_t *stats) {
    if (n_verts < 0 || n_tets < 0 || (mode != 0 && mode != 1)) return OR_ERR_ARG;
    if (z0 < 0 || z1 > res[2] || z0 > z1) return OR_ERR_ARG;
    int st = validate(xyz, n_verts, tets, n_tets);
    if (st != OR_OK) return st;
    const int64_t s = (int64_t)1 << (19 - k);
    const int64_t ry = res[1];
    const int64_t W = (res[0] + 31) / 32;
    const int64_t n_words = (int64_t)(z1 - z0) * ry * W;
    memset(out_bits, 0, (size_t)(n_words > 0 ? n_words : 0) * sizeof(uint32_t));
    tet_box *boxes = (tet_box *)malloc((size_t)(n_tets > 0 ? n_tets : 1) * sizeof(tet_box));
    if (!boxes) return OR_ERR_ARG;
    int64_t degenerate = 0;
    prepare(xyz, tets, n_tets, res, s, mode, n_threads, boxes, &degenerate);

    const int64_t depth = z1 - z0;
    int64_t chunk = 1;
    while (chunk * 64 < depth) chunk *= 2; /* at most 64 z-chunks */
    const int64_t n_chunks = depth > 0 ? (depth + chunk - 1) / chunk : 0;
    int64_t tested = 0, rows_hit = 0;
#pragma omp parallel num_threads(team_size(n_threads)) reduction(+ : tested, rows_hit)
    {
#pragma omp single
        note_team();
#pragma omp for schedule(dynamic, 1)
    for (int64_t ch = 0; ch < n_chunks; ++ch) {
        const int64_t c0 = z0 + ch * chunk;
        const int64_t c1 = (c0 + chunk - 1 < z1 - 1) ? c0 + chunk - 1 : z1 - 1;
        for (int64_t t = 0; t < n_tets; ++t) {
            const tet_box *b = &boxes[t];
            if (!b->live || b->hi[2] < c0 || b->lo[2] > c1) continue;
            int64_t V[4][3];
            for (int m = 0; m < 4; ++m) load_vertex(xyz, tets[4 * t + m], V[m]);
            const int64_t l0 = b->lo[2] > c0 ? b->lo[2] : c0;
            const int64_t l1 = b->hi[2] < c1 ? b->hi[2] : c1;
            for (int64_t l = l0; l <= l1; ++l)
                for (int64_t j = b->lo[1]; j <= b->hi[1]; ++j) {
                    int hit = 0;
                    for (int64_t i = b->lo[0]; i <= b->hi[0]; ++i) {
                        int64_t P[3] = {(2 * i + 1) * s, (2 * j + 1) * s, (2 * l + 1) * s};
                        tested += 1;
                        if (theorem1_inside(V[0], V[1], V[2], V[3], P, mode == 1)) {
                            out_bits[((l - z0) * ry + j) * W + (i >> 5)] |= (uint32_t)1u << (i & 31);
                            hit = 1;
                        }
                    }
                    rows_hit += hit;
                }
        }
    }
    }
    free(boxes);
    if (stats) {
        int64_t set = 0;
        for (int64_t w = 0; w < n_words; ++w) set += __builtin_popcount(out_bits[w]);
        stats[0] = degenerate;
        stats[1] = tested;
        stats[2] = set;
        stats[3] = rows_hit;
    }
    return OR_OK;
}

/* Cubic grid of res = 2^k voxels per axis, slices z0 <= l < z1 (full grid: 0, res). */
int voxtet_oracle_voxelize_fixed_slab(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                                      int32_t res, int32_t mode, int32_t n_threads, int32_t z0, int32_t z1,
                                      uint32_t *out_bits,
                                      int64_t *stats /* [4]: degenerate tets, samples tested, bits set, (tet, x-row) pairs holding a sample */) {
    int k = log2_res(res);
    if (k < 0) return OR_ERR_RES;
    const int32_t r3[3] = {res, res, res};
    return voxelize_core(xyz, n_verts, tets, n_tets, r3, k, mode, n_threads, z0, z1, out_bits, stats);
}

/* General grid (rx, ry, rz), slices z0 <= l < z1, lattice coordinates on the
 * grid's lattice (exponent K = ceil(log2(max side))). */
int voxtet_oracle_voxelize_grid_fixed(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                                      const int32_t res[3], int32_t mode, int32_t n_threads, int32_t z0, int32_t z1,
                                      uint32_t *out_bits, int64_t *stats) {
    int K = grid_exponent(res);
    if (K < 0) return OR_ERR_RES;
    return voxelize_core(xyz, n_verts, tets, n_tets, res, K, mode, n_threads, z0, z1, out_bits, stats);
}

/* General grid from float vertices: snap_grid, then voxelize_grid_fixed. */
int voxtet_oracle_voxelize_grid(const float *verts, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                                const float origin[3], float voxel_size, const int32_t res[3], int32_t mode,
                                int32_t n_threads, int32_t z0, int32_t z1, uint32_t *out_bits, int64_t *stats) {
    if (n_verts < 0) return OR_ERR_ARG;
    int32_t *xyz = (int32_t *)malloc((size_t)(n_verts > 0 ? n_verts : 1) * 3 * sizeof(int32_t));
    if (!xyz) return OR_ERR_ARG;
    int st = voxtet_oracle_snap_grid(verts, n_verts, origin, voxel_size, res, xyz);
    if (st == OR_OK)
        st = voxtet_oracle_voxelize_grid_fixed(xyz, n_verts, tets, n_tets, res, mode, n_threads, z0, z1, out_bits,
                                               stats);
    free(xyz);
    return st;
}

int voxtet_oracle_voxelize_fixed(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                                 int32_t res, int32_t mode, int32_t n_threads, uint32_t *out_bits,
                                 int64_t *stats) {
    if (log2_res(res) < 0) return OR_ERR_RES;
    return voxtet_oracle_voxelize_fixed_slab(xyz, n_verts, tets, n_tets, res, mode, n_threads, 0, res, out_bits,
                                             stats);
}

int voxtet_oracle_voxelize(const float *verts, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                           const float origin[3], float voxel_size, int32_t res, int32_t mode, int32_t n_threads,
                           uint32_t *out_bits, int64_t *stats) {
    if (n_verts < 0) return OR_ERR_ARG;
    int32_t *xyz = (int32_t *)malloc((size_t)(n_verts > 0 ? n_verts : 1) * 3 * sizeof(int32_t));
    if (!xyz) return OR_ERR_ARG;
    int st = voxtet_oracle_snap(verts, n_verts, origin, voxel_size, res, xyz);
    if (st == OR_OK)
        st = voxtet_oracle_voxelize_fixed(xyz, n_verts, tets, n_tets, res, mode, n_threads, out_bits, stats);
    free(xyz);
    return st;
}

/* Every sample against every tet, no bounding-box pruning, one thread.  Used
 * to pin the pruned loop above on tiny inputs. */
static int all_pairs_core(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                          const int32_t res[3], int k, int32_t mode, uint32_t *out_bits) {
    if (n_verts < 0 || n_tets < 0 || (mode != 0 && mode != 1)) return OR_ERR_ARG;
    int st = validate(xyz, n_verts, tets, n_tets);
    if (st != OR_OK) return st;
    const int64_t s = (int64_t)1 << (19 - k);
    const int64_t rx = res[0], ry = res[1], rz = res[2];
    const int64_t W = (rx + 31) / 32;
    memset(out_bits, 0, (size_t)(rz * ry * W) * sizeof(uint32_t));
    for (int64_t l = 0; l < rz; ++l)
        for (int64_t j = 0; j < ry; ++j)
            for (int64_t i = 0; i < rx; ++i) {
                int64_t P[3] = {(2 * i + 1) * s, (2 * j + 1) * s, (2 * l + 1) * s};
                for (int64_t t = 0; t < n_tets; ++t) {
                    int64_t V[4][3];
                    for (int m = 0; m < 4; ++m) load_vertex(xyz, tets[4 * t + m], V[m]);
                    if (mode == 0 && signed_volume6(V[0], V[1], V[2], V[3]) == 0) continue;
                    if (theorem1_inside(V[0], V[1], V[2], V[3], P, mode == 1)) {
                        out_bits[(l * ry + j) * W + (i >> 5)] |= (uint32_t)1u << (i & 31);
                        break;
                    }
                }
            }
    return OR_OK;
}

int voxtet_oracle_all_pairs(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                            int32_t res, int32_t mode, uint32_t *out_bits) {
    int k = log2_res(res);
    if (k < 0) return OR_ERR_RES;
    const int32_t r3[3] = {res, res, res};
    return all_pairs_core(xyz, n_verts, tets, n_tets, r3, k, mode, out_bits);
}

int voxtet_oracle_all_pairs_grid(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                                 const int32_t res[3], int32_t mode, uint32_t *out_bits) {
    int K = grid_exponent(res);
    if (K < 0) return OR_ERR_RES;
    return all_pairs_core(xyz, n_verts, tets, n_tets, res, K, mode, out_bits);
}

/* The four determinants of Theorem 1 for one point, as (hi, lo) halves of the
 * 128-bit values: out[2m] = high 64 bits, out[2m+1] = low 64 bits, m = a,b,c,d. */
void voxtet_oracle_theorem1_dets(const int64_t A[3], const int64_t B[3], const int64_t C[3], const int64_t D[3],
                                 const int64_t P[3], int64_t out[8]) {
    int64_t a[3], b[3], c[3], d[3];
    for (int q = 0; q < 3; ++q) {
        a[q] = A[q] - P[q];
        b[q] = B[q] - P[q];
        c[q] = C[q] - P[q];
        d[q] = D[q] - P[q];
    }
    i128 D4[4] = {det3(b, c, d), det3(a, c, d), det3(a, b, d), det3(a, b, c)};
    for (int m = 0; m < 4; ++m) {
        out[2 * m] = (int64_t)(D4[m] >> 64);
        out[2 * m + 1] = (int64_t)(uint64_t)D4[m];
    }
}

/* Threads a call with n_threads = 0 uses (the OpenMP default; no call changes it). */
int voxtet_oracle_num_threads(void) { return team_size(0); }

/* Team size of the last voxelization or paper-method region that ran. */
int voxtet_oracle_last_threads(void) { return voxtet_oracle_last_team; }
