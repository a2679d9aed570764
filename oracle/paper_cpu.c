/*
 * paper_cpu.c -- the paper's own CPU voxelization, in binary floating point.
 *
 * TEST INFRASTRUCTURE ONLY, and not a reference: it re-creates the method as a
 * CPU program would ordinarily write it, so that its answers can be counted
 * against the exact oracle (voxtet_oracle.c).  Nothing in the library uses it;
 * only the test suite and the benchmark's CPU-baseline leg load it.
 *
 * Method (arXiv 2106.01326): Section 3 "Voxelization" visits the bounding box of
 * every tetrahedron and applies the point-in-tetrahedron test of Section 4,
 * Theorem 1, to each sample; "Parallelization" spreads the tetrahedra over CPU
 * threads with OpenMP.  Theorem 1: with a = A-P, b = B-P, c = C-P, d = D-P and
 * D_a = det(b,c,d), D_b = det(a,c,d), D_c = det(a,b,d), D_d = det(a,b,c) (rows),
 * P is inside iff (D_a>0, D_b<0, D_c>0, D_d<0) or the reverse pattern.  The
 * determinants here are evaluated in float or double (cofactor expansion along
 * the first row), so signs near zero can come out wrong.  mode 1 is the
 * theorem as stated; mode 0 the closed reading (non-strict comparisons, and a
 * tetrahedron whose computed signed volume is zero marks nothing).
 *
 * Inputs are the oracle's: lattice coordinates (|X| <= 2^21) and a cubic grid of
 * res = 2^k, samples at (2i+1)s with s = 2^(19-k).  Coordinates and their
 * differences are exact in both precisions, so every difference from the oracle
 * comes from the rounding of the determinant products and sums.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Team size of the last region (defined in voxtet_oracle.c, same library). */
extern int voxtet_oracle_last_team;

/* n_threads > 0: that many threads for this call's region; 0: the OpenMP default.  A
 * num_threads clause, so the count never leaks into later calls. */
static int pc_team_size(int32_t n_threads) {
#ifdef _OPENMP
    return n_threads > 0 ? n_threads : omp_get_max_threads();
#else
    (void)n_threads;
    return 1;
#endif
}

static void pc_note_team(void) {
#ifdef _OPENMP
    voxtet_oracle_last_team = omp_get_num_threads();
#else
    voxtet_oracle_last_team = 1;
#endif
}

#define PC_OK 0
#define PC_ERR_ARG (-1)
#define PC_ERR_RES (-2)
#define PC_ERR_INDEX (-3)

#define DEFINE_DET3(T)                                                                          \
    static T det3_##T(const T r0[3], const T r1[3], const T r2[3]) {                           \
        return r0[0] * (r1[1] * r2[2] - r1[2] * r2[1]) - r0[1] * (r1[0] * r2[2] - r1[2] * r2[0]) + \
               r0[2] * (r1[0] * r2[1] - r1[1] * r2[0]);                                        \
    }
DEFINE_DET3(float)
DEFINE_DET3(double)

#define DEFINE_INSIDE(T)                                                                        \
    static int inside_##T(const T A[3], const T B[3], const T C[3], const T D[3], const T P[3],  \
                          int strict) {                                                         \
        T a[3], b[3], c[3], d[3];                                                               \
        for (int q = 0; q < 3; ++q) {                                                           \
            a[q] = A[q] - P[q];                                                                 \
            b[q] = B[q] - P[q];                                                                 \
            c[q] = C[q] - P[q];                                                                 \
            d[q] = D[q] - P[q];                                                                 \
        }                                                                                       \
        const T Da = det3_##T(b, c, d), Db = det3_##T(a, c, d);                                 \
        const T Dc = det3_##T(a, b, d), Dd = det3_##T(a, b, c);                                 \
        if (strict)                                                                             \
            return (Da > 0 && Db < 0 && Dc > 0 && Dd < 0) || (Da < 0 && Db > 0 && Dc < 0 && Dd > 0); \
        return (Da >= 0 && Db <= 0 && Dc >= 0 && Dd <= 0) || (Da <= 0 && Db >= 0 && Dc <= 0 && Dd >= 0); \
    }
DEFINE_INSIDE(float)
DEFINE_INSIDE(double)

static int64_t floor_div(int64_t a, int64_t b) {
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

int voxtet_paper_cpu(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets, int32_t res,
                     int32_t precision, int32_t mode, int32_t n_threads, uint32_t *out_bits) {
    if (res < 1 || res > (1 << 19) || (res & (res - 1))) return PC_ERR_RES;
    if (n_verts < 0 || n_tets < 0 || (mode != 0 && mode != 1) || (precision != 0 && precision != 1))
        return PC_ERR_ARG;
    for (int64_t t = 0; t < 4 * n_tets; ++t)
        if (tets[t] < 0 || (int64_t)tets[t] >= n_verts) return PC_ERR_INDEX;
    int k = 0;
    while ((1 << k) != res) ++k;
    const int64_t s = (int64_t)1 << (19 - k);
    const int64_t W = (res + 31) / 32;
    memset(out_bits, 0, (size_t)((int64_t)res * res * W) * sizeof(uint32_t));
#pragma omp parallel num_threads(pc_team_size(n_threads))
    {
#pragma omp single
        pc_note_team();
#pragma omp for schedule(dynamic, 64)
    for (int64_t t = 0; t < n_tets; ++t) {
        int64_t V[4][3];
        for (int m = 0; m < 4; ++m)
            for (int q = 0; q < 3; ++q) V[m][q] = xyz[3 * (int64_t)tets[4 * t + m] + q];
        int64_t lo[3], hi[3];
        int empty = 0;
        for (int q = 0; q < 3; ++q) {
            int64_t mn = V[0][q], mx = V[0][q];
            for (int m = 1; m < 4; ++m) {
                if (V[m][q] < mn) mn = V[m][q];
                if (V[m][q] > mx) mx = V[m][q];
            }
            lo[q] = -floor_div(-(mn - s), 2 * s);
            hi[q] = floor_div(mx - s, 2 * s);
            if (lo[q] < 0) lo[q] = 0;
            if (hi[q] > res - 1) hi[q] = res - 1;
            if (lo[q] > hi[q]) empty = 1;
        }
        if (empty) continue;
        float Vf[4][3];
        double Vd[4][3];
        for (int m = 0; m < 4; ++m)
            for (int q = 0; q < 3; ++q) {
                Vf[m][q] = (float)V[m][q];
                Vd[m][q] = (double)V[m][q];
            }
        if (mode == 0) { /* closed reading: a tet of zero computed volume marks nothing */
            float ef[3][3];
            double ed[3][3];
            for (int m = 0; m < 3; ++m)
                for (int q = 0; q < 3; ++q) {
                    ef[m][q] = Vf[m + 1][q] - Vf[0][q];
                    ed[m][q] = Vd[m + 1][q] - Vd[0][q];
                }
            if (precision == 0 ? det3_float(ef[0], ef[1], ef[2]) == 0.0f : det3_double(ed[0], ed[1], ed[2]) == 0.0)
                continue;
        }
        for (int64_t l = lo[2]; l <= hi[2]; ++l)
            for (int64_t j = lo[1]; j <= hi[1]; ++j)
                for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                    const int64_t Pi[3] = {(2 * i + 1) * s, (2 * j + 1) * s, (2 * l + 1) * s};
                    int in;
                    if (precision == 0) {
                        const float P[3] = {(float)Pi[0], (float)Pi[1], (float)Pi[2]};
                        in = inside_float(Vf[0], Vf[1], Vf[2], Vf[3], P, mode == 1);
                    } else {
                        const double P[3] = {(double)Pi[0], (double)Pi[1], (double)Pi[2]};
                        in = inside_double(Vd[0], Vd[1], Vd[2], Vd[3], P, mode == 1);
                    }
                    if (in)
                        __atomic_fetch_or(&out_bits[(l * res + j) * W + (i >> 5)], (uint32_t)1u << (i & 31),
                                          __ATOMIC_RELAXED);
                }
    }
    }
    return PC_OK;
}

/* Per-test disagreements: for every (tetrahedron, sample in its box) pair with
 * slices z0 <= l < z1, Theorem 1 in float and in double against the same test
 * in exact 128-bit integers (written out here, independent of the oracle file).
 * counts[0] tests, [1] exact closed-inside, [2] float closed differs, [3] float
 * strict differs, [4] double closed differs, [5] double strict differs. */
typedef __int128 i128;

static i128 det3_exact(const int64_t r0[3], const int64_t r1[3], const int64_t r2[3]) {
    return (i128)r0[0] * ((i128)r1[1] * r2[2] - (i128)r1[2] * r2[1]) -
           (i128)r0[1] * ((i128)r1[0] * r2[2] - (i128)r1[2] * r2[0]) +
           (i128)r0[2] * ((i128)r1[0] * r2[1] - (i128)r1[1] * r2[0]);
}

static int sign_pattern(int sa, int sb, int sc, int sd, int strict) {
    if (strict) return (sa > 0 && sb < 0 && sc > 0 && sd < 0) || (sa < 0 && sb > 0 && sc < 0 && sd > 0);
    return (sa >= 0 && sb <= 0 && sc >= 0 && sd <= 0) || (sa <= 0 && sb >= 0 && sc <= 0 && sd >= 0);
}

#define SGN(x) (((x) > 0) - ((x) < 0))

int voxtet_paper_cpu_disagreements(const int32_t *xyz, int64_t n_verts, const int32_t *tets, int64_t n_tets,
                                   int32_t res, int32_t z0, int32_t z1, int32_t n_threads, int64_t counts[6]) {
    if (res < 1 || res > (1 << 19) || (res & (res - 1))) return PC_ERR_RES;
    if (n_verts < 0 || n_tets < 0 || z0 < 0 || z1 > res || z0 > z1) return PC_ERR_ARG;
    for (int64_t t = 0; t < 4 * n_tets; ++t)
        if (tets[t] < 0 || (int64_t)tets[t] >= n_verts) return PC_ERR_INDEX;
    int k = 0;
    while ((1 << k) != res) ++k;
    const int64_t s = (int64_t)1 << (19 - k);
    int64_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0, c5 = 0;
#pragma omp parallel num_threads(pc_team_size(n_threads)) reduction(+ : c0, c1, c2, c3, c4, c5)
    {
#pragma omp single
        pc_note_team();
#pragma omp for schedule(dynamic, 64)
    for (int64_t t = 0; t < n_tets; ++t) {
        int64_t V[4][3];
        for (int m = 0; m < 4; ++m)
            for (int q = 0; q < 3; ++q) V[m][q] = xyz[3 * (int64_t)tets[4 * t + m] + q];
        int64_t lo[3], hi[3];
        int empty = 0;
        for (int q = 0; q < 3; ++q) {
            int64_t mn = V[0][q], mx = V[0][q];
            for (int m = 1; m < 4; ++m) {
                if (V[m][q] < mn) mn = V[m][q];
                if (V[m][q] > mx) mx = V[m][q];
            }
            lo[q] = -floor_div(-(mn - s), 2 * s);
            hi[q] = floor_div(mx - s, 2 * s);
            if (lo[q] < 0) lo[q] = 0;
            if (hi[q] > res - 1) hi[q] = res - 1;
        }
        if (lo[2] < z0) lo[2] = z0;
        if (hi[2] > z1 - 1) hi[2] = z1 - 1;
        for (int q = 0; q < 3; ++q)
            if (lo[q] > hi[q]) empty = 1;
        if (empty) continue;
        for (int64_t l = lo[2]; l <= hi[2]; ++l)
            for (int64_t j = lo[1]; j <= hi[1]; ++j)
                for (int64_t i = lo[0]; i <= hi[0]; ++i) {
                    const int64_t P[3] = {(2 * i + 1) * s, (2 * j + 1) * s, (2 * l + 1) * s};
                    int64_t e[4][3];
                    float f[4][3];
                    double d[4][3];
                    for (int m = 0; m < 4; ++m)
                        for (int q = 0; q < 3; ++q) {
                            e[m][q] = V[m][q] - P[q];
                            f[m][q] = (float)e[m][q];
                            d[m][q] = (double)e[m][q];
                        }
                    /* rows: D_a = (b,c,d), D_b = (a,c,d), D_c = (a,b,d), D_d = (a,b,c) */
                    const int xs[4] = {SGN(det3_exact(e[1], e[2], e[3])), SGN(det3_exact(e[0], e[2], e[3])),
                                       SGN(det3_exact(e[0], e[1], e[3])), SGN(det3_exact(e[0], e[1], e[2]))};
                    const int fs[4] = {SGN(det3_float(f[1], f[2], f[3])), SGN(det3_float(f[0], f[2], f[3])),
                                       SGN(det3_float(f[0], f[1], f[3])), SGN(det3_float(f[0], f[1], f[2]))};
                    const int ds[4] = {SGN(det3_double(d[1], d[2], d[3])), SGN(det3_double(d[0], d[2], d[3])),
                                       SGN(det3_double(d[0], d[1], d[3])), SGN(det3_double(d[0], d[1], d[2]))};
                    const int xc = sign_pattern(xs[0], xs[1], xs[2], xs[3], 0);
                    const int xst = sign_pattern(xs[0], xs[1], xs[2], xs[3], 1);
                    c0 += 1;
                    c1 += xc;
                    c2 += sign_pattern(fs[0], fs[1], fs[2], fs[3], 0) != xc;
                    c3 += sign_pattern(fs[0], fs[1], fs[2], fs[3], 1) != xst;
                    c4 += sign_pattern(ds[0], ds[1], ds[2], ds[3], 0) != xc;
                    c5 += sign_pattern(ds[0], ds[1], ds[2], ds[3], 1) != xst;
                }
    }
    }
    counts[0] = c0;
    counts[1] = c1;
    counts[2] = c2;
    counts[3] = c3;
    counts[4] = c4;
    counts[5] = c5;
    return PC_OK;
}
