/*
 * ecc_oracle.c -- plain, slow, single-threaded CPU oracle for the Euler
 * characteristic curve (ECC) of a d-dimensional integer grayscale image.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library's product path may link,
 * load or call this file: only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py use it.  It shares no code,
 * header, table or constant with the CUDA path.
 *
 * What it computes (Wang, Wagner, Chen, "GPU Computation of the Euler
 * Characteristic Curve for Imaging Data", SoCG 2022):
 *
 *   ECC_t = chi(K_{<=t}) = sum_j (-1)^j c_j(K_{<=t})           (Sec. 2.2, Eq. 1)
 *   VCEC_0 = ECC_0,  VCEC_t = ECC_t - ECC_{t-1},  ECC = prefix sum of VCEC
 *                                                               (Sec. 2.3)
 *
 * so VCEC_t is the signed count sum (-1)^dim(sigma) over all cells sigma whose
 * filtration value equals t.  The oracle enumerates every cell explicitly,
 * gives it its filtration value, and adds (-1)^dim to that gray level's bin.
 * No tie-break is needed: a cell's value does not depend on which voxel
 * "introduces" it (Sec. 2.3), so this is the plain definition, not the
 * per-voxel regrouping of Algorithm 1.
 *
 * Two complexes are supported.
 *
 *  vertex construction ("V-mode"): every voxel is a vertex of the cubical
 *    grid; a cell is a base point p plus a set A of axes, with vertex set
 *    p + {0,1}^A lying entirely inside the grid; dim = |A|; its value is the
 *    MAX of its vertex values; sublevel sets.  This is the complex "with
 *    pixels as vertices" whose cells enter at the max of their vertices.
 *
 *  top-cell construction ("T-mode", Sec. 2.1): voxels are the top-
 *    dimensional cells; a cell is a product of elementary intervals [k,k] or
 *    [k,k+1] (k integer) over the lattice 0..n_a on each axis; dim = number
 *    of non-degenerate intervals; its value is the MIN over the voxels that
 *    contain it (its top-dimensional cofaces); sublevel sets.
 *
 * Gray levels: bin g holds level lo+g, g = 0..hi-lo.  ECC[g] = chi(K_{<=lo+g})
 * for every level g, so the paper's sequence indexed by the values present in
 * the image (Eq. 1, t_i) is the subsequence of ECC at present levels.
 *
 * Layout: dense row-major, dims[0] slowest (the chunking of Sec. 3.4 cuts
 * along dims[0]).  Element types: 1 = uint8, 2 = uint16.
 *
 * Chunking (Sec. 3.4): the *_rows entry points only count cells whose
 * coordinate along dims[0] lies in a half-open range, reading the one extra
 * layer of the image they need (the one-voxel collar).  Summing the VCEC of
 * disjoint ranges that cover the axis gives the VCEC of the whole image; the
 * tests use this to run the oracle on slabs in parallel at full size.
 *
 * Return codes: 0 ok, 1 invalid arguments, 2 a value outside [lo, hi].
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

#define ORACLE_MAX_DIM 4

static int64_t voxel_value(const void *img, int dtype, int64_t lin)
{
    if (dtype == 1) return (int64_t)((const uint8_t *)img)[lin];
    return (int64_t)((const uint16_t *)img)[lin];
}

static int check_args(const void *img, int dtype, int ndim, const int64_t *dims,
                      int32_t lo, int32_t hi, const int64_t *vcec)
{
    if (!img || !dims || !vcec) return 1;
    if (dtype != 1 && dtype != 2) return 1;
    if (ndim < 1 || ndim > ORACLE_MAX_DIM) return 1;
    if (hi < lo) return 1;
    for (int a = 0; a < ndim; ++a)
        if (dims[a] < 1) return 1;
    return 0;
}

/* Row-major linear index of a coordinate vector. */
static int64_t linear_index(int ndim, const int64_t *dims, const int64_t *x)
{
    int64_t lin = 0;
    for (int a = 0; a < ndim; ++a) lin = lin * dims[a] + x[a];
    return lin;
}

/* Advance the mixed-radix counter x over [lo_a, hi_a) per axis, last axis
 * fastest.  Returns 0 once every coordinate has been visited. */
static int next_coord(int ndim, const int64_t *lo_a, const int64_t *hi_a, int64_t *x)
{
    for (int a = ndim - 1; a >= 0; --a) {
        if (++x[a] < hi_a[a]) return 1;
        x[a] = lo_a[a];
    }
    return 0;
}

/*
 * V-mode VCEC over the cells whose base point has dims[0]-coordinate in
 * [row_begin, row_end).  Accumulates into vcec[0 .. hi-lo].
 */
int oracle_vcec_vertex_rows(const void *img, int dtype, int ndim, const int64_t *dims,
                            int64_t row_begin, int64_t row_end,
                            int32_t lo, int32_t hi, int64_t *vcec)
{
    if (check_args(img, dtype, ndim, dims, lo, hi, vcec)) return 1;
    if (row_begin < 0 || row_end > dims[0] || row_begin > row_end) return 1;
    if (row_begin == row_end) return 0;

    int64_t lo_a[ORACLE_MAX_DIM], hi_a[ORACLE_MAX_DIM], p[ORACLE_MAX_DIM];
    for (int a = 0; a < ndim; ++a) { lo_a[a] = 0; hi_a[a] = dims[a]; p[a] = 0; }
    lo_a[0] = row_begin; hi_a[0] = row_end; p[0] = row_begin;

    const unsigned n_subsets = 1u << ndim;
    do {
        for (unsigned A = 0; A < n_subsets; ++A) {
            /* The cell p + {0,1}^A exists only if every vertex is in the grid. */
            int exists = 1, dim = 0;
            for (int a = 0; a < ndim; ++a) {
                if (A & (1u << a)) {
                    ++dim;
                    if (p[a] + 1 >= dims[a]) exists = 0;
                }
            }
            if (!exists) continue;

            /* Filtration value: the max over the 2^|A| vertices p + e_B, B subset of A. */
            int64_t value = -1;
            for (unsigned B = 0; B < n_subsets; ++B) {
                if (B & ~A) continue;
                int64_t q[ORACLE_MAX_DIM];
                for (int a = 0; a < ndim; ++a) q[a] = p[a] + ((B >> a) & 1u);
                int64_t v = voxel_value(img, dtype, linear_index(ndim, dims, q));
                if (v > value) value = v;
            }
            if (value < lo || value > hi) return 2;
            vcec[value - lo] += (dim % 2 == 0) ? 1 : -1;
        }
    } while (next_coord(ndim, lo_a, hi_a, p));
    return 0;
}

/*
 * T-mode VCEC over the cells whose elementary interval along dims[0] has
 * index e in [e_begin, e_end), where e = 2k is the degenerate interval [k,k]
 * and e = 2k+1 is [k,k+1]; e runs over 0 .. 2*dims[0].  Accumulates into vcec.
 */
int oracle_vcec_topcell_rows(const void *img, int dtype, int ndim, const int64_t *dims,
                             int64_t e_begin, int64_t e_end,
                             int32_t lo, int32_t hi, int64_t *vcec)
{
    if (check_args(img, dtype, ndim, dims, lo, hi, vcec)) return 1;
    if (e_begin < 0 || e_end > 2 * dims[0] + 1 || e_begin > e_end) return 1;
    if (e_begin == e_end) return 0;

    int64_t lo_a[ORACLE_MAX_DIM], hi_a[ORACLE_MAX_DIM], e[ORACLE_MAX_DIM];
    for (int a = 0; a < ndim; ++a) { lo_a[a] = 0; hi_a[a] = 2 * dims[a] + 1; e[a] = 0; }
    lo_a[0] = e_begin; hi_a[0] = e_end; e[0] = e_begin;

    do {
        /* Per axis, the voxel coordinates of the top-dimensional cofaces:
         * [k,k+1] lies only in voxel k; [k,k] lies in voxels k-1 and k,
         * whichever of them exist. */
        int64_t first[ORACLE_MAX_DIM], last[ORACLE_MAX_DIM];
        int dim = 0;
        for (int a = 0; a < ndim; ++a) {
            int64_t k = e[a] / 2;
            if (e[a] % 2 == 1) {
                ++dim;
                first[a] = k; last[a] = k;
            } else {
                first[a] = (k - 1 < 0) ? 0 : k - 1;
                last[a] = (k > dims[a] - 1) ? dims[a] - 1 : k;
            }
        }
        /* Filtration value: the min over all cofaces (a box of voxels). */
        int64_t value = INT64_MAX, v_hi[ORACLE_MAX_DIM], q[ORACLE_MAX_DIM];
        for (int a = 0; a < ndim; ++a) { q[a] = first[a]; v_hi[a] = last[a] + 1; }
        do {
            int64_t v = voxel_value(img, dtype, linear_index(ndim, dims, q));
            if (v < value) value = v;
        } while (next_coord(ndim, first, v_hi, q));

        if (value < lo || value > hi) return 2;
        vcec[value - lo] += (dim % 2 == 0) ? 1 : -1;
    } while (next_coord(ndim, lo_a, hi_a, e));
    return 0;
}

int oracle_vcec_vertex(const void *img, int dtype, int ndim, const int64_t *dims,
                       int32_t lo, int32_t hi, int64_t *vcec)
{
    if (check_args(img, dtype, ndim, dims, lo, hi, vcec)) return 1;
    memset(vcec, 0, sizeof(int64_t) * (size_t)(hi - lo + 1));
    return oracle_vcec_vertex_rows(img, dtype, ndim, dims, 0, dims[0], lo, hi, vcec);
}

int oracle_vcec_topcell(const void *img, int dtype, int ndim, const int64_t *dims,
                        int32_t lo, int32_t hi, int64_t *vcec)
{
    if (check_args(img, dtype, ndim, dims, lo, hi, vcec)) return 1;
    memset(vcec, 0, sizeof(int64_t) * (size_t)(hi - lo + 1));
    return oracle_vcec_topcell_rows(img, dtype, ndim, dims, 0, 2 * dims[0] + 1, lo, hi, vcec);
}

/* ECC_i = sum_{j <= i} VCEC_j (Sec. 2.3, "basic dynamic programming"). */
void oracle_ecc_from_vcec(const int64_t *vcec, int64_t nbins, int64_t *ecc)
{
    int64_t run = 0;
    for (int64_t g = 0; g < nbins; ++g) {
        run += vcec[g];
        ecc[g] = run;
    }
}

/*
 * Thresholds on float32 images (Eq. 1 with the levels t_i given).
 *
 * ECC_i = chi(K_{<= t_i}) = sum over cells sigma with value(sigma) <= t_i of
 * (-1)^dim(sigma), for ascending levels t_0 <= ... <= t_{m-1}.  Each cell is
 * enumerated exactly as above, its value computed in floating point (max of
 * its vertices, or min of its top cofaces), and (-1)^dim added to bin i =
 * the first index whose level is >= the value; a cell above t_{m-1} lies in
 * no sublevel set and is skipped.  The prefix sum of the m bins is then the
 * ECC at the m thresholds.  A NaN voxel is in no sublevel set (v <= t is
 * false for it at every t): it lies above every level, +infinity included,
 * so a cell with a NaN vertex (vertex complex) or with only NaN cofaces
 * (top-cell complex) is counted at no level.
 */
static double float_value(const float *img, int64_t lin)
{
    return (double)img[lin];
}

/* First index i in [0, m] with levels[i] >= v (m if none). */
static int64_t first_level_at_or_above(const double *levels, int64_t m, double v)
{
    int64_t lo = 0, hi = m;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (levels[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

int oracle_levels_vertex_rows(const float *img, int ndim, const int64_t *dims, int64_t row_begin, int64_t row_end,
                              const double *levels, int64_t m, int64_t *bins)
{
    if (!img || !dims || !levels || !bins || m < 1 || ndim < 1 || ndim > ORACLE_MAX_DIM) return 1;
    for (int a = 0; a < ndim; ++a)
        if (dims[a] < 1) return 1;
    for (int64_t i = 1; i < m; ++i)
        if (!(levels[i - 1] <= levels[i])) return 1;
    if (row_begin < 0 || row_end > dims[0] || row_begin > row_end) return 1;
    if (row_begin == row_end) return 0;

    int64_t lo_a[ORACLE_MAX_DIM], hi_a[ORACLE_MAX_DIM], p[ORACLE_MAX_DIM];
    for (int a = 0; a < ndim; ++a) { lo_a[a] = 0; hi_a[a] = dims[a]; p[a] = 0; }
    lo_a[0] = row_begin; hi_a[0] = row_end; p[0] = row_begin;

    const unsigned n_subsets = 1u << ndim;
    do {
        for (unsigned A = 0; A < n_subsets; ++A) {
            int exists = 1, dim = 0;
            for (int a = 0; a < ndim; ++a) {
                if (A & (1u << a)) {
                    ++dim;
                    if (p[a] + 1 >= dims[a]) exists = 0;
                }
            }
            if (!exists) continue;
            double value = -(double)INFINITY;
            int nan_vertex = 0;
            for (unsigned B = 0; B < n_subsets; ++B) {
                if (B & ~A) continue;
                int64_t q[ORACLE_MAX_DIM];
                for (int a = 0; a < ndim; ++a) q[a] = p[a] + ((B >> a) & 1u);
                const double v = float_value(img, linear_index(ndim, dims, q));
                if (v != v) nan_vertex = 1;
                else if (v > value) value = v;
            }
            if (nan_vertex) continue;
            const int64_t i = first_level_at_or_above(levels, m, value);
            if (i < m) bins[i] += (dim % 2 == 0) ? 1 : -1;
        }
    } while (next_coord(ndim, lo_a, hi_a, p));
    return 0;
}

int oracle_levels_topcell_rows(const float *img, int ndim, const int64_t *dims, int64_t e_begin, int64_t e_end,
                               const double *levels, int64_t m, int64_t *bins)
{
    if (!img || !dims || !levels || !bins || m < 1 || ndim < 1 || ndim > ORACLE_MAX_DIM) return 1;
    for (int a = 0; a < ndim; ++a)
        if (dims[a] < 1) return 1;
    for (int64_t i = 1; i < m; ++i)
        if (!(levels[i - 1] <= levels[i])) return 1;
    if (e_begin < 0 || e_end > 2 * dims[0] + 1 || e_begin > e_end) return 1;
    if (e_begin == e_end) return 0;

    int64_t lo_a[ORACLE_MAX_DIM], hi_a[ORACLE_MAX_DIM], e[ORACLE_MAX_DIM];
    for (int a = 0; a < ndim; ++a) { lo_a[a] = 0; hi_a[a] = 2 * dims[a] + 1; e[a] = 0; }
    lo_a[0] = e_begin; hi_a[0] = e_end; e[0] = e_begin;

    do {
        int64_t first[ORACLE_MAX_DIM], last[ORACLE_MAX_DIM];
        int dim = 0;
        for (int a = 0; a < ndim; ++a) {
            int64_t k = e[a] / 2;
            if (e[a] % 2 == 1) {
                ++dim;
                first[a] = k; last[a] = k;
            } else {
                first[a] = (k - 1 < 0) ? 0 : k - 1;
                last[a] = (k > dims[a] - 1) ? dims[a] - 1 : k;
            }
        }
        double value = (double)INFINITY;
        int any_coface = 0;  /* a coface that is not NaN */
        int64_t v_hi[ORACLE_MAX_DIM], q[ORACLE_MAX_DIM];
        for (int a = 0; a < ndim; ++a) { q[a] = first[a]; v_hi[a] = last[a] + 1; }
        do {
            const double v = float_value(img, linear_index(ndim, dims, q));
            if (v == v) {
                any_coface = 1;
                if (v < value) value = v;
            }
        } while (next_coord(ndim, first, v_hi, q));
        if (!any_coface) continue;
        const int64_t i = first_level_at_or_above(levels, m, value);
        if (i < m) bins[i] += (dim % 2 == 0) ? 1 : -1;
    } while (next_coord(ndim, lo_a, hi_a, e));
    return 0;
}
