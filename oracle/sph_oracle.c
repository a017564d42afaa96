/*
 * sph_oracle.c -- plain FP64 CPU oracle for the neighbour-search + density path.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct statement of
 * what the CUDA path computes.  Only tests/, __graft_entry__.smoke() and the
 * CPU-baseline legs of bench.py load it.  The product library never links,
 * loads or calls it, and it shares no code, header, table or constant with the
 * CUDA sources.
 *
 * Build with -O2 -ffp-contract=off: the squared distance must be the plain
 * left-to-right FP64 expression, with no fused multiply-add.
 *
 * What each function follows (section / equation of arXiv 2401.08586):
 *   oracle_kernel_alpha / oracle_kernel_w / oracle_kernel_dwdr
 *       cubic B-spline kernel W(R, h), Eq. 3, with alpha_d = 1/h, 15/(7 pi h^2),
 *       3/(2 pi h^3) for d = 1, 2, 3 (text under Eq. 3); R = r / h; and its
 *       derivative dW/dR, Eq. 3 differentiated term by term.
 *   oracle_allpairs
 *       all-list search ("SPH method", all-list paragraph; Fig. 3a): every
 *       particle is compared with every other one, N(N-1) ordered comparisons,
 *       and kept when it lies inside the search radius kh = 2h.
 *   oracle_cll
 *       cell link-list search (same section, link-list paragraph; Fig. 3b):
 *       uniform background cells sized to the search radius, particles assigned
 *       to cells, and only the same and adjacent cells searched.  It finds the
 *       same set as oracle_allpairs (the paper notes the two give identical
 *       neighbour decisions, Table 2).
 *   oracle_cll_rows / oracle_density_rows
 *       the same two computations for a listed subset of rows (sampled
 *       checks of workloads too large for a full oracle pass).
 *   oracle_density
 *       summation density rho_i = sum_j m_j W(r_ij / h, h) over the neighbour
 *       list plus the self term j = i (the textbook SPH density; W from Eq. 3).
 *   oracle_gradient_a5
 *       volume-free normalised first-order gradient operator, Appendix Eq. A5:
 *       <f_i^a> = sum_j (f_j - f_i) dW_ij/dx^a / sum_j (x_j^a - x_i^a) dW_ij/dx^a
 *       for each axis a, with dW/dx^a = W'(R) / h * (x_i^a - x_j^a) / r.
 *
 * Readings where the paper is silent (the same readings the CUDA path uses):
 *   - neighbour test is strict: r_ij^2 < kh^2; self is excluded from the list;
 *   - r_ij^2 = (dx0*dx0 + dx1*dx1) + dx2*dx2 with dxk = x_i[k] - x_j[k], FP64;
 *     kh^2 = kh*kh in FP64;
 *   - CSR output: rows in input order, columns ascending;
 *   - cell size h_c = kh * (1 + 2^-30); n_k = max(1, ceil((hi_k - lo_k)/h_c));
 *     cell index = clamp(floor((x_k - lo_k)/h_c), 0, n_k - 1) over the particle
 *     bounding box [lo, hi].  The 2^-30 margin keeps every pair with r < kh at
 *     most one cell apart per axis after FP64 rounding, for up to 2^20 cells
 *     per axis.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_PI 3.14159265358979323846

/* alpha_d of Eq. 3. */
double oracle_kernel_alpha(int dim, double h)
{
    if (dim == 1) return 1.0 / h;
    if (dim == 2) return 15.0 / (7.0 * ORACLE_PI * h * h);
    return 3.0 / (2.0 * ORACLE_PI * h * h * h);
}

/* W(R, h) of Eq. 3. */
double oracle_kernel_w(int dim, double R, double h)
{
    double a = oracle_kernel_alpha(dim, h);
    if (R < 0.0) R = -R;
    if (R < 1.0) return a * (2.0 / 3.0 - R * R + 0.5 * R * R * R);
    if (R < 2.0) {
        double t = 2.0 - R;
        return a * (t * t * t / 6.0);
    }
    return 0.0;
}

/* dW/dR of Eq. 3 (used by the gradient operator of Appendix Eq. A5):
 * alpha_d (-2R + 3R^2/2) on [0, 1), -alpha_d (2 - R)^2 / 2 on [1, 2), 0 beyond. */
double oracle_kernel_dwdr(int dim, double R, double h)
{
    double a = oracle_kernel_alpha(dim, h);
    if (R < 1.0) return a * (-2.0 * R + 1.5 * R * R);
    if (R < 2.0) {
        double t = 2.0 - R;
        return a * (-0.5 * t * t);
    }
    return 0.0;
}

void oracle_kernel_w_array(int dim, int64_t n, const double *R, double h, double *out)
{
    for (int64_t k = 0; k < n; ++k) out[k] = oracle_kernel_w(dim, R[k], h);
}

/* Squared distance, the one expression every oracle function uses. */
static double pair_r2(int dim, const double *xi, const double *xj)
{
    double d0 = xi[0] - xj[0];
    double d1 = xi[1] - xj[1];
    double r2 = d0 * d0 + d1 * d1;
    if (dim == 3) {
        double d2 = xi[2] - xj[2];
        r2 = r2 + d2 * d2;
    }
    return r2;
}

/*
 * All-list search.  Returns nnz.  row_ptr[n+1] is always written; col is
 * written only when col != NULL and cap >= nnz.
 */
int64_t oracle_allpairs(int dim, int64_t n, const double *xyz, double kh,
                        int64_t *row_ptr, int32_t *col, int64_t cap)
{
    double kh2 = kh * kh;
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c = 0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (pair_r2(dim, xyz + i * dim, xyz + j * dim) < kh2) ++c;
        }
        row_ptr[i + 1] = row_ptr[i] + c;
    }
    int64_t nnz = row_ptr[n];
    if (col == NULL || cap < nnz) return nnz;
    for (int64_t i = 0; i < n; ++i) {
        int64_t w = row_ptr[i];
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            if (pair_r2(dim, xyz + i * dim, xyz + j * dim) < kh2) col[w++] = (int32_t)j;
        }
    }
    return nnz;
}

/* Background-cell grid of the link-list search. */
typedef struct {
    int dim;
    double lo[3], hc;
    int64_t nk[3];
    int64_t ncell;
    int64_t *cell_start; /* ncell + 1 */
    int32_t *members;    /* particle ids, cell by cell, ascending within a cell */
} oracle_grid;

static int64_t cell_coord(double x, double lo, double hc, int64_t nk)
{
    double t = floor((x - lo) / hc);
    if (t < 0.0) t = 0.0;
    if (t > (double)(nk - 1)) t = (double)(nk - 1);
    return (int64_t)t;
}

/* Returns 0 on success, -1 when the grid would be too large. */
static int grid_build(int dim, int64_t n, const double *xyz, double kh, oracle_grid *g)
{
    memset(g, 0, sizeof(*g));
    g->dim = dim;
    g->hc = kh * (1.0 + 0x1p-30);
    double hi[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k) { g->lo[k] = 0.0; g->nk[k] = 1; }
    for (int k = 0; k < dim; ++k) {
        double lo = INFINITY, h = -INFINITY;
        for (int64_t i = 0; i < n; ++i) {
            double x = xyz[i * dim + k];
            if (x < lo) lo = x;
            if (x > h) h = x;
        }
        if (n == 0) { lo = 0.0; h = 0.0; }
        g->lo[k] = lo;
        hi[k] = h;
        double span = ceil((h - lo) / g->hc);
        if (span > (double)(1 << 20)) return -1;
        g->nk[k] = span < 1.0 ? 1 : (int64_t)span;
    }
    g->ncell = g->nk[0] * g->nk[1] * g->nk[2];
    if (g->ncell > ((int64_t)1 << 28)) return -1;
    g->cell_start = (int64_t *)calloc((size_t)g->ncell + 1, sizeof(int64_t));
    g->members = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
    int64_t *cid = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    int64_t *fill = (int64_t *)malloc((size_t)g->ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3] = {0, 0, 0};
        for (int k = 0; k < dim; ++k) c[k] = cell_coord(xyz[i * dim + k], g->lo[k], g->hc, g->nk[k]);
        cid[i] = (c[2] * g->nk[1] + c[1]) * g->nk[0] + c[0];
        g->cell_start[cid[i] + 1] += 1;
    }
    for (int64_t c = 0; c < g->ncell; ++c) g->cell_start[c + 1] += g->cell_start[c];
    memcpy(fill, g->cell_start, (size_t)g->ncell * sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) g->members[fill[cid[i]]++] = (int32_t)i;
    free(cid);
    free(fill);
    (void)hi;
    return 0;
}

static void grid_free(oracle_grid *g)
{
    free(g->cell_start);
    free(g->members);
}

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Neighbours of particle i from the 3^d cells around its own cell, sorted
 * ascending into buf.  Returns how many were found.
 */
static int64_t cll_row(const oracle_grid *g, int64_t n, const double *xyz, double kh2,
                       int64_t i, int32_t *buf)
{
    int dim = g->dim;
    const double *xi = xyz + i * dim;
    int64_t c[3] = {0, 0, 0};
    for (int k = 0; k < dim; ++k) c[k] = cell_coord(xi[k], g->lo[k], g->hc, g->nk[k]);
    int64_t zlo = dim == 3 ? -1 : 0, zhi = dim == 3 ? 1 : 0;
    int64_t found = 0;
    for (int64_t dz = zlo; dz <= zhi; ++dz)
        for (int64_t dy = -1; dy <= 1; ++dy)
            for (int64_t dx = -1; dx <= 1; ++dx) {
                int64_t a = c[0] + dx, b = c[1] + dy, e = c[2] + dz;
                if (a < 0 || a >= g->nk[0] || b < 0 || b >= g->nk[1] || e < 0 || e >= g->nk[2])
                    continue;
                int64_t cell = (e * g->nk[1] + b) * g->nk[0] + a;
                for (int64_t s = g->cell_start[cell]; s < g->cell_start[cell + 1]; ++s) {
                    int64_t j = g->members[s];
                    if (j == i) continue;
                    if (pair_r2(dim, xi, xyz + j * dim) < kh2) buf[found++] = (int32_t)j;
                }
            }
    qsort(buf, (size_t)found, sizeof(int32_t), cmp_i32);
    (void)n;
    return found;
}

/* Largest candidate count over all particles (sizes the per-row buffer). */
static int64_t max_candidates(const oracle_grid *g)
{
    int dim = g->dim;
    int64_t best = 0;
    int64_t zn = dim == 3 ? g->nk[2] : 1;
    for (int64_t e = 0; e < zn; ++e)
        for (int64_t b = 0; b < g->nk[1]; ++b)
            for (int64_t a = 0; a < g->nk[0]; ++a) {
                int64_t tot = 0;
                for (int64_t dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
                    for (int64_t dy = -1; dy <= 1; ++dy)
                        for (int64_t dx = -1; dx <= 1; ++dx) {
                            int64_t x = a + dx, y = b + dy, z = e + dz;
                            if (x < 0 || x >= g->nk[0] || y < 0 || y >= g->nk[1] || z < 0 || z >= zn)
                                continue;
                            int64_t cell = (z * g->nk[1] + y) * g->nk[0] + x;
                            tot += g->cell_start[cell + 1] - g->cell_start[cell];
                        }
                if (tot > best) best = tot;
            }
    return best;
}

/*
 * Cell link-list search.  Same contract as oracle_allpairs.  nthreads > 1
 * splits the independent rows over OpenMP threads (used only to time the
 * oracle on all host cores); the result does not depend on it.
 * Returns -1 when the grid would exceed 2^20 cells per axis or 2^28 cells.
 */
int64_t oracle_cll(int dim, int64_t n, const double *xyz, double kh, int nthreads,
                   int64_t *row_ptr, int32_t *col, int64_t cap)
{
    oracle_grid g;
    if (grid_build(dim, n, xyz, kh, &g) != 0) return -1;
    double kh2 = kh * kh;
    int64_t maxc = max_candidates(&g) + 1;
    if (nthreads < 1) nthreads = 1;
    int64_t *cnt = (int64_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int32_t *buf = (int32_t *)malloc((size_t)maxc * sizeof(int32_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 512)
#endif
        for (int64_t i = 0; i < n; ++i) cnt[i] = cll_row(&g, n, xyz, kh2, i, buf);
        free(buf);
    }
    row_ptr[0] = 0;
    for (int64_t i = 0; i < n; ++i) row_ptr[i + 1] = row_ptr[i] + cnt[i];
    int64_t nnz = row_ptr[n];
    if (col != NULL && cap >= nnz) {
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
        {
            int32_t *buf = (int32_t *)malloc((size_t)maxc * sizeof(int32_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 512)
#endif
            for (int64_t i = 0; i < n; ++i) {
                int64_t f = cll_row(&g, n, xyz, kh2, i, buf);
                memcpy(col + row_ptr[i], buf, (size_t)f * sizeof(int32_t));
            }
            free(buf);
        }
    }
    free(cnt);
    grid_free(&g);
    return nnz;
}

/*
 * The cell link-list search restricted to the listed rows (input indices
 * rows[0..nrows)): row r of the output is particle rows[r]'s neighbour list,
 * ascending.  Same grid and decisions as oracle_cll, for checking sampled rows
 * of a workload too large to search in full.  Returns the total count, or -1
 * as oracle_cll; col is written only when cap is large enough.
 */
int64_t oracle_cll_rows(int dim, int64_t n, const double *xyz, double kh, int nthreads,
                        const int64_t *rows, int64_t nrows, int64_t *row_ptr, int32_t *col, int64_t cap)
{
    oracle_grid g;
    if (grid_build(dim, n, xyz, kh, &g) != 0) return -1;
    double kh2 = kh * kh;
    int64_t maxc = max_candidates(&g) + 1;
    if (nthreads < 1) nthreads = 1;
    int64_t *cnt = (int64_t *)malloc((size_t)(nrows > 0 ? nrows : 1) * sizeof(int64_t));
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int32_t *buf = (int32_t *)malloc((size_t)maxc * sizeof(int32_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t r = 0; r < nrows; ++r) cnt[r] = cll_row(&g, n, xyz, kh2, rows[r], buf);
        free(buf);
    }
    row_ptr[0] = 0;
    for (int64_t r = 0; r < nrows; ++r) row_ptr[r + 1] = row_ptr[r] + cnt[r];
    int64_t nnz = row_ptr[nrows];
    if (col != NULL && cap >= nnz) {
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
        {
            int32_t *buf = (int32_t *)malloc((size_t)maxc * sizeof(int32_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
            for (int64_t r = 0; r < nrows; ++r) {
                int64_t f = cll_row(&g, n, xyz, kh2, rows[r], buf);
                memcpy(col + row_ptr[r], buf, (size_t)f * sizeof(int32_t));
            }
            free(buf);
        }
    }
    free(cnt);
    grid_free(&g);
    return nnz;
}

/*
 * Summation density of the listed rows only: rho[r] for particle rows[r],
 * whose neighbours are col[row_ptr[r] .. row_ptr[r + 1]) (input indices).
 * Same sum, order and arithmetic as oracle_density.
 */
void oracle_density_rows(int dim, const double *xyz, double h, double mass, const int64_t *rows, int64_t nrows,
                         const int64_t *row_ptr, const int32_t *col, double *rho)
{
    for (int64_t r = 0; r < nrows; ++r) {
        int64_t i = rows[r];
        double s = mass * oracle_kernel_w(dim, 0.0, h);
        for (int64_t k = row_ptr[r]; k < row_ptr[r + 1]; ++k) {
            int64_t j = col[k];
            double d = sqrt(pair_r2(dim, xyz + i * dim, xyz + j * dim));
            s += mass * oracle_kernel_w(dim, d / h, h);
        }
        rho[r] = s;
    }
}

/*
 * Summation density in FP64: rho_i = m W(0, h) + sum_{j in N(i)} m W(r_ij / h, h),
 * accumulated in CSR order.  nthreads as in oracle_cll.
 */
void oracle_density(int dim, int64_t n, const double *xyz, double h, double mass,
                    const int64_t *row_ptr, const int32_t *col, int nthreads, double *rho)
{
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 512)
#endif
    for (int64_t i = 0; i < n; ++i) {
        double s = mass * oracle_kernel_w(dim, 0.0, h);
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            double r = sqrt(pair_r2(dim, xyz + i * dim, xyz + j * dim));
            s += mass * oracle_kernel_w(dim, r / h, h);
        }
        rho[i] = s;
    }
}

/*
 * Appendix Eq. A5, one axis at a time.  grad is n x dim.  An axis whose
 * denominator is zero (no neighbour offset along it) yields 0.
 */
void oracle_gradient_a5(int dim, int64_t n, const double *xyz, double h, const double *f,
                        const int64_t *row_ptr, const int32_t *col, double *grad)
{
    for (int64_t i = 0; i < n; ++i) {
        const double *xi = xyz + i * dim;
        double num[3] = {0, 0, 0}, den[3] = {0, 0, 0};
        for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
            int64_t j = col[k];
            const double *xj = xyz + j * dim;
            double r = sqrt(pair_r2(dim, xi, xj));
            if (r == 0.0) continue;
            double dwdr = oracle_kernel_dwdr(dim, r / h, h) / h;
            for (int a = 0; a < dim; ++a) {
                double dwdx = dwdr * (xi[a] - xj[a]) / r;
                num[a] += (f[j] - f[i]) * dwdx;
                den[a] += (xj[a] - xi[a]) * dwdx;
            }
        }
        for (int a = 0; a < dim; ++a) grad[i * dim + a] = den[a] != 0.0 ? num[a] / den[a] : 0.0;
    }
}

int oracle_openmp_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
