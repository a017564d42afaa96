/*
 * sph.h -- C ABI of libsph: FP16 relative-coordinate cell link-list (RCLL)
 * neighbour search and SPH summation density on one NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2401.08586 ("A GPU accelerated mixed-precision Smoothed
 * Particle Hydrodynamics framework with cell-based relative coordinates").
 * Given N particle positions and a search radius kh (= 2h in the paper), the
 * library finds, for every particle i, all particles j != i with
 * |x_i - x_j|^2 < kh^2 (the neighbour definition of the all-list and cell
 * link-list searches, Section "SPH method", Fig. 3) and can sum the SPH
 * density rho_i = m W(0, h) + sum_j m W(r_ij / h, h) with the cubic B-spline
 * W of Eq. 3.
 *
 * Precision contract (FP16-RCLL mode): the bulk of the distance tests run in
 * FP16 on cell-relative coordinates (Eq. 6-7); every pair the FP16 test cannot
 * reject is re-decided in FP32, and the few pairs inside the FP32 error band
 * are decided by the FP64 expression (dx0*dx0 + dx1*dx1) + dx2*dx2 < kh*kh on
 * the caller's coordinates.  The neighbour lists are therefore identical to
 * an FP64 evaluation of that expression.  Density is accumulated in FP32 in
 * CSR order.
 *
 * Conventions for every entry point:
 *  - Return value: SPH_OK (0), SPH_PENDING (1, serving only) or a negative
 *    SPH_ERR_* code.  No C++ exception crosses the ABI.  sph_last_error()
 *    gives a human-readable message for the calling thread's last failure.
 *  - "device" pointers are CUDA device memory owned by the caller; "host"
 *    pointers are ordinary host memory owned by the caller.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy
 *    default stream.  All device work of a call is enqueued on it; calls
 *    return without waiting unless the description says they synchronise.
 *  - Layouts: coordinates are N x dim row-major FP64 (x0 y0 [z0] x1 y1 ...).
 *    CSR: row_ptr int64[N+1], col int32[nnz].
 */
#ifndef SPH_H
#define SPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SPH_OK 0
#define SPH_PENDING 1
#define SPH_ERR_INVALID (-1)      /* bad argument or input (non-finite coordinate, kh <= 0, ...) */
#define SPH_ERR_CAPACITY (-2)     /* col_capacity < nnz; nothing was written past the end */
#define SPH_ERR_BUDGET (-3)       /* request exceeds the serving HBM budget */
#define SPH_ERR_CUDA (-4)         /* a CUDA runtime call failed */
#define SPH_ERR_TIMEOUT (-5)      /* a bounded device or host wait ran out */
#define SPH_ERR_DEVICE_CHECK (-6) /* a device-side consistency check fired */
#define SPH_ERR_NOMEM (-7)        /* device or host allocation failed */
#define SPH_ERR_NOT_FOUND (-8)    /* unknown handle or ticket */

/* ---- output row order -------------------------------------------------- */
/* SPH_ORDER_CELL: rows are the particles in the grid's cell-sorted order
 *   (row r is input particle orig_id[r], see sph_grid_info) and columns are
 *   cell-sorted positions, ascending within each row.  This is the order the
 *   search produces natively.
 * SPH_ORDER_CANONICAL: rows in input order, columns are input indices,
 *   ascending within each row (costs an extra permute + per-row sort). */
#define SPH_ORDER_CELL 0
#define SPH_ORDER_CANONICAL 1

/* ---- arithmetic of the search ---------------------------------------- */
/* SPH_PREC_FP16_RCLL: FP16 cell-relative coordinates (Eq. 6), FP16 distance
 *   test (Eq. 7 with the scale reading h_c/2), FP32 re-decision, FP64 tie tier.
 * SPH_PREC_FP64_CLL: plain FP64 cell link-list (the paper's high-precision
 *   approach I, Table 4): FP64 coordinates in cell order, FP64 test, FP64
 *   density (written out as FP32).  Used as the same-GPU baseline. */
#define SPH_PREC_FP16_RCLL 0
#define SPH_PREC_FP64_CLL 1

/* Parameters of one particle system (Eq. 3 and the cell link-list, Fig. 3b). */
typedef struct sph_params {
    int32_t dim;        /* 2 or 3 */
    int32_t order;      /* SPH_ORDER_* of sph_nnps_query / sph_density_sum output */
    int32_t precision;  /* SPH_PREC_* */
    int32_t have_box;   /* 1: box_lo/box_hi bound every particle (checked on the
                           device); 0: the bounding box is computed */
    double h;           /* smoothing length of W (Eq. 3), > 0 */
    double kh;          /* search radius, > 0 (the paper uses kh = 2h) */
    double cell_size;   /* background cell size h_c; 0 selects kh * (1 + 2^-30);
                           otherwise must be >= kh * (1 + 2^-30) */
    double box_lo[3];   /* used when have_box == 1 */
    double box_hi[3];
    double mass;        /* uniform particle mass m of the density sum */
} sph_params;

/* Opaque binned particle system.  It owns its device buffers (allocated
 * stream-ordered on the stream of the call that creates or grows them) and
 * keeps a reference to the caller's coordinate array, which must stay valid
 * and unchanged until the grid is re-binned or freed. */
typedef struct sph_grid_s *sph_grid_t;

typedef struct sph_grid_info {
    int64_t n;               /* particles binned */
    int64_t ncell;           /* background cells */
    int32_t nk[3];           /* cells per axis (nk[2] = 1 in 2D) */
    int32_t dim;
    double lo[3];            /* grid origin (box lower corner) */
    double cell_size;        /* h_c */
    const int32_t *cell_start; /* device int32[ncell+1]: first sorted position of each cell */
    const int32_t *orig_id;  /* device int32[n]: sorted position -> input index */
    const int32_t *rank;     /* device int32[n]: input index -> sorted position */
    int64_t stat_fp32_pairs; /* pairs re-decided in FP32 by the last query (if counted) */
    int64_t stat_fp64_pairs; /* pairs decided by the FP64 tier by the last query (if counted) */
} sph_grid_info;

/*
 * Bin N particles into background cells and build the search structure
 * (cell link-list, Section "SPH method" Fig. 3b; normalised cell-relative
 * coordinates, Eq. 5-6, with the cell centre as reference and unit h_c/2).
 *   p      host: parameters (copied).
 *   xyz    device: FP64 coordinates, n x p->dim row-major.  Must stay valid
 *          and unchanged until *grid is re-binned or freed (the FP64 tier of
 *          the search reads it).  Must be finite.
 *   n      number of particles, 0 <= n < 2^31 - 1.
 *   grid   host: in/out.  If *grid is NULL a new grid is created; otherwise
 *          the existing grid is re-binned in place (its buffers are reused and
 *          grown when needed).
 * Synchronises `stream` once when the bounding box must be computed (to size
 * the cell array).  Errors: SPH_ERR_INVALID (bad parameters, non-finite
 * coordinate, more than 2^20 cells per axis or 2^28 cells), SPH_ERR_NOMEM,
 * SPH_ERR_CUDA.  A particle outside a caller-supplied box is reported by the
 * next synchronising call as SPH_ERR_INVALID.
 */
int sph_bin_cells(const sph_params *p, const double *xyz, int64_t n, void *stream,
                  sph_grid_t *grid);

/*
 * Neighbour search over a binned grid: emits the CSR neighbour list
 * (all-list definition, Section "SPH method"; searched over the 3^d cells
 * around each particle as in the cell link-list, Fig. 3b; pair distance from
 * cell-relative coordinates as in Eq. 7).  Self is excluded; the test is
 * strict (r^2 < kh^2).
 *   row_ptr      device int64[n+1]: written.  row_ptr[n] = nnz.
 *   col          device int32[col_capacity] or NULL.  NULL: only row_ptr (and
 *                *nnz_out) are produced.
 *   col_capacity entries available in col.  If nnz > col_capacity no entry at
 *                or past col[col_capacity] is written (the contents of col
 *                are then unspecified; row_ptr is complete), and the call (or
 *                the next synchronising call when nnz_out is NULL) returns
 *                SPH_ERR_CAPACITY.
 *   nnz_out      host int64 or NULL.  Non-NULL: the call synchronises `stream`
 *                and stores nnz.  NULL: the call does not synchronise.
 *   rho          device float[n] or NULL.  Non-NULL (and col non-NULL): the
 *                density sum is fused into the search and written in the
 *                output row order.
 * Row order follows the grid's sph_params.order.
 */
int sph_nnps_query(sph_grid_t grid, int64_t *row_ptr, int32_t *col, int64_t col_capacity,
                   int64_t *nnz_out, float *rho, void *stream);

/*
 * SPH summation density over an existing CSR neighbour list (in the grid's
 * output order, as produced by sph_nnps_query on this grid):
 * rho_i = m W(0, h) + sum_{j in N(i)} m W(r_ij / h, h), W from Eq. 3,
 * accumulated in FP32 in CSR order.
 *   row_ptr device int64[n+1], col device int32[nnz], rho device float[n].
 */
int sph_density_sum(sph_grid_t grid, const int64_t *row_ptr, const int32_t *col, float *rho,
                    void *stream);

/*
 * SPH summation density without a neighbour list, over a half stencil:
 * rho_i = m W(0, h) + sum_{j in N(i)} m W(r_ij / h, h) (Eq. 3), each pair
 * tested once and its weight added to both particles -- the reuse of
 * computed distances raised in the paper's conclusions.  The pairs are
 * decided exactly as by sph_nnps_query (FP32 with the FP64 definition inside
 * the band); weights in FP32.  The partner's share is added atomically, so
 * the order of the FP32 additions varies between calls (results agree to
 * ~1e-7 relative).  rho: device float[n], indexed by sorted position (row r
 * is input particle orig_id[r]).  FP16-RCLL grids in cell order only
 * (SPH_ERR_INVALID otherwise).  Enqueued on `stream`.
 */
int sph_density_half(sph_grid_t grid, float *rho, void *stream);

/*
 * Volume-free normalised first-order gradient of a particle field f
 * (Appendix Eq. A5): for each axis a,
 *   grad_a f_i = sum_j (f_j - f_i) dW_ij/dx^a / sum_j (x_j^a - x_i^a) dW_ij/dx^a
 * over the neighbour list of sph_nnps_query (same row order and column
 * convention as the grid's order), W from Eq. 3.  f: device FP64[n] in input
 * order; grad: device FP64[n * dim], rows in the CSR's row order.  Distances
 * from the FP32 relative coordinates, f_j - f_i from a float hi/lo split of f,
 * sums in FP32 (relative error ~1e-6 of the result's scale); an axis whose
 * denominator is zero gives 0.  FP16-RCLL grids only.  Enqueued on `stream`.
 */
int sph_gradient_a5(sph_grid_t grid, const int64_t *row_ptr, const int32_t *col, const double *f, double *grad,
                    void *stream);

/*
 * Precision study of the neighbour decision (Tables 1-2, approach II of
 * Table 4): over every candidate pair (i, j != i) of the cell link-list with
 * i's input index in [row_begin, row_end), count the decisions that differ
 * from the FP64 definition when made with FP16 or FP32 absolute coordinates,
 * with FP16 cell-relative coordinates alone (the paper's FP16 RCLL), and with
 * this library's tiered decision (0 by construction).  An instrument, not a
 * search: one thread per particle.  FP16-RCLL grids.  Synchronises `stream`.
 */
typedef struct {
    int64_t candidates;       /* ordered pairs tested */
    int64_t neighbours;       /* pairs with r^2 < kh^2 in FP64 */
    int64_t wrong_fp16_abs;   /* FP16 absolute coordinates: decisions != FP64 */
    int64_t wrong_fp32_abs;   /* FP32 absolute coordinates */
    int64_t wrong_fp16_rcll;  /* FP16 relative coordinates, FP16 decision alone */
    int64_t wrong_tiered;     /* FP16 band, FP32 band, FP64 tier */
} sph_precision_counts;
int sph_precision_study(sph_grid_t grid, int64_t row_begin, int64_t row_end, sph_precision_counts *out,
                        void *stream);

/*
 * The neighbour search of sph_nnps_query (cell order, FP16-RCLL, fused
 * density, single pass over row tiles) for callers that cannot allocate
 * device memory when they call it.  Typical such callers: a process whose
 * device memory is all handed out up front by its own allocator or an HBM
 * budget (a cudaMalloc from inside the library would fail or break that
 * accounting), and latency-critical loops that cannot afford the implicit
 * synchronisation and unbounded time of an allocation.  sph_nnps_query may
 * grow grid-owned buffers with cudaMallocAsync; this call never allocates
 * and calls no allocating routine.  (The paper has no counterpart; this is an
 * interface addition.)
 *
 * Its working memory (tile list, its row offsets, look-back state: about 3.1
 * MiB) is one fixed array inside the library.  Every GPU that loads the
 * library holds that array until the process exits.  The first call in each
 * CUDA context (per device; again after a device reset) looks up the array's
 * device address with cudaGetSymbolAddress (no allocation) and caches it;
 * make that first call before any stream capture.  All calls share the one array and it keeps the
 * last call's contents (the call clears what must start at zero), so calls
 * whose GPU work overlaps -- different streams, or concurrent host threads on
 * one device -- race and give wrong results: serialise them.
 *
 *   grid         binned by sph_bin_cells with precision SPH_PREC_FP16_RCLL and
 *                order SPH_ORDER_CELL (the grid's own buffers are read, not
 *                grown).
 *   row_ptr      device int64[n+1], written; row_ptr[n] = nnz.
 *   col          device int32[col_capacity], written (cell-sorted indices,
 *                ascending per row); nothing at or past col_capacity.
 *   rho          device float[n] or NULL: fused density, cell order.
 * The call does not synchronise; an nnz above col_capacity is reported as
 * SPH_ERR_CAPACITY by the next sph_grid_check.
 * Limits: n <= 1048576 particles and nk[1] * nk[2] <= 65536 rows of cells;
 * larger grids, another precision or order, or a NULL row_ptr/col give
 * SPH_ERR_INVALID without any GPU work.
 */
int sph_nnps_query_static(sph_grid_t grid, int64_t *row_ptr, int32_t *col, int64_t col_capacity, float *rho,
                          void *stream);

/* Per-grid switches (host call, no GPU work).
 *   SPH_OPT_FUSED selects the search (all give identical neighbour lists):
 *       1 (default) single pass, one warp per 32-particle tile of a row of
 *         cells, CSR offsets found by a look-back across tiles; every query
 *         (count only, cell or canonical order) of either precision: FP16
 *         test with FP32/FP64 re-decision on FP16-RCLL grids, the FP64 test
 *         and FP64 density on FP64-CLL grids;
 *       2 single pass, one thread block per cell, look-back across cells
 *         (cell-order FP16-RCLL queries with col != NULL; other queries take
 *         two passes);
 *       0 two passes (count pass, row scan, fill pass), one thread block per
 *         cell. */
#define SPH_OPT_FUSED 1
/*   SPH_OPT_STAGING: bytes of shared memory the tile search (SPH_OPT_FUSED 1)
 *     adds to its output staging area: -1 (default) sizes it from the
 *     neighbours per particle of the grid's last query that reported nnz
 *     (else from the particle density), 0 .. 65536 in multiples of 16 fix it.
 *     A tile whose output does not fit writes its rows directly (same
 *     result); more staging lowers the number of resident warps. */
#define SPH_OPT_STAGING 2
/*   SPH_OPT_TILE_SHAPE: shared-memory shape of the tile search: -1 (default)
 *     chosen from the neighbours per particle, 0 sparse (up to 672 kept
 *     candidates per pass of a tile, 20 resident warps per SM, output staged
 *     for tiles of up to ~80 neighbours per row), 1 dense (832 kept
 *     candidates, 16 warps); other values are refused (SPH_ERR_INVALID).
 *     Same CSR and the same density bits either way: every row's Eq. 3 sum
 *     adds its pairs in column order whatever the shape. */
#define SPH_OPT_TILE_SHAPE 3
/*   SPH_OPT_TEST_LOOKBACK: for tests of the bounded device waits only.  0
 *     (default): normal queries.  k in 1 .. 2^20: the next queries run the
 *     single-pass tile search with its first tile left out, so every later
 *     tile's look-back wait on it runs out after k polls (each at most ~1 us
 *     apart); the query's results are then wrong by design, nothing is
 *     written at or past col_capacity, the query reports SPH_ERR_TIMEOUT (or
 *     sph_grid_check does) and the GPU context stays usable.  Set 0 to go
 *     back to normal queries. */
#define SPH_OPT_TEST_LOOKBACK 4
/*   SPH_OPT_SM_SHARE: percent (1 .. 100, default 100) of the device's resident
 *     thread-block slots the tile search's persistent grid takes.  Below 100
 *     the search leaves room for kernels of other streams to run beside it
 *     (the request server gives large requests a share so that small ones
 *     are not queued behind them); results are unchanged. */
#define SPH_OPT_SM_SHARE 5
int sph_grid_set_option(sph_grid_t grid, int option, int64_t value);

/* The neighbour list over a half stencil: every pair decided once (from the
 * particle whose cell comes first in (z, y, x) order, or in one cell from
 * the lower sorted index, exactly as sph_nnps_query decides it) and written
 * into both rows.  A count pass (with the density when rho != NULL, summed
 * as sph_density_half sums it: an FP32 atomic adds the partner's share, so
 * its last bits vary between calls), a scan, a fill pass at atomic row
 * cursors and a per-row sort give the same CSR as sph_nnps_query (cell
 * order).  Cell-order FP16-RCLL grids only; col == NULL counts only.
 * Synchronises; SPH_ERR_CAPACITY (nothing written to col) when nnz exceeds
 * col_capacity.  This is the symmetric "distance reuse" of the paper's
 * conclusions applied to the full neighbour list; it is slower than
 * sph_nnps_query on GB300 (see the measurement in the bench line). */
int sph_nnps_query_half(sph_grid_t grid, int64_t *row_ptr, int32_t *col, int64_t col_capacity, int64_t *nnz_out,
                        float *rho, void *stream);

/* Fill *info (host) with the grid's sizes and device pointers.  The pointers
 * stay valid until the grid is re-binned or freed. */
int sph_grid_info_get(sph_grid_t grid, sph_grid_info *info);

/* Copy the grid's permutation and cell arrays into caller buffers (device
 * memory, any may be NULL): orig_id int32[n] (sorted position -> input index),
 * rank int32[n] (input index -> sorted position), cell_start int32[ncell+1]
 * (first sorted position of each cell).  Enqueued on `stream`. */
int sph_grid_export(sph_grid_t grid, int32_t *orig_id, int32_t *rank, int32_t *cell_start,
                    void *stream);

/* Copy the stored cell-relative coordinates (Eq. 6, SPH_PREC_FP16_RCLL grids
 * only) in sorted order into caller buffers (device memory, either may be
 * NULL): rel16 uint16[n][4] (FP16 bit patterns of x, y, z, then the cell x
 * index modulo 2^16 as an unsigned integer), rel32 float[n][4] (x, y, z, 0).  Units u = h_c / 2 relative to the centre of the particle's
 * cell: for s = 2 (x - lo) / h_c rounded to FP64 (one fused multiply-add
 * when every coordinate lies within 2^17 u of the origin, else a subtraction
 * and a multiplication) and c = min(floor(s / 2), n_k - 1), the FP32 value is
 * s - (2c + 1) rounded to nearest and the FP16 value is the FP32 value
 * rounded to nearest.  Enqueued on `stream`.  SPH_ERR_INVALID for other
 * precisions. */
int sph_grid_export_rel(sph_grid_t grid, uint16_t *rel16, float *rel32, void *stream);

/* Synchronise `stream` and report any error a device-side check recorded for
 * this grid since the last synchronising call (SPH_OK if none). */
int sph_grid_check(sph_grid_t grid, void *stream);

/* Release the grid and its device buffers (stream-ordered on the stream the
 * grid last used).  NULL is accepted. */
int sph_grid_free(sph_grid_t grid);

/* Message for the calling thread's last failed call ("" if none). */
const char *sph_last_error(void);

/*
 * One call from host memory: copy xyz (host, n x p->dim FP64, preferably
 * pinned) into a device buffer owned by the grid, bin it (as
 * sph_bin_cells), search with the fused density (as sph_nnps_query), copy
 * the density (host float[n], may be NULL; in the grid's output row order)
 * and nnz (host, may be NULL) back.  The CSR stays on the device in
 * grid-owned buffers (sph_grid_csr); the grid grows them as needed.
 * *grid as in sph_bin_cells.  Synchronises `stream`.  Errors as
 * sph_bin_cells and sph_nnps_query.
 */
int sph_search_host(const sph_params *p, const double *xyz_host, int64_t n, float *rho_host,
                    int64_t *nnz_host, sph_grid_t *grid, void *stream);

/* sph_search_host without the final wait, for callers that overlap
 * consecutive searches (two grids on two streams: one search's copies run
 * while the other's kernels do).  The call copies xyz in, bins (reading the
 * bounds back waits for this stream's copy and bounds kernel only), searches
 * with the grid's column buffer as it is, and queues the copy of the density
 * to rho_host (pinned host memory) and of nnz into the grid's host record;
 * it returns without waiting for them.  xyz_host and rho_host must stay
 * valid until sph_search_host_finish.  The first call on a grid, or a call
 * whose n or dim differs from the grid's last, runs sph_search_host instead
 * (it sizes the column buffer and waits).  A call on a grid whose previous
 * asynchronous search is unfinished finishes that one first. */
int sph_search_host_async(const sph_params *p, const double *xyz_host, int64_t n, float *rho_host,
                          int64_t *nnz_host, sph_grid_t *grid, void *stream);
/* Wait for the grid's last sph_search_host_async; then nnz (here, or to the
 * nnz_host given to that call when this one is NULL), the density and the CSR
 * are complete.  SPH_ERR_CAPACITY when the neighbours outgrew the grid's
 * column buffer (the CSR is then incomplete: call sph_search_host, which
 * grows it); the status errors of sph_nnps_query otherwise.  When nothing
 * is pending (the last call ran synchronously) it returns SPH_OK and that
 * search's nnz. */
int sph_search_host_finish(sph_grid_t grid, int64_t *nnz_host);

/* Device pointers of the grid-owned CSR and density written by the last
 * sph_search_host on this grid (host out-pointers; any may be NULL). */
/* Copy the CSR written by the last sph_search_host on this grid into caller
 * buffers (host -- preferably pinned -- or device; any may be NULL): row_ptr
 * int64[n + 1], col int32[nnz], on `stream`, then synchronise it.
 * SPH_ERR_INVALID when the grid holds no sph_search_host result. */
int sph_grid_csr_copy(sph_grid_t grid, int64_t *row_ptr, int32_t *col, void *stream);
int sph_grid_csr(sph_grid_t grid, const int64_t **row_ptr, const int32_t **col, const float **rho,
                 int64_t *nnz);

/* Mixed-precision time step (Eq. 8-9): advance a binned FP16-RCLL grid by
 * one step of its particles' motion without converting the absolute
 * coordinates again.  The cell-relative coordinates move by 2 v dt / h_c
 * (Eq. 8, displacement v dt of Eq. 9, kept in FP64 and rounded once to
 * FP16 / FP32 as binning rounds them); a particle whose coordinate leaves
 * [-1, 1] moves to the adjacent cell; the cell order is then rebuilt from the
 * integer cell ids (no bounds pass).  The grid's box is kept: if a particle
 * leaves it the grid is binned again from xyz_new (with a caller box that is
 * SPH_ERR_INVALID instead).
 *   xyz_new  device FP64 n x dim (input order): the positions after the step,
 *            x + v dt as the caller computes them.  FP64 decisions use them
 *            from now on; the array must stay valid like sph_bin_cells' xyz.
 *   vel      device FP64 n x dim (input order), dt the step.
 * The FP64 relative coordinates accumulate rounding apart from xyz_new; the
 * library bounds that drift each step and derives them again from the
 * positions before it could reach 1e-7 u (u = h_c / 2), far inside the bands,
 * so the neighbour lists stay those of the FP64 definition on xyz_new.
 * Other grids (FP64-CLL, n == 0) are binned again from xyz_new.
 * Synchronises `stream` once.  SPH_ERR_INVALID for non-finite velocities. */
int sph_advance(sph_grid_t grid, const double *xyz_new, const double *vel, double dt, void *stream);

/* ---- Batched runs: many independent systems in one pass ----------------------
 *
 * sph_batch_run bins, searches and sums the density of nsys independent
 * particle systems (all of one dimension, FP16-RCLL, cell order) as one
 * concatenated problem: one launch per binning step and one persistent
 * launch of the tile search for all systems.  The paper searches one system
 * at a time; batching is this library's way of filling the GPU with many
 * small ones.
 *
 * The output is one block-diagonal CSR over the concatenation in cell order:
 * system s owns sorted positions (= rows) [sys_first[s], sys_first[s+1]),
 * its columns are sorted positions of the same range, ascending within each
 * row, and orig_id maps a sorted position to the system's own input index.
 *
 * per_system, xyz (host array of nsys device pointers, each n[s] x dim FP64),
 * n (host) describe the systems; params as for sph_bin_cells (have_box per
 * system; order must be SPH_ORDER_CELL, precision SPH_PREC_FP16_RCLL).
 * *batch: workspace, created on first use (pass a pointer to NULL) and reused;
 * it owns the device buffers, the recorded CUDA graph and the tuning cache.
 * The call synchronises `stream` (it reads the systems' bounds and nnz).
 *
 * Errors: SPH_ERR_INVALID (parameters, mixed dims, more than 2^31 - 1
 * particles or cells in total), SPH_ERR_CAPACITY (nnz > col_capacity: out->nnz
 * is set, no entry at or past col_capacity is written), others as
 * sph_bin_cells.
 */
typedef struct sph_batch_s *sph_batch_t;

typedef struct {
    int64_t *row_ptr;     /* device int64[n_total + 1], written (global offsets into col) */
    int32_t *col;         /* device int32[col_capacity], or NULL: row_ptr, rho and nnz only */
    int64_t col_capacity;
    float *rho;           /* device float[n_total] (sorted positions), or NULL; needs col */
    int32_t *orig_id;     /* device int32[n_total] or NULL: sorted position -> the system's input index */
    int64_t *sys_first;   /* host int64[nsys + 1] or NULL: first sorted position of each system */
    int64_t nnz;          /* written: total neighbour count */
} sph_batch_out;

/* Create an empty workspace (host call; binds to the current CUDA device). */
int sph_batch_create(sph_batch_t *batch);

int sph_batch_run(sph_batch_t *batch, const sph_params *per_system, const double *const *xyz, const int64_t *n,
                  int nsys, sph_batch_out *out, void *stream);

/* Counters of a workspace (host struct). */
typedef struct {
    int64_t runs;             /* sph_batch_run calls */
    int64_t graph_captures;   /* launch sequences recorded as CUDA graphs */
    int64_t graph_replays;    /* runs that replayed the recorded graph */
    int32_t tuned_staging;    /* staging bytes chosen by the last tuning, -1: none yet */
    int32_t tuned_candidates; /* candidates timed by the last tuning */
    int32_t tuned_shape;      /* tile shape chosen by the last tuning (SPH_OPT_TILE_SHAPE values), -1: none */
    int32_t reserved;
    int64_t fp32_pairs;       /* last run: pairs re-decided in FP32 */
    int64_t fp64_pairs;       /* last run: pairs decided in FP64 */
    int64_t direct_launches;  /* last run: kernels launched outside the replayed graph */
    int64_t graph_launched;   /* last run: 1 if it launched the recorded graph, else 0 */
} sph_batch_stats;
int sph_batch_get_stats(sph_batch_t batch, sph_batch_stats *stats);

/* SPH_BATCH_OPT_GRAPH: 1 (default) record the launches after the bounds --
 *   binning, tile list, counter reset and the persistent tile search with the
 *   shape and staging chosen for the batch -- as one CUDA graph and replay it
 *   while the batch's sizes, buffers and chosen shape are unchanged (a run
 *   that tunes the shape runs directly and records the graph with its
 *   choice); 0 launch directly every time.
 * SPH_BATCH_OPT_STAGING: -1 (default) tune the tile search's shape and
 *   staging bytes by timing five candidates (sparse 0 / 2048, dense 0 / 2048 /
 *   4096) on the first run of each density class (dimension and neighbours per
 *   particle to a quarter octave) and reuse the winner; -2 choose both from
 *   the particle density without timing; 0 .. 65536 in multiples of 16 fix the
 *   staging (shape from the density). */
#define SPH_BATCH_OPT_GRAPH 1
#define SPH_BATCH_OPT_STAGING 2
int sph_batch_set_option(sph_batch_t batch, int option, int64_t value);

/* Free a workspace (synchronises the device).  NULL is a no-op. */
int sph_batch_free(sph_batch_t batch);

/* ---- Serving: a request server over the search ----------------------------
 *
 * A server owns worker threads (one CUDA stream each) on the device current
 * at creation.  Clients submit particle systems; each request is binned,
 * searched and its density summed, and its results stay in device memory
 * owned by the server until the client releases them.  Admission keeps the
 * device memory reserved for running requests plus held results within
 * hbm_budget_bytes (each running request reserves an estimate for up to 128
 * neighbours per particle in 3D, 40 in 2D; a finished one holds its exact
 * result).  Requests start in submission order, except that younger requests
 * that fit may pass one that does not, until it has waited max_wait_ns.
 * Small cell-order requests (n <= small_n) waiting together of one dimension
 * are searched as one batch (up to max_batch requests) and their results
 * split afterwards (continuous batching).  A request that fails (for example
 * a non-finite coordinate) reports its error alone; the others are unaffected.
 * Requests of more than large_n particles run on a low-priority stream and
 * their persistent search takes only large_sm_percent of the GPU's resident
 * thread-block slots; the others run on high-priority streams, so that small
 * requests arriving next to a large one start at once instead of queueing
 * behind it.  Unless reserve_pool is -1, the server grows the device's
 * stream-ordered memory pool to the budget (or, failing that, as far as it
 * can) once at creation, so that no request waits on the pool growing.
 * The paper serves no requests; this is the library's serving layer.
 */
typedef struct sph_server_s *sph_server_t;

typedef struct {
    int64_t hbm_budget_bytes; /* > 0 */
    int32_t streams;          /* worker threads / CUDA streams, 0: 2 (max 16) */
    int32_t max_batch;        /* requests per batched search, 0: 64 */
    int64_t small_n;          /* batching threshold in particles, 0: 32768 */
    int64_t max_wait_ns;      /* passing limit, 0: 20 ms */
    int64_t large_n;          /* requests above it run beside the others on a share of the GPU, 0: 262144 */
    int32_t large_sm_percent; /* that share in percent (1 .. 100), 0: 75 */
    int32_t reserve_pool;     /* 0: grow the memory pool to the budget at creation, -1: do not */
} sph_server_cfg;

typedef struct {
    sph_params params;      /* as for sph_bin_cells (order and precision are honoured) */
    const double *xyz;      /* n x dim FP64; must stay valid and unchanged until the request completes */
    int64_t n;
    int32_t xyz_on_device;  /* 1: device pointer; 0: host pointer (copied when the request starts) */
    int32_t want_density;   /* 1: compute rho */
} sph_request;

typedef struct {
    int32_t status;            /* SPH_OK or the request's error code */
    int64_t n, nnz;
    const int64_t *row_ptr;    /* device int64[n + 1] (rows in the request's order: see params.order) */
    const int32_t *col;        /* device int32[nnz] */
    const float *rho;          /* device float[n] or NULL */
    const int32_t *orig_id;    /* device int32[n] (cell order: sorted position -> input index) or NULL */
    int64_t t_submit_ns, t_admit_ns, t_done_ns; /* steady clock: submitted, started, results ready */
} sph_result;

typedef struct {
    int64_t submitted, completed, failed; /* requests */
    int64_t batches, batched_requests;    /* batched searches and the requests they served */
    int64_t held_bytes, peak_held_bytes;  /* reserved + held device bytes now / at most */
    int64_t queued;                       /* requests waiting for admission */
} sph_server_stats;

/* Create a server (host call; starts the worker threads). */
int sph_server_create(const sph_server_cfg *cfg, sph_server_t *server);
/* Queue a request; *ticket identifies it.  SPH_ERR_INVALID for bad
 * parameters, SPH_ERR_BUDGET when the request alone exceeds the budget. */
int sph_serve_submit(sph_server_t server, const sph_request *req, uint64_t *ticket);
/* SPH_PENDING while the request is queued or running; SPH_OK once it has
 * finished (then *result is filled, result->status tells success or the
 * request's error); SPH_ERR_NOT_FOUND for an unknown or released ticket. */
int sph_serve_poll(sph_server_t server, uint64_t ticket, sph_result *result);
/* As sph_serve_poll, waiting up to timeout_ns (< 0: without limit). */
int sph_serve_wait(sph_server_t server, uint64_t ticket, int64_t timeout_ns, sph_result *result);
/* Copy a finished request's results into caller buffers (device or host
 * memory, any may be NULL; sizes n + 1, nnz, n, n) on `stream` (not
 * synchronised).  SPH_ERR_INVALID before the request has finished, its own
 * error code if it failed. */
int sph_result_copy(sph_server_t server, uint64_t ticket, int64_t *row_ptr, int32_t *col, float *rho,
                    int32_t *orig_id, void *stream);
/* Free a finished request's device results; the ticket becomes unknown.
 * The caller's own work on the result buffers must have completed. */
int sph_result_release(sph_server_t server, uint64_t ticket);
int sph_server_get_stats(sph_server_t server, sph_server_stats *stats);
/* Stop the workers (running requests finish, queued ones are dropped), free
 * every result and the server. */
int sph_server_destroy(sph_server_t server);

/* Per-kernel device timing of the library's own launches.  While enabled,
 * every launch is bracketed by CUDA events recorded on its stream.
 * sph_profile_read waits for the recorded events and returns the summed
 * milliseconds and launch count for one kernel tag since the last reset:
 * "bounds", "hash", "scan", "scatter", "sort", "convert", "count", "fill",
 * "density", "canon", "fused", "batch", "step".
 * sph_profile_select enables the events for the listed tags only
 * (comma-separated, e.g. "fused"; NULL: all), so that a timed loop pays for
 * events around the kernels it reports and no others.  SPH_ERR_INVALID for an
 * unknown tag (the selection is then unchanged). */
int sph_profile_enable(int on);
int sph_profile_select(const char *kernels);
int sph_profile_reset(void);
int sph_profile_read(const char *kernel, double *total_ms, int64_t *launches);

/* Measured FP64 fused multiply-add throughput of the current CUDA device in
 * FLOP/s (two per FMA): a short kernel of independent FMA chains timed with
 * CUDA events on the legacy default stream (synchronises the device).  A
 * diagnostic beside the FP64 cell link-list baseline; the paper's case for
 * FP16 rests on the FP64 rate.  *flops: host pointer. */
int sph_device_fp64_rate(double *flops);

/* Number of kernels the library has launched since it was loaded. */
int64_t sph_launch_count(void);

/* Error bands of the FP16-RCLL search, in units of u^2 with u = h_c / 2 (the
 * unit of the normalised relative coordinates of Eq. 6; the threshold is
 * T = kh^2 / u^2).  A pair is kept by the FP16 test when
 * r2_fp16 - T < *tau16; a kept pair is a neighbour when r2_fp32 < T - *tau32,
 * not one when r2_fp32 > T + *tau32, and is decided in FP64 otherwise.
 * Host pointers; either may be NULL.  No GPU needed. */
int sph_precision_bands(double *tau16, double *tau32);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int sph_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
