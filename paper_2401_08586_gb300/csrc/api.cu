// api.cu -- C ABI of libsph (declared in include/sph.h): grid objects,
// parameter validation, the launch sequence of the binning and search steps,
// and error reporting.  No exception crosses the ABI.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "host.cuh"
#include "launch.cuh"
#include "profile.cuh"
#include "sph_internal.cuh"


using namespace sph;

struct sph_grid_s {
    sph_params p;
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    long long n = 0;
    int nk[3] = {1, 1, 1};
    long long ncell = 1;
    double lo[3] = {0, 0, 0};
    double hc = 0;
    const double *xyz = nullptr;
    DevBuf cell_start, cnt, cid, slot, orig_id, rank, scell, rel16, rel32, rel16u, rel32u, x64, scan_tmp, big_list,
        rowcnt, tmp_rp, tmp_col, tmp_rho, status, own_xyz, own_rp, own_col, own_rho, tstate, scell_x, tcount,
        toff, tiles;
    int fused_enabled = 1;  // search variant for cell-order FP16 queries (SPH_OPT_FUSED)
    int staging = -1;       // extra staging bytes of the tile search (SPH_OPT_STAGING; -1: automatic)
    int tile_shape = -1;    // shared-memory shape of the tile search (SPH_OPT_TILE_SHAPE; -1: automatic)
    double last_nbr = 0;    // neighbours per particle of the last query whose nnz reached the host
    int test_lookback = 0;  // SPH_OPT_TEST_LOOKBACK: > 0 skips the first tile, waits give up after that many polls
    int sm_percent = 100;   // SPH_OPT_SM_SHARE
    DevBuf rel64, rel64u;   // FP64 relative coordinates kept across time steps (cell / input order)
    DevBuf fsplit;          // gradient: the field as float hi + lo in cell order
    DevBuf study;           // precision study counters
    bool rel64_valid = false;
    double drift = 0;       // bound on |rel64 - conversion of xyz| in units of u
    long long own_nnz = 0;
    DevStatus *h_status = nullptr;  // pinned host mirror, followed by the read-back flag
    unsigned int status_seq = 0;    // sequence number of the last flagged read-back
    bool async_pending = false;     // sph_search_host_async enqueued, sph_search_host_finish not yet called
    int64_t *async_nnz = nullptr;   // where sph_search_host_finish reports nnz
};

static unsigned int *status_flag(sph_grid_s *g) {
    return reinterpret_cast<unsigned int *>(reinterpret_cast<char *>(g->h_status) + sizeof(DevStatus));
}

static GridDev make_dev(sph_grid_s *g) {
    GridDev d;
    memset(&d, 0, sizeof(d));
    d.dim = g->p.dim;
    d.n = (int)g->n;
    for (int k = 0; k < 3; ++k) {
        d.nk[k] = g->nk[k];
        d.lo[k] = g->lo[k];
    }
    d.ncell = g->ncell;
    set_divisors(d);
    d.hc = g->hc;
    d.two_over_hc = 2.0 / g->hc;
    // one-FMA binning when every coordinate of the grid lies within 2^17 u of
    // the origin (|x| 2/h_c <= 2^17 for x in [lo, lo + n h_c])
    d.fma_bin = 1;
    for (int k = 0; k < 3; ++k) {
        d.neg_lo_t[k] = -g->lo[k] * d.two_over_hc;
        const double far = fmax(fabs(g->lo[k]), fabs(g->lo[k] + g->nk[k] * g->hc)) * d.two_over_hc;
        if (!(far <= 131072.0)) d.fma_bin = 0;
    }
    d.cell_start = P<int>(g->cell_start);
    d.rel16 = P<uint2>(g->rel16);
    d.rel32 = P<float4>(g->rel32);
    d.x64 = P<double>(g->x64);
    d.orig_id = P<int>(g->orig_id);
    d.scell_x = P<int>(g->scell_x);
    d.xyz = g->xyz;
    set_constants(d, g->p, g->hc);
    d.status = P<DevStatus>(g->status);
    return d;
}

// Copy the status record (and, if rp_nnz != NULL, the nnz at rp_nnz) to
// the pinned host mirror and wait.  A kernel writes the mirror: no copy
// engine on the control path.
static int read_status(sph_grid_s *g, const long long *rp_nnz = nullptr) {
    SPH_CUDA(status_to_host(g->h_status, P<DevStatus>(g->status), rp_nnz, g->stream));
    SPH_CUDA(cudaStreamSynchronize(g->stream));
    return SPH_OK;
}

// The status record when nothing else the host reads is pending on the
// stream (binning's bounds): the host spins on a flag the read-back kernel
// sets after the record, which wakes it sooner than a stream
// synchronisation; if the flag does not come within 0.2 s (a failed
// earlier launch, a device that is far behind) the stream is synchronised,
// which reports any error.
static int read_status_flagged(sph_grid_s *g) {
    const unsigned int seq = ++g->status_seq;
    SPH_CUDA(status_to_host_flag(g->h_status, P<DevStatus>(g->status), status_flag(g), seq, g->stream));
    if (!wait_host_flag(status_flag(g), seq, 2e5)) SPH_CUDA(cudaStreamSynchronize(g->stream));
    return SPH_OK;
}

extern "C" int sph_version(void) { return 100; }

extern "C" int sph_precision_bands(double *tau16, double *tau32) {
    if (tau16) *tau16 = TAU16;
    if (tau32) *tau32 = TAU32;
    return SPH_OK;
}

extern "C" const char *sph_last_error(void) { return last_error(); }

static int grid_create(sph_grid_s **out) {
    sph_grid_s *g = new (std::nothrow) sph_grid_s();
    if (!g) return fail(SPH_ERR_NOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&g->h_status, sizeof(DevStatus) + 16);
    if (e == cudaSuccess) *status_flag(g) = 0;
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete g;
        return fail(SPH_ERR_CUDA, "CUDA initialisation failed: %s", cudaGetErrorString(e));
    }
    *out = g;
    return SPH_OK;
}

extern "C" int sph_bin_cells(const sph_params *p, const double *xyz, int64_t n, void *stream,
                             sph_grid_t *grid) {
    if (!grid) return fail(SPH_ERR_INVALID, "grid is NULL");
    SPH_TRY(validate_params(p, n, xyz));
    bool created = false;
    if (*grid == nullptr) {
        SPH_TRY(grid_create(grid));
        created = true;
    }
    sph_grid_s *g = *grid;
    cudaStream_t s = (cudaStream_t)stream;
    g->p = *p;
    g->stream = s;
    g->n = n;
    g->xyz = xyz;
    g->hc = p->cell_size != 0 ? p->cell_size : p->kh * (1.0 + 0x1p-30);
    g->rel64_valid = false;
    const int dim = p->dim;
    int rc = SPH_OK;
    do {
        if ((rc = ensure(g->status, sizeof(DevStatus), s)) != SPH_OK) break;
        if (launch_status_init(P<DevStatus>(g->status), s) != cudaSuccess) {
            cudaGetLastError();
            rc = fail(SPH_ERR_CUDA, "status launch failed");
            break;
        }
        double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
        if (p->have_box) {
            for (int k = 0; k < dim; ++k) {
                lo[k] = p->box_lo[k];
                hi[k] = p->box_hi[k];
            }
        } else if (n > 0) {
            if (launch_bounds(xyz, n, dim, P<DevStatus>(g->status), g->sm_count, s) != cudaSuccess) {
                rc = fail(SPH_ERR_CUDA, "bounds launch failed");
                break;
            }
            if ((rc = read_status_flagged(g)) != SPH_OK) break;
            if (g->h_status->flags & ST_NONFINITE) {
                rc = fail(SPH_ERR_INVALID, "non-finite particle coordinate");
                break;
            }
            for (int k = 0; k < dim; ++k) {
                lo[k] = dkey_inv(g->h_status->min_key[k]);
                hi[k] = dkey_inv(g->h_status->max_key[k]);
            }
        }
        long long ncell = 1;
        for (int k = 0; k < 3; ++k) {
            g->lo[k] = lo[k];
            g->nk[k] = 1;
            if (k < dim) {
                double span = ceil((hi[k] - lo[k]) / g->hc);
                if (!(span <= (double)(1 << 20))) {
                    rc = fail(SPH_ERR_INVALID, "more than 2^20 cells along axis %d", k);
                    break;
                }
                g->nk[k] = span < 1.0 ? 1 : (int)span;
            }
            ncell *= g->nk[k];
        }
        if (rc != SPH_OK) break;
        if (ncell > (1LL << 28)) {
            rc = fail(SPH_ERR_INVALID, "grid of %lld cells exceeds 2^28", ncell);
            break;
        }
        g->ncell = ncell;
        const long long nn = n > 0 ? n : 1;
        const long long big = ncell > nn ? ncell : nn;
        if ((rc = ensure(g->cell_start, (ncell + 1) * sizeof(int), s)) ||
            (rc = ensure(g->cnt, cnt_bytes(ncell), s)) || (rc = ensure(g->cid, nn * sizeof(int), s)) ||
            (rc = ensure(g->slot, nn * sizeof(int), s)) || (rc = ensure(g->orig_id, nn * sizeof(int), s)) ||
            (rc = ensure(g->rank, nn * sizeof(int), s)) || (rc = ensure(g->scell, nn * sizeof(int), s)) ||
            (rc = ensure(g->scan_tmp, scan_tmp_bytes(big + 1), s)) ||
            (rc = ensure(g->big_list, big * sizeof(int), s)) || (rc = ensure(g->scell_x, nn * sizeof(int), s)))
            break;
        if (p->precision == SPH_PREC_FP16_RCLL) {
            if ((rc = ensure(g->rel16, nn * sizeof(uint2), s)) || (rc = ensure(g->rel32, nn * sizeof(float4), s)) ||
                (rc = ensure(g->rel16u, nn * sizeof(uint2), s)) || (rc = ensure(g->rel32u, nn * sizeof(float4), s)))
                break;
        } else {
            if ((rc = ensure(g->x64, nn * sizeof(double4_32a), s))) break;
        }
        if (n == 0) {
            if (cudaMemsetAsync(g->cell_start.p, 0, (ncell + 1) * sizeof(int), s) != cudaSuccess) {
                rc = fail(SPH_ERR_CUDA, "memset failed");
                break;
            }
            break;
        }
        GridDev d = make_dev(g);
        cudaError_t e = launch_hash_scatter_convert(
            d, xyz, (int)n, dim, p->precision, P<int>(g->cnt), P<int>(g->cid), P<int>(g->slot),
            P<int>(g->cell_start), P<int>(g->orig_id), P<int>(g->rank), P<int>(g->scell), P<uint2>(g->rel16),
            P<float4>(g->rel32), P<uint2>(g->rel16u), P<float4>(g->rel32u), P<double4_32a>(g->x64), P<int>(g->scell_x),
            g->scan_tmp.p, P<int>(g->big_list),
            &P<DevStatus>(g->status)->big_cells, p->have_box, g->sm_count, s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(SPH_ERR_CUDA, "binning launch failed: %s", cudaGetErrorString(e));
        }
    } while (0);
    if (rc != SPH_OK && created) {
        sph_grid_free(*grid);
        *grid = nullptr;
    }
    return rc;
}

// Largest drift of the FP64 relative coordinates from the caller's positions
// (units of u) that the search's bands absorb: the FP32 band keeps 2.5e-6 u^2
// of slack over its worst case, and a drift d moves r^2 by at most ~14 d.
static const double DRIFT_BUDGET = 1e-7;

extern "C" int sph_advance(sph_grid_t grid, const double *xyz_new, const double *vel, double dt, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (!isfinite(dt)) return fail(SPH_ERR_INVALID, "dt must be finite");
    const long long n = g->n;
    if (n > 0 && (!xyz_new || !vel)) return fail(SPH_ERR_INVALID, "xyz_new and vel are needed");
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    if (g->p.precision != SPH_PREC_FP16_RCLL || n == 0) return sph_bin_cells(&g->p, xyz_new, n, stream, &grid);
    SPH_TRY(ensure(g->rel64, (size_t)n * sizeof(double4_32a), s));
    SPH_TRY(ensure(g->rel64u, (size_t)n * sizeof(double4_32a), s));
    GridDev d = make_dev(g);
    if (!g->rel64_valid || g->drift > DRIFT_BUDGET) {
        // derive the FP64 relative coordinates from the current positions
        SPH_CUDA(launch_rel64_sync(d, P<int>(g->scell), g->xyz, P<double4_32a>(g->rel64), g->sm_count, s));
        g->rel64_valid = true;
        g->drift = 0;
    }
    SPH_CUDA(launch_status_init(P<DevStatus>(g->status), s));
    SPH_CUDA(launch_advance(d, P<int>(g->scell), P<double4_32a>(g->rel64), vel, dt, P<int>(g->cnt), P<int>(g->cid),
                            P<int>(g->slot), P<uint2>(g->rel16u), P<float4>(g->rel32u), P<double4_32a>(g->rel64u),
                            g->sm_count, s));
    SPH_TRY(read_status(g));
    if (g->h_status->flags & ST_NONFINITE) return fail(SPH_ERR_INVALID, "non-finite velocity or displacement");
    if (g->h_status->flags & ST_OUT_OF_BOX) {
        if (g->p.have_box) return fail(SPH_ERR_INVALID, "a particle left the given box");
        // a particle left the grid: bin again with the new bounds
        return sph_bin_cells(&g->p, xyz_new, n, stream, &grid);
    }
    // drift bound of this step: the FMA of Eq. 8, the rounding of v dt and of
    // 2/h_c, and the caller's rounding of x + v dt, relative 2^-53 each
    double dmax = 0;
    {
        const unsigned long long b = g->h_status->max_key[0];
        memcpy(&dmax, &b, 8);
    }
    double xmax = 0;
    for (int k = 0; k < g->p.dim; ++k) {
        const double a = fabs(g->lo[k]), b = fabs(g->lo[k] + g->nk[k] * g->hc);
        xmax = fmax(xmax, fmax(a, b));
    }
    const double du = dmax * d.two_over_hc, xu = xmax * d.two_over_hc;
    g->drift += 0x1p-53 * (3.0 + 2.0 * du + 2.0 * (xu + du));
    SPH_CUDA(launch_order_convert(d, (int)n, g->p.dim, SPH_PREC_FP16_RCLL, P<int>(g->cnt), P<int>(g->cid),
                                  P<int>(g->slot), P<int>(g->cell_start), P<int>(g->orig_id), P<int>(g->rank),
                                  P<int>(g->scell), P<uint2>(g->rel16), P<float4>(g->rel32), P<uint2>(g->rel16u),
                                  P<float4>(g->rel32u), P<double4_32a>(g->rel64u), P<double4_32a>(g->rel64), nullptr,
                                  P<int>(g->scell_x),
                                  g->scan_tmp.p, P<int>(g->big_list), &P<DevStatus>(g->status)->big_cells,
                                  g->sm_count, s));
    g->xyz = xyz_new;
    return SPH_OK;
}

// Single pass, one warp per 32-particle row tile, look-back across tiles
// (nnps_tile.cu; FP64 grids: nnps_tile64.cu), in cell order: row pointers
// always; columns and the fused density when col / rho are given (col ==
// NULL: the count only).
static int run_tile_search(sph_grid_s *g, long long *rp_cell, int *col, long long cap, float *rho, bool test_lb,
                           cudaStream_t s) {
    const long long n = g->n;
    const long long nrow = (long long)g->nk[1] * g->nk[2];
    const long long ntiles_max = tiles_max(n, g->ncell, nrow);
    SPH_TRY(ensure(g->tcount, nrow * sizeof(int), s));
    SPH_TRY(ensure(g->toff, (nrow + 1) * sizeof(long long), s));
    SPH_TRY(ensure(g->tiles, ntiles_max * sizeof(int4), s));
    // look-back state of the search (ntiles_max entries), then of the
    // tile-list builder's chunks of rows (at most nrow + 1), cleared at once
    const long long nstate = ntiles_max + nrow + 1;
    SPH_TRY(ensure(g->tstate, nstate * sizeof(unsigned long long), s));
    SPH_CUDA(cudaMemsetAsync(g->tstate.p, 0, nstate * sizeof(unsigned long long), s));
    unsigned long long *tstate = P<unsigned long long>(g->tstate);
    GridDev d = make_dev(g);
    if (test_lb) d.spin_limit = g->test_lookback;
    SPH_CUDA(launch_tiles(d, true, P<int>(g->tcount), P<long long>(g->toff), g->scan_tmp.p, P<int4>(g->tiles),
                          tstate + ntiles_max, g->sm_count, s));
    if (g->p.precision == SPH_PREC_FP64_CLL) {
        SPH_CUDA(launch_nnps_tile64(d, P<int4>(g->tiles), P<long long>(g->toff) + nrow, ntiles_max, rp_cell, col, cap,
                                    rho, tstate, g->sm_count, s));
        return SPH_OK;
    }
    const TileLaunch tv = tile_choose_grid(g->last_nbr, n, g->ncell, g->p.dim, g->p.kh, g->hc, g->tile_shape,
                                           g->staging, g->sm_percent);
    SPH_CUDA(launch_nnps_tile(d, nullptr, P<int4>(g->tiles), P<long long>(g->toff) + nrow, ntiles_max, rp_cell, col,
                              cap, rho, tstate, tv, true, g->sm_count, s));
    return SPH_OK;
}

// nnz of a finished cell-order search (rp_cell[n]); synchronises the stream.
static int read_nnz(sph_grid_s *g, const long long *rp_cell, long long *nnz) {
    SPH_TRY(read_status(g, rp_cell + g->n));
    *nnz = g->h_status->nnz;
    if (g->n > 0) g->last_nbr = (double)*nnz / (double)g->n;
    return SPH_OK;
}

extern "C" int sph_nnps_query(sph_grid_t grid, int64_t *row_ptr, int32_t *col, int64_t col_capacity,
                              int64_t *nnz_out, float *rho, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (!row_ptr) return fail(SPH_ERR_INVALID, "row_ptr is NULL");
    if (col && col_capacity < 0) return fail(SPH_ERR_INVALID, "negative col_capacity");
    if (rho && !col) return fail(SPH_ERR_INVALID, "rho needs col (the density is fused into the fill)");
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    const long long n = g->n;
    if (n == 0) {
        SPH_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s));
        if (nnz_out) {
            SPH_CUDA(cudaStreamSynchronize(s));
            *nnz_out = 0;
        }
        return SPH_OK;
    }
    GridDev d = make_dev(g);
    const bool test_lb = g->test_lookback > 0;
    SPH_CUDA(launch_status_reset_counters(P<DevStatus>(g->status), s, test_lb ? 1ull : 0ull));
    SPH_TRY(ensure(g->rowcnt, n * sizeof(int), s));
    const bool canonical = g->p.order == SPH_ORDER_CANONICAL;
    const int prec = g->p.precision;
    // the single-pass tile search (FP16-RCLL, or its FP64 form on FP64-CLL
    // grids) serves every query unless another search variant is asked for
    // (SPH_OPT_FUSED 0: two passes; 2: one CTA per cell, FP16 cell-order
    // queries with columns only; other FP64 queries then take two passes)
    const bool tile = g->fused_enabled == 1 || test_lb;
    long long *rp_cell = reinterpret_cast<long long *>(row_ptr);
    if (canonical) {
        SPH_TRY(ensure(g->tmp_rp, (n + 1) * sizeof(long long), s));
        rp_cell = P<long long>(g->tmp_rp);
    }
    if (!canonical) {
        const bool cell_cta = col != nullptr && prec == SPH_PREC_FP16_RCLL && g->fused_enabled == 2 && !test_lb;
        if (cell_cta) {
            // single pass, one CTA per cell, row offsets by look-back across cells
            SPH_TRY(ensure(g->tstate, (size_t)g->ncell * sizeof(unsigned long long), s));
            SPH_CUDA(launch_nnps_fused(d, rp_cell, col, col_capacity, rho, P<unsigned long long>(g->tstate),
                                       P<int>(g->rowcnt), g->sm_count, s));
        } else if (tile) {
            SPH_TRY(run_tile_search(g, rp_cell, col, col ? col_capacity : 0, rho, test_lb, s));
        } else {
            SPH_CUDA(launch_nnps(d, prec, 0, P<int>(g->rowcnt), nullptr, nullptr, 0, nullptr, g->sm_count, s));
            SPH_CUDA(exclusive_scan_i64(P<int>(g->rowcnt), rp_cell, n, g->scan_tmp.p, s));
            if (col) SPH_CUDA(launch_nnps(d, prec, 1, nullptr, rp_cell, col, col_capacity, rho, g->sm_count, s));
        }
        if (nnz_out) {
            long long nnz_host = 0;
            SPH_TRY(read_nnz(g, rp_cell, &nnz_host));  // the status record comes with it
            *nnz_out = nnz_host;
            int rc = status_to_code(g->h_status->flags);
            if (rc == SPH_OK && col && nnz_host > col_capacity)
                rc = fail(SPH_ERR_CAPACITY, "nnz %lld exceeds col_capacity %lld", nnz_host,
                          (long long)col_capacity);
            return rc;
        }
        return SPH_OK;
    }
    // Canonical order: search in cell order into the grid's own buffers, then
    // permute the rows, map the columns to input indices and sort each row
    // (this path always synchronises: it needs nnz on the host).
    long long nnz = 0;
    bool have_cols = false;  // tmp_col / tmp_rho already hold the cell-order result
    if (tile && col) {
        // capacity guess from the last query (else the uniform-density
        // estimate), one more search if the guess was short
        double nbr = g->last_nbr;
        if (nbr <= 0) {
            const double ppc = (double)n / (double)g->ncell, r = g->p.kh / g->hc;
            nbr = g->p.dim == 3 ? ppc * 4.18879 * r * r * r : ppc * 3.14159 * r * r;
        }
        long long cap_t = (long long)(nbr * (double)n * 1.1) + 4096;
        SPH_TRY(ensure(g->tmp_col, (size_t)cap_t * sizeof(int), s));
        cap_t = (long long)(g->tmp_col.cap / sizeof(int));
        if (rho) SPH_TRY(ensure(g->tmp_rho, n * sizeof(float), s));
        SPH_TRY(run_tile_search(g, rp_cell, P<int>(g->tmp_col), cap_t, rho ? P<float>(g->tmp_rho) : nullptr, test_lb,
                                s));
        SPH_TRY(read_nnz(g, rp_cell, &nnz));
        have_cols = nnz <= cap_t;
        if (!have_cols && nnz <= col_capacity) {
            SPH_TRY(ensure(g->tmp_col, (size_t)nnz * sizeof(int), s));
            SPH_CUDA(launch_status_reset_counters(P<DevStatus>(g->status), s, test_lb ? 1ull : 0ull));
            SPH_TRY(run_tile_search(g, rp_cell, P<int>(g->tmp_col), nnz, rho ? P<float>(g->tmp_rho) : nullptr,
                                    test_lb, s));
            have_cols = true;
        }
    } else if (tile) {
        SPH_TRY(run_tile_search(g, rp_cell, nullptr, 0, nullptr, test_lb, s));
        SPH_TRY(read_nnz(g, rp_cell, &nnz));
    } else {
        SPH_CUDA(launch_nnps(d, prec, 0, P<int>(g->rowcnt), nullptr, nullptr, 0, nullptr, g->sm_count, s));
        SPH_CUDA(exclusive_scan_i64(P<int>(g->rowcnt), rp_cell, n, g->scan_tmp.p, s));
        SPH_TRY(read_nnz(g, rp_cell, &nnz));
    }
    if (nnz_out) *nnz_out = nnz;
    if (col && nnz > col_capacity) {
        SPH_TRY(launch_canon((int)n, P<int>(g->rank), P<int>(g->orig_id), rp_cell, nullptr, nullptr,
                             P<int>(g->rowcnt), g->scan_tmp.p, reinterpret_cast<long long *>(row_ptr), nullptr,
                             nullptr, P<int>(g->big_list), &P<DevStatus>(g->status)->big_cells, g->sm_count, s) ==
                        cudaSuccess
                    ? SPH_OK
                    : fail(SPH_ERR_CUDA, "canonical row pointer launch failed"));
        SPH_CUDA(cudaStreamSynchronize(s));
        return fail(SPH_ERR_CAPACITY, "nnz %lld exceeds col_capacity %lld", nnz, (long long)col_capacity);
    }
    if (col && !have_cols) {
        SPH_TRY(ensure(g->tmp_col, (nnz > 0 ? nnz : 1) * sizeof(int), s));
        if (rho) SPH_TRY(ensure(g->tmp_rho, n * sizeof(float), s));
        SPH_CUDA(launch_nnps(d, prec, 1, nullptr, rp_cell, P<int>(g->tmp_col), nnz, rho ? P<float>(g->tmp_rho) : nullptr,
                             g->sm_count, s));
    }
    // row lengths are needed again: rowcnt is reused as scratch by launch_canon
    SPH_CUDA(launch_canon((int)n, P<int>(g->rank), P<int>(g->orig_id), rp_cell, col ? P<int>(g->tmp_col) : nullptr,
                          rho ? P<float>(g->tmp_rho) : nullptr, P<int>(g->rowcnt), g->scan_tmp.p,
                          reinterpret_cast<long long *>(row_ptr), col, rho, P<int>(g->big_list),
                          &P<DevStatus>(g->status)->big_cells, g->sm_count, s));
    SPH_TRY(read_status(g));
    return status_to_code(g->h_status->flags);
}

extern "C" int sph_density_half(sph_grid_t grid, float *rho, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (g->p.precision != SPH_PREC_FP16_RCLL) return fail(SPH_ERR_INVALID, "FP16-RCLL grids only");
    if (g->p.order != SPH_ORDER_CELL) return fail(SPH_ERR_INVALID, "cell-order grids only");
    if (g->n > 0 && !rho) return fail(SPH_ERR_INVALID, "rho is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    if (g->n == 0) return SPH_OK;
    const GridDev d = make_dev(g);
    SPH_CUDA(launch_status_reset_counters(P<DevStatus>(g->status), s));
    SPH_CUDA(launch_density_half(d, P<int>(g->scell), rho, g->sm_count, s));
    return SPH_OK;
}

extern "C" int sph_nnps_query_half(sph_grid_t grid, int64_t *row_ptr, int32_t *col, int64_t col_capacity,
                                   int64_t *nnz_out, float *rho, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (!row_ptr) return fail(SPH_ERR_INVALID, "row_ptr is NULL");
    if (g->p.precision != SPH_PREC_FP16_RCLL) return fail(SPH_ERR_INVALID, "FP16-RCLL grids only");
    if (g->p.order != SPH_ORDER_CELL) return fail(SPH_ERR_INVALID, "cell-order grids only");
    if (col && col_capacity < 0) return fail(SPH_ERR_INVALID, "negative col_capacity");
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    const long long n = g->n;
    if (n == 0) {
        SPH_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t), s));
        SPH_CUDA(cudaStreamSynchronize(s));
        if (nnz_out) *nnz_out = 0;
        return SPH_OK;
    }
    const GridDev d = make_dev(g);
    long long *rp = reinterpret_cast<long long *>(row_ptr);
    SPH_CUDA(launch_status_reset_counters(P<DevStatus>(g->status), s));
    SPH_TRY(ensure(g->rowcnt, n * sizeof(int), s));
    SPH_CUDA(launch_half_count(d, P<int>(g->scell), P<int>(g->rowcnt), rho, g->sm_count, s));
    SPH_CUDA(exclusive_scan_i64(P<int>(g->rowcnt), rp, n, g->scan_tmp.p, s));
    long long nnz = 0;
    SPH_TRY(read_nnz(g, rp, &nnz));
    if (nnz_out) *nnz_out = nnz;
    SPH_TRY(status_to_code(g->h_status->flags));
    if (!col) return SPH_OK;
    if (nnz > col_capacity)
        return fail(SPH_ERR_CAPACITY, "nnz %lld exceeds col_capacity %lld", nnz, (long long)col_capacity);
    SPH_TRY(ensure(g->tmp_rp, (size_t)(n + 1) * sizeof(long long), s));
    SPH_CUDA(copy_d2d_kernel(g->tmp_rp.p, rp, (size_t)n * sizeof(long long), s));
    SPH_CUDA(launch_half_fill(d, P<int>(g->scell), P<unsigned long long>(g->tmp_rp), col, g->sm_count, s));
    SPH_CUDA(segmented_sort_rows(col, rp, n, P<int>(g->big_list), &P<DevStatus>(g->status)->big_cells, g->sm_count,
                                 s));
    SPH_TRY(read_status(g));
    return status_to_code(g->h_status->flags);
}

extern "C" int sph_density_sum(sph_grid_t grid, const int64_t *row_ptr, const int32_t *col, float *rho,
                               void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (!row_ptr || !rho || (!col && g->n > 0)) return fail(SPH_ERR_INVALID, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    if (g->n == 0) return SPH_OK;
    GridDev d = make_dev(g);
    SPH_CUDA(launch_density(d, g->p.precision, P<int>(g->rank), P<int>(g->scell),
                            reinterpret_cast<const long long *>(row_ptr), col,
                            g->p.order == SPH_ORDER_CANONICAL, rho, g->sm_count, s));
    return SPH_OK;
}

extern "C" int sph_gradient_a5(sph_grid_t grid, const int64_t *row_ptr, const int32_t *col, const double *f,
                               double *grad, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (!row_ptr || !f || !grad || (!col && g->n > 0)) return fail(SPH_ERR_INVALID, "NULL argument");
    if (g->p.precision != SPH_PREC_FP16_RCLL) return fail(SPH_ERR_INVALID, "the gradient needs an FP16-RCLL grid");
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    if (g->n == 0) return SPH_OK;
    SPH_TRY(ensure(g->fsplit, (size_t)g->n * sizeof(float2), s));
    GridDev d = make_dev(g);
    SPH_CUDA(launch_gradient_a5(d, P<int>(g->rank), P<int>(g->scell), reinterpret_cast<const long long *>(row_ptr),
                                col, g->p.order == SPH_ORDER_CANONICAL, f, P<float2>(g->fsplit), grad, g->sm_count,
                                s));
    return SPH_OK;
}

extern "C" int sph_precision_study(sph_grid_t grid, int64_t row_begin, int64_t row_end, sph_precision_counts *out,
                                   void *stream) {
    sph_grid_s *g = grid;
    if (!g || !out) return fail(SPH_ERR_INVALID, "NULL argument");
    if (g->p.precision != SPH_PREC_FP16_RCLL) return fail(SPH_ERR_INVALID, "the study needs an FP16-RCLL grid");
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    memset(out, 0, sizeof(*out));
    if (g->n == 0) return SPH_OK;
    SPH_TRY(ensure(g->study, 6 * sizeof(unsigned long long), s));
    GridDev d = make_dev(g);
    SPH_CUDA(launch_precision_study(d, P<int>(g->scell), row_begin, row_end, g->p.kh, P<unsigned long long>(g->study),
                                    g->sm_count, s));
    unsigned long long h[6];
    SPH_CUDA(cudaMemcpyAsync(h, g->study.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    out->candidates = (int64_t)h[0];
    out->neighbours = (int64_t)h[1];
    out->wrong_fp16_abs = (int64_t)h[2];
    out->wrong_fp32_abs = (int64_t)h[3];
    out->wrong_fp16_rcll = (int64_t)h[4];
    out->wrong_tiered = (int64_t)h[5];
    return SPH_OK;
}

extern "C" int sph_grid_info_get(sph_grid_t grid, sph_grid_info *info) {
    sph_grid_s *g = grid;
    if (!g || !info) return fail(SPH_ERR_INVALID, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n = g->n;
    info->ncell = g->ncell;
    info->dim = g->p.dim;
    for (int k = 0; k < 3; ++k) {
        info->nk[k] = g->nk[k];
        info->lo[k] = g->lo[k];
    }
    info->cell_size = g->hc;
    info->cell_start = P<int>(g->cell_start);
    info->orig_id = P<int>(g->orig_id);
    info->rank = P<int>(g->rank);
    if (g->h_status) {
        info->stat_fp32_pairs = (int64_t)g->h_status->fp32_pairs;
        info->stat_fp64_pairs = (int64_t)g->h_status->fp64_pairs;
    }
    return SPH_OK;
}

extern "C" int sph_grid_export(sph_grid_t grid, int32_t *orig_id, int32_t *rank, int32_t *cell_start,
                               void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    if (orig_id && g->n)
        SPH_CUDA(copy_d2d_kernel(orig_id, g->orig_id.p, g->n * sizeof(int), s));
    if (rank && g->n)
        SPH_CUDA(copy_d2d_kernel(rank, g->rank.p, g->n * sizeof(int), s));
    if (cell_start && g->cell_start.p)
        SPH_CUDA(cudaMemcpyAsync(cell_start, g->cell_start.p, (g->ncell + 1) * sizeof(int),
                                 cudaMemcpyDeviceToDevice, s));
    return SPH_OK;
}

extern "C" int sph_grid_export_rel(sph_grid_t grid, uint16_t *rel16, float *rel32, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (g->p.precision != SPH_PREC_FP16_RCLL) return fail(SPH_ERR_INVALID, "the grid stores no relative coordinates");
    cudaStream_t s = (cudaStream_t)stream;
    if (rel16 && g->n)
        SPH_CUDA(cudaMemcpyAsync(rel16, g->rel16.p, g->n * sizeof(uint2), cudaMemcpyDeviceToDevice, s));
    if (rel32 && g->n)
        SPH_CUDA(cudaMemcpyAsync(rel32, g->rel32.p, g->n * sizeof(float4), cudaMemcpyDeviceToDevice, s));
    return SPH_OK;
}

extern "C" int sph_grid_set_option(sph_grid_t grid, int option, int64_t value) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (option == SPH_OPT_FUSED) {
        if (value < 0 || value > 2) return fail(SPH_ERR_INVALID, "SPH_OPT_FUSED takes 0, 1 or 2");
        g->fused_enabled = (int)value;
        return SPH_OK;
    }
    if (option == SPH_OPT_TILE_SHAPE) {
        if (value < -1 || value > 1) return fail(SPH_ERR_INVALID, "SPH_OPT_TILE_SHAPE takes -1, 0 or 1");
        g->tile_shape = (int)value;
        return SPH_OK;
    }
    if (option == SPH_OPT_SM_SHARE) {
        if (value < 1 || value > 100) return fail(SPH_ERR_INVALID, "SPH_OPT_SM_SHARE takes 1 .. 100 (percent)");
        g->sm_percent = (int)value;
        return SPH_OK;
    }
    if (option == SPH_OPT_TEST_LOOKBACK) {
        if (value < 0 || value > (1 << 20)) return fail(SPH_ERR_INVALID, "SPH_OPT_TEST_LOOKBACK takes 0 .. 2^20");
        g->test_lookback = (int)value;
        return SPH_OK;
    }
    if (option == SPH_OPT_STAGING) {
        if (value < -1 || value > 65536 || (value > 0 && value % 16 != 0))
            return fail(SPH_ERR_INVALID, "SPH_OPT_STAGING takes -1 or a multiple of 16 in [0, 65536]");
        g->staging = (int)value;
        return SPH_OK;
    }
    return fail(SPH_ERR_INVALID, "unknown option %d", option);
}

extern "C" int sph_grid_check(sph_grid_t grid, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    g->stream = (cudaStream_t)stream;
    if (!g->status.p) return SPH_OK;
    SPH_TRY(read_status(g));
    return status_to_code(g->h_status->flags);
}

extern "C" int sph_search_host(const sph_params *p, const double *xyz_host, int64_t n, float *rho_host,
                               int64_t *nnz_host, sph_grid_t *grid, void *stream) {
    if (!grid) return fail(SPH_ERR_INVALID, "grid is NULL");
    SPH_TRY(validate_params(p, n, xyz_host));
    cudaStream_t s = (cudaStream_t)stream;
    if (*grid == nullptr) SPH_TRY(grid_create(grid));
    sph_grid_s *g = *grid;
    g->stream = s;
    const size_t xbytes = (size_t)(n > 0 ? n : 1) * p->dim * sizeof(double);
    SPH_TRY(ensure(g->own_xyz, xbytes, s));
    if (n > 0) SPH_CUDA(cudaMemcpyAsync(g->own_xyz.p, xyz_host, (size_t)n * p->dim * sizeof(double),
                                        cudaMemcpyHostToDevice, s));
    SPH_TRY(sph_bin_cells(p, P<double>(g->own_xyz), n, stream, grid));
    SPH_TRY(ensure(g->own_rp, (size_t)(n + 1) * sizeof(long long), s));
    SPH_TRY(ensure(g->own_rho, (size_t)(n > 0 ? n : 1) * sizeof(float), s));
    int64_t nnz = 0;
    const long long cap = (long long)(g->own_col.cap / sizeof(int));
    int rc = sph_nnps_query(g, P<int64_t>(g->own_rp), g->own_col.p ? P<int32_t>(g->own_col) : nullptr, cap,
                            &nnz, g->own_col.p ? P<float>(g->own_rho) : nullptr, stream);
    if (rc == SPH_ERR_CAPACITY || (rc == SPH_OK && !g->own_col.p)) {
        SPH_TRY(ensure(g->own_col, (size_t)(nnz > 0 ? nnz : 1) * sizeof(int), s));
        rc = sph_nnps_query(g, P<int64_t>(g->own_rp), P<int32_t>(g->own_col),
                            (long long)(g->own_col.cap / sizeof(int)), &nnz, P<float>(g->own_rho), stream);
    }
    if (rc != SPH_OK) return rc;
    g->own_nnz = nnz;
    if (rho_host && n > 0)
        SPH_CUDA(cudaMemcpyAsync(rho_host, g->own_rho.p, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    if (nnz_host) *nnz_host = nnz;
    return SPH_OK;
}

extern "C" int sph_search_host_async(const sph_params *p, const double *xyz_host, int64_t n, float *rho_host,
                                     int64_t *nnz_host, sph_grid_t *grid, void *stream) {
    if (!grid) return fail(SPH_ERR_INVALID, "grid is NULL");
    SPH_TRY(validate_params(p, n, xyz_host));
    sph_grid_s *g = *grid;
    // the first call on a grid (or one with a different shape) sizes the
    // grid-owned CSR: the synchronous form does that and leaves nothing pending
    if (g == nullptr || g->async_pending || !g->own_col.p || g->n != n || g->p.dim != p->dim) {
        if (g && g->async_pending) SPH_TRY(sph_search_host_finish(g, nullptr));
        return sph_search_host(p, xyz_host, n, rho_host, nnz_host, grid, stream);
    }
    cudaStream_t s = (cudaStream_t)stream;
    g->stream = s;
    if (n > 0) SPH_CUDA(cudaMemcpyAsync(g->own_xyz.p, xyz_host, (size_t)n * p->dim * sizeof(double),
                                        cudaMemcpyHostToDevice, s));
    // binning reads the bounds back (this waits for the copy and the bounds
    // kernel of this stream only); the search then runs with the grid's column
    // capacity and no host read; the density and the status record (with nnz)
    // come back asynchronously
    SPH_TRY(sph_bin_cells(p, P<double>(g->own_xyz), n, stream, grid));
    const long long cap = (long long)(g->own_col.cap / sizeof(int));
    SPH_TRY(sph_nnps_query(g, P<int64_t>(g->own_rp), P<int32_t>(g->own_col), cap, nullptr, P<float>(g->own_rho),
                           stream));
    if (rho_host && n > 0)
        SPH_CUDA(cudaMemcpyAsync(rho_host, g->own_rho.p, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
    SPH_CUDA(status_to_host(g->h_status, P<DevStatus>(g->status), P<long long>(g->own_rp) + n, s));
    g->async_pending = true;
    g->async_nnz = nnz_host;
    return SPH_OK;
}

extern "C" int sph_search_host_finish(sph_grid_t grid, int64_t *nnz_host) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (!g->async_pending) {
        // nothing queued (the last call ran synchronously): its nnz
        if (nnz_host) *nnz_host = g->own_nnz;
        return SPH_OK;
    }
    g->async_pending = false;
    SPH_CUDA(cudaStreamSynchronize(g->stream));
    const long long nnz = g->h_status->nnz;
    int64_t *out = nnz_host ? nnz_host : g->async_nnz;
    if (out) *out = nnz;
    g->own_nnz = nnz;
    if (g->n > 0) g->last_nbr = (double)nnz / (double)g->n;
    int rc = status_to_code(g->h_status->flags & ~(unsigned)ST_CAPACITY);
    if (rc != SPH_OK) return rc;
    if (nnz > (long long)(g->own_col.cap / sizeof(int)))
        return fail(SPH_ERR_CAPACITY, "nnz %lld exceeds the grid's column buffer: call sph_search_host", nnz);
    return SPH_OK;
}

extern "C" int sph_grid_csr_copy(sph_grid_t grid, int64_t *row_ptr, int32_t *col, void *stream) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (!g->own_rp.p) return fail(SPH_ERR_INVALID, "the grid holds no sph_search_host result");
    cudaStream_t s = (cudaStream_t)stream;
    if (row_ptr)
        SPH_CUDA(cudaMemcpyAsync(row_ptr, g->own_rp.p, (size_t)(g->n + 1) * sizeof(int64_t), cudaMemcpyDefault, s));
    if (col && g->own_nnz > 0)
        SPH_CUDA(cudaMemcpyAsync(col, g->own_col.p, (size_t)g->own_nnz * sizeof(int32_t), cudaMemcpyDefault, s));
    SPH_CUDA(cudaStreamSynchronize(s));
    return SPH_OK;
}

extern "C" int sph_grid_csr(sph_grid_t grid, const int64_t **row_ptr, const int32_t **col, const float **rho,
                            int64_t *nnz) {
    sph_grid_s *g = grid;
    if (!g) return fail(SPH_ERR_INVALID, "grid is NULL");
    if (row_ptr) *row_ptr = P<int64_t>(g->own_rp);
    if (col) *col = P<int32_t>(g->own_col);
    if (rho) *rho = P<float>(g->own_rho);
    if (nnz) *nnz = g->own_nnz;
    return SPH_OK;
}

extern "C" int sph_profile_enable(int on) {
    prof_enable(on);
    return SPH_OK;
}

extern "C" int sph_profile_select(const char *kernels) {
    if (prof_select(kernels) != 0) return fail(SPH_ERR_INVALID, "unknown kernel tag in \"%s\"", kernels);
    return SPH_OK;
}

extern "C" int sph_device_fp64_rate(double *flops) {
    if (!flops) return fail(SPH_ERR_INVALID, "NULL argument");
    if (fp64_fma_rate(flops) != 0) {
        cudaGetLastError();
        return fail(SPH_ERR_CUDA, "FP64 rate measurement failed");
    }
    return SPH_OK;
}

extern "C" int sph_profile_reset(void) {
    prof_reset();
    return SPH_OK;
}

extern "C" int sph_profile_read(const char *kernel, double *total_ms, int64_t *launches) {
    if (!kernel) return fail(SPH_ERR_INVALID, "kernel name is NULL");
    long long c = 0;
    if (prof_read(kernel, total_ms, &c) != 0) return fail(SPH_ERR_NOT_FOUND, "unknown kernel tag %s", kernel);
    if (launches) *launches = c;
    return SPH_OK;
}

extern "C" int64_t sph_launch_count(void) { return launch_count(); }

namespace sph {

int grid_view(sph_grid_t grid, GridView *v) {
    sph_grid_s *g = grid;
    if (!g || !v) return fail(SPH_ERR_INVALID, "grid is NULL");
    v->d = make_dev(g);
    v->scell = P<int>(g->scell);
    v->sm_count = g->sm_count;
    v->precision = g->p.precision;
    v->order = g->p.order;
    v->n = g->n;
    v->nrow = (long long)g->nk[1] * g->nk[2];
    const TileLaunch tv =
        tile_choose_grid(g->last_nbr, g->n, g->ncell, g->p.dim, g->p.kh, g->hc, g->tile_shape, g->staging);
    v->tile_shape = tv.shape;
    v->tile_extra = tv.extra;
    return SPH_OK;
}

int set_error(int code, const char *msg) { return fail(code, "%s", msg); }

cudaError_t reset_counters_async(DevStatus *st, cudaStream_t s) { return launch_status_reset_counters(st, s); }

}  // namespace sph

extern "C" int sph_grid_free(sph_grid_t grid) {
    sph_grid_s *g = grid;
    if (!g) return SPH_OK;
    cudaStream_t s = g->stream;
    DevBuf *bufs[] = {&g->cell_start, &g->cnt, &g->cid, &g->slot, &g->orig_id, &g->rank, &g->scell,
                      &g->rel16, &g->rel32, &g->rel16u, &g->rel32u, &g->rel64, &g->rel64u, &g->fsplit, &g->study, &g->x64, &g->scan_tmp, &g->big_list,
                      &g->rowcnt, &g->tmp_rp, &g->tmp_col, &g->tmp_rho, &g->status, &g->own_xyz, &g->own_rp, &g->own_col, &g->own_rho,
                      &g->tstate, &g->scell_x, &g->tcount, &g->toff, &g->tiles};
    for (DevBuf *b : bufs) release(*b, s);
    if (g->h_status) {
        cudaStreamSynchronize(s);
        cudaFreeHost(g->h_status);
    }
    cudaGetLastError();
    delete g;
    return SPH_OK;
}
