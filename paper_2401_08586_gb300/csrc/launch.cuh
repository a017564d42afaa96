// launch.cuh -- host launchers of the library's kernels, one per step of the
// path (defined next to their kernels: bin.cu, search.cu, nnps_fused.cu,
// nnps_tile.cu, batch.cu).  All enqueue on stream s and return the launch
// status; none synchronises.
#pragma once

#include "sph_internal.cuh"

namespace sph {

// Blocks of kernel `kern` (nt threads, smem bytes of dynamic shared memory)
// that one SM holds at once, at least 1 (the per-cell sort of binning runs
// one wave of these).
inline int resident_blocks(const void *kern, int nt, size_t smem = 0) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, nt, smem) != cudaSuccess) {
        (void)cudaGetLastError();  // a failed query is not a launch error: the threads' limit
        b = 2048 / nt;
    }
    return b < 1 ? 1 : b;
}

// Binning (bin.cu).
cudaError_t launch_bounds(const double *xyz, long long n, int dim, DevStatus *st, int sm_count, cudaStream_t s);
cudaError_t launch_hash_scatter_convert(const GridDev &g, const double *xyz, int n, int dim, int prec, int *cnt,
                                        int *cid, int *slot, int *cell_start, int *orig_id, int *rank, int *scell,
                                        uint2 *rel16, float4 *rel32, uint2 *rel16u, float4 *rel32u, double4_32a *x64,
                                        int *scell_x, void *scan_tmp, int *big_list, unsigned int *big_count,
                                        int check_box, int sm_count, cudaStream_t s);
// Scan of the cell histogram, scatter, per-cell sort and the gather of the
// input-order arrays (cid, rel16u, rel32u and, if not NULL, rel64u) into
// cell order: the second half of binning, shared with the time step.  cnt
// has cnt_bytes(ncell) bytes, cleared (with its scan state) before the
// histogram was counted.
cudaError_t launch_order_convert(const GridDev &g, int n, int dim, int prec, int *cnt, int *cid, int *slot,
                                 int *cell_start, int *orig_id, int *rank, int *scell, uint2 *rel16, float4 *rel32,
                                 const uint2 *rel16u, const float4 *rel32u, const double4_32a *rel64u, double4_32a *rel64,
                                 double4_32a *x64, int *scell_x, void *scan_tmp, int *big_list, unsigned int *big_count,
                                 int sm_count, cudaStream_t s);
cudaError_t launch_scatter(int n, const int *cell_start, const int *cid, const int *slot, int *orig_id,
                           int sm_count, cudaStream_t s);

// Time step of Eq. 8-9 (advance.cu).  Relative coordinates of the sorted
// particles (rel64) advanced by 2 v dt / h_c, cell shifts where they leave
// [-1, 1]; input-order outputs (cid, slot with the histogram cnt, rel16u,
// rel32u, rel64u) ready for launch_order_convert.  Status: ST_OUT_OF_BOX when
// a particle leaves the grid, max |v dt| as a key in max_key[0].
cudaError_t launch_advance(const GridDev &g, const int *scell, const double4_32a *rel64, const double *vel, double dt,
                           int *cnt, int *cid, int *slot, uint2 *rel16u, float4 *rel32u, double4_32a *rel64u,
                           int sm_count, cudaStream_t s);
// FP64 relative coordinates of the sorted particles from positions xyz in
// their current cells (the conversion of binning, cells unchanged).
cudaError_t launch_rel64_sync(const GridDev &g, const int *scell, const double *xyz, double4_32a *rel64, int sm_count,
                              cudaStream_t s);

// Two-pass search, unfused density, canonical order (search.cu).
cudaError_t launch_nnps(const GridDev &g, int prec, int mode_fill, int *cnt, const long long *row_ptr, int *col,
                        long long cap, float *rho, int sm_count, cudaStream_t s);
cudaError_t launch_density(const GridDev &g, int prec, const int *rank, const int *scell, const long long *row_ptr,
                           const int *col, int canonical, float *rho, int sm_count, cudaStream_t s);
cudaError_t launch_canon(int n, const int *rank, const int *orig_id, const long long *rp_cell, const int *col_cell,
                         const float *rho_cell, int *cnt_tmp, void *scan_tmp, long long *rp, int *col, float *rho,
                         int *big_list, unsigned int *big_count, int sm_count, cudaStream_t s);

// Appendix Eq. A5 gradient over a CSR (gradient.cu); fs: float2 scratch of n.
// Summation density over a half stencil, rho in sorted order (density_half.cu).
cudaError_t launch_density_half(const GridDev &g, const int *scell, float *rho, int sm_count, cudaStream_t s);
// Half-stencil CSR (density_half.cu): row lengths into cnt (zeroed here) and
// the density (rho != NULL); then both entries of every pair at the row
// cursors cur (a copy of the row starts), rows unsorted.
cudaError_t launch_half_count(const GridDev &g, const int *scell, int *cnt, float *rho, int sm_count, cudaStream_t s);
cudaError_t launch_half_fill(const GridDev &g, const int *scell, unsigned long long *cur, int *col, int sm_count,
                             cudaStream_t s);
cudaError_t launch_gradient_a5(const GridDev &g, const int *rank, const int *scell, const long long *row_ptr,
                               const int *col, int canonical, const double *f, float2 *fs, double *grad,
                               int sm_count, cudaStream_t s);

// Precision study of the neighbour decision (study.cu): out[0..5] =
// candidates, neighbours, wrong FP16 absolute, wrong FP32 absolute, wrong
// FP16 RCLL alone, wrong tiered; rows restricted to input indices
// [row_begin, row_end).
cudaError_t launch_precision_study(const GridDev &g, const int *scell, long long row_begin, long long row_end,
                                   double kh, unsigned long long *out, int sm_count, cudaStream_t s);

// Single-pass search, one CTA per cell (nnps_fused.cu).
cudaError_t launch_nnps_fused(const GridDev &g, long long *row_ptr, int *col, long long cap, float *rho,
                              unsigned long long *tstate, int *rowcnt, int sm_count, cudaStream_t s);

// Single-pass search, one warp per row tile (nnps_tile.cu).
// Tile list: span_limited tiles (at most TILE_SPAN cells each; the search's
// own list) or plain runs of 32 particles per row (the no-allocation path,
// whose fixed scratch bounds the tile count by n / 32 + nrow + 1).  cstate
// (nrow + 1 zeroed entries, or nullptr): build the list in one launch with a
// look-back over chunks of rows instead of count, scan and write.
cudaError_t launch_tiles(const GridDev &g, bool span_limited, int *tcount, long long *toff, void *scan_tmp,
                         int4 *tiles, unsigned long long *cstate, int sm_count, cudaStream_t s);
// Shared-memory shape of a tile-search launch: TILE_SPARSE (672 kept
// candidates per pass, 20 warps per SM) or TILE_DENSE (832, 16 per SM), and
// extra dynamic shared memory for output staging.
enum { TILE_SPARSE = 0, TILE_DENSE = 1 };
struct TileLaunch {
    int shape;
    int extra;
    int sm_percent = 100;  // share of the device's resident CTA slots the persistent grid takes (1 .. 100)
};
cudaError_t launch_nnps_tile(const GridDev &g, const GridDev *gsys, const int4 *tiles, const long long *ntiles_dev,
                             long long ntiles_max, long long *row_ptr, int *col, long long cap, float *rho,
                             unsigned long long *tstate, TileLaunch v, bool zeroed, int sm_count, cudaStream_t s);
// The same search with the FP64 test and density on the cell-ordered FP64
// coordinates (SPH_PREC_FP64_CLL grids; nnps_tile64.cu); tstate zeroed.
cudaError_t launch_nnps_tile64(const GridDev &g, const int4 *tiles, const long long *ntiles_dev,
                               long long ntiles_max, long long *row_ptr, int *col, long long cap, float *rho,
                               unsigned long long *tstate, int sm_count, cudaStream_t s);
// Shape (shape < 0: chosen from nbr) and staging for about nbr neighbours per particle.
TileLaunch tile_choose(double neighbours_per_particle, int shape);
// The same for a grid: its last measured neighbours per particle (else the
// uniform-density estimate) and its SPH_OPT_TILE_SHAPE / SPH_OPT_STAGING settings.
TileLaunch tile_choose_grid(double last_nbr, long long n, long long ncell, int dim, double kh, double hc,
                            int tile_shape, int staging, int sm_percent = 100);

}  // namespace sph
