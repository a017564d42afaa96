// tile_rows.cuh -- the candidate rows of a row tile, shared by the FP16 and
// FP64 tile searches: the 3^d rows of cells around the tile's row (cy, cz)
// (3 in 2D), each the contiguous sorted range of cells [xlo, xhi] (the
// tile's cells widened by one per side; cell link-list, same and adjacent
// cells only).
#pragma once

#include "sph_internal.cuh"

namespace sph {

// For each candidate row r: rt[r] = (sorted index minus the flat index of
// the row's first candidate, code bits (dy + 1) << 3 | (dz + 1) << 5, frame
// shifts 2 dy and 2 dz as float bits), rcum[r] = candidates in rows before r
// (rcum[nrows] = all).  Called by a whole warp; ends with __syncwarp.
template <int DIM>
__device__ __forceinline__ void tile_candidate_rows(int4 *rt, int *rcum, const GridDev &g, int cy, int cz, int xlo,
                                                    int xhi) {
    constexpr int NROWS = DIM == 3 ? 9 : 3;
    const int lane = threadIdx.x & 31;
    const int nx = g.nk[0], ny = g.nk[1], nz = g.nk[2];
    // lane 2r + e loads the start (e = 0) or end (e = 1) of row r
    int v = -1;
    const int r = lane >> 1, e = lane & 1;
    if (r < NROWS) {
        const int dy = DIM == 3 ? (r % 3) - 1 : r - 1;
        const int dz = DIM == 3 ? (r / 3) - 1 : 0;
        const int yy = cy + dy, zz = cz + dz;
        if (yy >= 0 && yy < ny && zz >= 0 && zz < nz)
            v = g.cell_start[((long long)zz * ny + yy) * nx + (e ? xhi + 1 : xlo)];
    }
    const int vend = __shfl_down_sync(0xffffffffu, v, 1);
    const int mylen = (e == 0 && v >= 0) ? vend - v : 0;
    // rows to lanes 0 .. NROWS-1: start and length
    const int src = 2 * (lane < NROWS ? lane : 0);
    const int st = __shfl_sync(0xffffffffu, v, src);
    int len = __shfl_sync(0xffffffffu, mylen, src);
    if (lane >= NROWS) len = 0;
    // flat index of the candidates: rcum[r] = candidates in rows before r
    int inc = len;
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
        const int up = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += up;
    }
    if (lane < NROWS) {
        const int dy = DIM == 3 ? (lane % 3) - 1 : lane - 1;
        const int dz = DIM == 3 ? (lane / 3) - 1 : 0;
        rt[lane] = make_int4((st >= 0 ? st : 0) - (inc - len), ((dy + 1) << 3) | ((dz + 1) << 5),
                             __float_as_int(2.f * (float)dy), __float_as_int(2.f * (float)dz));
        rcum[lane + 1] = inc;
    }
    if (lane == 0) rcum[0] = 0;
    __syncwarp();
}

// Row of flat candidate index k: the rows before it end at or below k.
template <int DIM>
__device__ __forceinline__ int tile_row_of(int k, const int (&rc)[DIM == 3 ? 9 : 3]) {
    constexpr int NROWS = DIM == 3 ? 9 : 3;
    int r = 0;
#pragma unroll
    for (int t = 0; t < NROWS - 1; ++t) r += k >= rc[t] ? 1 : 0;
    return r;
}

}  // namespace sph
