// Host-only test shim for the row tiles of the single-pass search
// (row_tile_end and tiles_max in paper_2401_08586_gb300/csrc/sph_internal.cuh),
// built by tests/test_tile_cuts.py with nvcc (the header is CUDA source).
#include "../../paper_2401_08586_gb300/csrc/sph_internal.cuh"

extern "C" int tc_tile_rows() { return sph::TILE_ROWS; }
extern "C" int tc_tile_span() { return sph::TILE_SPAN; }

// Cuts one row (cs: its nx + 1 cell starts) into tiles as the tile-list
// builder does; writes the end of every tile to ends (at most cap) and
// returns the number of tiles.
extern "C" int tc_cut_row(const int *cs, int nx, int *ends, int cap) {
    int count = 0, c = 0;
    for (int p = cs[0]; p < cs[nx]; ++count) {
        p = sph::row_tile_end(cs, nx, p, c);
        if (count < cap) ends[count] = p;
    }
    return count;
}

extern "C" long long tc_tiles_max(long long n, long long ncell, long long nrow) {
    return sph::tiles_max(n, ncell, nrow);
}
