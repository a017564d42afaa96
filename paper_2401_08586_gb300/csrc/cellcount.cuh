// cellcount.cuh -- per-cell counting of a warp's particles during binning,
// shared by the single-grid, batched and time-step hash kernels.
#pragma once

namespace sph {

// Slot of each live lane among its cell's particles: every run of
// consecutive lanes with the same cell adds its length to cnt[c] once and
// its lanes take consecutive slots from the count it found.  Input in
// spatial order puts a cell's particles in runs; any order stays correct (a
// cell split over several runs takes one atomic per run, and the per-cell
// sort afterwards restores input order).  Dead lanes (live false) must be
// the warp's last lanes and hold a cell no live lane holds (-1).  Called by
// a whole warp.
__device__ __forceinline__ int cell_run_slot(int c, bool live, int *cnt) {
    const int lane = threadIdx.x & 31;
    const int up = __shfl_up_sync(0xffffffffu, c, 1);
    const unsigned int heads = __ballot_sync(0xffffffffu, lane == 0 || up != c);
    const unsigned int upto = 0xffffffffu >> (31 - lane);  // lanes 0 .. lane
    const int head = 31 - __clz(heads & upto);              // first lane of this lane's run
    const unsigned int later = heads & ~upto;
    const int end = later ? __ffs(later) - 1 : 32;          // one past the run
    int old = 0;
    if (live && lane == head) old = atomicAdd(&cnt[c], end - head);
    old = __shfl_sync(0xffffffffu, old, head);
    return old + (lane - head);
}

}  // namespace sph
