// lookback.cuh -- decoupled look-back: the exclusive prefix of a unit's total
// over all earlier units, where units (tiles of a search, chunks of rows,
// tiles of a scan) are taken in ticket order by running warps.  Each unit
// publishes its total as soon as it knows it, then sums the published states
// of its predecessors 32 at a time, stopping at the first inclusive prefix.
// State word per unit: flag in the top two bits (0 not yet published, 1
// aggregate, 2 inclusive prefix), value below.  The states of a launch must
// start at zero.
#pragma once

#include "sph_internal.cuh"

namespace sph {
namespace lb {

constexpr unsigned long long ST_AGG = 1ull << 62;
constexpr unsigned long long ST_INCL = 2ull << 62;
constexpr unsigned long long ST_VAL = (1ull << 62) - 1;
constexpr int LOOKBACK_SPIN_LIMIT = 1 << 20;

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}

// Publish unit t's total (an aggregate, or already the inclusive prefix for
// unit 0).  Successors can use it before unit t has resolved its own prefix.
// Called by a whole warp.
__device__ __forceinline__ void look_back_publish(unsigned long long *tstate, long long t, long long agg) {
    if ((threadIdx.x & 31) == 0)
        atomicExch(&tstate[t], (t == 0 ? ST_INCL : ST_AGG) | (unsigned long long)agg);
}

// Sum of all earlier units' totals, by looking back over their published
// states 32 at a time (stopping at the first inclusive prefix); then publish
// unit t's inclusive prefix.  Called by a whole warp.  Every wait is bounded:
// after spin_limit polls (each at most ~1 us apart) the unit records
// ST_TIMEOUT in *flags, publishes the prefix it has (so later units do not
// wait on the missing one) and continues.
__device__ __forceinline__ long long look_back_resolve(unsigned long long *tstate, long long t, long long agg,
                                                       unsigned int *flags, int spin_limit = LOOKBACK_SPIN_LIMIT) {
    const int lane = threadIdx.x & 31;
    if (t == 0) return 0;
    long long excl = 0, j = t - 1;
    int spins = 0, backoff = 32;
    bool timed_out = false;
    while (true) {
        const long long idx = j - lane;
        const unsigned long long s = idx >= 0 ? ld_volatile(&tstate[idx]) : ST_INCL;
        const unsigned int flag = (unsigned int)(s >> 62);
        const unsigned int m2 = __ballot_sync(0xffffffffu, flag == 2u);
        const unsigned int m0 = __ballot_sync(0xffffffffu, flag == 0u);
        const int stop = m2 ? __ffs(m2) - 1 : 31;
        const unsigned int need = stop == 31 ? 0xffffffffu : ((2u << stop) - 1u);
        if (m0 & need) {
            if (++spins > spin_limit) {
                timed_out = true;
                break;
            }
            __nanosleep(backoff);
            backoff = min(backoff * 2, 1024);
            continue;
        }
        long long v = lane <= stop ? (long long)(s & ST_VAL) : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        excl += v;
        if (m2) break;
        j -= 32;
        backoff = 32;
    }
    if (timed_out && lane == 0) atomicOr(flags, ST_TIMEOUT);
    if (lane == 0) atomicExch(&tstate[t], ST_INCL | (unsigned long long)(excl + agg));
    return excl;
}

}  // namespace lb
}  // namespace sph
