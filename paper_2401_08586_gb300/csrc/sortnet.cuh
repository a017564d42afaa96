// sortnet.cuh -- sorting networks for short segments of int keys: one warp
// in registers (up to 32 keys) and a compare-exchange network over any
// memory run by cooperating threads.  Every comparator puts the minimum at
// the lower index (the first step of each merge compares i with i ^ (k - 1)),
// so positions past the segment end behave as +infinity and are skipped.
#pragma once

namespace sph {
namespace net {

// One warp sorts keys[0, len) (len <= 32) held one per lane.
__device__ __forceinline__ int warp_sort32(int v, int lane, int len) {
    const int INF = 0x7fffffff;
    if (lane >= len) v = INF;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            int partner = (j == (k >> 1)) ? (lane ^ (k - 1)) : (lane ^ j);
            int o = __shfl_sync(0xffffffffu, v, partner);
            bool lower = lane < partner;
            v = lower ? min(v, o) : max(v, o);
        }
    }
    return v;
}

// Compare-exchange network over keys[0, len) in any memory, executed by
// `nthr` cooperating threads with index `t`; `sync` orders the steps.
template <typename Sync>
__device__ void bitonic_all_ascending(int *keys, long long len, int t, int nthr, Sync sync) {
    long long P = 1;
    while (P < len) P <<= 1;
    for (long long k = 2; k <= P; k <<= 1) {
        for (long long j = k >> 1; j > 0; j >>= 1) {
            for (long long i = t; i < P; i += nthr) {
                long long partner = (j == (k >> 1)) ? (i ^ (k - 1)) : (i ^ j);
                if (partner > i && partner < len) {
                    int a = keys[i], b = keys[partner];
                    if (a > b) {
                        keys[i] = b;
                        keys[partner] = a;
                    }
                }
            }
            sync();
        }
    }
}

struct WarpSync {
    __device__ void operator()() const { __syncwarp(); }
};
struct BlockSync {
    __device__ void operator()() const { __syncthreads(); }
};

}  // namespace net
}  // namespace sph
