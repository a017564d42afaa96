// fastdiv.h -- division of non-negative 32-bit integers by a divisor fixed
// for a whole launch, as a multiply-high and shifts (Granlund and Montgomery,
// "Division by invariant integers using multiplication", PLDI 1994, the
// round-up method for unsigned division).  For d >= 1 with l = ceil(log2 d):
//   m = floor(2^32 (2^l - d) / d) + 1,  t = mulhi(m, n),
//   n / d = (t + ((n - t) >> 1)) >> (l - 1)   (l >= 1),  n / 1 = n,
// exact for every 32-bit unsigned n.  Host and device; no CUDA headers.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define SPH_HD __host__ __device__ __forceinline__
#else
#define SPH_HD inline
#endif

namespace sph {

struct FastDiv {
    uint32_t d, m;
    int32_t l;
};

inline FastDiv fastdiv_make(uint32_t d) {
    FastDiv f;
    f.d = d;
    int l = 0;
    while (l < 32 && ((uint64_t)1 << l) < d) ++l;
    f.l = l;
    f.m = (uint32_t)((((uint64_t)1 << 32) * (((uint64_t)1 << l) - d)) / d + 1);
    return f;
}

SPH_HD uint32_t fastdiv_mulhi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

SPH_HD uint32_t fastdiv_div(uint32_t n, const FastDiv &f) {
    if (f.l == 0) return n;
    const uint32_t t = fastdiv_mulhi(f.m, n);
    return (t + ((n - t) >> 1)) >> (f.l - 1);
}

}  // namespace sph
