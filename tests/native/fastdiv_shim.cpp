// Host-only test shim for paper_2401_08586_gb300/csrc/fastdiv.h, built by
// tests/test_fastdiv.py with the host compiler.
#include <stdint.h>

#include "../../paper_2401_08586_gb300/csrc/fastdiv.h"

// Checks n / d for the given n against the division operator; returns the
// number of mismatches.
extern "C" long long fd_check(uint32_t d, const uint32_t *n, long long count) {
    const sph::FastDiv f = sph::fastdiv_make(d);
    long long bad = 0;
    for (long long k = 0; k < count; ++k) bad += sph::fastdiv_div(n[k], f) != n[k] / d;
    return bad;
}
