// advance.cu -- the mixed-precision time step of Eq. 8-9 (arXiv 2401.08586,
// "Mixed-precision SPH framework"): the cell-relative coordinates are
// advanced by the displacement itself, x_rel += 2 v dt / h_c, instead of
// being converted again from the absolute coordinates; a coordinate that
// leaves [-1, 1] moves its particle to the adjacent cell (by as many cells as
// it takes) and is shifted back by 2 per cell.
//
// The relative coordinates are kept in FP64 (rel64, cell order) and rounded
// once to FP16 / FP32 after each step, exactly as binning rounds them.  The
// new cells are then put in order by the integer half of binning (histogram,
// scan, scatter, per-cell sort, gather): no bounds pass, no FP64 conversion.
#include "cellcount.cuh"
#include "launch.cuh"
#include "profile.cuh"
#include "sph_internal.cuh"

namespace sph {
namespace {

__device__ __forceinline__ void cell_xyz(const GridDev &g, int c, int cc[3]) {
    cell_decompose(g, c, cc[0], cc[1], cc[2]);
}

// RN32(a) from the bits of a for 2^-95 <= |a| < 2^101: the significand is
// normalised to bit 63, every bit below the top 32 is ORed into the lowest
// of them (sticky: the FP32 rounding looks at no more than the 8 bits below
// its 24), the 32-bit value is converted and scaled by an exact power of two.
// Other values (zero, tiny, huge, non-finite) take the FP64 conversion.
__device__ __forceinline__ float f64_to_f32_rn(double a) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(a);
    const int e = (int)((b >> 52) & 0x7ffull) - 1023;
    if (e < -95 || e > 100) return __double2float_rn(a);
    const unsigned long long t = ((b & ((1ull << 52) - 1ull)) | (1ull << 52)) << 11;
    const unsigned int hi = (unsigned int)(t >> 32) | ((unsigned int)t != 0u ? 1u : 0u);
    const float r = __uint2float_rn(hi) * __int_as_float((96 + e) << 23);
    return (b >> 63) ? -r : r;
}

// rel64[s] from the positions, each particle in its current cell:
// s_k = 2 (x_k - lo_k) / h_c, a_k = s_k - (2 c_k + 1) (the binning formula).
__global__ void k_rel64_sync(GridDev g, const int *__restrict__ scell, const double *__restrict__ xyz,
                             double4_32a *__restrict__ rel64) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.n;
         s += (long long)gridDim.x * blockDim.x) {
        const int i = g.orig_id[s];
        int cc[3];
        cell_xyz(g, scell[s], cc);
        double a[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < g.dim; ++k) {
            const double sk = __dmul_rn(__dsub_rn(xyz[(long long)i * g.dim + k], g.lo[k]), g.two_over_hc);
            a[k] = __dsub_rn(sk, (double)(2 * cc[k] + 1));
        }
        rel64[s] = make_double4_32a(a[0], a[1], a[2], 0.0);
    }
}

// Eq. 8 with the displacement of Eq. 9 for every sorted particle, its new
// cell, the warp-aggregated histogram of the new cells, and the rounded
// relative coordinates, all in input order for the gather of the re-sort.
template <int DIM>
__global__ void k_advance(GridDev g, const int *__restrict__ scell, const double4_32a *__restrict__ rel64,
                          const double *__restrict__ vel, double dt, int *__restrict__ cnt, int *__restrict__ cid,
                          int *__restrict__ slot, uint2 *__restrict__ rel16u, float4 *__restrict__ rel32u,
                          double4_32a *__restrict__ rel64u) {
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < g.n; base += (long long)gridDim.x * blockDim.x) {
        const long long s = base + threadIdx.x;
        const bool live = s < g.n;
        int c = -1, i = 0;
        bool out = false, bad = false;
        unsigned long long dkey_max = 0ull;
        if (live) {
            i = g.orig_id[s];
            int cc[3];
            cell_xyz(g, scell[s], cc);
            const double4_32a r = rel64[s];
            double a[3] = {r.x, r.y, r.z};
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                const double d = __dmul_rn(vel[(long long)i * DIM + k], dt);  // Eq. 9
                unsigned long long db = (unsigned long long)__double_as_longlong(d) & 0x7fffffffffffffffull;
                dkey_max = db > dkey_max ? db : dkey_max;  // |d| as bits: order-preserving for d >= 0
                a[k] = __fma_rn(d, g.two_over_hc, a[k]);   // Eq. 8 in units of u = h_c / 2
                bad |= ((__double_as_longlong(a[k]) >> 52) & 0x7ff) == 0x7ff;
                // cells crossed: floor((a + 1) / 2), none while |a| < 1 (the
                // common case, told from the exponent without FP64 work); the
                // remainder is exact (a conversion that saturates only
                // happens far outside the grid)
                int sh = 0;
                if (!bad && ((__double_as_longlong(a[k]) >> 52) & 0x7ff) >= 1023) {
                    sh = __double2int_rd(__dmul_rn(__dadd_rn(a[k], 1.0), 0.5));
                    a[k] = __dsub_rn(a[k], 2.0 * (double)sh);
                }
                const long long ck = (long long)cc[k] + sh;
                if (ck < 0 || ck >= g.nk[k]) out = true;
                cc[k] = (int)(ck < 0 ? 0 : (ck >= g.nk[k] ? g.nk[k] - 1 : ck));
            }
            c = (cc[2] * g.nk[1] + cc[1]) * g.nk[0] + cc[0];
            rel64u[i] = make_double4_32a(a[0], a[1], a[2], 0.0);
            uint2 q;
            float4 f;
            round_rel_f(f64_to_f32_rn(a[0]), f64_to_f32_rn(a[1]), f64_to_f32_rn(a[2]), cc[0], q, f);
            rel16u[i] = q;
            rel32u[i] = f;
        }
        if (__any_sync(0xffffffffu, out) && lane == 0) atomicOr(&g.status->flags, ST_OUT_OF_BOX);
        if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(&g.status->flags, ST_NONFINITE);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long v = __shfl_xor_sync(0xffffffffu, dkey_max, o);
            dkey_max = v > dkey_max ? v : dkey_max;
        }
        if (lane == 0 && dkey_max) atomicMax(&g.status->max_key[0], dkey_max);
        const int sl = cell_run_slot(c, live, cnt);
        if (live) {
            cid[i] = c;
            slot[i] = sl;
        }
    }
}

unsigned grid_blocks(long long n, int nt, int sm_count) {
    long long b = (n + nt - 1) / nt;
    if (b > (long long)sm_count * 16) b = (long long)sm_count * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

}  // namespace

cudaError_t launch_rel64_sync(const GridDev &g, const int *scell, const double *xyz, double4_32a *rel64, int sm_count,
                              cudaStream_t s) {
    ProfScope ps(TAG_CONVERT, s);
    note_launch(1);
    k_rel64_sync<<<grid_blocks(g.n, 256, sm_count), 256, 0, s>>>(g, scell, xyz, rel64);
    return cudaGetLastError();
}

cudaError_t launch_advance(const GridDev &g, const int *scell, const double4_32a *rel64, const double *vel, double dt,
                           int *cnt, int *cid, int *slot, uint2 *rel16u, float4 *rel32u, double4_32a *rel64u,
                           int sm_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(cnt, 0, cnt_bytes(g.ncell), s);  // counters and their scan state
    if (e != cudaSuccess) return e;
    ProfScope ps(TAG_HASH, s);
    note_launch(1);
    (g.dim == 2 ? k_advance<2> : k_advance<3>)<<<grid_blocks(g.n, 256, sm_count), 256, 0, s>>>(g, scell, rel64, vel, dt, cnt, cid, slot, rel16u,
                                                              rel32u, rel64u);
    return cudaGetLastError();
}

}  // namespace sph
