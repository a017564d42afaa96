// density_half.cu -- the half-stencil forms of the search.
//
// Summation density (Eq. 3) over a half stencil: every
// pair of particles is tested once, from the particle whose cell comes first
// (or, in one cell, from the lower sorted index), and its weight is added to
// both densities.  This is the reuse of computed distances that the paper's
// conclusions ("Conclusions and discussions") point to, for callers that
// need the density but not the neighbour list: the full CSR cannot be
// emitted this way without writing every pair a second time into another
// particle's row.
//
// Forward cells of a particle in cell (cx, cy, cz): its own cell after it and
// the cell at +x (contiguous in sorted order), the three cells of the row at
// +y, and in 3D the nine cells of the plane at +z: 13 in 3D, 4 in 2D, the
// half of the 3^d - 1 neighbour cells whose offset is positive in
// (z, y, x) order.  Each unordered pair is visited exactly once.
//
// The neighbour decision is the search's: FP32 distance from the FP32
// relative coordinates with the cell offset, and the FP64 definition on the
// caller's coordinates inside the FP32 band, so the pairs are exactly those
// of the FP64 definition.  The partner's share is added with an FP32 atomic:
// the densities match the FP64 oracle within the search's tolerance, but the
// order of the FP32 additions (and so the last bits) is not fixed.
//
// The neighbour list over the same half stencil (sph_nnps_query_half): a
// count pass (each pair decided once, the row lengths of both particles
// incremented, the density as above), a scan of the row lengths, a fill pass
// that decides every pair again and writes it into both rows at atomic row
// cursors, and a per-row sort that restores ascending columns.  The result is
// the search's CSR exactly; it is kept to measure what the half stencil costs
// when the full CSR is wanted.
#include "launch.cuh"
#include "nnps_common.cuh"
#include "profile.cuh"

namespace sph {

namespace {

using namespace nn;

// The self term m W(0, h) of every particle.
__global__ void k_density_self(long long n, float w0, float *__restrict__ rho) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (long long)gridDim.x * blockDim.x)
        rho[s] = w0;
}

template <int DIM>
__global__ void __launch_bounds__(256) k_density_half(GridDev g, const int *__restrict__ scell,
                                                      float *__restrict__ rho) {
    const int nx = g.nk[0], ny = g.nk[1], nz = g.nk[2];
    unsigned int n32 = 0, n64 = 0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.n;
         s += (long long)gridDim.x * blockDim.x) {
        const int i = (int)s;
        int cx, cy, cz;
        cell_decompose(g, scell[i], cx, cy, cz);
        const float4 ri = g.rel32[i];
        float acc = 0.f;
        // rows of forward cells: (dy, dz) = (0, 0) from i + 1 through the
        // cell at +x; (1, 0) over x - 1 .. x + 1; in 3D (-1..1, 1) likewise
        constexpr int NROW = DIM == 3 ? 5 : 2;
#pragma unroll 1
        for (int r = 0; r < NROW; ++r) {
            const int dy = r == 0 ? 0 : (r == 1 ? 1 : r - 3);
            const int dz = r < 2 ? 0 : 1;
            const int yy = cy + dy, zz = cz + dz;
            if (yy >= ny || zz >= nz || yy < 0) continue;
            const long long rowc = ((long long)zz * ny + yy) * nx;
            const int xb = min(cx + 1, nx - 1);
            const int j0 = r == 0 ? i + 1 : g.cell_start[rowc + max(cx - 1, 0)];
            const int j1 = g.cell_start[rowc + xb + 1];
            const float sy = 2.f * (float)dy, sz = 2.f * (float)dz;
            for (int j = j0; j < j1; ++j) {
                const float sx = 2.f * (float)(g.scell_x[j] - cx);
                float r2;
                if (decide_fp32<DIM>(g, ri, g.rel32[j], sx, sy, sz, i, j, &r2, n32, n64)) {
                    const float w = g.w_norm * w_poly(sqrtf(r2) * g.r_scale);
                    acc += w;
                    atomicAdd(&rho[j], w);
                }
            }
        }
        atomicAdd(&rho[i], acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n32 += __shfl_xor_sync(0xffffffffu, n32, o);
        n64 += __shfl_xor_sync(0xffffffffu, n64, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n32) atomicAdd(&g.status->fp32_pairs, (unsigned long long)n32);
        if (n64) atomicAdd(&g.status->fp64_pairs, (unsigned long long)n64);
    }
}

// The forward pairs of particle i (its neighbours in the forward cells, each
// unordered pair once), decided as the search decides them: f(j, r2) for
// each.
template <int DIM, class F>
__device__ __forceinline__ void forward_pairs(const GridDev &g, const int *scell, int i, unsigned int &n32,
                                              unsigned int &n64, F f) {
    const int nx = g.nk[0], ny = g.nk[1], nz = g.nk[2];
    int cx, cy, cz;
    cell_decompose(g, scell[i], cx, cy, cz);
    const float4 ri = g.rel32[i];
    constexpr int NROW = DIM == 3 ? 5 : 2;
#pragma unroll 1
    for (int r = 0; r < NROW; ++r) {
        const int dy = r == 0 ? 0 : (r == 1 ? 1 : r - 3);
        const int dz = r < 2 ? 0 : 1;
        const int yy = cy + dy, zz = cz + dz;
        if (yy >= ny || zz >= nz || yy < 0) continue;
        const long long rowc = ((long long)zz * ny + yy) * nx;
        const int xb = min(cx + 1, nx - 1);
        const int j0 = r == 0 ? i + 1 : g.cell_start[rowc + max(cx - 1, 0)];
        const int j1 = g.cell_start[rowc + xb + 1];
        const float sy = 2.f * (float)dy, sz = 2.f * (float)dz;
        for (int j = j0; j < j1; ++j) {
            const float sx = 2.f * (float)(g.scell_x[j] - cx);
            float r2;
            if (decide_fp32<DIM>(g, ri, g.rel32[j], sx, sy, sz, i, j, &r2, n32, n64)) f(j, r2);
        }
    }
}

__device__ __forceinline__ void add_tier_counts(const GridDev &g, unsigned int n32, unsigned int n64) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n32 += __shfl_xor_sync(0xffffffffu, n32, o);
        n64 += __shfl_xor_sync(0xffffffffu, n64, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n32) atomicAdd(&g.status->fp32_pairs, (unsigned long long)n32);
        if (n64) atomicAdd(&g.status->fp64_pairs, (unsigned long long)n64);
    }
}

// Half-stencil CSR, pass 1: row lengths (the particle's own forward pairs in
// a register, the partner's by an atomic) and, when rho != NULL, the density
// as k_density_half computes it.  cnt must be zero, rho the self terms.
template <int DIM>
__global__ void __launch_bounds__(256) k_half_count(GridDev g, const int *__restrict__ scell, int *__restrict__ cnt,
                                                    float *__restrict__ rho) {
    unsigned int n32 = 0, n64 = 0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.n;
         s += (long long)gridDim.x * blockDim.x) {
        const int i = (int)s;
        int own = 0;
        float acc = 0.f;
        forward_pairs<DIM>(g, scell, i, n32, n64, [&](int j, float r2) {
            ++own;
            atomicAdd(&cnt[j], 1);
            if (rho != nullptr) {
                const float w = g.w_norm * w_poly(sqrtf(r2) * g.r_scale);
                acc += w;
                atomicAdd(&rho[j], w);
            }
        });
        atomicAdd(&cnt[i], own);
        if (rho != nullptr) atomicAdd(&rho[i], acc);
    }
    add_tier_counts(g, n32, n64);
}

// Pass 2: every pair written into both rows at the rows' atomic cursors
// (cur: a copy of the row starts), in no particular order within a row.
template <int DIM>
__global__ void __launch_bounds__(256) k_half_fill(GridDev g, const int *__restrict__ scell,
                                                   unsigned long long *__restrict__ cur, int *__restrict__ col) {
    unsigned int n32 = 0, n64 = 0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.n;
         s += (long long)gridDim.x * blockDim.x) {
        const int i = (int)s;
        forward_pairs<DIM>(g, scell, i, n32, n64, [&](int j, float) {
            col[atomicAdd(&cur[i], 1ull)] = j;
            col[atomicAdd(&cur[j], 1ull)] = i;
        });
    }
    (void)n32;
    (void)n64;
}

}  // namespace

cudaError_t launch_half_count(const GridDev &g, const int *scell, int *cnt, float *rho, int sm_count, cudaStream_t s) {
    const int nt = 256;
    long long blocks = (g.n + nt - 1) / nt;
    if (blocks > (long long)sm_count * 8) blocks = (long long)sm_count * 8;
    if (blocks < 1) blocks = 1;
    ProfScope ps(TAG_COUNT, s);
    cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)g.n * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (rho != nullptr) {
        note_launch(1);
        k_density_self<<<(unsigned)blocks, nt, 0, s>>>(g.n, g.w_norm * (2.f / 3.f), rho);
    }
    note_launch(1);
    if (g.dim == 2)
        k_half_count<2><<<(unsigned)blocks, nt, 0, s>>>(g, scell, cnt, rho);
    else
        k_half_count<3><<<(unsigned)blocks, nt, 0, s>>>(g, scell, cnt, rho);
    return cudaGetLastError();
}

cudaError_t launch_half_fill(const GridDev &g, const int *scell, unsigned long long *cur, int *col, int sm_count,
                             cudaStream_t s) {
    const int nt = 256;
    long long blocks = (g.n + nt - 1) / nt;
    if (blocks > (long long)sm_count * 8) blocks = (long long)sm_count * 8;
    if (blocks < 1) blocks = 1;
    ProfScope ps(TAG_FILL, s);
    note_launch(1);
    if (g.dim == 2)
        k_half_fill<2><<<(unsigned)blocks, nt, 0, s>>>(g, scell, cur, col);
    else
        k_half_fill<3><<<(unsigned)blocks, nt, 0, s>>>(g, scell, cur, col);
    return cudaGetLastError();
}

cudaError_t launch_density_half(const GridDev &g, const int *scell, float *rho, int sm_count, cudaStream_t s) {
    const int nt = 256;
    long long blocks = (g.n + nt - 1) / nt;
    if (blocks > (long long)sm_count * 8) blocks = (long long)sm_count * 8;
    if (blocks < 1) blocks = 1;
    ProfScope ps(TAG_FILL, s);
    note_launch(2);
    k_density_self<<<(unsigned)blocks, nt, 0, s>>>(g.n, g.w_norm * (2.f / 3.f), rho);
    if (g.dim == 2)
        k_density_half<2><<<(unsigned)blocks, nt, 0, s>>>(g, scell, rho);
    else
        k_density_half<3><<<(unsigned)blocks, nt, 0, s>>>(g, scell, rho);
    return cudaGetLastError();
}

}  // namespace sph
