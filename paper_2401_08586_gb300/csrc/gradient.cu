// gradient.cu -- the volume-free normalised first-order SPH gradient of the
// Appendix (Eq. A5 of arXiv 2401.08586) over an existing neighbour list:
//   <f_i^a> = sum_j (f_j - f_i) dW_ij/dx^a / sum_j (x_j^a - x_i^a) dW_ij/dx^a
// for each axis a, with dW_ij/dx^a = W'(R) / h * (x_i^a - x_j^a) / r.
// Every constant factor of dW (alpha_d, 1/h, the length unit) cancels in the
// ratio, so with d = x_j - x_i in units of u = h_c / 2 and q_j = P'(R_j) / r_j
// (P the polynomial of Eq. 3 without alpha_d):
//   <f_i^a> = (2 / h_c) * sum_j (f_j - f_i) d_a q_j / sum_j d_a^2 q_j.
// Distances come from the FP32 relative coordinates as in the density;
// f_j - f_i is taken from a float hi + lo split of the FP64 field (both
// subtractions in FP32), which keeps the difference accurate to about 2^-24
// of itself plus 2^-48 of |f|, without FP64 arithmetic per pair.  Sums in
// FP32 in CSR order; q < 0 for every pair, so the denominator has no
// cancellation.  A pair at r = 0 contributes nothing, an axis with a zero
// denominator gives 0.
#include "launch.cuh"
#include "profile.cuh"
#include "sph_internal.cuh"

namespace sph {
namespace {

// f in cell order as (hi, lo) with hi = fl32(f), lo = fl32(f - hi).
__global__ void k_f_split(GridDev g, const double *__restrict__ f, float2 *__restrict__ fs) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.n;
         s += (long long)gridDim.x * blockDim.x) {
        const double v = f[g.orig_id[s]];
        const float hi = __double2float_rn(v);
        fs[s] = make_float2(hi, __double2float_rn(__dsub_rn(v, (double)hi)));
    }
}

// dP/dR of Eq. 3's polynomial (without alpha_d): -2R + 1.5R^2 on [0, 1),
// -(2 - R)^2 / 2 on [1, 2), 0 beyond.
__device__ __forceinline__ float dpoly(float R) {
    const float t = fmaxf(2.f - R, 0.f);
    return R < 1.f ? R * fmaf(1.5f, R, -2.f) : -0.5f * t * t;
}

template <int DIM>
__global__ void k_gradient_a5(GridDev g, const int *__restrict__ rank, const int *__restrict__ scell,
                              const long long *__restrict__ row_ptr, const int *__restrict__ col, int canonical,
                              const float2 *__restrict__ fs, double *__restrict__ grad) {
    for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < g.n;
         r += (long long)gridDim.x * blockDim.x) {
        const int si = canonical ? rank[r] : (int)r;
        const float4 ri = g.rel32[si];
        const float2 fi = fs[si];
        const int ci = scell[si];
        int cix, ciy, ciz;
        cell_decompose(g, ci, cix, ciy, ciz);
        float num[3] = {0.f, 0.f, 0.f}, den[3] = {0.f, 0.f, 0.f};
        for (long long q = row_ptr[r]; q < row_ptr[r + 1]; ++q) {
            const int sj = canonical ? rank[col[q]] : col[q];
            const int cj = scell[sj];
            int cjx, cjy, cjz;
            cell_decompose(g, cj, cjx, cjy, cjz);
            const float4 rj = g.rel32[sj];
            float d[3];
            d[0] = __fsub_rn(__fadd_rn(rj.x, 2.f * (float)(cjx - cix)), ri.x);
            d[1] = __fsub_rn(__fadd_rn(rj.y, 2.f * (float)(cjy - ciy)), ri.y);
            d[2] = DIM == 3 ? __fsub_rn(__fadd_rn(rj.z, 2.f * (float)(cjz - ciz)), ri.z) : 0.f;
            const float r2 = __fmaf_rn(d[2], d[2], __fmaf_rn(d[1], d[1], __fmul_rn(d[0], d[0])));
            if (r2 == 0.f) continue;
            const float rr = sqrtf(r2);
            const float qj = dpoly(rr * g.r_scale) / rr;
            const float2 fj = fs[sj];
            const float df = __fadd_rn(__fsub_rn(fj.x, fi.x), __fsub_rn(fj.y, fi.y));
#pragma unroll
            for (int a = 0; a < DIM; ++a) {
                const float dq = d[a] * qj;
                num[a] = fmaf(df, dq, num[a]);
                den[a] = fmaf(d[a], dq, den[a]);
            }
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a)
            grad[r * DIM + a] = den[a] != 0.f ? g.two_over_hc * (double)(num[a] / den[a]) : 0.0;
    }
}

}  // namespace

cudaError_t launch_gradient_a5(const GridDev &g, const int *rank, const int *scell, const long long *row_ptr,
                               const int *col, int canonical, const double *f, float2 *fs, double *grad,
                               int sm_count, cudaStream_t s) {
    const int nt = 128;
    long long blocks = (g.n + nt - 1) / nt;
    if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
    if (blocks < 1) blocks = 1;
    ProfScope ps(TAG_DENSITY, s);
    note_launch(2);
    k_f_split<<<(unsigned)blocks, nt, 0, s>>>(g, f, fs);
    if (g.dim == 2)
        k_gradient_a5<2><<<(unsigned)blocks, nt, 0, s>>>(g, rank, scell, row_ptr, col, canonical, fs, grad);
    else
        k_gradient_a5<3><<<(unsigned)blocks, nt, 0, s>>>(g, rank, scell, row_ptr, col, canonical, fs, grad);
    return cudaGetLastError();
}

}  // namespace sph
