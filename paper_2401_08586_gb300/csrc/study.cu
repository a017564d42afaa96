// study.cu -- precision study of the neighbour decision (Tables 1-2 and
// approach II of Table 4 in arXiv 2401.08586): over the candidate pairs of
// the cell link-list (the 3^d cells around each particle), count how often
// each reduced-precision decision differs from the FP64 definition
// r^2 = (dx0^2 + dx1^2) + dx2^2 < kh^2 on the caller's coordinates:
//   FP16 / FP32 absolute: coordinates rounded to FP16 / FP32, differences,
//       squares and sums in that precision, compared with kh^2 rounded to it;
//   FP16 RCLL: the cell-relative coordinates of Eq. 6 in FP16 (rel16), the
//       difference d = (x_rel,j - x_rel,i) + 2 dc, r^2 in FP16, compared
//       with T = kh^2 / u^2 rounded to FP16 -- the FP16 decision alone;
//   tiered: this library's decision (FP16 band, FP32 band, FP64 tier).
// Not on the search path: an accuracy instrument (every pair, thread per
// particle, FP64 conversions per pair).
#include "launch.cuh"
#include "nnps_common.cuh"
#include "profile.cuh"

namespace sph {
namespace {

using nn::r2_fp64;

struct Counts {
    unsigned long long cand, nbr, w16, w32, wrc, wtier;
};

__device__ __forceinline__ bool fp16_abs(int dim, const double *a, const double *b, __half kh2) {
    __half r2 = __float2half(0.f);
    for (int k = 0; k < dim; ++k) {
        const __half d = __hsub(__double2half(a[k]), __double2half(b[k]));
        r2 = __hfma(d, d, r2);
    }
    return __hlt(r2, kh2);
}

__device__ __forceinline__ bool fp32_abs(int dim, const double *a, const double *b, float kh2) {
    float r2 = 0.f;
    for (int k = 0; k < dim; ++k) {
        const float d = __fsub_rn(__double2float_rn(a[k]), __double2float_rn(b[k]));
        r2 = __fmaf_rn(d, d, r2);
    }
    return r2 < kh2;
}

__global__ void k_precision_study(GridDev g, const int *__restrict__ scell, long long row_begin, long long row_end,
                                  __half kh2_16, float kh2_32, __half t16, unsigned long long *__restrict__ out) {
    Counts c = {0, 0, 0, 0, 0, 0};
    const int dim = g.dim;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < g.n;
         s += (long long)gridDim.x * blockDim.x) {
        const int oi = g.orig_id[s];
        if (oi < row_begin || oi >= row_end) continue;
        const double *xi = g.xyz + (long long)oi * dim;
        const int ci = scell[s];
        int cx, cy, cz;
        cell_decompose(g, ci, cx, cy, cz);
        const uint2 qi = g.rel16[s];
        const float4 fi = g.rel32[s];
        const __half2 qixy = *reinterpret_cast<const __half2 *>(&qi.x);
        const __half2 qiz = *reinterpret_cast<const __half2 *>(&qi.y);
        for (int dz = (dim == 3 ? -1 : 0); dz <= (dim == 3 ? 1 : 0); ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    const int x = cx + dx, y = cy + dy, z = cz + dz;
                    if (x < 0 || x >= g.nk[0] || y < 0 || y >= g.nk[1] || z < 0 || z >= g.nk[2]) continue;
                    const long long cell = ((long long)z * g.nk[1] + y) * g.nk[0] + x;
                    for (int t = g.cell_start[cell]; t < g.cell_start[cell + 1]; ++t) {
                        if (t == s) continue;
                        const int oj = g.orig_id[t];
                        const double *xj = g.xyz + (long long)oj * dim;
                        const bool ex = r2_fp64(dim, xi, xj) < g.kh2;
                        ++c.cand;
                        c.nbr += ex;
                        c.w16 += fp16_abs(dim, xi, xj, kh2_16) != ex;
                        c.w32 += fp32_abs(dim, xi, xj, kh2_32) != ex;
                        // FP16 RCLL alone
                        const uint2 qj = g.rel16[t];
                        const __half2 qjxy = *reinterpret_cast<const __half2 *>(&qj.x);
                        const __half2 qjz = *reinterpret_cast<const __half2 *>(&qj.y);
                        __half2 dxy = __hsub2(qjxy, qixy);
                        dxy = __hadd2(dxy, __floats2half2_rn(2.f * dx, 2.f * dy));
                        __half r2 = __hmul(__low2half(dxy), __low2half(dxy));
                        r2 = __hfma(__high2half(dxy), __high2half(dxy), r2);
                        if (dim == 3) {
                            const __half d2 = __hadd(__hsub(__low2half(qjz), __low2half(qiz)), __float2half(2.f * dz));
                            r2 = __hfma(d2, d2, r2);
                        }
                        c.wrc += __hlt(r2, t16) != ex;
                        // tiered decision: FP16 "maybe" band, FP32 band, FP64
                        const __half e = __hsub(r2, t16);
                        bool tier = false;
                        if (__hlt(e, __low2half(*reinterpret_cast<const __half2 *>(&g.tau16)))) {
                            const float4 fj = g.rel32[t];
                            const float e0 = __fsub_rn(__fadd_rn(fj.x, 2.f * dx), fi.x);
                            const float e1 = __fsub_rn(__fadd_rn(fj.y, 2.f * dy), fi.y);
                            const float e2 = dim == 3 ? __fsub_rn(__fadd_rn(fj.z, 2.f * dz), fi.z) : 0.f;
                            const float q = __fmaf_rn(e2, e2, __fmaf_rn(e1, e1, __fmul_rn(e0, e0)));
                            tier = q < g.t32_in ? true : (q > g.t32_out ? false : ex);
                        }
                        c.wtier += tier != ex;
                    }
                }
    }
    // warp sums, one atomic per warp and counter
    unsigned long long v[6] = {c.cand, c.nbr, c.w16, c.w32, c.wrc, c.wtier};
#pragma unroll
    for (int k = 0; k < 6; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        if ((threadIdx.x & 31) == 0 && v[k]) atomicAdd(&out[k], v[k]);
    }
}

}  // namespace

cudaError_t launch_precision_study(const GridDev &g, const int *scell, long long row_begin, long long row_end,
                                   double kh, unsigned long long *out, int sm_count, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(out, 0, 6 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const double u = g.hc * 0.5;
    const __half kh2_16 = __double2half(kh * kh);
    const float kh2_32 = (float)(kh * kh);
    const __half t16 = __double2half(kh * kh / (u * u));
    long long blocks = (g.n + 127) / 128;
    if (blocks > (long long)sm_count * 16) blocks = (long long)sm_count * 16;
    if (blocks < 1) blocks = 1;
    note_launch(1);
    k_precision_study<<<(unsigned)blocks, 128, 0, s>>>(g, scell, row_begin, row_end, kh2_16, kh2_32, t16, out);
    return cudaGetLastError();
}

}  // namespace sph
