// bin.cu -- binning of particles into background cells (cell link-list,
// Section "SPH method" / Fig. 3b of arXiv 2401.08586) and conversion to the
// normalised cell-relative coordinates of Eq. 6.
//
// Steps (one pass each over the particles):
//   k_bounds   per-axis min/max of the FP64 coordinates (Eq. 5 uses the
//              domain extent), finiteness check;
//   k_hash     cell index c_k = clamp(floor((x_k - lo_k) / h_c), 0, n_k - 1),
//              linear id (c_z n_y + c_y) n_x + c_x, warp-aggregated histogram
//              whose returned counter value is the particle's provisional slot;
//   (exclusive scan of the histogram -> cell_start)
//   k_scatter  orig_id[cell_start[cell] + slot] = i;
//   (per-cell sort of orig_id, so the order inside a cell is the input order
//    and the result does not depend on atomic timing)
//   k_convert  for every sorted position: rank, cell id, and the relative
//              coordinate x_rel = 2 (x - x_cc) / h_c with x_cc the cell centre,
//              computed in FP64 and rounded once to FP16 (rel16) and FP32
//              (rel32); or, for the FP64 cell link-list, the FP64 coordinate.
#include "profile.cuh"
#include "sph_internal.cuh"

namespace sph {

__global__ void k_bounds(const double *__restrict__ xyz, long long total, int dim,
                         DevStatus *st) {
    // Launched with a thread count that is a multiple of dim, so each thread
    // always reads the same axis.
    long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long stride = (long long)gridDim.x * blockDim.x;
    const int axis = (int)(t % dim);
    double mn = INFINITY, mx = -INFINITY;
    bool bad = false;
    for (long long f = t; f < total; f += stride) {
        double x = xyz[f];
        bad |= !isfinite(x);
        mn = fmin(mn, x);
        mx = fmax(mx, x);
    }
    if (bad) atomicOr(&st->flags, ST_NONFINITE);
    // Reduce lanes that read the same axis: with 32 lanes and dim in {2,3} the
    // lanes of one axis are lane = axis0 + k*dim; simplest is a shared-memory
    // reduction per axis.
    __shared__ double smin[3][32], smax[3][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int a = 0; a < 3; ++a) {
        double vmn = (axis == a) ? mn : INFINITY;
        double vmx = (axis == a) ? mx : -INFINITY;
        for (int o = 16; o > 0; o >>= 1) {
            vmn = fmin(vmn, __shfl_xor_sync(0xffffffffu, vmn, o));
            vmx = fmax(vmx, __shfl_xor_sync(0xffffffffu, vmx, o));
        }
        if (lane == 0) {
            smin[a][w] = vmn;
            smax[a][w] = vmx;
        }
    }
    __syncthreads();
    if (threadIdx.x < dim) {
        int a = threadIdx.x;
        double vmn = INFINITY, vmx = -INFINITY;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            vmn = fmin(vmn, smin[a][k]);
            vmx = fmax(vmx, smax[a][k]);
        }
        if (vmn <= vmx) {
            atomicMin(&st->min_key[a], dkey(vmn));
            atomicMax(&st->max_key[a], dkey(vmx));
        }
    }
}

__global__ void k_hash(const double *__restrict__ xyz, int n, int dim, GridDev g,
                       int *__restrict__ cnt, int *__restrict__ cid, int *__restrict__ slot) {
    const int lane = threadIdx.x & 31;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < n;
         base += (long long)gridDim.x * blockDim.x) {
        long long i = base + threadIdx.x;
        bool live = i < n;
        int c = -1;
        if (live) {
            int cc[3] = {0, 0, 0};
            for (int k = 0; k < dim; ++k)
                cc[k] = cell_coord(xyz[i * dim + k], g.lo[k], g.hc, g.nk[k]);
            c = (cc[2] * g.nk[1] + cc[1]) * g.nk[0] + cc[0];
        }
        // Lanes with the same cell add to its counter once.
        unsigned int peers = __match_any_sync(0xffffffffu, c);
        int leader = __ffs(peers) - 1;
        int old = 0;
        if (live && lane == leader) old = atomicAdd(&cnt[c], __popc(peers));
        old = __shfl_sync(0xffffffffu, old, leader);
        if (live) {
            cid[i] = c;
            slot[i] = old + __popc(peers & ((1u << lane) - 1u));
        }
    }
}

__global__ void k_scatter(int n, const int *__restrict__ cell_start, const int *__restrict__ cid,
                          const int *__restrict__ slot, int *__restrict__ orig_id) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        orig_id[cell_start[cid[i]] + slot[i]] = (int)i;
}

template <int PREC>
__global__ void k_convert(int n, int dim, GridDev g, const int *__restrict__ cid_in,
                          int *__restrict__ rank, int *__restrict__ scell, uint2 *__restrict__ rel16,
                          float4 *__restrict__ rel32, double4 *__restrict__ x64, int check_box) {
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < n;
         s += (long long)gridDim.x * blockDim.x) {
        int i = g.orig_id[s];
        rank[i] = (int)s;
        scell[s] = cid_in[i];
        double x[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < dim; ++k) x[k] = g.xyz[(long long)i * dim + k];
        if (PREC == SPH_PREC_FP64_CLL) {
            x64[s] = make_double4(x[0], x[1], x[2], 0.0);
            if (check_box) {
                for (int k = 0; k < dim; ++k)
                    if (x[k] < g.lo[k] || x[k] > g.lo[k] + g.nk[k] * g.hc)
                        atomicOr(&g.status->flags, ST_OUT_OF_BOX);
            }
            continue;
        }
        double a[3] = {0.0, 0.0, 0.0};
        bool out = false;
        for (int k = 0; k < dim; ++k) {
            int c = cell_coord(x[k], g.lo[k], g.hc, g.nk[k]);
            // x - x_cc with x_cc = lo + (c + 1/2) h_c: one rounding for the
            // difference to lo, one for the fused subtraction of the centre.
            double t = __dsub_rn(x[k], g.lo[k]);
            double r = __fma_rn(-((double)c + 0.5), g.hc, t);
            a[k] = __dmul_rn(r, g.two_over_hc);
            out |= fabs(a[k]) > 1.0 + 1e-6;
        }
        if (out && check_box) atomicOr(&g.status->flags, ST_OUT_OF_BOX);
        __half2 xy = __halves2half2(__double2half(a[0]), __double2half(a[1]));
        __half2 z0 = __halves2half2(__double2half(a[2]), __double2half(0.0));
        uint2 q;
        q.x = *reinterpret_cast<unsigned int *>(&xy);
        q.y = *reinterpret_cast<unsigned int *>(&z0);
        rel16[s] = q;
        rel32[s] = make_float4(__double2float_rn(a[0]), __double2float_rn(a[1]),
                               __double2float_rn(a[2]), 0.f);
    }
}

// ---- host launchers ---------------------------------------------------------

static unsigned grid_for(long long n, int nt, int sm_count, int per_sm) {
    long long b = (n + nt - 1) / nt;
    if (b > (long long)sm_count * per_sm) b = (long long)sm_count * per_sm;
    return (unsigned)(b < 1 ? 1 : b);
}

cudaError_t launch_bounds(const double *xyz, long long n, int dim, DevStatus *st, int sm_count,
                          cudaStream_t s) {
    const int nt = 192;  // multiple of 2 and 3: each thread keeps one axis
    ProfScope ps(TAG_BOUNDS, s);
    note_launch(1);
    k_bounds<<<grid_for(n * dim, nt, sm_count, 8), nt, 0, s>>>(xyz, n * dim, dim, st);
    return cudaGetLastError();
}

cudaError_t launch_hash_scatter_convert(const GridDev &g, const double *xyz, int n, int dim, int prec,
                                        int *cnt, int *cid, int *slot, int *cell_start, int *orig_id,
                                        int *rank, int *scell, uint2 *rel16, float4 *rel32, double4 *x64,
                                        void *scan_tmp, int *big_list, unsigned int *big_count,
                                        int check_box, int sm_count, cudaStream_t s) {
    const int nt = 256;
    const unsigned blocks = grid_for(n, nt, sm_count, 16);
    cudaError_t e = cudaMemsetAsync(cnt, 0, g.ncell * sizeof(int), s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(TAG_HASH, s);
        note_launch(1);
        k_hash<<<blocks, nt, 0, s>>>(xyz, n, dim, g, cnt, cid, slot);
    }
    e = exclusive_scan_i32(cnt, cell_start, g.ncell, scan_tmp, s);
    if (e != cudaSuccess) return e;
    {
        ProfScope ps(TAG_SCATTER, s);
        note_launch(1);
        k_scatter<<<blocks, nt, 0, s>>>(n, cell_start, cid, slot, orig_id);
    }
    e = segmented_sort_i32(orig_id, cell_start, g.ncell, big_list, big_count, s);
    if (e != cudaSuccess) return e;
    ProfScope ps(TAG_CONVERT, s);
    note_launch(1);
    if (prec == SPH_PREC_FP16_RCLL)
        k_convert<SPH_PREC_FP16_RCLL><<<blocks, nt, 0, s>>>(n, dim, g, cid, rank, scell, rel16, rel32,
                                                            nullptr, check_box);
    else
        k_convert<SPH_PREC_FP64_CLL><<<blocks, nt, 0, s>>>(n, dim, g, cid, rank, scell, nullptr, nullptr,
                                                           x64, check_box);
    return cudaGetLastError();
}

}  // namespace sph
