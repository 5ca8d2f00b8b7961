// msft_simt.cu -- CUDA-core direct sum of Eq. 9 in FP32 or FP64.
//
// Each thread owns two detector pixels.  For a chunk of YC consecutive y it
// keeps e^{-i q_y y} of both pixels in registers; the slices s[z][x][y-chunk]
// of a group of (z, x) columns are staged in shared memory and read as
// broadcasts.  Per column the y-sum G = sum_y e^{-i q_y y} s is formed with
// complex FMAs and accumulated with the column phase e^{-i (q_x x + q_z z)}
// (re-anchored every 16 columns and after a skipped column, stepped in
// between).  With the voxeliser's per-slice occupied boxes, columns outside
// their slice's x range and y chunks outside its y range are skipped (their
// slice values are zero).  The (z, x) columns can be split across blocks;
// partial fields are summed in a fixed order by a second kernel, so the
// result does not depend on scheduling.
#include "internal.cuh"

namespace scm {

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

template <typename R>
__device__ __forceinline__ typename Cplx<R>::T expmi(double q, double c);
template <> __device__ __forceinline__ float2 expmi<float>(double q, double c) { return expmi_f(q, c); }
template <> __device__ __forceinline__ double2 expmi<double>(double q, double c) { return expmi_d(q, c); }

constexpr int kSimtThreads = 128;
constexpr int kPPT = 2;        // pixels per thread
constexpr int kCols = 64;      // (z, x) columns staged per round

template <typename R, int YC>
__global__ void __launch_bounds__(kSimtThreads) msft_simt_kernel(const typename Cplx<R>::T *__restrict__ s,
                                                                 const double *__restrict__ q, long long n_pix,
                                                                 int nx, int ny, int nz, double voxel,
                                                                 int cols_per_split,
                                                                 const int *__restrict__ bounds,
                                                                 typename Cplx<R>::T *__restrict__ partial) {
    using C = typename Cplx<R>::T;
    __shared__ C tile[kCols][YC];
    __shared__ int s_live[kCols];         // per staged column: 1 if its slice is occupied there in this y chunk
    const long long pix0 = (long long)blockIdx.x * (kSimtThreads * kPPT) + threadIdx.x;
    const int ncol = nx * nz;
    const int col_begin = blockIdx.y * cols_per_split;
    const int col_end = min(ncol, col_begin + cols_per_split);

    double qx[kPPT], qy[kPPT], qz[kPPT];
#pragma unroll
    for (int pp = 0; pp < kPPT; ++pp) {
        long long p = pix0 + pp * kSimtThreads;
        if (p < n_pix) {
            qx[pp] = q[3 * p];
            qy[pp] = q[3 * p + 1];
            qz[pp] = q[3 * p + 2];
        } else {
            qx[pp] = qy[pp] = qz[pp] = 0.0;
        }
    }
    C wx[kPPT];
#pragma unroll
    for (int pp = 0; pp < kPPT; ++pp) wx[pp] = expmi<R>(qx[pp], voxel);
    // FP32: q as float pairs and FP32 coordinates, so the phase anchors do no
    // FP64 work (FP64 runs at a small fraction of the FP32 rate here)
    float qxh[kPPT], qxl[kPPT], qyh[kPPT], qyl[kPPT], qzh[kPPT], qzl[kPPT];
#pragma unroll
    for (int pp = 0; pp < kPPT; ++pp) {
        qxh[pp] = (float)qx[pp];
        qxl[pp] = (float)(qx[pp] - (double)qxh[pp]);
        qyh[pp] = (float)qy[pp];
        qyl[pp] = (float)(qy[pp] - (double)qyh[pp]);
        qzh[pp] = (float)qz[pp];
        qzl[pp] = (float)(qz[pp] - (double)qzh[pp]);
    }
    const float vf = (float)voxel;
    const float xoff = 0.5f * (float)(nx - 1), yoff = 0.5f * (float)(ny - 1), zoff = 0.5f * (float)(nz - 1);

    C acc[kPPT];
#pragma unroll
    for (int pp = 0; pp < kPPT; ++pp) acc[pp].x = acc[pp].y = (R)0;

    for (int y0 = 0; y0 < ny; y0 += YC) {
        C py[kPPT][YC];
#pragma unroll
        for (int k = 0; k < YC; ++k) {
            const bool in = (y0 + k) < ny;
            const double yc = (y0 + k - 0.5 * (ny - 1)) * voxel;
#pragma unroll
            for (int pp = 0; pp < kPPT; ++pp) {
                C e;
                if constexpr (sizeof(R) == 4)
                    e = expmi_fs(qyh[pp], qyl[pp], ((float)(y0 + k) - yoff) * vf);
                else
                    e = expmi<R>(qy[pp], yc);
                py[pp][k].x = in ? e.x : (R)0;
                py[pp][k].y = in ? e.y : (R)0;
            }
        }
        C accz[kPPT], ph[kPPT];
#pragma unroll
        for (int pp = 0; pp < kPPT; ++pp) {
            accz[pp].x = accz[pp].y = (R)0;
            ph[pp].x = (R)1;
            ph[pp].y = (R)0;
        }
        int zcur = -1, xprev = -2;
        C Z[kPPT];
        for (int c0 = col_begin; c0 < col_end; c0 += kCols) {
            __syncthreads();
            for (int cl = threadIdx.x; cl < kCols; cl += kSimtThreads) {
                const int col = c0 + cl;
                bool live = col < col_end;
                if (live && bounds) {
                    const int z = col / nx, x = col - z * nx;
                    live = x >= bounds[z] && x < bounds[nz + z] && y0 < bounds[3 * nz + z] &&
                           y0 + YC > bounds[2 * nz + z];
                }
                s_live[cl] = live ? 1 : 0;
            }
            __syncthreads();
            for (int it = threadIdx.x; it < kCols * YC; it += kSimtThreads) {
                const int cl = it / YC, k = it % YC;
                const int col = c0 + cl;
                C v;
                v.x = v.y = (R)0;
                if (s_live[cl] && y0 + k < ny) v = s[(size_t)col * ny + y0 + k];
                tile[cl][k] = v;
            }
            __syncthreads();
            const int nc = min(kCols, col_end - c0);
            for (int cl = 0; cl < nc; ++cl) {
                if (!s_live[cl]) continue;             // block-uniform: no divergence
                const int col = c0 + cl;
                const int z = col / nx, x = col - z * nx;
                if (z != zcur) {
#pragma unroll
                    for (int pp = 0; pp < kPPT; ++pp) {
                        acc[pp].x += accz[pp].x;
                        acc[pp].y += accz[pp].y;
                        accz[pp].x = accz[pp].y = (R)0;
                        if constexpr (sizeof(R) == 4)
                            Z[pp] = expmi_fs(qzh[pp], qzl[pp], ((float)z - zoff) * vf);
                        else
                            Z[pp] = expmi<R>(qz[pp], (z - 0.5 * (nz - 1)) * voxel);
                    }
                    zcur = z;
                    xprev = -2;
                }
                const bool anchor = (x % 16 == 0) || (x != xprev + 1);
                xprev = x;
#pragma unroll
                for (int pp = 0; pp < kPPT; ++pp) {
                    if (anchor) {
                        if constexpr (sizeof(R) == 4)
                            ph[pp] = cmul(Z[pp], expmi_fs(qxh[pp], qxl[pp], ((float)x - xoff) * vf));
                        else
                            ph[pp] = cmul(Z[pp], expmi<R>(qx[pp], (x - 0.5 * (nx - 1)) * voxel));
                    } else {
                        ph[pp] = cmul(ph[pp], wx[pp]);
                    }
                }
                C g[kPPT];
#pragma unroll
                for (int pp = 0; pp < kPPT; ++pp) g[pp].x = g[pp].y = (R)0;
#pragma unroll
                for (int k = 0; k < YC; ++k) {
                    const C sv = tile[cl][k];
#pragma unroll
                    for (int pp = 0; pp < kPPT; ++pp) {
                        g[pp].x = fma(py[pp][k].x, sv.x, g[pp].x);
                        g[pp].x = fma(-py[pp][k].y, sv.y, g[pp].x);
                        g[pp].y = fma(py[pp][k].x, sv.y, g[pp].y);
                        g[pp].y = fma(py[pp][k].y, sv.x, g[pp].y);
                    }
                }
#pragma unroll
                for (int pp = 0; pp < kPPT; ++pp) {
                    accz[pp].x = fma(ph[pp].x, g[pp].x, accz[pp].x);
                    accz[pp].x = fma(-ph[pp].y, g[pp].y, accz[pp].x);
                    accz[pp].y = fma(ph[pp].x, g[pp].y, accz[pp].y);
                    accz[pp].y = fma(ph[pp].y, g[pp].x, accz[pp].y);
                }
            }
        }
#pragma unroll
        for (int pp = 0; pp < kPPT; ++pp) {
            acc[pp].x += accz[pp].x;
            acc[pp].y += accz[pp].y;
        }
    }
#pragma unroll
    for (int pp = 0; pp < kPPT; ++pp) {
        long long p = pix0 + pp * kSimtThreads;
        if (p < n_pix) partial[(size_t)blockIdx.y * n_pix + p] = acc[pp];
    }
}

// Sums the column splits in order, applies n^2 - 1 and forms I = |A|^2.
template <typename R>
__global__ void msft_reduce_kernel(const typename Cplx<R>::T *__restrict__ partial, int splits, long long n_pix,
                                   R str_re, R str_im, typename Cplx<R>::T *__restrict__ A,
                                   R *__restrict__ I) {
    using C = typename Cplx<R>::T;
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_pix) return;
    C a;
    a.x = a.y = (R)0;
    for (int k = 0; k < splits; ++k) {
        C v = partial[(size_t)k * n_pix + p];
        a.x += v.x;
        a.y += v.y;
    }
    C st;
    st.x = str_re;
    st.y = str_im;
    a = cmul(st, a);
    A[p] = a;
    I[p] = a.x * a.x + a.y * a.y;
}

double simt_issued_flops(const int *bounds, int nz, int ny, long long n_pix, bool fp64) {
    const int yc = fp64 ? 8 : 16;       // the y chunk of the FP64 / FP32 kernel
    double cols_y = 0.0;
    for (int z = 0; z < nz; ++z) {
        const int xlo = bounds[z], xhi = bounds[nz + z], ylo = bounds[2 * nz + z], yhi = bounds[3 * nz + z];
        if (xlo >= xhi || ylo >= yhi) continue;
        int chunks = 0;
        for (int y0 = 0; y0 < ny; y0 += yc) chunks += (y0 < yhi && y0 + yc > ylo) ? 1 : 0;
        cols_y += (double)(xhi - xlo) * chunks * yc;
    }
    return 8.0 * cols_y * (double)n_pix;
}

int simt_splits(long long n_pix, int nx, int nz, int sm_count) {
    long long pblocks = (n_pix + kSimtThreads * kPPT - 1) / (kSimtThreads * kPPT);
    int ncol_groups = (nx * nz + kCols - 1) / kCols;
    long long want = (4LL * sm_count + pblocks - 1) / pblocks;
    if (want < 1) want = 1;
    if (want > ncol_groups) want = ncol_groups;
    if (want > 64) want = 64;
    return (int)want;
}

cudaError_t launch_msft_simt(bool fp64, const void *s, const double *q, long long n_pix, int nx, int ny, int nz,
                             double voxel, double str_re, double str_im, void *A, void *I, void *partial,
                             int splits, cudaStream_t st, const int *bounds) {
    long long pblocks = (n_pix + kSimtThreads * kPPT - 1) / (kSimtThreads * kPPT);
    int ncol = nx * nz;
    int groups = (ncol + kCols - 1) / kCols;
    int per = (groups + splits - 1) / splits * kCols;
    int used = (ncol + per - 1) / per;
    dim3 grid((unsigned)pblocks, used);
    int rthreads = 256;
    unsigned rblocks = (unsigned)((n_pix + rthreads - 1) / rthreads);
    if (fp64) {
        msft_simt_kernel<double, 8><<<grid, kSimtThreads, 0, st>>>(
            (const double2 *)s, q, n_pix, nx, ny, nz, voxel, per, bounds, (double2 *)partial);
        msft_reduce_kernel<double><<<rblocks, rthreads, 0, st>>>((const double2 *)partial, used, n_pix, str_re,
                                                                 str_im, (double2 *)A, (double *)I);
    } else {
        msft_simt_kernel<float, 16><<<grid, kSimtThreads, 0, st>>>(
            (const float2 *)s, q, n_pix, nx, ny, nz, voxel, per, bounds, (float2 *)partial);
        msft_reduce_kernel<float><<<rblocks, rthreads, 0, st>>>((const float2 *)partial, used, n_pix,
                                                                (float)str_re, (float)str_im, (float2 *)A,
                                                                (float *)I);
    }
    return cudaGetLastError();
}

}  // namespace scm
