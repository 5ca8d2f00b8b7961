// msft_uniform.cu -- Eq. 9 on the paper's uniform-q virtual detector (Block 1,
// Block 6's per-slice DFT), where q_x depends on the pixel column u only and
// q_y on the row v only, so the transverse sum separates:
//   U1:  H[v][j][x] = sum_y s_j(x, y) e^{-i q_y(v) y}
//   U2:  A(u, v)    = (n^2-1) sum_j e^{-i q_z(u,v) z_j} sum_x e^{-i q_x(u) x} H[v][j][x]
// Both stages are shared-memory tiled complex GEMMs on the CUDA cores (FP32
// or FP64); U2 applies the per-pixel slice phase e^{-i q_z z_j} and reduces
// over j in a fixed order.  Pixels with q_x^2 + q_y^2 > k0^2 have no
// scattering direction and get A = 0.
#include "internal.cuh"

namespace scm {

template <typename R> struct UC;
template <> struct UC<float> { using T = float2; };
template <> struct UC<double> { using T = double2; };
template <typename R> __device__ __forceinline__ typename UC<R>::T uexp(double q, double c);
template <> __device__ __forceinline__ float2 uexp<float>(double q, double c) { return expmi_f(q, c); }
template <> __device__ __forceinline__ double2 uexp<double>(double q, double c) { return expmi_d(q, c); }

// Transverse momentum of pixel index i of n on the uniform grid.
__device__ __forceinline__ double uq_of(int i, int n, double qmax) {
    return qmax * (double)(2 * i + 1 - n) / (double)n;
}

// Per-block table of the 64 transverse momenta of a tile's rows or columns:
// FP32 sums take them as float pairs (no FP64 in the inner loops), FP64 sums
// as doubles.
template <typename R> struct UQTab;
template <> struct UQTab<float> {
    float2 q[64];
    __device__ void set(int i, double v) {
        const float h = (float)v;
        q[i] = make_float2(h, (float)(v - (double)h));
    }
    // e^{-i q_i (k - off) voxel}
    __device__ float2 phase(int i, int k, float off, float vox) const {
        return expmi_fs(q[i].x, q[i].y, ((float)k - off) * vox);
    }
};
template <> struct UQTab<double> {
    double q[64];
    __device__ void set(int i, double v) { q[i] = v; }
    __device__ double2 phase(int i, int k, double off, double vox) const { return expmi_d(q[i], (k - off) * vox); }
};

// a1 for the uniform-q detector: q for every pixel (q_z = -k0 where the pixel
// has no scattering direction).
__global__ void detector_q_uniform_kernel(int det_nx, int det_ny, double qmax, double k0, double *q) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)det_nx * det_ny) return;
    const int u = (int)(p % det_nx), v = (int)(p / det_nx);
    const double qx = uq_of(u, det_nx, qmax), qy = uq_of(v, det_ny, qmax);
    const double s2 = __ddiv_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(k0, k0));
    q[3 * p] = qx;
    q[3 * p + 1] = qy;
    q[3 * p + 2] = s2 <= 1.0 ? k0 * (sqrt(1.0 - s2) - 1.0) : -k0;
}

// q_z of every pixel as a float pair, or the off-sphere marker: decided from
// the detector's stored q with the same FP64 operations that set q_z.
__global__ void uq_qz_table_kernel(const double *q, long long n, double k0, float2 *tab) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
    const double s2 = __ddiv_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(k0, k0));
    const float h = (float)qz;
    tab[p] = s2 <= 1.0 ? make_float2(h, (float)(qz - (double)h)) : make_float2(__uint_as_float(kUqOffSphereBits), 0.f);
}

cudaError_t launch_uq_qz_table(const double *q, long long n, double k0, float2 *tab, cudaStream_t st) {
    uq_qz_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(q, n, k0, tab);
    return cudaGetLastError();
}

cudaError_t launch_detector_q_uniform(int det_nx, int det_ny, double theta_max_deg, double k0, double *q,
                                      cudaStream_t st) {
    const double qmax = k0 * sin(theta_max_deg * kPi / 180.0);
    const long long n = (long long)det_nx * det_ny;
    detector_q_uniform_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(det_nx, det_ny, qmax, k0, q);
    return cudaGetLastError();
}

constexpr int kUT = 64;        // tile edge
constexpr int kUK = 16;        // K chunk

// U1: H[v][c] = sum_y s[c][y] P(v, y), c = (j, x).  Block tile 64 v x 64 c,
// thread 4 v x 4 c (c strided by 16 so shared reads are conflict-free).
// (In the tensor-core modes this stage runs on the tensor cores instead: the
// flat contraction kernel in store mode, csrc/msft_tc.cu.)
template <typename R>
__global__ void __launch_bounds__(256) uq_y_kernel(const typename UC<R>::T *__restrict__ s, int ny, int ncol,
                                                   int ndv, double qmax, double voxel,
                                                   typename UC<R>::T *__restrict__ H) {
    using C = typename UC<R>::T;
    __shared__ C Ps[kUK][kUT];
    __shared__ C Ss[kUK][kUT];
    __shared__ UQTab<R> qy;
    const int v0 = blockIdx.y * kUT, c0 = blockIdx.x * kUT;
    const int tv = threadIdx.x / 16, tc = threadIdx.x % 16;
    if (threadIdx.x < kUT) qy.set(threadIdx.x, uq_of(min(v0 + (int)threadIdx.x, ndv - 1), ndv, qmax));
    const R yoff = (R)(0.5 * (ny - 1)), vox = (R)voxel;
    C acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b].x = acc[a][b].y = (R)0;
    for (int y0 = 0; y0 < ny; y0 += kUK) {
        __syncthreads();
        for (int it = threadIdx.x; it < kUK * kUT; it += 256) {
            const int k = it / kUT, i = it % kUT;
            const int y = y0 + k;
            C pv, sv;
            pv.x = pv.y = sv.x = sv.y = (R)0;
            if (y < ny) {
                if (v0 + i < ndv) pv = qy.phase(i, y, yoff, vox);
                if (c0 + i < ncol) sv = s[(size_t)(c0 + i) * ny + y];
            }
            Ps[k][i] = pv;
            Ss[k][i] = sv;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kUK; ++k) {
            C p[4], q[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) p[a] = Ps[k][4 * tv + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) q[b] = Ss[k][tc + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    acc[a][b].x = fma(p[a].x, q[b].x, fma(-p[a].y, q[b].y, acc[a][b].x));
                    acc[a][b].y = fma(p[a].x, q[b].y, fma(p[a].y, q[b].x, acc[a][b].y));
                }
        }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int v = v0 + 4 * tv + a;
        if (v >= ndv) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = c0 + tc + 16 * b;
            if (c < ncol) H[(size_t)v * ncol + c] = acc[a][b];
        }
    }
}

// U2: for one detector row v and 64 columns u: F[u][j] = sum_x E(u, x) H[v][j][x],
// then A(u, v) = str * sum_j e^{-i q_z(u,v) z_j} F[u][j].  Thread: 4 u x JP j.
template <typename R, int JP, int KC>
__global__ void __launch_bounds__(256) uq_xz_kernel(const typename UC<R>::T *__restrict__ H, int nx, int nz,
                                                    int ndu, int ndv, double qmax, double k0, double voxel,
                                                    R str_re, R str_im, const float2 *__restrict__ qz_tab,
                                                    typename UC<R>::T *__restrict__ A, R *__restrict__ I) {
    using C = typename UC<R>::T;
    __shared__ C Es[KC][kUT];
    __shared__ C Hs[KC][16 * JP];
    __shared__ C red[16][kUT + 1];
    __shared__ UQTab<R> qx;
    const int v = blockIdx.y, u0 = blockIdx.x * kUT;
    const int tu = threadIdx.x % 16, tj = threadIdx.x / 16;     // u = u0 + tu + 16 a ; j = tj + 16 b
    if (threadIdx.x < kUT) qx.set(threadIdx.x, uq_of(min(u0 + (int)threadIdx.x, ndu - 1), ndu, qmax));
    const R xoff = (R)(0.5 * (nx - 1)), vox = (R)voxel;
    C acc[4][JP];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < JP; ++b) acc[a][b].x = acc[a][b].y = (R)0;
    const C *Hv = H + (size_t)v * nz * nx;
    for (int x0 = 0; x0 < nx; x0 += KC) {
        __syncthreads();
        for (int it = threadIdx.x; it < KC * kUT; it += 256) {
            const int k = it / kUT, i = it % kUT;
            C e;
            e.x = e.y = (R)0;
            if (x0 + k < nx && u0 + i < ndu) e = qx.phase(i, x0 + k, xoff, vox);
            Es[k][i] = e;
        }
        for (int it = threadIdx.x; it < KC * 16 * JP; it += 256) {
            const int j = it / KC, k = it % KC;
            C h;
            h.x = h.y = (R)0;
            if (x0 + k < nx && j < nz) h = Hv[(size_t)j * nx + x0 + k];
            Hs[k][j] = h;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < KC; ++k) {
            C e[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) e[a] = Es[k][tu + 16 * a];
#pragma unroll
            for (int b = 0; b < JP; ++b) {
                const C h = Hs[k][tj + 16 * b];
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    acc[a][b].x = fma(e[a].x, h.x, fma(-e[a].y, h.y, acc[a][b].x));
                    acc[a][b].y = fma(e[a].x, h.y, fma(e[a].y, h.x, acc[a][b].y));
                }
            }
        }
    }
    // slice phases and the sum over this thread's j; FP32 takes q_z from the
    // handle's table (float pair, marker off the Ewald sphere), FP64 forms it
    const double qy = uq_of(v, ndv, qmax);
    const R zoff = (R)(0.5 * (nz - 1));
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int u = u0 + tu + 16 * a;
        C part;
        part.x = part.y = (R)0;
        if constexpr (sizeof(R) == 4) {
            const float2 t = u < ndu ? qz_tab[(size_t)v * ndu + u] : make_float2(0.f, 0.f);
#pragma unroll
            for (int b = 0; b < JP; ++b) {
                const int j = tj + 16 * b;
                if (j < nz) {
                    const float2 z = expmi_fs(t.x, t.y, ((float)j - zoff) * vox);
                    part.x = fmaf(z.x, acc[a][b].x, fmaf(-z.y, acc[a][b].y, part.x));
                    part.y = fmaf(z.x, acc[a][b].y, fmaf(z.y, acc[a][b].x, part.y));
                }
            }
        } else {
            const double qxu = uq_of(u < ndu ? u : 0, ndu, qmax);
            const double s2 = __ddiv_rn(__dadd_rn(__dmul_rn(qxu, qxu), __dmul_rn(qy, qy)), __dmul_rn(k0, k0));
            const double qz = s2 <= 1.0 ? k0 * (sqrt(1.0 - s2) - 1.0) : -k0;
#pragma unroll
            for (int b = 0; b < JP; ++b) {
                const int j = tj + 16 * b;
                if (j < nz) {
                    const C z = uexp<R>(qz, (j - 0.5 * (nz - 1)) * voxel);
                    part.x = fma(z.x, acc[a][b].x, fma(-z.y, acc[a][b].y, part.x));
                    part.y = fma(z.x, acc[a][b].y, fma(z.y, acc[a][b].x, part.y));
                }
            }
        }
        red[tj][tu + 16 * a] = part;
    }
    __syncthreads();
    if (threadIdx.x < kUT) {
        const int i = threadIdx.x, u = u0 + i;
        if (u < ndu) {
            C sum;
            sum.x = sum.y = (R)0;
            for (int t = 0; t < 16; ++t) {
                sum.x += red[t][i].x;
                sum.y += red[t][i].y;
            }
            bool valid;
            if constexpr (sizeof(R) == 4) {
                valid = __float_as_uint(qz_tab[(size_t)v * ndu + u].x) != kUqOffSphereBits;
            } else {
                const double qxu = uq_of(u, ndu, qmax);
                const double s2 = __ddiv_rn(__dadd_rn(__dmul_rn(qxu, qxu), __dmul_rn(qy, qy)), __dmul_rn(k0, k0));
                valid = s2 <= 1.0;
            }
            C out;
            if (valid) {
                out.x = str_re * sum.x - str_im * sum.y;
                out.y = str_re * sum.y + str_im * sum.x;
            } else {
                out.x = out.y = (R)0;
            }
            const size_t p = (size_t)v * ndu + u;
            A[p] = out;
            I[p] = out.x * out.x + out.y * out.y;
        }
    }
}

template <typename R, int KC>
static void launch_uq_xz(int JP, dim3 g2, cudaStream_t st, const void *H, int nx, int nz, int det_nx, int det_ny,
                         double qmax, double k0, double voxel, double str_re, double str_im, const float2 *qz,
                         void *A, void *I) {
    using C = typename UC<R>::T;
    const C *Hc = (const C *)H;
    C *Ac = (C *)A;
    R *Ir = (R *)I;
    // j per thread = JP: the smallest power of two with 16 JP >= nz
    if (JP == 1)
        uq_xz_kernel<R, 1, KC><<<g2, 256, 0, st>>>(Hc, nx, nz, det_nx, det_ny, qmax, k0, voxel, (R)str_re, (R)str_im, qz, Ac, Ir);
    else if (JP == 2)
        uq_xz_kernel<R, 2, KC><<<g2, 256, 0, st>>>(Hc, nx, nz, det_nx, det_ny, qmax, k0, voxel, (R)str_re, (R)str_im, qz, Ac, Ir);
    else if (JP == 4)
        uq_xz_kernel<R, 4, KC><<<g2, 256, 0, st>>>(Hc, nx, nz, det_nx, det_ny, qmax, k0, voxel, (R)str_re, (R)str_im, qz, Ac, Ir);
    else
        uq_xz_kernel<R, 8, KC><<<g2, 256, 0, st>>>(Hc, nx, nz, det_nx, det_ny, qmax, k0, voxel, (R)str_re, (R)str_im, qz, Ac, Ir);
}

cudaError_t launch_msft_uniform(bool fp64, const void *s, int nx, int ny, int nz, int det_nx, int det_ny,
                                double theta_max_deg, double k0, double voxel, double str_re, double str_im,
                                const float2 *qz, void *H, void *A, void *I, cudaStream_t st) {
    const double qmax = k0 * sin(theta_max_deg * kPi / 180.0);
    const int ncol = nx * nz;
    dim3 g1((ncol + kUT - 1) / kUT, (det_ny + kUT - 1) / kUT);
    dim3 g2((det_nx + kUT - 1) / kUT, det_ny);
    if (nz > 128) return cudaErrorInvalidValue;
    const int JP = nz <= 16 ? 1 : nz <= 32 ? 2 : nz <= 64 ? 4 : 8;
    if (fp64) {
        uq_y_kernel<double><<<g1, 256, 0, st>>>((const double2 *)s, ny, ncol, det_ny, qmax, voxel, (double2 *)H);
        launch_uq_xz<double, 8>(JP, g2, st, H, nx, nz, det_nx, det_ny, qmax, k0, voxel, str_re, str_im, qz, A, I);
    } else {
        uq_y_kernel<float><<<g1, 256, 0, st>>>((const float2 *)s, ny, ncol, det_ny, qmax, voxel, (float2 *)H);
        launch_uq_xz<float, 16>(JP, g2, st, H, nx, nz, det_nx, det_ny, qmax, k0, voxel, str_re, str_im, qz, A, I);
    }
    return cudaGetLastError();
}

}  // namespace scm
