// adjoint.cu -- gradient of a loss L(I) with respect to the shape parameters.
//
// With A_q = c F_q, c = n^2 - 1, F_q = sum_v s_v e^{-i q.r_v}, s_v = chi_v T_v:
//   dL/dtheta = 2 Re[(c'/c) sum_q w_q |A_q|^2] + 2 Re sum_v R_v ds_v/dtheta,
//   R_v = c conj(S_v),  S_v = sum_q w_q A_q e^{+i q.r_v}   (adjoint field),
// w = dL/dI.  Through the exclusive transmission scan (Eq. 8) the occupancy
// of voxel v also enters every later voxel of its column, so its weight is
//   chibar_v = R_v T_v + i k0 dz (n-1) sum_{v' after v} R_v' s_v'
// (a reverse, suffix scan along z).  Occupancy and transmission are
// recomputed here from the shape, not stored by the forward pass.
#include "internal.cuh"
#include "shape_device.cuh"

namespace scm {

template <typename R> struct Cx;
template <> struct Cx<float> { using T = float2; };
template <> struct Cx<double> { using T = double2; };

template <typename R>
__device__ __forceinline__ typename Cx<R>::T expmi_t(double q, double c);
template <> __device__ __forceinline__ float2 expmi_t<float>(double q, double c) { return expmi_f(q, c); }
template <> __device__ __forceinline__ double2 expmi_t<double>(double q, double c) { return expmi_d(q, c); }

constexpr int kAdjPix = 32;      // pixels staged per round
constexpr int kAdjX = 16;        // x values per block
constexpr int kAdjRun = 16;      // y values per thread

// S[z][x][y] = sum_q w_q A_q e^{+i q.r}.  Block: one z, 16 x, all y; thread
// (xl, y-run).  Per staged pixel the thread forms
//   base = (w A e^{i q_z z}) e^{i q_x x} e^{i q_y y0}
// from shared tables and steps e^{i q_y dy} along its 16 y values.
template <typename R>
__global__ void adjoint_field_kernel(const typename Cx<R>::T *__restrict__ A, const R *__restrict__ w,
                                     const double *__restrict__ q, long long n_pix, int nx, int ny, int nz,
                                     double voxel, typename Cx<R>::T *__restrict__ S) {
    using C = typename Cx<R>::T;
    const int ych = (ny + kAdjRun - 1) / kAdjRun;
    extern __shared__ __align__(16) unsigned char smem[];
    C *gz = reinterpret_cast<C *>(smem);                    // [kAdjPix]
    C *ex = gz + kAdjPix;                                   // [kAdjPix][kAdjX]
    C *ey = ex + kAdjPix * kAdjX;                           // [kAdjPix][ych]
    C *es = ey + kAdjPix * ych;                             // [kAdjPix]

    const int z = blockIdx.y, x0 = blockIdx.x * kAdjX;
    const int xl = threadIdx.x % kAdjX, yc = threadIdx.x / kAdjX;
    const int nthr = blockDim.x;
    const double zc = (z - 0.5 * (nz - 1)) * voxel;
    C acc[kAdjRun];
#pragma unroll
    for (int k = 0; k < kAdjRun; ++k) acc[k].x = acc[k].y = (R)0;

    const int per_pix = 1 + kAdjX + ych + 1;
    for (long long p0 = 0; p0 < n_pix; p0 += kAdjPix) {
        __syncthreads();
        for (int it = threadIdx.x; it < kAdjPix * per_pix; it += nthr) {
            const int pl = it / per_pix, f = it % per_pix;
            const long long p = p0 + pl;
            C v;
            v.x = v.y = (R)0;
            if (p < n_pix) {
                const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
                if (f == 0) {
                    C a = A[p];
                    R wp = w[p];
                    a.x *= wp;
                    a.y *= wp;
                    v = cmul(a, expmi_t<R>(qz, -zc));
                } else if (f <= kAdjX) {
                    v = expmi_t<R>(qx, -((x0 + f - 1) - 0.5 * (nx - 1)) * voxel);
                } else if (f <= kAdjX + ych) {
                    v = expmi_t<R>(qy, -((f - 1 - kAdjX) * kAdjRun - 0.5 * (ny - 1)) * voxel);
                } else {
                    v = expmi_t<R>(qy, -voxel);
                }
            }
            if (f == 0) gz[pl] = v;
            else if (f <= kAdjX) ex[pl * kAdjX + (f - 1)] = v;
            else if (f <= kAdjX + ych) ey[pl * ych + (f - 1 - kAdjX)] = v;
            else es[pl] = v;
        }
        __syncthreads();
        const int np = (int)min((long long)kAdjPix, n_pix - p0);
        for (int pl = 0; pl < np; ++pl) {
            C b = cmul(cmul(gz[pl], ex[pl * kAdjX + xl]), ey[pl * ych + yc]);
            const C st = es[pl];
#pragma unroll
            for (int k = 0; k < kAdjRun; ++k) {
                acc[k].x += b.x;
                acc[k].y += b.y;
                b = cmul(b, st);
            }
        }
    }
    const int x = x0 + xl;
    if (x < nx) {
#pragma unroll
        for (int k = 0; k < kAdjRun; ++k) {
            const int y = yc * kAdjRun + k;
            if (y < ny) S[((size_t)z * nx + x) * ny + y] = acc[k];
        }
    }
}

cudaError_t launch_adjoint_field(bool fp64, const void *A, const void *dLdI, const double *q, long long n_pix,
                                 int nx, int ny, int nz, double voxel, void *S, cudaStream_t st) {
    const int ych = (ny + kAdjRun - 1) / kAdjRun;
    dim3 grid((nx + kAdjX - 1) / kAdjX, nz);
    const int threads = kAdjX * ych;
    if (threads > 1024) return cudaErrorInvalidValue;
    const size_t cx = fp64 ? sizeof(double2) : sizeof(float2);
    const size_t smem = cx * (size_t)kAdjPix * (2 + kAdjX + ych);
    // the largest size (64 y-runs, 1024 threads), so concurrent launches never race on the attribute
    const int smem_max = (int)(cx * kAdjPix * (2 + kAdjX + 64));
    if (fp64) {
        cudaError_t e = cudaFuncSetAttribute(adjoint_field_kernel<double>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
        if (e != cudaSuccess) return e;
        adjoint_field_kernel<double><<<grid, threads, smem, st>>>((const double2 *)A, (const double *)dLdI, q, n_pix,
                                                                  nx, ny, nz, voxel, (double2 *)S);
    } else {
        cudaError_t e = cudaFuncSetAttribute(adjoint_field_kernel<float>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
        if (e != cudaSuccess) return e;
        adjoint_field_kernel<float><<<grid, threads, smem, st>>>((const float2 *)A, (const float *)dLdI, q, n_pix,
                                                                 nx, ny, nz, voxel, (float2 *)S);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Per-voxel chain rule.  Geometric parameters: sphere [r]; ellipsoid
// [a, b, c]; harmonics [a_lm (l >= 1), R0].  Two extra accumulators hold
// D = sum_v R_v s_v C_v (complex), which carries the delta/beta dependence
// of the transmission.
// ---------------------------------------------------------------------------
int grad_param_count(const ShapeParams &sp) { return n_geom_params(sp.kind, sp.lmax); }

constexpr int kGradThreads = 256;
constexpr int kGradMaxRun = 16;
constexpr int kMaxGeom = (SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 1);
constexpr int kGradWarpSlots = (kMaxGeom + 31) / 32;

// Soft occupancy of one voxel with its surface radius and clip state: the
// forward voxeliser's soft branch in FP64; in FP32 with FP32 body coordinates
// (the occupancy is smooth, so this moves chi by ~1e-7, far inside the FP32
// gradient's tolerance, and keeps FP64 off the per-voxel path).
// kMaxL: compile-time bound on the harmonics' degree (sp.lmax <= kMaxL).
template <typename R, int kMaxL>
__device__ __forceinline__ void soft_voxel(const ShapeParams &sp, const GridParams &gp, int ix, int iy, int iz, R &chi,
                                           R &rs, int &clip, R &ux, R &uy, R &uz) {
    R px, py, pz;
    if constexpr (sizeof(R) == 8) {
        if (sp.kind == SCATMAN_SPHERE) {
            px = (ix - 0.5 * (gp.nx - 1)) * gp.voxel - sp.cx;
            py = (iy - 0.5 * (gp.ny - 1)) * gp.voxel - sp.cy;
            pz = (iz - 0.5 * (gp.nz - 1)) * gp.voxel - sp.cz;
        } else {
            body_coords(sp, gp, ix, iy, iz, px, py, pz);
        }
    } else {
        const float vox = gp.voxf;
        const float dx = ((float)ix - 0.5f * (float)(gp.nx - 1)) * vox - sp.cxf;
        const float dy = ((float)iy - 0.5f * (float)(gp.ny - 1)) * vox - sp.cyf;
        const float dz = ((float)iz - 0.5f * (float)(gp.nz - 1)) * vox - sp.czf;
        if (sp.kind == SCATMAN_SPHERE) {
            px = dx;
            py = dy;
            pz = dz;
        } else {
            px = sp.Rf[0] * dx + sp.Rf[3] * dy + sp.Rf[6] * dz;
            py = sp.Rf[1] * dx + sp.Rf[4] * dy + sp.Rf[7] * dz;
            pz = sp.Rf[2] * dx + sp.Rf[5] * dy + sp.Rf[8] * dz;
        }
    }
    const R rr = sqrt(px * px + py * py + pz * pz);
    ux = (R)0;
    uy = (R)0;
    uz = (R)1;
    if (rr > (R)0) {
        ux = px / rr;
        uy = py / rr;
        uz = pz / rr;
    }
    clip = 0;
    if (sp.kind == SCATMAN_SPHERE) {
        rs = (R)sp.r;
    } else if (sp.kind == SCATMAN_ELLIPSOID) {
        const R ia = sizeof(R) == 4 ? (R)sp.inv_af : (R)(1.0 / sp.a);
        const R ib = sizeof(R) == 4 ? (R)sp.inv_bf : (R)(1.0 / sp.b);
        const R ic = sizeof(R) == 4 ? (R)sp.inv_cf : (R)(1.0 / sp.c);
        rs = (R)1 / sqrt(ux * ux * ia * ia + uy * uy * ib * ib + uz * uz * ic * ic);
    } else {
        const ShTab<R> tb(sp);
        R raw = sh_radius_unclipped<R, kMaxL>(sp, px, py, pz, rr);
        rs = raw;
        if (raw < tb.rmin) {
            rs = tb.rmin;
            clip = -1;
        } else if (raw > tb.rmax) {
            rs = tb.rmax;
            clip = 1;
        }
    }
    const R inv_w = sizeof(R) == 4 ? (R)sp.inv_w_f : (R)sp.inv_w;
    const R t = (rs - rr) * inv_w;
    // the forward's FP32 cut (soft_zero): chi = 0 there, and so is its derivative
    chi = (sizeof(R) == 4 && soft_zero((float)t)) ? (R)0 : (R)1 / ((R)1 + exp(-t));
}

// kRun: voxels per lane along z (nz <= 32 kRun), a compile-time bound so the
// per-lane runs stay in registers.  kMaxL: bound on the harmonics' degree, so
// shapes of low degree run a kernel whose unrolled harmonic code is short.
template <typename R, int kRun, int kMaxL>
__global__ void __launch_bounds__(kGradThreads, sizeof(R) == 4 ? 3 : 2) grad_voxel_kernel(ShapeParams sp, GridParams gp,
                                                                  const typename Cx<R>::T *__restrict__ S,
                                                                  double *__restrict__ partials) {
    using C = typename Cx<R>::T;
    const int ng = n_geom_params(sp.kind, sp.lmax);
    // Sphere / ellipsoid parameters and the harmonics' R0 accumulate per
    // thread (acc[0..2]).  The harmonics' a_lm (index j = l^2 + l + m - 1):
    // FP32 keeps one running sum per lane and coefficient in shared memory
    // (s_alm[warp][j][lane], consecutive lanes in consecutive banks), so a
    // voxel adds with one read-modify-write per coefficient and the lanes are
    // summed once, at the end; FP64 sums each term over the warp right away,
    // coefficient j held by lane j % 32 in slot j / 32.
    constexpr bool kSmemAlm = sizeof(R) == 4;
    extern __shared__ float s_alm[];
    R acc[3] = {(R)0, (R)0, (R)0};
    R aw[kGradWarpSlots];
#pragma unroll
    for (int k = 0; k < kGradWarpSlots; ++k) aw[k] = (R)0;
    const bool sh = sp.kind == SCATMAN_SPHHARM;
    C D;
    D.x = D.y = (R)0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float *my_alm = s_alm + (size_t)warp * (ng - 1) * 32;
    if (kSmemAlm && sh)
        for (int j = 0; j < ng - 1; ++j) my_alm[j * 32 + lane] = 0.f;
    const int nz = gp.nz, run = (nz + 31) / 32;
    // c = n^2 - 1 and n - 1 for n = 1 - delta + i beta
    const double d = gp.delta, b = gp.beta;
    C cst, nm1;
    cst.x = (R)(-2.0 * d + d * d - b * b);
    cst.y = (R)(2.0 * b - 2.0 * d * b);
    nm1.x = (R)(-d);
    nm1.y = (R)b;
    const R kdz = (R)(gp.k0 * gp.voxel);
    // per-voxel constants converted once (FP64 stays off the voxel loop)
    const R inv_w = sizeof(R) == 4 ? (R)sp.inv_w_f : (R)sp.inv_w;
    const R R0 = (R)sp.R0, inv_R0 = (R)(1.0 / sp.R0);
    const R inv_a3 = sp.kind == SCATMAN_ELLIPSOID ? (R)(1.0 / (sp.a * sp.a * sp.a)) : (R)0;
    const R inv_b3 = sp.kind == SCATMAN_ELLIPSOID ? (R)(1.0 / (sp.b * sp.b * sp.b)) : (R)0;
    const R inv_c3 = sp.kind == SCATMAN_ELLIPSOID ? (R)(1.0 / (sp.c * sp.c * sp.c)) : (R)0;
    const long long ncols = (long long)gp.nx * gp.ny;
    const long long wstride = (long long)gridDim.x * (kGradThreads / 32);
    for (long long col = (long long)blockIdx.x * (kGradThreads / 32) + warp; col < ncols; col += wstride) {
        const int ix = (int)(col / gp.ny), iy = (int)(col % gp.ny);
        R chi[kRun], rs[kRun], ux[kRun], uy[kRun], uz[kRun];
        int clip[kRun];
        C T[kRun], Rv[kRun];
        R local = (R)0;
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
            const int iz = lane * run + k;
            chi[k] = (R)0;
            if (k < run && iz < nz)
                soft_voxel<R, kMaxL>(sp, gp, ix, iy, iz, chi[k], rs[k], clip[k], ux[k], uy[k], uz[k]);
            local += chi[k];
        }
        R incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            R nb = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += nb;
        }
        R Cz = incl - local;
        C rsum;
        rsum.x = rsum.y = (R)0;
#pragma unroll
        for (int k = 0; k < kRun; ++k) {
            const int iz = lane * run + k;
            T[k].x = T[k].y = (R)0;
            Rv[k].x = Rv[k].y = (R)0;
            if (k < run && iz < nz) {
                // T = exp(i kdz (n-1) C) = e^{-kdz beta C} e^{-i kdz delta C}
                const R mag = exp(-kdz * nm1.y * Cz);
                R sn, cs;
                sincos(kdz * nm1.x * Cz, &sn, &cs);
                T[k].x = mag * cs;
                T[k].y = mag * sn;
                const C Sv = S[((size_t)iz * gp.nx + ix) * gp.ny + iy];
                C Sc;
                Sc.x = Sv.x;
                Sc.y = -Sv.y;
                Rv[k] = cmul(cst, Sc);
                C sv;
                sv.x = chi[k] * T[k].x;
                sv.y = chi[k] * T[k].y;
                const C rsv = cmul(Rv[k], sv);
                rsum.x += rsv.x;
                rsum.y += rsv.y;
                D.x += rsv.x * Cz;
                D.y += rsv.y * Cz;
                Cz += chi[k];
            }
        }
        // suffix over the lanes above: sum of rsum for lanes > lane
        C above = rsum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            R nx_ = __shfl_down_sync(0xffffffffu, above.x, o);
            R ny_ = __shfl_down_sync(0xffffffffu, above.y, o);
            if (lane + o < 32) {
                above.x += nx_;
                above.y += ny_;
            }
        }
        C suffix;
        suffix.x = above.x - rsum.x;
        suffix.y = above.y - rsum.y;
#pragma unroll
        for (int k = kRun - 1; k >= 0; --k) {
            if (k >= run) continue;                       // warp-uniform
            const int iz = lane * run + k;
            R w0 = (R)0, ct = (R)1, st = (R)0, cph = (R)1, sph = (R)0;
            if (iz < nz) {
                // chibar = R T + i kdz (n-1) suffix
                C t1 = cmul(Rv[k], T[k]);
                C t2 = cmul(nm1, suffix);
                const R re_chibar = t1.x - kdz * t2.y;
                const R coef = re_chibar * chi[k] * ((R)1 - chi[k]) * inv_w;
                C sv;
                sv.x = chi[k] * T[k].x;
                sv.y = chi[k] * T[k].y;
                const C rsv = cmul(Rv[k], sv);
                suffix.x += rsv.x;
                suffix.y += rsv.y;
                if (sp.kind == SCATMAN_SPHERE) {
                    acc[0] += coef;
                } else if (sp.kind == SCATMAN_ELLIPSOID) {
                    const R r3 = rs[k] * rs[k] * rs[k];
                    acc[0] += coef * r3 * ux[k] * ux[k] * inv_a3;
                    acc[1] += coef * r3 * uy[k] * uy[k] * inv_b3;
                    acc[2] += coef * r3 * uz[k] * uz[k] * inv_c3;
                } else if (clip[k] == 0) {
                    w0 = coef * R0;
                    ct = uz[k];
                    st = sqrt(ux[k] * ux[k] + uy[k] * uy[k]);
                    if (st > (R)0) {
                        cph = ux[k] / st;
                        sph = uy[k] / st;
                    }
                    acc[0] += coef * rs[k] * inv_R0;
                } else if (clip[k] < 0) {
                    acc[0] += coef * (R)0.1;
                }
            }
            // d radius / d a_lm = R0 Y_lm: every lane evaluates its direction (w0 = 0
            // where the voxel does not contribute)
            if (sh && __any_sync(0xffffffffu, w0 != (R)0)) {
                const ShTab<R> tb(sp);
                real_sh_all<R, kMaxL>(tb, sp.lmax, ct, st, cph, sph, [&](int idx, R y) {
                    if (idx == 0) return;
                    const int j = idx - 1;
                    if constexpr (kSmemAlm) {
                        my_alm[j * 32 + lane] += w0 * y;
                    } else {
                        R v = w0 * y;
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                        if (lane == (j & 31)) {
#pragma unroll
                            for (int q = 0; q < kGradWarpSlots; ++q)
                                if (q == (j >> 5)) aw[q] += v;
                        }
                    }
                });
            }
        }
    }
    // deterministic reduction: warp tree, then warps in order
    __shared__ double red[kGradThreads / 32][kMaxGeom + 2];
    // per-thread sums: sphere / ellipsoid parameters, or R0 (the last index)
    const int n_thread = sh ? 1 : ng;
    for (int k = 0; k < n_thread + 2; ++k) {
        double v = k < n_thread ? (double)acc[k] : (k == n_thread ? (double)D.x : (double)D.y);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        const int at = k < n_thread ? (sh ? ng - 1 : k) : ng + (k - n_thread);
        if (lane == 0) red[warp][at] = v;
    }
    if (sh && kSmemAlm) {
        // lane sums of coefficient j, added in the fixed order t = 0..31 over
        // lanes (j + t) % 32 (the rotation keeps the 32 reading lanes in 32 banks)
        __syncwarp();
        for (int j = lane; j < ng - 1; j += 32) {
            float v = 0.f;
#pragma unroll 8
            for (int t = 0; t < 32; ++t) v += my_alm[j * 32 + ((j + t) & 31)];
            red[warp][j] = (double)v;
        }
    } else if (sh) {
        // a_lm sums are already warp totals
#pragma unroll
        for (int q = 0; q < kGradWarpSlots; ++q) {
            const int j = 32 * q + lane;
            if (j < ng - 1) red[warp][j] = (double)aw[q];
        }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ng + 2; k += kGradThreads) {
        double s = 0.0;
        for (int w = 0; w < kGradThreads / 32; ++w) s += red[w][k];
        partials[(size_t)blockIdx.x * (ng + 2) + k] = s;
    }
}

// Dynamic shared memory of the FP32 voxel gradient: the harmonics' per-lane
// a_lm sums (8 warps x ((lmax + 1)^2 - 1) x 32 floats; 172 KB at lmax 12).
static size_t grad_voxel_smem(const ShapeParams &sp) {
    if (sp.kind != SCATMAN_SPHHARM) return 0;
    return (size_t)(kGradThreads / 32) * (size_t)(n_geom_params(sp.kind, sp.lmax) - 1) * 32 * sizeof(float);
}

template <typename R>
using GradVoxelFn = void (*)(ShapeParams, GridParams, const typename Cx<R>::T *, double *);

// The instantiation for this shape and grid: z run per lane from nz, and the
// short harmonic code (degree <= 6) for FP32 shapes that need no more.
template <typename R, int kMaxL>
static GradVoxelFn<R> grad_voxel_fn_l(int run) {
    if (run <= 2) return grad_voxel_kernel<R, 2, kMaxL>;
    if (run <= 4) return grad_voxel_kernel<R, 4, kMaxL>;
    if (run <= 8) return grad_voxel_kernel<R, 8, kMaxL>;
    return grad_voxel_kernel<R, 16, kMaxL>;
}

template <typename R>
static GradVoxelFn<R> grad_voxel_fn(const ShapeParams &sp, const GridParams &gp) {
    const int run = (gp.nz + 31) / 32;
    if constexpr (sizeof(R) == 8) {
        // FP64 (the accuracy mode, nz <= 256): two instantiations keep the build
        // short (the FP64 8-voxel form alone took minutes in ptxas); runs above
        // 2 take the 16-voxel form, whose per-lane arrays live in local memory
        (void)sp;
        return run <= 2 ? grad_voxel_kernel<R, 2, SCATMAN_MAX_LMAX> : grad_voxel_kernel<R, 16, SCATMAN_MAX_LMAX>;
    } else {
        if (sp.kind == SCATMAN_SPHHARM && sp.lmax > 6) return grad_voxel_fn_l<R, SCATMAN_MAX_LMAX>(run);
        return grad_voxel_fn_l<R, 6>(run);
    }
}

// Blocks of the voxel gradient: one per 8 columns, at most the resident count
// of the instantiation that runs (whole waves), and never above 608 (the
// serving footprint's bound on the partial sums).
int grad_voxel_blocks(bool fp64, const ShapeParams &sp, const GridParams &gp, int sm_count) {
    const long long cols = (long long)gp.nx * gp.ny;
    const long long b = (cols + (kGradThreads / 32) - 1) / (kGradThreads / 32);
    int per_sm = 0;
    bool ok;
    if (fp64) {
        ok = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, grad_voxel_fn<double>(sp, gp), kGradThreads, 0) ==
             cudaSuccess;
    } else {
        const auto fn = grad_voxel_fn<float>(sp, gp);
        const size_t smem = grad_voxel_smem(sp);
        ok = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
             cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kGradThreads, smem) == cudaSuccess;
    }
    if (!ok) {
        // a failed query only costs the whole-wave sizing; the launch reports real errors
        (void)cudaGetLastError();
        per_sm = 1;
    }
    long long cap = (long long)(sm_count > 0 ? sm_count : 1) * (per_sm > 0 ? per_sm : 1);
    if (cap > 608) cap = 608;
    return (int)(b < cap ? b : cap);
}

cudaError_t launch_grad_voxels(bool fp64, const ShapeParams &sp, const GridParams &gp, const void *S,
                               double *partials, int n_blocks, cudaStream_t st) {
    if (gp.nz > 32 * kGradMaxRun) return cudaErrorInvalidValue;
    if (fp64) {
        grad_voxel_fn<double>(sp, gp)<<<n_blocks, kGradThreads, 0, st>>>(sp, gp, (const double2 *)S, partials);
        return cudaGetLastError();
    }
    const auto fn = grad_voxel_fn<float>(sp, gp);
    const size_t smem = grad_voxel_smem(sp);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<n_blocks, kGradThreads, smem, st>>>(sp, gp, (const float2 *)S, partials);
    return cudaGetLastError();
}

// sum_q w_q |A_q|^2 per block.
template <typename R>
__global__ void grad_pixel_kernel(const typename Cx<R>::T *__restrict__ A, const R *__restrict__ w, long long n_pix,
                                  double *__restrict__ partials) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n_pix;
         p += (long long)gridDim.x * blockDim.x) {
        const auto a = A[p];
        s += (double)w[p] * ((double)a.x * a.x + (double)a.y * a.y);
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

int grad_pixel_blocks(long long n_pix) {
    long long b = (n_pix + 255) / 256;
    return (int)(b < 256 ? b : 256);
}

cudaError_t launch_grad_pixels(bool fp64, const void *A, const void *dLdI, long long n_pix, double *partials,
                               int n_blocks, cudaStream_t st) {
    if (fp64)
        grad_pixel_kernel<double><<<n_blocks, 256, 0, st>>>((const double2 *)A, (const double *)dLdI, n_pix, partials);
    else
        grad_pixel_kernel<float><<<n_blocks, 256, 0, st>>>((const float2 *)A, (const float *)dLdI, n_pix, partials);
    return cudaGetLastError();
}

}  // namespace scm

namespace scm {

// Least-squares fit residual: w = dL/dI = 2 (I - target) and per-block
// partial sums of (I - target)^2 (summed on the host in block order).
template <typename R>
__global__ void l2_residual_kernel(const R *__restrict__ I, const float *__restrict__ target, long long n,
                                   R *__restrict__ w, double *__restrict__ partials) {
    __shared__ double red[256];
    double s = 0.0;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const R d = I[p] - (R)target[p];
        w[p] = (R)2 * d;
        s += (double)d * (double)d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

int l2_residual_blocks(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 256 ? b : 256);
}

cudaError_t launch_l2_residual(bool fp64, const void *I, const float *target, long long n, void *w, double *partials,
                               int n_blocks, cudaStream_t st) {
    if (fp64)
        l2_residual_kernel<double><<<n_blocks, 256, 0, st>>>((const double *)I, target, n, (double *)w, partials);
    else
        l2_residual_kernel<float><<<n_blocks, 256, 0, st>>>((const float *)I, target, n, (float *)w, partials);
    return cudaGetLastError();
}

}  // namespace scm
