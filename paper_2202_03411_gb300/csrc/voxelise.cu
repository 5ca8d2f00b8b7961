// voxelise.cu -- detector q (Eq. 3) and the fused voxeliser + transmission
// scan (Block 5 + Block 9, Eq. 8 of arXiv 2202.03411).
//
// One CTA owns one x column-plane strip: a fixed x and 32 consecutive y lines.
// Each warp takes whole lines along z, 32 consecutive z per step (one per
// lane), and the exclusive prefix C_j = sum_{j'<j} chi is a warp-shuffle scan
// per step plus the running total of the earlier steps.  The slice strength
// s_j = chi_j exp(i k0 dz (n-1) C_j) is staged in shared memory and then
// written out so that consecutive threads store consecutive y -- the
// contraction's operand rows are y-contiguous.
#include "internal.cuh"
#include "shape_device.cuh"

namespace scm {

// ---------------------------------------------------------------------------
// a1: transfer momentum of every flat-detector pixel (Eq. 3).  The pixel sits
// at (X, Y, 1); k_out = k0 (X, Y, 1)/r and q = k_out - k0 z^.  q_z is written
// as -k0 (X^2+Y^2) / (r (1 + r)) to avoid cancellation near the axis.
// ---------------------------------------------------------------------------
__global__ void detector_q_kernel(int det_nx, int det_ny, double h, double k0, double *q) {
    long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long n = (long long)det_nx * det_ny;
    if (p >= n) return;
    int u = (int)(p % det_nx);
    int v = (int)(p / det_nx);
    double X = h * (double)(2 * u + 1 - det_nx) / (double)det_nx;
    double Y = h * (double)(2 * v + 1 - det_ny) / (double)det_ny;
    double rho2 = X * X + Y * Y;
    double r = sqrt(rho2 + 1.0);
    q[3 * p + 0] = k0 * X / r;
    q[3 * p + 1] = k0 * Y / r;
    q[3 * p + 2] = -k0 * rho2 / (r * (1.0 + r));
}

cudaError_t launch_detector_q(int det_nx, int det_ny, double theta_max_deg, double k0, double *q,
                              cudaStream_t st) {
    long long n = (long long)det_nx * det_ny;
    double h = tan(theta_max_deg * kPi / 180.0);
    int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    detector_q_kernel<<<(unsigned)blocks, threads, 0, st>>>(det_nx, det_ny, h, k0, q);
    return cudaGetLastError();
}

constexpr int kLinesPerCta = 32;
constexpr int kVoxThreads = 256;
constexpr int kMaxRun = 16;         // z values per lane: nz <= 512 (256 in the FP64 mode)
constexpr int kVoxQueue = 512;      // binary voxels per CTA whose FP64 decision is batched

// s_j = chi_j T_j with T_j = exp(i k0 dz (n-1) C_j) = e^{-k0 dz beta C} e^{-i k0 dz delta C}.
// A warp takes one (x, y) line at a time; its lanes take 32 consecutive z per
// step, so neighbouring lanes hold neighbouring voxels (and binary shapes can
// skip the surface radius where the whole step is clearly inside or outside).
// Pass 1 renders chi into shared memory for all of the CTA's lines; in the
// FP32 modes the few binary voxels too close to the surface for the FP32 test
// are queued and decided in FP64 afterwards by whole warps (a lone lane in
// the FP64 path would hold its warp for the full FP64 radius).  Pass 2 forms
// the exclusive prefix C_j with a warp scan per step plus the running total
// of earlier steps, then T_j and s_j.  Tiles are [line][z] with a padded row,
// so both the z-walk and the line-fastest output loop are free of bank
// conflicts.
// Per-launch constants of the scan, formed on the host in FP64 and handed
// over in both precisions (no FP64 arithmetic in the kernel's prologue).
struct VoxConst {
    double att, ph, kdz, inv_scale;         // k0 dz beta, k0 dz delta, k0 dz, 1 / nscale
    float att_f, ph_f, kdz_f, inv_scale_f;
};
template <typename T> __device__ __forceinline__ T vc_pick(double d, float f);
template <> __device__ __forceinline__ double vc_pick<double>(double d, float) { return d; }
template <> __device__ __forceinline__ float vc_pick<float>(double, float f) { return f; }

template <bool kFp64, typename ScanT, bool kMaps>
__global__ void __launch_bounds__(kVoxThreads, 3) voxelise_scan_kernel(ShapeParams sp, GridParams gp,
                                                                    SliceOut out, VoxConst vc) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nz = gp.nz;
    const int zs = nz + 1;                                                    // padded row
    using Cx = typename std::conditional<kFp64, double2, float2>::type;
    using Re = typename std::conditional<kFp64, double, float>::type;
    Cx *s_tile = reinterpret_cast<Cx *>(smem);                                // [32][zs]
    float *chi_tile = reinterpret_cast<float *>(smem + sizeof(Cx) * zs * kLinesPerCta);
    int *queue = reinterpret_cast<int *>(chi_tile + (size_t)zs * kLinesPerCta);   // (line << 16) | z
    __shared__ int s_qn;
    if (threadIdx.x == 0) s_qn = 0;
    __syncthreads();

    const int ix = blockIdx.x;
    const int y0 = blockIdx.y * kLinesPerCta;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int steps = (nz + 31) / 32;
    const ScanT a_att = vc_pick<ScanT>(vc.att, vc.att_f);         // attenuation per unit C
    const ScanT a_ph = vc_pick<ScanT>(vc.ph, vc.ph_f);             // phase per unit C
    const bool varn = kMaps && sp.varn != 0;                      // per-cell index of a volume map
    const ScanT kdz = vc_pick<ScanT>(vc.kdz, vc.kdz_f);
    const Re inv_scale = vc_pick<Re>(vc.inv_scale, vc.inv_scale_f);
    // radius band (harmonics, radii maps, soft spheres and ellipsoids): inside below lo, outside above hi
    // (the host sets none for FP64 soft occupancy)
    const bool band = (!kFp64 || !sp.soft) && sp.band_hi > 0.f;
    const float vox = gp.voxf;
    const float xo = ((float)ix - 0.5f * (float)(gp.nx - 1)) * vox - sp.cxf;

    for (int yl = warp; yl < kLinesPerCta; yl += kVoxThreads / 32) {
        const int iy = y0 + yl;
        if (iy >= gp.ny) break;
        const float yo = ((float)iy - 0.5f * (float)(gp.ny - 1)) * vox - sp.cyf;
        const float r2xy = xo * xo + yo * yo;
        Cx *srow = s_tile + (size_t)yl * zs;
        float *crow = chi_tile + (size_t)yl * zs;
        // pass 1: occupancy (and, with a per-cell index, the cells' delta and beta)
#pragma unroll 1
        for (int st = 0; st < steps; ++st) {
            const int iz = 32 * st + lane;
            Re c = (Re)0;                       // FP32 in the FP32 modes: no FP64 on the common path
            if (iz < nz) {
                bool decided = false;
                if (band) {
                    // |p| = |d|: the rotation keeps lengths; margins cover FP32 rounding
                    const float zo = ((float)iz - 0.5f * (float)(nz - 1)) * vox - sp.czf;
                    const float d = sqrtf(r2xy + zo * zo);
                    const float m = 1e-3f * vox + 1e-5f * d;
                    if (d + m < sp.band_lo) {
                        c = (Re)1;
                        decided = true;
                    } else if (d - m > sp.band_hi) {
                        decided = true;
                    }
                }
                if (!decided) {
                    if (varn) {
                        const int cell = vmap_cell<kFp64>(sp, gp, ix, iy, iz);
                        c = (cell >= 0 && sp.vmap[cell] != 0) ? (Re)1 : (Re)0;
                    } else {
                        c = (Re)occupancy<kFp64, kMaps, true>(sp, gp, ix, iy, iz);
                        if (!kFp64 && c < (Re)0) {
                            // too close to the surface for FP32: queue it (inline when full)
                            const int slot = atomicAdd(&s_qn, 1);
                            if (slot < kVoxQueue)
                                queue[slot] = (yl << 16) | iz;
                            else
                                c = (Re)occupancy_binary_fp64(sp, gp, ix, iy, iz);
                        }
                    }
                }
                if (kFp64) srow[iz].x = c;                                // exact copy until pass 2
                crow[iz] = (float)c;
            }
        }
    }
    __syncthreads();
    if (!kFp64) {
        // the queued voxels' FP64 decisions: harmonics one voxel per warp (its
        // lanes split the orders; coefficient tables staged in the slice tile,
        // which the FP32 modes leave unused until pass 2, when it is large
        // enough), other kinds one voxel per thread
        const int qn = min(s_qn, kVoxQueue);
        const bool warp_sh = !kMaps && sp.kind == SCATMAN_SPHHARM &&
                             sizeof(Cx) * (size_t)zs * kLinesPerCta >= kShTabDoubles * sizeof(double);
        if (warp_sh && qn > 0) {
            double *tab = reinterpret_cast<double *>(s_tile);
            sh_stage_tables(sp, tab);
            __syncthreads();
            for (int k = warp; k < qn; k += kVoxThreads / 32) {
                const int e = queue[k];
                const int yl = e >> 16, iz = e & 0xffff;
                const double in = sh_binary_fp64_warp(sp, gp, ix, y0 + yl, iz, tab);
                if (lane == 0) chi_tile[(size_t)yl * zs + iz] = (float)in;
            }
        } else {
            for (int k = threadIdx.x; k < qn; k += kVoxThreads) {
                const int e = queue[k];
                const int yl = e >> 16, iz = e & 0xffff;
                chi_tile[(size_t)yl * zs + iz] = (float)occupancy_binary_fp64(sp, gp, ix, y0 + yl, iz);
            }
        }
        __syncthreads();
    }

    for (int yl = warp; yl < kLinesPerCta; yl += kVoxThreads / 32) {
        const int iy = y0 + yl;
        if (iy >= gp.ny) break;
        Cx *srow = s_tile + (size_t)yl * zs;
        float *crow = chi_tile + (size_t)yl * zs;
        // pass 2: exclusive prefix along z, transmission, slice value
        ScanT carry = (ScanT)0, carry_d = (ScanT)0, carry_b = (ScanT)0;
#pragma unroll 1
        for (int st = 0; st < steps; ++st) {
            const int iz = 32 * st + lane;
            const Re chi = iz < nz ? (kFp64 ? (Re)srow[iz].x : (Re)crow[iz]) : (Re)0;
            if (varn) {
                // voxel-resolved index: T_j = exp(i k0 dz sum_{j'<j} chi (n_v - 1)),
                // s = chi (n_v^2 - 1) T / nscale (Eq. 8-9 with one n per voxel)
                double dl = 0.0, bt = 0.0;
                if (chi != (Re)0) {
                    const int cell = vmap_cell<kFp64>(sp, gp, ix, iy, iz);
                    dl = sp.mdelta[cell];
                    bt = sp.mbeta[cell];
                }
                const ScanT ed = (ScanT)(chi * (Re)dl), eb = (ScanT)(chi * (Re)bt);
                ScanT id = ed, ib = eb;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const ScanT a = __shfl_up_sync(0xffffffffu, id, o);
                    const ScanT b = __shfl_up_sync(0xffffffffu, ib, o);
                    if (lane >= o) {
                        id += a;
                        ib += b;
                    }
                }
                const ScanT Cd = carry_d + id - ed, Cb = carry_b + ib - eb;
                carry_d += __shfl_sync(0xffffffffu, id, 31);
                carry_b += __shfl_sync(0xffffffffu, ib, 31);
                if (iz < nz) {
                    Cx v;
                    v.x = v.y = (Re)0;
                    if (chi != (Re)0) {
                        const ScanT mag = exp(-kdz * Cb);
                        ScanT sn, cs;
                        sincos(kdz * Cd, &sn, &cs);
                        const Re sr = (Re)((-2.0 * dl + dl * dl - bt * bt)) * inv_scale;
                        const Re si = (Re)((2.0 * bt - 2.0 * dl * bt)) * inv_scale;
                        const Re tr = (Re)(mag * cs), ti = -(Re)(mag * sn);
                        v.x = chi * (sr * tr - si * ti);
                        v.y = chi * (sr * ti + si * tr);
                    }
                    srow[iz] = v;
                }
                continue;
            }
            ScanT incl = (ScanT)chi;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const ScanT nb = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += nb;
            }
            const ScanT C = carry + incl - (ScanT)chi;
            carry += __shfl_sync(0xffffffffu, incl, 31);
            if (iz < nz) {
                Cx v;
                v.x = v.y = (Re)0;                 // s = chi T vanishes with chi: no T needed
                if (chi != (Re)0) {
                    const ScanT mag = exp(-a_att * C);
                    ScanT sn, cs;
                    sincos(a_ph * C, &sn, &cs);
                    v.x = chi * (Re)(mag * cs);
                    v.y = -chi * (Re)(mag * sn);
                }
                srow[iz] = v;
            }
        }
    }
    __syncthreads();

    const int ny_here = min(kLinesPerCta, gp.ny - y0);
    const long long nxy = (long long)gp.nx * gp.ny;
    if (out.bounds) {
        // occupied box of each slice (order-independent min/max)
        for (int iz = threadIdx.x; iz < nz; iz += kVoxThreads) {
            int lo = kLinesPerCta, hi = -1;
            for (int yl = 0; yl < ny_here; ++yl)
                if (chi_tile[(size_t)yl * (nz + 1) + iz] != 0.f) {
                    lo = min(lo, yl);
                    hi = yl;
                }
            if (hi >= 0) {
                atomicMin(&out.bounds[iz], ix);
                atomicMax(&out.bounds[nz + iz], ix + 1);
                atomicMin(&out.bounds[2 * nz + iz], y0 + lo);
                atomicMax(&out.bounds[3 * nz + iz], y0 + hi + 1);
                if (out.chunk_y) {
                    // y range of this slice's 8-column chunk (tensor-core grids: ix < 8 kGeomChunks)
                    const int c = iz * kGeomChunks + (ix >> 3);
                    atomicMin(&out.chunk_y[c], y0 + lo);
                    atomicMax(&out.chunk_y[kGeomChunks * nz + c], y0 + hi + 1);
                }
            }
        }
    }
    for (int it = threadIdx.x; it < nz * kLinesPerCta; it += kVoxThreads) {
        const int iz = it / kLinesPerCta, yl = it % kLinesPerCta;
        if (yl >= ny_here) continue;
        const int iy = y0 + yl;
        const Cx v = s_tile[(size_t)yl * (nz + 1) + iz];
        const long long vidx = iz * nxy + (long long)ix * gp.ny + iy;
        out.chi[vidx] = chi_tile[(size_t)yl * (nz + 1) + iz];
        if (out.layout == kLayoutC64) {
            reinterpret_cast<double2 *>(out.s)[vidx] = make_double2((double)v.x, (double)v.y);
        } else if (out.layout == kLayoutC32) {
            reinterpret_cast<float2 *>(out.s)[vidx] = make_float2((float)v.x, (float)v.y);
        } else {
            // tensor-core slice operand: three planes per slice, rows
            // (3j + 0) Nxp + x = -Im s, (3j + 1) Nxp + x = Re s, (3j + 2) Nxp + x = Im s,
            // each row running over y (msft_tc.cu reads [Re | Im] and [-Im | Re] windows)
            const size_t row_n = (size_t)iz * 3 * out.Nxp + ix;
            const size_t row_r = row_n + out.Nxp;
            const size_t row_i = row_r + out.Nxp;
            const float sr = (float)v.x, si = (float)v.y;
            if (out.layout == kLayoutTcF16) {
                __half *B = reinterpret_cast<__half *>(out.s);
                B[row_n * out.Kp + iy] = __float2half_rn(-si);
                B[row_r * out.Kp + iy] = __float2half_rn(sr);
                B[row_i * out.Kp + iy] = __float2half_rn(si);
            } else {
                __nv_bfloat16 *B = reinterpret_cast<__nv_bfloat16 *>(out.s);
                B[row_n * out.Kp + iy] = __float2bfloat16_rn(-si);
                B[row_r * out.Kp + iy] = __float2bfloat16_rn(sr);
                B[row_i * out.Kp + iy] = __float2bfloat16_rn(si);
            }
        }
    }
}

__global__ void bounds_init_kernel(int *b, int nz, int *cy) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 4 * nz) {
        const int part = i / nz;
        b[i] = (part == 0 || part == 2) ? 0x7fffffff : 0;     // lo parts start high, hi parts low
    }
    if (cy && i < 2 * kGeomChunks * nz) cy[i] = i < kGeomChunks * nz ? 0x7fffffff : 0;
}

cudaError_t launch_voxelise(const ShapeParams &sp, const GridParams &gp, const SliceOut &out, bool scan_fp64,
                            bool fp64_mode, cudaStream_t st) {
    if (gp.nz > 32 * kMaxRun || (fp64_mode && gp.nz > 256)) return cudaErrorInvalidValue;
    if (out.chunk_y && (out.bounds == nullptr || gp.nx > 8 * kGeomChunks)) return cudaErrorInvalidValue;
    if (out.bounds)
        bounds_init_kernel<<<(2 * kGeomChunks * gp.nz + 255) / 256, 256, 0, st>>>(out.bounds, gp.nz, out.chunk_y);
    dim3 grid(gp.nx, (gp.ny + kLinesPerCta - 1) / kLinesPerCta);
    size_t cx = fp64_mode ? sizeof(double2) : sizeof(float2);
    size_t smem = (cx + sizeof(float)) * (size_t)(gp.nz + 1) * kLinesPerCta + kVoxQueue * sizeof(int);
    // per-function attribute shared by all threads: set it to the largest size
    // (nz = 256) so a concurrent launch from another thread is never rejected
    const int smem_max = (int)((cx + sizeof(float)) * ((fp64_mode ? 256 : 32 * kMaxRun) + 1) * kLinesPerCta +
                               kVoxQueue * sizeof(int));
    const bool maps = sp.kind == SCATMAN_RADIALMAP || sp.kind == SCATMAN_VOLUMEMAP;
    auto k = fp64_mode   ? (maps ? voxelise_scan_kernel<true, double, true> : voxelise_scan_kernel<true, double, false>)
             : scan_fp64 ? (maps ? voxelise_scan_kernel<false, double, true> : voxelise_scan_kernel<false, double, false>)
                         : (maps ? voxelise_scan_kernel<false, float, true> : voxelise_scan_kernel<false, float, false>);
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_max);
    if (e != cudaSuccess) return e;
    VoxConst vc;
    vc.att = gp.k0 * gp.voxel * gp.beta;
    vc.ph = gp.k0 * gp.voxel * gp.delta;
    vc.kdz = gp.k0 * gp.voxel;
    vc.inv_scale = sp.nscale != 0.0 ? 1.0 / sp.nscale : 0.0;
    vc.att_f = (float)vc.att;
    vc.ph_f = (float)vc.ph;
    vc.kdz_f = (float)vc.kdz;
    vc.inv_scale_f = (float)vc.inv_scale;
    k<<<grid, kVoxThreads, smem, st>>>(sp, gp, out, vc);
    return cudaGetLastError();
}

}  // namespace scm
