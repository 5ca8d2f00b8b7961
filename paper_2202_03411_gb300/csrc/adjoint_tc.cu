// adjoint_tc.cu -- tensor-core (tcgen05) form of the adjoint field
//   S[j, x, y] = sum_q g_q e^{+i (q_x x + q_y y + q_z z_j)},   g_q = w_q A_q,
// the transpose of Eq. 9's contraction that the gradient needs.
//
// Per slice j it is one complex GEMM over the pixels:
//   S_j[x, y] = sum_q L_j[x, q] R[q, y],
//   L_j[x, q] = (g_q / g_max) e^{+i q_z z_j} e^{+i q_x x},   R[q, y] = e^{+i q_y y},
// real-ified with K = pixels x {re, im} (the re/im pair of one pixel adjacent
// in K) and N = [Re S: y | Im S: y]:
//   A[x, 2p] = Re L, A[x, 2p+1] = Im L,
//   B[(y,re), 2p] = Re R, B[(y,re), 2p+1] = -Im R,
//   B[(y,im), 2p] = Im R, B[(y,im), 2p+1] = Re R.
// The y-phase operand R depends only on the pixels, so it is built once per
// handle as the tile image the MMA reads (128-byte swizzle, FP16, |R| <= 1) and
// copied into each stage with one bulk copy; the x-phase operand L depends on
// the slice and the weights, so eight generator warps build it in shared
// memory (phase recurrences, FP16 with |L| <= 1), rows x < nx only (padding
// rows feed output rows that are never written back), in teams of two that
// take successive chunks, while one MMA warp consumes the finished stages.  Per-pixel constants (q split into FP32 pairs,
// one-voxel rotations) come from a table built once per handle, so the
// generators do no FP64 work.  A CTA owns two slices (two TMEM accumulators
// sharing every R tile) and a contiguous range of pixels; the pixel ranges'
// partial fields are summed in a fixed order afterwards.
//
// Order mode.  The slice factor e^{+i q_z z_j} is the only part of L_j that
// depends on j.  With q_z = q_c + D u (u in [-1, 1] over the pixels) the
// Jacobi-Anger expansion
//   e^{+i q_z z_j} = e^{+i q_c z_j} sum_{n >= 0} eps_n i^n J_n(D z_j) T_n(u),
//   T_n(u) = cos(n theta), theta = acos(u), eps_0 = 1, eps_n = 2,
// truncated after N orders (|J_n(w)| <= (|w|/2)^n / n!, so the tail is below
// 1e-7 of sum_q |g_q| for the N chosen on the host) turns the nz slice GEMMs into
// N order GEMMs S~_n[x, y] = sum_q g_q cos(n theta_q) e^{+i (q_x x + q_y y)}: the
// same kernel, with the order n in place of the slice and the real factor
// cos(n theta_q) in place of the slice phase; adj_orders_combine_kernel then
// forms S_j = sum_n a[j, n] S~_n with a[j, n] = e^{+i q_c z_j} eps_n i^n J_n(D z_j).
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace scm {

constexpr int kAdjGenWarps = 8;             // build the x-phase operand, then the epilogue
constexpr int kAdjLoadWarp = kAdjGenWarps;  // bulk-copies the y-phase operand
constexpr int kAdjMmaWarp = kAdjGenWarps + 1;
constexpr int kAdjThreads = (kAdjGenWarps + 2) * 32;
constexpr int kAdjChunk = 32;                 // pixels per K block (64 real K = 128 bytes)
constexpr int kAdjMaxStages = 6;
constexpr int kAdjRows = 128;                 // M: x rows
constexpr int kAdjTileA = kAdjRows * 128;     // one A tile: 128 rows x 128 bytes
constexpr int kAdjMaxSplits = 8;             // bounds the partial-field memory to 8 fields (slice mode)
constexpr int kAdjMaxSplitsOrders = 32;      // order mode: few order pairs, 2D partial fields

struct AdjParams {
    const float4 *tab;          // per pixel: (qxh, qxl, qyh, qyl), (qzh, qzl, e^{+i qx dv}), (e^{+i qy dv}, e^{+i qz dv});
                                // order mode: theta (hi, lo) in place of q_z and e^{+i theta} in place of e^{+i qz dv}
    int orders;                 // 1: order mode (nz below is the number of orders N)
    const uint8_t *rtile;       // per 32-pixel chunk: the y-phase operand tile (2 Nyp rows x 128 bytes)
    int stages;
    int teams;                  // generator teams (1, 2 or 4; never more than stages)
    const float2 *A;            // forward field (FP32)
    const float *w;             // dL/dI
    const unsigned *gmax_bits;  // max |w A| as float bits
    long long n_pix;
    int nx, ny, nz, Nyp;
    int pix_per_split;          // multiple of kAdjChunk
    double voxel;
    uint32_t idesc;
    uint32_t tmem_cols;
    float2 *partial;            // [split][z][x][y]
    long long nvox;
    int *err;
};

// Byte offset of the 4-byte (re, im) pair of pixel i in row r of a
// 128-byte-swizzled K-major tile (k = 2i).
__device__ __forceinline__ uint32_t pair_offset(int r, int i) {
    return (uint32_t)(r * 128 + ((((i >> 2) ^ (r & 7))) << 4) + ((i & 3) << 2));
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Per-pixel constants of the generators: q as FP32 pairs and e^{+i q dv}; in
// order mode (inv_d > 0) theta = acos((q_z - q_c) inv_d) replaces q_z and
// e^{+i theta} replaces e^{+i q_z dv}.
__global__ void adj_pixel_table_kernel(const double *__restrict__ q, long long n, double voxel, int orders,
                                       double qc, double inv_d, float4 *__restrict__ tab) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double qx = q[3 * p], qy = q[3 * p + 1];
    double qz = q[3 * p + 2];
    const float vf = (float)voxel;
    float zstep = vf;
    if (orders) {
        const double u = fmin(1.0, fmax(-1.0, (qz - qc) * inv_d));
        qz = acos(u);
        zstep = 1.0f;
    }
    const float qxh = (float)qx, qxl = (float)(qx - (double)qxh);
    const float qyh = (float)qy, qyl = (float)(qy - (double)qyh);
    const float qzh = (float)qz, qzl = (float)(qz - (double)qzh);
    // e^{+i t} = conj(e^{-i t}) = expmi(q, -c)
    const float2 ex = expmi_fs(qxh, qxl, -vf), ey = expmi_fs(qyh, qyl, -vf), ez = expmi_fs(qzh, qzl, -zstep);
    tab[3 * p] = make_float4(qxh, qxl, qyh, qyl);
    tab[3 * p + 1] = make_float4(qzh, qzl, ex.x, ex.y);
    tab[3 * p + 2] = make_float4(ey.x, ey.y, ez.x, ez.y);
}

cudaError_t launch_adj_pixel_table(const double *q, long long n, double voxel, int orders, double qc, double inv_d,
                                   float4 *tab, cudaStream_t st) {
    adj_pixel_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(q, n, voxel, orders, qc, inv_d, tab);
    return cudaGetLastError();
}

// The y-phase operand, per 32-pixel chunk, as the tile image the MMA reads:
// row y holds (Re R, -Im R) and row Nyp + y holds (Im R, Re R) for each pixel,
// R = e^{+i q_y y} (zero past the last pixel).
__global__ void adj_rtile_kernel(const float4 *__restrict__ tab, long long n_pix, int Nyp, int ny, double voxel,
                                 uint8_t *__restrict__ rt, long long total) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    const int i = (int)(idx % kAdjChunk);
    const int y = (int)((idx / kAdjChunk) % Nyp);
    const long long cg = idx / ((long long)kAdjChunk * Nyp);
    const long long p = cg * kAdjChunk + i;
    float2 R = make_float2(0.f, 0.f);
    if (p < n_pix) {
        const float4 ta = tab[3 * p];
        const float yv = ((float)y - 0.5f * (float)(ny - 1)) * (float)voxel;
        R = expmi_fs(ta.z, ta.w, -yv);           // e^{+i q_y y}
    }
    uint8_t *tile = rt + cg * (long long)(2 * Nyp * 128);
    *reinterpret_cast<uint32_t *>(tile + pair_offset(y, i)) = pack_half2(R.x, -R.y);
    *reinterpret_cast<uint32_t *>(tile + pair_offset(Nyp + y, i)) = pack_half2(R.y, R.x);
}

size_t adj_rtile_bytes(long long n_pix, int ny) {
    const int Nyp = ((ny + 7) / 8 * 8 + 15) / 16 * 16;
    return (size_t)((n_pix + kAdjChunk - 1) / kAdjChunk) * 2 * Nyp * 128;
}

cudaError_t launch_adj_rtile(const float4 *tab, long long n_pix, int ny, double voxel, uint8_t *rt, cudaStream_t st) {
    const int Nyp = ((ny + 7) / 8 * 8 + 15) / 16 * 16;
    const long long total = (n_pix + kAdjChunk - 1) / kAdjChunk * kAdjChunk * Nyp;
    adj_rtile_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(tab, n_pix, Nyp, ny, voxel, rt, total);
    return cudaGetLastError();
}

__global__ void __launch_bounds__(kAdjThreads, 1) adjoint_tc_kernel(const AdjParams P) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int Nn = 2 * P.Nyp;                               // real output columns per slice
    const uint32_t b_bytes = (uint32_t)Nn * 128;
    const uint32_t stage_bytes = 2 * kAdjTileA + b_bytes;
    const int NS = P.stages;
    uint64_t *bars = reinterpret_cast<uint64_t *>(base + NS * stage_bytes);
    uint64_t *full = bars;                          // x-phase operand written (generator warps)
    uint64_t *bfull = bars + kAdjMaxStages;         // y-phase operand copied (bytes)
    uint64_t *empty = bars + 2 * kAdjMaxStages;
    uint64_t *done = bars + 3 * kAdjMaxStages;
    uint64_t *never = done + 1;                     // no thread arrives here (the failure-path test waits on it)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(never + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = 2 * blockIdx.x;                          // slices j0, j0 + 1
    const long long p_begin = (long long)blockIdx.y * P.pix_per_split;
    const long long p_end = min(P.n_pix, p_begin + P.pix_per_split);
    const int n_chunks = p_end > p_begin ? (int)((p_end - p_begin + kAdjChunk - 1) / kAdjChunk) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), kAdjGenWarps / P.teams);
            mbar_init(smem_u32(&bfull[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(done), 1);
        mbar_init(smem_u32(never), 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == kAdjMmaWarp) {
        tmem_alloc(smem_u32(tmem_slot), P.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == kAdjMmaWarp) {
        // warp-wide loop; one elected lane issues the MMAs and commits
        const uint32_t d0 = tmem_base, d1 = tmem_base + (uint32_t)Nn;
        const uint64_t desc0 = sw128_desc(smem_u32(base));
        const bool stalled =
            stall_requested(P.err) && !warp_wait(smem_u32(never), 0, abort_flag, P.err, kErrTimeoutMma);
        for (int c = 0; c < (stalled ? 0 : n_chunks); ++c) {
            const uint32_t s = c % NS, ph = (c / NS) & 1;
            if (!warp_wait(smem_u32(&full[s]), ph, abort_flag, P.err, kErrTimeoutMma)) break;
            if (!warp_wait(smem_u32(&bfull[s]), ph, abort_flag, P.err, kErrTimeoutMma)) break;
            tc_fence_after();
            // descriptors advance by encoded (>> 4) byte offsets
            const uint64_t a0 = desc0 + (uint64_t)((s * stage_bytes) >> 4);
            const uint64_t a1 = a0 + (uint64_t)(kAdjTileA >> 4), bb = a0 + (uint64_t)((2 * kAdjTileA) >> 4);
            if (elect_one()) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint32_t acc = (c | kk) != 0;
                    mma_f16(d0, a0 + (uint64_t)(2 * kk), bb + (uint64_t)(2 * kk), P.idesc, acc);
                    mma_f16(d1, a1 + (uint64_t)(2 * kk), bb + (uint64_t)(2 * kk), P.idesc, acc);
                }
                mma_commit(smem_u32(&empty[s]));
            }
            __syncwarp();
        }
        if (elect_one()) mma_commit(smem_u32(done));
        __syncwarp();
    } else if (warp == kAdjLoadWarp) {
        // ---------------- y-phase operand: one bulk copy per chunk ----------------
        const uint8_t *src = P.rtile + (size_t)(p_begin / kAdjChunk) * b_bytes;
        int issued = 0;
        for (int c = 0; c < n_chunks; ++c) {
            const uint32_t s = c % NS, ph = (c / NS) & 1;
            if (!warp_wait(smem_u32(&empty[s]), ph ^ 1, abort_flag, P.err, kErrTimeoutProducer)) break;
            if (elect_one()) {
                const uint32_t fb = smem_u32(&bfull[s]);
                mbar_arrive_expect_tx(fb, b_bytes);
                bulk_load(smem_u32(base + s * stage_bytes + 2 * kAdjTileA), src + (size_t)c * b_bytes, b_bytes, fb);
            }
            __syncwarp();
            ++issued;
        }
        // copies still in flight land before the CTA exits
        if (*abort_flag && lane == 0) {
            volatile int dummy = 0;
            for (int c = issued > NS ? issued - NS : 0; c < issued; ++c)
                mbar_wait(smem_u32(&bfull[c % NS]), (c / NS) & 1, &dummy, P.err, kErrTimeoutDrain);
        }
        __syncwarp();
    } else {
        // ---------------- generator warps: the x-phase operand ----------------
        // Teams of warps take whole chunks in turn (chunk c: team c % teams),
        // each warp a share of the rows, so a lane's per-chunk set-up (weights,
        // start phases) serves more rows.  A team's next chunk reuses a stage
        // only after the chunk `stages` earlier has been consumed, which with
        // teams <= stages keeps every stage barrier within one phase of its
        // waiters (the parity waits need that).
        const float inv_g = 1.0f / fmaxf(__uint_as_float(*P.gmax_bits), 1e-30f);
        const int i = lane;                      // pixel within the chunk
        const int per_team = kAdjGenWarps / P.teams;
        const int team = warp / per_team;
        // rows r0 .. r1 - 1 of both slices' L tiles (x < nx only)
        const int ra = (P.nx + per_team - 1) / per_team;
        const int r0 = (warp % per_team) * ra, r1 = min(P.nx, r0 + ra);
        const float vox = (float)P.voxel;
        const float x0 = ((float)r0 - 0.5f * (float)(P.nx - 1)) * vox;
        // slice mode: z of slice j0 (the factor e^{+i q_z z}); order mode: the order
        // j0 (the factor e^{+i j0 theta}, stepped by e^{+i theta} to order j0 + 1)
        const float zj = P.orders ? (float)j0 : ((float)j0 - 0.5f * (P.nz - 1)) * vox;
        // this lane's pixel data, loaded one chunk ahead so the L2 latency
        // overlaps the previous chunk's generation
        float2 a_n = make_float2(0.f, 0.f);
        float w_n = 0.f;
        float4 ta_n = make_float4(0.f, 0.f, 0.f, 0.f), tb_n = ta_n, tc_n = ta_n;
        auto load_pixel = [&](int c) {
            const long long p = p_begin + (long long)c * kAdjChunk + i;
            if (c < n_chunks && p < p_end && r0 < r1) {
                a_n = P.A[p];
                w_n = P.w[p];
                ta_n = P.tab[3 * p];
                tb_n = P.tab[3 * p + 1];
                tc_n = P.tab[3 * p + 2];
            } else {
                a_n = make_float2(0.f, 0.f);
                w_n = 0.f;
                ta_n = tb_n = tc_n = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        load_pixel(team);
        for (int c = team; c < n_chunks; c += P.teams) {
            const float2 a_c = a_n;
            const float w_c = w_n;
            const float4 ta = ta_n, tb = tb_n, tcv = tc_n;
            load_pixel(c + P.teams);
            const uint32_t s = c % NS, ph = (c / NS) & 1;
            if (!warp_wait(smem_u32(&empty[s]), ph ^ 1, abort_flag, P.err, kErrTimeoutEpilogue)) break;
            uint8_t *sA0 = base + s * stage_bytes;
            uint8_t *sA1 = sA0 + kAdjTileA;
            if (r0 < r1) {
                const float wp = w_c * inv_g;
                const float2 g = make_float2(a_c.x * wp, a_c.y * wp);
                // e^{+i t} = conj(e^{-i t}) = expmi(q, -c)
                const float2 ez = expmi_fs(tb.x, tb.y, -zj);
                const float2 ezs = make_float2(tcv.z, tcv.w);
                const float2 ex = expmi_fs(ta.x, ta.y, -x0);
                const float2 exs = make_float2(tb.z, tb.w);
                if (P.orders) {
                    // orders j0 and j0 + 1: real factors c0 = cos(j0 theta), c1 = cos((j0 + 1) theta)
                    // of one complex row value G_r = g e^{+i q_x x_r}, rotated row by row
                    const float c0 = ez.x, c1 = ez.x * ezs.x - ez.y * ezs.y;
                    float2 G = cmul(g, ex);
                    auto put = [&](uint8_t *d0, uint8_t *d1) {
                        *reinterpret_cast<uint32_t *>(d0) = pack_half2(c0 * G.x, c0 * G.y);
                        *reinterpret_cast<uint32_t *>(d1) = pack_half2(c1 * G.x, c1 * G.y);
                        G = cmul(G, exs);
                    };
                    int r = r0;
                    for (; r < r1 && (r & 7) != 0; ++r) put(sA0 + pair_offset(r, i), sA1 + pair_offset(r, i));
                    if (r + 8 <= r1) {
                        // whole groups of 8 rows (one swizzle period): this lane's offsets
                        // within a group, the group base advancing by 1 KB
                        uint32_t o[8];
#pragma unroll
                        for (int k = 0; k < 8; ++k) o[k] = pair_offset(k, i);
                        uint8_t *g0 = sA0 + (size_t)r * 128, *g1 = sA1 + (size_t)r * 128;
                        for (; r + 8 <= r1; r += 8, g0 += 1024, g1 += 1024) {
#pragma unroll
                            for (int k = 0; k < 8; ++k) put(g0 + o[k], g1 + o[k]);
                        }
                    }
                    for (; r < r1; ++r) put(sA0 + pair_offset(r, i), sA1 + pair_offset(r, i));
                } else {
                    float2 L0 = cmul(cmul(g, ez), ex);       // slice j0, row r0
#pragma unroll 4
                    for (int r = r0; r < r1; ++r) {
                        const float2 L1 = cmul(L0, ezs);
                        const uint32_t off = pair_offset(r, i);
                        *reinterpret_cast<uint32_t *>(sA0 + off) = pack_half2(L0.x, L0.y);
                        *reinterpret_cast<uint32_t *>(sA1 + off) = pack_half2(L1.x, L1.y);
                        L0 = cmul(L0, exs);
                    }
                }
            }
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&full[s]));
        }
        // ---------------- epilogue: accumulators -> partial field ----------------
        volatile int dummy = 0;
        const bool ok = n_chunks == 0 ? false : mbar_wait(smem_u32(done), 0, abort_flag, P.err, kErrTimeoutEpilogue);
        (void)dummy;
        tc_fence_after();
        const int quarter = warp & 3, part = warp >> 2;   // TMEM lane quarter; column groups part, part + 4, ...
        const int x = quarter * 32 + lane;
        const float gmax = fmaxf(__uint_as_float(*P.gmax_bits), 1e-30f);
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        const int ych = P.Nyp / 16;                       // 16-column groups per part
        float2 *out = P.partial + (size_t)blockIdx.y * P.nvox;
        for (int sl = 0; sl < 2; ++sl) {
            const int j = j0 + sl;
            for (int gq = part; gq < ych; gq += kAdjGenWarps / 4) {
                float re[16], im[16];
                tmem_ld16(lane_base + (uint32_t)(sl * Nn + 16 * gq), re);
                tmem_ld16(lane_base + (uint32_t)(sl * Nn + P.Nyp + 16 * gq), im);
                tmem_ld_wait(re, im);
                if (ok && j < P.nz && x < P.nx) {
                    float2 *row = out + ((size_t)j * P.nx + x) * P.ny;
#pragma unroll
                    for (int k = 0; k < 16; ++k) {
                        const int y = 16 * gq + k;
                        if (y < P.ny) row[y] = make_float2(re[k] * gmax, im[k] * gmax);
                    }
                } else if (j < P.nz && x < P.nx && n_chunks == 0) {
                    float2 *row = out + ((size_t)j * P.nx + x) * P.ny;
                    for (int k = 0; k < 16; ++k) {
                        const int y = 16 * gq + k;
                        if (y < P.ny) row[y] = make_float2(0.f, 0.f);
                    }
                }
            }
        }
        tc_fence_before();
    }
    __syncthreads();
    if (*abort_flag && warp == kAdjMmaWarp && lane == 0) {
        // make sure no MMA is still writing tensor memory before it is freed
        volatile int dummy = 0;
        mma_commit(smem_u32(done));
        mbar_wait(smem_u32(done), 1, &dummy, P.err, kErrTimeoutDrain);
    }
    __syncthreads();
    if (warp == kAdjMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem_base, P.tmem_cols);
    }
}

// max_q |w_q A_q| as float bits (non-negative floats order like their bits).
__global__ void adj_gmax_kernel(const float2 *__restrict__ A, const float *__restrict__ w, long long n,
                                unsigned *__restrict__ gmax_bits) {
    float m = 0.f;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (long long)gridDim.x * blockDim.x) {
        const float2 a = A[p];
        m = fmaxf(m, fabsf(w[p]) * sqrtf(a.x * a.x + a.y * a.y));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(gmax_bits, __float_as_uint(m));
}

// S = sum over pixel ranges of the partial fields, in range order.
__global__ void adj_sum_kernel(const float2 *__restrict__ partial, int splits, long long nvox, float2 *__restrict__ S) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    float2 s = partial[v];
    for (int k = 1; k < splits; ++k) {
        const float2 t = partial[(size_t)k * nvox + v];
        s.x += t.x;
        s.y += t.y;
    }
    S[v] = s;
}

static size_t adj_stage_bytes(int Nyp) { return 2 * (size_t)kAdjTileA + (size_t)2 * Nyp * 128; }
static size_t adj_fixed_bytes() { return 1024 + 256; }   // alignment, barriers
// Stages that fit beside the barriers (at most kAdjMaxStages).
static int adj_stages(int Nyp) {
    const size_t n = (232448 - adj_fixed_bytes()) / adj_stage_bytes(Nyp);
    return (int)(n > (size_t)kAdjMaxStages ? kAdjMaxStages : n);
}
static size_t adj_smem_bytes(int Nyp) { return adj_fixed_bytes() + (size_t)adj_stages(Nyp) * adj_stage_bytes(Nyp); }

static int adj_nyp(int ny) {
    const int Nyp = (ny + 7) / 8 * 8;
    return Nyp % 16 != 0 ? (Nyp + 15) / 16 * 16 : Nyp;   // 16-column epilogue groups
}

bool adjoint_tc_supported(int nx, int ny) {
    const int Nyp = adj_nyp(ny);
    return nx <= kAdjRows && Nyp <= 128 && adj_stages(Nyp) >= 2;
}

// Pixel ranges per slice (or order) pair: balance the grid over the SMs (1 CTA per SM).
int adjoint_tc_splits(long long n_pix, int nz, int sm_count, bool orders) {
    const int pairs = (nz + 1) / 2;
    const long long max_split = (n_pix + kAdjChunk - 1) / kAdjChunk;
    const int cap = orders ? kAdjMaxSplitsOrders : kAdjMaxSplits;
    int best = 1;
    double best_score = -1.0;
    for (int ks = 1; ks <= cap && ks <= max_split; ++ks) {
        const long long total = (long long)pairs * ks;
        const long long waves = (total + sm_count - 1) / sm_count;
        const double eff = (double)total / (double)(waves * sm_count);
        const double score = eff - 0.004 * ks;
        if (score > best_score) {
            best_score = score;
            best = ks;
        }
    }
    return best;
}

cudaError_t launch_adjoint_tc(const float2 *A, const float *w, const float4 *tab, const uint8_t *rtile, long long n_pix,
                              int nx, int ny, int nz, int orders, double voxel, int splits, float2 *partial,
                              unsigned *gmax_bits, float2 *S, int *err, cudaStream_t st) {
    AdjParams P;
    P.tab = tab;
    P.orders = orders ? 1 : 0;
    P.rtile = rtile;
    P.A = A;
    P.w = w;
    P.gmax_bits = gmax_bits;
    P.n_pix = n_pix;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.Nyp = adj_nyp(ny);
    if (!adjoint_tc_supported(nx, ny)) return cudaErrorInvalidValue;
    P.stages = adj_stages(P.Nyp);
    P.teams = P.stages >= 4 ? 4 : P.stages >= 2 ? 2 : 1;
    const long long chunks = (n_pix + kAdjChunk - 1) / kAdjChunk;
    P.pix_per_split = (int)((chunks + splits - 1) / splits) * kAdjChunk;
    P.voxel = voxel;
    const uint32_t N = (uint32_t)(2 * P.Nyp), M = kAdjRows;
    P.idesc = (1u << 4) | ((N >> 3) << 17) | ((M >> 4) << 24);     // F32 accumulate, F16 A and B
    uint32_t cols = 32;
    while (cols < 2 * N) cols <<= 1;
    P.tmem_cols = cols;
    P.partial = partial;
    P.nvox = (long long)nx * ny * nz;
    P.err = err;
    cudaError_t e = cudaMemsetAsync(gmax_bits, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    adj_gmax_kernel<<<(unsigned)std::min<long long>((n_pix + 255) / 256, 1024), 256, 0, st>>>(A, w, n_pix, gmax_bits);
    e = cudaFuncSetAttribute(adjoint_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    dim3 grid((nz + 1) / 2, splits);
    adjoint_tc_kernel<<<grid, kAdjThreads, adj_smem_bytes(P.Nyp), st>>>(P);
    adj_sum_kernel<<<(unsigned)((P.nvox + 255) / 256), 256, 0, st>>>(partial, splits, P.nvox, S);
    return cudaGetLastError();
}

// Order mode: S[j][x][y] = sum_n coef[j][n] S~[n][x][y], summed in order n = 0, 1, ...
// A thread holds one (x, y) column's N order values in registers and forms
// kAdjCombineZ consecutive slices of it from the block's coefficients, staged
// in shared memory; blockIdx.y picks the slice group.
constexpr int kAdjCombineZ = 8;
template <int kMaxN>
__global__ void __launch_bounds__(128) adj_orders_combine_kernel(const float2 *__restrict__ Sord,
                                                                 const float2 *__restrict__ coef, int N, int nz,
                                                                 long long nxy, float2 *__restrict__ S) {
    __shared__ float2 s_coef[kAdjCombineZ * kMaxN];
    const int j0 = blockIdx.y * kAdjCombineZ, nj = min(kAdjCombineZ, nz - j0);
    for (int i = threadIdx.x; i < nj * N; i += blockDim.x) s_coef[i] = coef[(size_t)j0 * N + i];
    __syncthreads();
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nxy) return;
    float2 v[kMaxN];
#pragma unroll
    for (int n = 0; n < kMaxN; ++n) v[n] = n < N ? Sord[(size_t)n * nxy + c] : make_float2(0.f, 0.f);
    for (int jj = 0; jj < nj; ++jj) {
        const float2 *a = s_coef + jj * N;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int n = 0; n < kMaxN; ++n) {
            if (n < N) {
                const float2 t = a[n];
                acc.x = fmaf(t.x, v[n].x, fmaf(-t.y, v[n].y, acc.x));
                acc.y = fmaf(t.x, v[n].y, fmaf(t.y, v[n].x, acc.y));
            }
        }
        S[(size_t)(j0 + jj) * nxy + c] = acc;
    }
}

cudaError_t launch_adj_orders_combine(const float2 *Sord, const float2 *coef, int N, int nz, int nx, int ny, float2 *S,
                                      cudaStream_t st) {
    const long long nxy = (long long)nx * ny;
    const dim3 blocks((unsigned)((nxy + 127) / 128), (unsigned)((nz + kAdjCombineZ - 1) / kAdjCombineZ));
    if (N <= 0) return cudaErrorInvalidValue;
    if (N <= 16)
        adj_orders_combine_kernel<16><<<blocks, 128, 0, st>>>(Sord, coef, N, nz, nxy, S);
    else if (N <= 24)
        adj_orders_combine_kernel<24><<<blocks, 128, 0, st>>>(Sord, coef, N, nz, nxy, S);
    else if (N <= 32)
        adj_orders_combine_kernel<32><<<blocks, 128, 0, st>>>(Sord, coef, N, nz, nxy, S);
    else if (N <= 48)
        adj_orders_combine_kernel<48><<<blocks, 128, 0, st>>>(Sord, coef, N, nz, nxy, S);
    else if (N <= 64)
        adj_orders_combine_kernel<64><<<blocks, 128, 0, st>>>(Sord, coef, N, nz, nxy, S);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace scm
