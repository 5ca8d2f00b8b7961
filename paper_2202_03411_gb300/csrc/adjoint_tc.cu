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
// Both operands depend on the pixel chunk, so sixteen generator warps build
// them in shared memory (phase recurrences, FP16 with |L|, |R| <= 1), one
// 16-row run each (the L runs cover only x < nx: rows beyond feed output rows
// that are never written back), while one MMA warp consumes the previous
// stages.  Per-pixel constants (q split into FP32
// pairs, one-voxel rotations) come from a table built once per handle, so the
// generators do no FP64 work and one reduced sincos per operand anchor.  A CTA owns two slices (two TMEM
// accumulators sharing every R tile) and a contiguous range of pixels; the
// pixel ranges' partial fields are summed in a fixed order afterwards.
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace scm {

constexpr int kAdjGenWarps = 16;            // one 16-row operand run each
constexpr int kAdjMmaWarp = kAdjGenWarps;
constexpr int kAdjThreads = (kAdjGenWarps + 1) * 32;
constexpr int kAdjChunk = 32;                 // pixels per K block (64 real K = 128 bytes)
constexpr int kAdjMaxStages = 6;
constexpr int kAdjRows = 128;                 // M: x rows
constexpr int kAdjTileA = kAdjRows * 128;     // one A tile: 128 rows x 128 bytes
constexpr int kAdjMaxSplits = 8;             // bounds the partial-field memory to 8 fields

struct AdjParams {
    const float4 *tab;          // per pixel: (qxh, qxl, qyh, qyl), (qzh, qzl, e^{+i qx dv}), (e^{+i qy dv}, e^{+i qz dv})
    int stages;
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

// Per-pixel constants of the generators: q as FP32 pairs and e^{+i q dv}.
__global__ void adj_pixel_table_kernel(const double *__restrict__ q, long long n, double voxel,
                                       float4 *__restrict__ tab) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
    const float qxh = (float)qx, qxl = (float)(qx - (double)qxh);
    const float qyh = (float)qy, qyl = (float)(qy - (double)qyh);
    const float qzh = (float)qz, qzl = (float)(qz - (double)qzh);
    const float vf = (float)voxel;
    // e^{+i t} = conj(e^{-i t}) = expmi(q, -c)
    const float2 ex = expmi_fs(qxh, qxl, -vf), ey = expmi_fs(qyh, qyl, -vf), ez = expmi_fs(qzh, qzl, -vf);
    tab[3 * p] = make_float4(qxh, qxl, qyh, qyl);
    tab[3 * p + 1] = make_float4(qzh, qzl, ex.x, ex.y);
    tab[3 * p + 2] = make_float4(ey.x, ey.y, ez.x, ez.y);
}

cudaError_t launch_adj_pixel_table(const double *q, long long n, double voxel, float4 *tab, cudaStream_t st) {
    adj_pixel_table_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(q, n, voxel, tab);
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
    uint64_t *full = bars;
    uint64_t *empty = bars + kAdjMaxStages;
    uint64_t *done = bars + 2 * kAdjMaxStages;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j0 = 2 * blockIdx.x;                          // slices j0, j0 + 1
    const long long p_begin = (long long)blockIdx.y * P.pix_per_split;
    const long long p_end = min(P.n_pix, p_begin + P.pix_per_split);
    const int n_chunks = p_end > p_begin ? (int)((p_end - p_begin + kAdjChunk - 1) / kAdjChunk) : 0;

    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            mbar_init(smem_u32(&full[s]), kAdjGenWarps);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        mbar_init(smem_u32(done), 1);
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
        for (int c = 0; c < n_chunks; ++c) {
            const uint32_t s = c % NS, ph = (c / NS) & 1;
            if (!warp_wait(smem_u32(&full[s]), ph, abort_flag, P.err, kErrTimeoutMma)) break;
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
    } else {
        // ---------------- generator warps ----------------
        const float inv_g = 1.0f / fmaxf(__uint_as_float(*P.gmax_bits), 1e-30f);
        const int i = lane;                      // pixel within the chunk
        // warp roles: runs 0 .. na-1 of the L tiles (x rows, both slices), then
        // runs of the R tile; a warp without a run only signals the stage
        const int na = (P.nx + 15) / 16, nb = P.Nyp / 16;
        const bool is_a = warp < na, is_b = !is_a && warp - na < nb;
        const int run = is_a ? warp : warp - na;  // rows 16*run .. 16*run + 15
        const float vox = (float)P.voxel;
        const float x0 = (16 * run - 0.5f * (P.nx - 1)) * vox;
        const float y0 = (16 * run - 0.5f * (P.ny - 1)) * vox;
        const float zj = ((float)j0 - 0.5f * (P.nz - 1)) * vox;
        const int rows_a = min(16, P.nx - 16 * run);
        // this lane's pixel data, loaded one chunk ahead so the L2 latency
        // overlaps the previous chunk's generation
        float2 a_n = make_float2(0.f, 0.f);
        float w_n = 0.f;
        float4 ta_n = make_float4(0.f, 0.f, 0.f, 0.f), tb_n = ta_n, tc_n = ta_n;
        auto load_pixel = [&](int c) {
            const long long p = p_begin + (long long)c * kAdjChunk + i;
            if (c < n_chunks && p < p_end && (is_a || is_b)) {
                ta_n = P.tab[3 * p];
                tc_n = P.tab[3 * p + 2];
                if (is_a) {
                    a_n = P.A[p];
                    w_n = P.w[p];
                    tb_n = P.tab[3 * p + 1];
                }
            } else {
                a_n = make_float2(0.f, 0.f);
                w_n = 0.f;
                ta_n = tb_n = tc_n = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        };
        load_pixel(0);
        for (int c = 0; c < n_chunks; ++c) {
            const float2 a_c = a_n;
            const float w_c = w_n;
            const float4 ta = ta_n, tb = tb_n, tcv = tc_n;
            load_pixel(c + 1);
            const uint32_t s = c % NS, ph = (c / NS) & 1;
            if (!warp_wait(smem_u32(&empty[s]), ph ^ 1, abort_flag, P.err, kErrTimeoutEpilogue)) break;
            uint8_t *sA0 = base + s * stage_bytes;
            uint8_t *sA1 = sA0 + kAdjTileA;
            uint8_t *sB = sA0 + 2 * kAdjTileA;
            const long long p = p_begin + (long long)c * kAdjChunk + i;
            const bool in = p < p_end;
            if (is_a) {
                const float wp = w_c * inv_g;
                const float2 g = make_float2(a_c.x * wp, a_c.y * wp);
                // e^{+i t} = conj(e^{-i t}) = expmi(q, -c)
                const float2 ez = expmi_fs(tb.x, tb.y, -zj);
                const float2 ezs = make_float2(tcv.z, tcv.w);
                const float2 ex = expmi_fs(ta.x, ta.y, -x0);
                const float2 exs = make_float2(tb.z, tb.w);
                float2 L0 = cmul(cmul(g, ez), ex);       // slice j0, row 16*run
#pragma unroll 4
                for (int k = 0; k < rows_a; ++k) {
                    const int r = 16 * run + k;
                    const float2 L1 = cmul(L0, ezs);
                    const uint32_t off = pair_offset(r, i);
                    *reinterpret_cast<uint32_t *>(sA0 + off) = pack_half2(L0.x, L0.y);
                    *reinterpret_cast<uint32_t *>(sA1 + off) = pack_half2(L1.x, L1.y);
                    L0 = cmul(L0, exs);
                }
            } else if (is_b) {
                // rows of the B tile: (y, re) and (y, im)
                const float2 eys = make_float2(tcv.x, tcv.y);
                float2 R = in ? expmi_fs(ta.z, ta.w, -y0) : make_float2(0.f, 0.f);
#pragma unroll 4
                for (int k = 0; k < 16; ++k) {
                    const int y = 16 * run + k;
                    *reinterpret_cast<uint32_t *>(sB + pair_offset(y, i)) = pack_half2(R.x, -R.y);
                    *reinterpret_cast<uint32_t *>(sB + pair_offset(P.Nyp + y, i)) = pack_half2(R.y, R.x);
                    R = cmul(R, eys);
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
static size_t adj_fixed_bytes() { return 1024 + 256; }
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

// Pixel ranges per slice pair: balance the grid over the SMs (1 CTA per SM).
int adjoint_tc_splits(long long n_pix, int nz, int sm_count) {
    const int pairs = (nz + 1) / 2;
    const long long max_split = (n_pix + kAdjChunk - 1) / kAdjChunk;
    int best = 1;
    double best_score = -1.0;
    for (int ks = 1; ks <= kAdjMaxSplits && ks <= max_split; ++ks) {
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

cudaError_t launch_adjoint_tc(const float2 *A, const float *w, const float4 *tab, long long n_pix, int nx, int ny,
                              int nz, double voxel, int splits, float2 *partial, unsigned *gmax_bits, float2 *S,
                              int *err, cudaStream_t st) {
    AdjParams P;
    P.tab = tab;
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

}  // namespace scm
