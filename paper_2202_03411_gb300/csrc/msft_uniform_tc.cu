// msft_uniform_tc.cu -- tensor-core form of the uniform-q detector's x/z sum
// (the paper's virtual detector, Block 1 and Block 6: q_x depends on the
// pixel column u only and q_y on the row v only):
//   G[u, (v, j)] = sum_x e^{-i q_x(u) x} H_v[j, x]          (one complex GEMM over all rows v)
//   A(u, v)      = (n^2-1) sum_j e^{-i q_z(u,v) z_j} G[u, (v, j)]
// H_v[j, x] = sum_y e^{-i q_y(v) y} s_j(x, y) comes from the y-contraction
// (msft_uniform.cu) as 16-bit planes [-Im | Re | Im].  Rows v are grouped
// Rg at a time (Rg Jp = Jg <= 128 GEMM columns per plane, Jp = nz padded to
// 16), so each K step of 16 x is two MMAs with N = 2 Jg:
//   [Re G | Im G] += Er [Hr | Hi] + Ei [-Hi | Hr],
// with the phase operand [Er | Ei] split hi + lo.  Each CTA takes one
// contiguous range of (tile of 128 pixel columns u, row group) pairs; a phase
// operand is built per tile and serves its run of groups.  Warp roles (320 threads): warps
// 0-7 build the phase tile and sum the z-phases, warps 0-3 on even groups
// and 4-7 on odd ones (each warp reads its TMEM lane quarter), warp 8 loads
// H tiles by TMA, warp 9 issues the MMAs and owns the tensor memory, whose
// two accumulators alternate between the groups.  Every wait is bounded: on
// time-out the kernel sets a bit in the error word, drains its own work,
// releases its tensor memory and returns.
#include "internal.cuh"
#include "tc_ptx.cuh"
#include "tc_tiles.cuh"

namespace scm {

constexpr int kUqThreads = 320;
constexpr int kUqEpiWarps = 8;
constexpr int kUqEpiThreads = kUqEpiWarps * 32;
constexpr int kUqProdWarp = 8;
constexpr int kUqMmaWarp = 9;
constexpr int kUqMaxSlots = 8;
constexpr int kUqMaxSmem = 232448;

struct UqParams {
    const float2 *qz;           // per pixel (q_z hi, lo); hi = NaN marker off the Ewald sphere
    int det_nx, det_ny;
    int nx, nz;
    int Kx, Jp, Jg;             // x padded to the K block, z padded to 16, Rg Jp
    int kbe, rb, kbs;           // K block: 16 / 32 / 64 elements (2^kbs) in rows of rb = 32 / 64 / 128 bytes
    int n_groups;               // ceil(det_ny / Rg)
    int nkb;                    // Kx / kbe
    int n_ut;                   // pixel tiles of 128 columns u
    int slots;
    uint32_t box_bytes;         // one K block of a group: 3 Jg rows of rb bytes
    uint32_t stage_bytes;       // box_bytes rounded up to 1024 (every stage swizzle-aligned)
    int split, bf16;
    uint32_t idesc;             // N = 2 Jg
    uint32_t tmem_cols;
    double qmax, voxel;
    float str_re, str_im;
    float2 *A;
    float *I;
    int *err;
};

__device__ __forceinline__ double uq_coord(int i, int n, double qmax) {
    return qmax * (double)(2 * i + 1 - n) / (double)n;
}

// Work split: the (pixel tile, row group) pairs, tile-major, cut into one
// contiguous range per CTA (sizes differ by at most one group).  A segment is
// the part of the range inside one pixel tile: one phase operand serves it.
struct UqSeg {
    int tile, gb, ge;
};
__device__ __forceinline__ bool uq_next_seg(const UqParams &P, long long &idx, long long hi, UqSeg &s) {
    if (idx >= hi) return false;
    s.tile = (int)(idx / P.n_groups);
    s.gb = (int)(idx - (long long)s.tile * P.n_groups);
    const long long end = min(hi, (long long)(s.tile + 1) * P.n_groups);
    s.ge = s.gb + (int)(end - idx);
    idx = end;
    return true;
}
__device__ __forceinline__ void uq_range(const UqParams &P, long long &lo, long long &hi) {
    const long long total = (long long)P.n_ut * P.n_groups;
    lo = total * blockIdx.x / gridDim.x;
    hi = total * (blockIdx.x + 1) / gridDim.x;
}

// Operand tiles in K blocks of kbe elements: rows of rb bytes with the
// matching swizzle (128, 64 or 32 bytes: the 16-byte chunk index XOR row
// bits, as TMA writes them and the MMA descriptors read them), so a small x
// extent pads to 16 or 32 instead of 64.
__device__ __forceinline__ uint32_t uq_chunk_offset(const UqParams &P, int m, int k) {
    const int kb = k >> P.kbs, c = (k & (P.kbe - 1)) >> 3;
    const int sw = P.rb == 128 ? (m & 7) : P.rb == 64 ? ((m >> 1) & 3) : ((m >> 2) & 1);
    return (uint32_t)(kb * kTileRows * P.rb + m * P.rb + ((c ^ sw) << 4));
}
// K-major shared-memory descriptor: 8-row groups rb x 8 bytes apart, layout
// 2 / 4 / 6 = 128 / 64 / 32-byte swizzle.
__device__ __forceinline__ uint64_t uq_desc(uint32_t saddr, int rb) {
    uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)((8 * rb) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(rb == 128 ? 2 : rb == 64 ? 4 : 6) << 61;
    return d;
}

// Phase operand E[m, k] = [cos(q_x x_k) | -sin(q_x x_k)] of pixel column
// u = u0 + m (zero beyond nx and beyond the detector), hi and lo parts: one
// reduced sincos per 8 x and FP32 rotations by 1..4 voxels.
__device__ __forceinline__ void build_uq_phase(const UqParams &P, int u0, uint8_t *sA_hi, uint8_t *sA_lo, int tid) {
    const int m = tid % kTileRows;
    const int u = u0 + m;
    const bool valid = u < P.det_nx;
    const double qx = valid ? uq_coord(u, P.det_nx, P.qmax) : 0.0;
    const float qh = (float)qx, ql = (float)(qx - (double)qh);
    const float xoff = 0.5f * (float)(P.nx - 1), vox = (float)P.voxel;
    const float2 s1 = expmi_fs(qh, ql, vox);
    const float2 s2 = cmul(s1, s1), s3 = cmul(s2, s1), s4 = cmul(s2, s2);
    const int nx8 = P.Kx >> 3;
#pragma unroll 2
    for (int x8 = tid / kTileRows; x8 < nx8; x8 += kUqEpiThreads / kTileRows) {
        const float2 p0 = expmi_fs(qh, ql, ((float)(8 * x8) - xoff) * vox);
        const float2 p4 = cmul(p0, s4);
        const float2 phs[8] = {p0, cmul(p0, s1), cmul(p0, s2), cmul(p0, s3),
                               p4, cmul(p4, s1), cmul(p4, s2), cmul(p4, s3)};
        uint32_t re_hi[4], im_hi[4], re_lo[4], im_lo[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const int x = 8 * x8 + e;
            const bool in0 = valid && x < P.nx, in1 = valid && x + 1 < P.nx;
            split_pair(in0 ? phs[e].x : 0.f, in1 ? phs[e + 1].x : 0.f, P.bf16, &re_hi[e >> 1], &re_lo[e >> 1]);
            split_pair(in0 ? phs[e].y : 0.f, in1 ? phs[e + 1].y : 0.f, P.bf16, &im_hi[e >> 1], &im_lo[e >> 1]);
        }
        const uint32_t o_re = uq_chunk_offset(P, m, 8 * x8);
        const uint32_t o_im = uq_chunk_offset(P, m, P.Kx + 8 * x8);
        *reinterpret_cast<uint4 *>(sA_hi + o_re) = make_uint4(re_hi[0], re_hi[1], re_hi[2], re_hi[3]);
        *reinterpret_cast<uint4 *>(sA_hi + o_im) = make_uint4(im_hi[0], im_hi[1], im_hi[2], im_hi[3]);
        if (P.split) {
            *reinterpret_cast<uint4 *>(sA_lo + o_re) = make_uint4(re_lo[0], re_lo[1], re_lo[2], re_lo[3]);
            *reinterpret_cast<uint4 *>(sA_lo + o_im) = make_uint4(im_lo[0], im_lo[1], im_lo[2], im_lo[3]);
        }
    }
}

template <int kR>
__global__ void __launch_bounds__(kUqThreads, 1) uq_tc_kernel(const __grid_constant__ CUtensorMap map, const UqParams P) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t a_bytes = (uint32_t)(2 * P.nkb * kTileRows * P.rb);        // [Er | Ei] over K = 2 Kx
    uint8_t *sA_hi = base;
    uint8_t *sA_lo = base + a_bytes;
    uint8_t *stages = base + (P.split ? 2 : 1) * a_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(stages + (size_t)P.slots * P.stage_bytes);
    uint64_t *full = bars;
    uint64_t *empty = bars + kUqMaxSlots;
    uint64_t *tfull = bars + 2 * kUqMaxSlots;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint64_t *a_full = drain + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(a_full + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P.slots; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), kUqEpiWarps / 2);
        }
        mbar_init(smem_u32(drain), 1);
        mbar_init(smem_u32(a_full), kUqEpiThreads);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == kUqMmaWarp) {
        tmem_alloc(smem_u32(tmem_slot), P.tmem_cols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    uint32_t prod_it = 0;

    if (warp == kUqProdWarp) {
        // ---------------- TMA producer: every group of every segment, every 64-x block ----------------
        long long idx, hi;
        uq_range(P, idx, hi);
        UqSeg sg;
        while (uq_next_seg(P, idx, hi, sg)) {
            bool ok = true;
            for (int g = sg.gb; g < sg.ge && ok; ++g)
                for (int kb = 0; kb < P.nkb; ++kb) {
                    const uint32_t s = prod_it % P.slots, ph = (prod_it / P.slots) & 1;
                    if (!warp_wait(smem_u32(&empty[s]), ph ^ 1, abort_flag, P.err, kErrTimeoutProducer)) {
                        ok = false;
                        break;
                    }
                    if (elect_one()) {
                        const uint32_t fb = smem_u32(&full[s]);
                        mbar_arrive_expect_tx(fb, P.box_bytes);
                        tma_load_3d(smem_u32(stages + (size_t)s * P.stage_bytes), &map, fb, kb * P.kbe, 0, 3 * g);
                    }
                    __syncwarp();
                    ++prod_it;
                }
            if (!ok) break;
        }
    } else if (warp == kUqMmaWarp) {
        // ---------------- MMA issuer (warp-wide loop, one elected lane issues) ----------------
        const uint64_t ahi0 = uq_desc(smem_u32(sA_hi), P.rb), alo0 = uq_desc(smem_u32(sA_lo), P.rb);
        const uint64_t st0 = uq_desc(smem_u32(stages), P.rb);
        uint32_t it = 0, acc_it = 0, tl = 0;
        bool ok = true;
        long long idx, hi;
        uq_range(P, idx, hi);
        UqSeg sg;
        for (; ok && uq_next_seg(P, idx, hi, sg); ++tl) {
            if (!warp_wait(smem_u32(a_full), tl & 1, abort_flag, P.err, kErrTimeoutMma)) break;
            tc_fence_after();
            for (int g = sg.gb; g < sg.ge && ok; ++g) {
                const uint32_t b = acc_it & 1, aph = (acc_it >> 1) & 1;
                if (!warp_wait(smem_u32(&tempty[b]), aph ^ 1, abort_flag, P.err, kErrTimeoutMma)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + b * (uint32_t)(2 * P.Jg);
                bool first = true;
                for (int kb = 0; kb < P.nkb; ++kb) {
                    const uint32_t s = it % P.slots, ph = (it / P.slots) & 1;
                    if (!warp_wait(smem_u32(&full[s]), ph, abort_flag, P.err, kErrTimeoutMma)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t w2 = st0 + (uint64_t)(((size_t)s * P.stage_bytes) >> 4);    // rows [0, 2 Jg): [-Hi | Hr]
                    const uint64_t w1 = w2 + (uint64_t)(((uint32_t)P.Jg * (uint32_t)P.rb) >> 4); // rows [Jg, 3 Jg): [Hr | Hi]
                    const int ksteps = P.kbe >> 4;
                    // K block kb of [Er] and block nkb + kb of [Ei]; 32 bytes per K step
                    const uint64_t blk_r = (uint64_t)(((uint32_t)kb * kTileRows * (uint32_t)P.rb) >> 4);
                    const uint64_t blk_i = (uint64_t)(((uint32_t)(P.nkb + kb) * kTileRows * (uint32_t)P.rb) >> 4);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        if (kk >= ksteps) break;
                        const uint64_t off_r = blk_r + (uint64_t)(2 * kk), off_i = blk_i + (uint64_t)(2 * kk);
                        const uint64_t b1 = w1 + (uint64_t)(kk * 2), b2 = w2 + (uint64_t)(kk * 2);
                        const uint32_t acc0 = first ? 0u : 1u;
                        if (elect_one()) {
                            mma_f16(d, ahi0 + off_r, b1, P.idesc, acc0);
                            mma_f16(d, ahi0 + off_i, b2, P.idesc, 1u);
                            if (P.split) {
                                mma_f16(d, alo0 + off_r, b1, P.idesc, 1u);
                                mma_f16(d, alo0 + off_i, b2, P.idesc, 1u);
                            }
                        }
                        __syncwarp();
                        first = false;
                    }
                    if (elect_one()) mma_commit(smem_u32(&empty[s]));
                    __syncwarp();
                    ++it;
                }
                if (!ok) break;
                if (elect_one()) mma_commit(smem_u32(&tfull[b]));
                __syncwarp();
                ++acc_it;
            }
        }
    } else {
        // ---------------- phase tile; z-phase sums, halves on alternate groups ----------------
        const int quarter = warp & 3, half = warp >> 2;
        const int m = quarter * 32 + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        const float vf = (float)P.voxel;
        const float z0 = -0.5f * (float)(P.nz - 1) * vf;   // z of slice 0
        const int cpr = P.Jp >> 4;                         // 16-column chunks per row
        const float2 str = make_float2(P.str_re, P.str_im);
        uint32_t git = 0;                                  // groups seen by this CTA (both halves count all)
        long long idx, hi;
        uq_range(P, idx, hi);
        UqSeg sg;
        while (uq_next_seg(P, idx, hi, sg)) {
            const int u0 = sg.tile * kTileRows;
            // Each half has seen the completion of its own last group; after
            // this barrier every MMA that read the previous phase tile is done.
            named_bar_sync(kUqEpiThreads);
            if (!*abort_flag) build_uq_phase(P, u0, sA_hi, sA_lo, threadIdx.x);
            fence_async_smem();
            mbar_arrive(smem_u32(a_full));
            const int u = u0 + m;
            const bool valid_u = u < P.det_nx;
            for (int g = sg.gb; g < sg.ge; ++g, ++git) {
                if ((int)(git & 1) != half) continue;
                // the rows' q_z before the accumulator wait, so the loads overlap it
                float2 tq[kR];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    const int v = g * kR + r;
                    tq[r] = (valid_u && v < P.det_ny) ? P.qz[(long long)v * P.det_nx + u]
                                                      : make_float2(__uint_as_float(kUqOffSphereBits), 0.f);
                }
                const uint32_t b = git & 1, ph = (git >> 1) & 1;
                const bool got = mbar_wait(smem_u32(&tfull[b]), ph, abort_flag, P.err, kErrTimeoutEpilogue);
                if (!__all_sync(0xffffffffu, got)) continue;
                tc_fence_after();
                float2 out[kR];
#pragma unroll
                for (int r = 0; r < kR; ++r) {
                    // sum_j e^{-i q_z z_j} G_j = e^{-i q_z z_0} sum_j w^j G_j with w = e^{-i q_z dz},
                    // the polynomial in w by Horner's rule from the top slice down
                    const float2 w = expmi_fs(tq[r].x, tq[r].y, vf);
                    float2 acc = make_float2(0.f, 0.f);
                    for (int cc = cpr - 1; cc >= 0; --cc) {
                        float gr[16], gi[16];
                        const uint32_t col = b * (uint32_t)(2 * P.Jg) + (uint32_t)(r * P.Jp + 16 * cc);
                        tmem_ld16(lane_base + col, gr);
                        tmem_ld16(lane_base + col + (uint32_t)P.Jg, gi);
                        tmem_ld_wait(gr, gi);
#pragma unroll
                        for (int k = 15; k >= 0; --k) {
                            const float ax = acc.x;
                            acc.x = fmaf(ax, w.x, fmaf(-acc.y, w.y, gr[k]));
                            acc.y = fmaf(ax, w.y, fmaf(acc.y, w.x, gi[k]));
                        }
                    }
                    out[r] = cmul(expmi_fs(tq[r].x, tq[r].y, z0), acc);
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
                if (valid_u) {
#pragma unroll
                    for (int r = 0; r < kR; ++r) {
                        const int v = g * kR + r;
                        if (v >= P.det_ny) break;
                        // a pixel with no scattering direction has no field
                        const bool on = __float_as_uint(tq[r].x) != kUqOffSphereBits;
                        const float2 a = on ? cmul(str, out[r]) : make_float2(0.f, 0.f);
                        const long long p = (long long)v * P.det_nx + u;
                        P.A[p] = a;
                        P.I[p] = a.x * a.x + a.y * a.y;
                    }
                }
            }
        }
    }

    // ---- teardown: no tensor-core or TMA work may be in flight ----
    __syncthreads();
    if (*abort_flag) {
        if (warp == kUqMmaWarp && lane == 0) {
            mma_commit(smem_u32(drain));
            volatile int dummy = 0;
            mbar_wait(smem_u32(drain), 0, &dummy, P.err, kErrTimeoutDrain);
        }
        if (warp == kUqProdWarp && lane == 0) {
            volatile int dummy = 0;
            const uint32_t first = prod_it > (uint32_t)P.slots ? prod_it - P.slots : 0;
            for (uint32_t i = first; i < prod_it; ++i)
                mbar_wait(smem_u32(&full[i % P.slots]), (i / P.slots) & 1, &dummy, P.err, kErrTimeoutDrain);
        }
    }
    __syncthreads();
    if (warp == kUqMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem_base, P.tmem_cols);
    }
}

// ---- host side ----------------------------------------------------------------------
// [Er | Ei] (and its low part): 128 rows x 2 Kx elements of 2 bytes.
static size_t uq_a_bytes(int Kx, bool split) { return (size_t)(split ? 2 : 1) * kTileRows * 2 * Kx * 2; }
static size_t uq_fixed_bytes() { return 1024 + 256; }

// K block of the x contraction: 16, 32 or 64 x (32-, 64- or 128-byte rows).
static int uq_kblock(int nx) { return nx <= 16 ? 16 : nx <= 32 ? 32 : 64; }
static size_t uq_stage_bytes(int Jg, int kbe) { return ((size_t)3 * Jg * kbe * 2 + 1023) / 1024 * 1024; }

void uq_tc_geometry(int nx, int nz, int *Kx, int *Jp, int *Rg) {
    const int kbe = uq_kblock(nx);
    *Kx = (nx + kbe - 1) / kbe * kbe;
    *Jp = (nz + 15) / 16 * 16;
    int r = 1;
    while (r < 8 && 2 * r * *Jp <= 128) r <<= 1;
    *Rg = r;
}

// Stage slots beside the phase operand (0 when fewer than two fit).
int uq_tc_slots(int nx, int nz, bool split) {
    int Kx, Jp, Rg;
    uq_tc_geometry(nx, nz, &Kx, &Jp, &Rg);
    if (Kx > 128 || Jp > 128) return 0;
    const size_t stage = uq_stage_bytes(Rg * Jp, uq_kblock(nx));
    const size_t used = uq_a_bytes(Kx, split) + uq_fixed_bytes();
    if (used + 2 * stage > (size_t)kUqMaxSmem) return 0;
    const size_t n = ((size_t)kUqMaxSmem - used) / stage;
    return (int)(n > (size_t)kUqMaxSlots ? kUqMaxSlots : n);
}

bool encode_tmap_uq(CUtensorMap *map, void *H, int nx, int nz, int det_ny, bool bf16, std::string *why) {
    int Kx, Jp, Rg;
    uq_tc_geometry(nx, nz, &Kx, &Jp, &Rg);
    const int Jg = Rg * Jp, n_groups = (det_ny + Rg - 1) / Rg;
    const uint64_t dims[3] = {(uint64_t)Kx, (uint64_t)Jg, (uint64_t)3 * n_groups};
    const uint64_t strides[2] = {(uint64_t)Kx * 2, (uint64_t)Jg * Kx * 2};
    const int kbe = uq_kblock(nx);
    const uint32_t box[3] = {(uint32_t)kbe, (uint32_t)Jg, 3u};
    return encode_tmap_3d_16bit(map, H, dims, strides, box, bf16, why, kbe * 2);
}

// Bytes of the y-contracted 16-bit operand: every row group, three planes.
size_t uq_tc_h_bytes(int nx, int nz, int det_ny) {
    int Kx, Jp, Rg;
    uq_tc_geometry(nx, nz, &Kx, &Jp, &Rg);
    return (size_t)((det_ny + Rg - 1) / Rg) * 3 * Rg * Jp * Kx * 2;
}

// Real flops the x/z launch issues: per row group and pixel tile, 4 MMAs of
// 128 x 2 Jg x 16 per K step of 16 x (2 with unsplit phases).
double uq_tc_issued_flops(int nx, int nz, int det_nx, int det_ny, bool split) {
    int Kx, Jp, Rg;
    uq_tc_geometry(nx, nz, &Kx, &Jp, &Rg);
    const double n_ut = (double)((det_nx + kTileRows - 1) / kTileRows);
    const double n_groups = (double)((det_ny + Rg - 1) / Rg);
    return n_ut * n_groups * (Kx / 16) * 2.0 * (split ? 2.0 : 1.0) * 2.0 * kTileRows * (2.0 * Rg * Jp) * 16.0;
}

cudaError_t launch_uq_tc(const CUtensorMap &map, const float2 *qz, int nx, int nz, int det_nx, int det_ny,
                         double theta_max_deg, double k0, double voxel, double str_re, double str_im, bool split,
                         bool bf16, float2 *A, float *I, int *err, int sm_count, cudaStream_t st) {
    UqParams P;
    int Rg;
    uq_tc_geometry(nx, nz, &P.Kx, &P.Jp, &Rg);
    P.qz = qz;
    P.det_nx = det_nx;
    P.det_ny = det_ny;
    P.nx = nx;
    P.nz = nz;
    P.Jg = Rg * P.Jp;
    P.n_groups = (det_ny + Rg - 1) / Rg;
    P.kbe = uq_kblock(nx);
    P.rb = 2 * P.kbe;
    P.kbs = P.kbe == 16 ? 4 : P.kbe == 32 ? 5 : 6;
    P.nkb = P.Kx / P.kbe;
    P.slots = uq_tc_slots(nx, nz, split);
    if (P.slots < 2) return cudaErrorInvalidValue;
    P.box_bytes = (uint32_t)(3 * P.Jg * P.rb);
    P.stage_bytes = (uint32_t)uq_stage_bytes(P.Jg, P.kbe);
    P.n_ut = (det_nx + kTileRows - 1) / kTileRows;
    const long long total = (long long)P.n_ut * P.n_groups;
    P.split = split ? 1 : 0;
    P.bf16 = bf16 ? 1 : 0;
    const uint32_t N = (uint32_t)(2 * P.Jg), M = kTileRows;
    P.idesc = (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((N >> 3) << 17) | ((M >> 4) << 24);
    uint32_t cols = 32;
    while (cols < 2 * N) cols <<= 1;
    P.tmem_cols = cols;
    P.qmax = k0 * sin(theta_max_deg * kPi / 180.0);
    P.voxel = voxel;
    P.str_re = (float)str_re;
    P.str_im = (float)str_im;
    P.A = A;
    P.I = I;
    P.err = err;
    const size_t smem = uq_a_bytes(P.Kx, split) + (size_t)P.slots * P.stage_bytes + uq_fixed_bytes();
    const int grid = (int)(total < sm_count ? total : sm_count);
    // per-function attribute shared by every thread of the process: always the maximum
    cudaError_t e;
    switch (Rg) {
    case 8:
        e = cudaFuncSetAttribute(uq_tc_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUqMaxSmem);
        if (e == cudaSuccess) uq_tc_kernel<8><<<grid, kUqThreads, smem, st>>>(map, P);
        break;
    case 4:
        e = cudaFuncSetAttribute(uq_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUqMaxSmem);
        if (e == cudaSuccess) uq_tc_kernel<4><<<grid, kUqThreads, smem, st>>>(map, P);
        break;
    case 2:
        e = cudaFuncSetAttribute(uq_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUqMaxSmem);
        if (e == cudaSuccess) uq_tc_kernel<2><<<grid, kUqThreads, smem, st>>>(map, P);
        break;
    default:
        e = cudaFuncSetAttribute(uq_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kUqMaxSmem);
        if (e == cudaSuccess) uq_tc_kernel<1><<<grid, kUqThreads, smem, st>>>(map, P);
        break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace scm
