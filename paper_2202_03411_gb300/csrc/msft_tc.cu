// msft_tc.cu -- tensor-core (tcgen05) form of Eq. 9's per-slice Fourier sum.
//
// Per slice j the 2D sum over (x, y) is factored as
//   G[q, (j,x)] = sum_y e^{-i q_y y} s_j(x, y)          (dense complex contraction)
//   A[q]        = (n^2-1) sum_j e^{-i q_z z_j} sum_x e^{-i q_x x} G[q, (j,x)]
// The first line is a complex GEMM per slice with K = y.  Each K step of 16 y
// takes two real MMAs per phase product:
//   [Re G | Im G] += Pr [Sr | Si] + Pi [-Si | Sr],
//   Pr[m, y] = cos(q_y y), Pi[m, y] = -sin(q_y y)   (e^{-i q_y y}),
//   Sr[x, y] = Re s_j(x, y), Si[x, y] = Im s_j(x, y).
// The slice operand is stored as three planes [-Si | Sr | Si], so both B
// operands are windows of one staged block.  The phase operand [Pr | Pi] of a
// pixel tile is built once per tile by the epilogue warps in shared memory
// (K-major, 128-byte swizzle); with split phases it is held as an FP16/BF16
// pair P = P_hi + P_lo and both halves accumulate into the same FP32 result.
//
// Work units.  A unit is one occupied slice's run of occupied 8-column chunks
// of x, at most 16 (128 x; wider slices, up to nx = 256, are cut evenly into
// two units): its MMAs have N = 16 nch <= 256, and it runs only the K
// steps its y range needs, shifted by 8 y when that saves one (the B box then
// starts 8 y later and the epilogue multiplies the unit's sum by
// e^{-i q_y 8 dy}).  Whole slices keep each unit's MMA work long enough to
// hide the hand-offs between the warp roles (holding a phase half in tensor
// memory makes each MMA cheaper but forces units of at most 96 x into the
// remaining columns, and then those hand-offs show).  Each stage of the shared
// memory ring is one 3D TMA box (64 y x 8 nch rows x 3 planes, 128-byte
// swizzle), as large as the unit.  Accumulators are double buffered, and
// eight epilogue warps apply the x- and z-phases (second line) while the next
// unit's MMAs run.
//
// Warp roles (352 threads): warps 0-7 build the phase operand and run the
// epilogue (two per TMEM lane quarter, alternating chunks), warp 8 is the TMA
// producer, warps 9 and 10 issue the MMAs of alternate units (warp 9 owns the
// tensor memory).  The roles meet only at mbarriers, so the producer runs
// ahead across pixel tiles.  Work is handed out per pixel tile and a range of
// its units: whole tiles, except that the last partial wave's tiles are cut
// into up to four unit ranges whose partial fields tc_tail_sum_kernel adds,
// so that wave fills the SMs.  The same kernel in store mode is the
// uniform-q detector's y-sum: its rows are detector rows, every tile is cut
// into unit ranges (units are independent there) and the epilogue writes the
// accumulators as 16-bit operand planes instead of reducing them.
// Every wait is bounded: on time-out the kernel sets a bit in the error word,
// drains its own TMA copies and MMAs, releases its tensor memory and returns.
#include "internal.cuh"
#include "tc_ptx.cuh"
#include "tc_tiles.cuh"

#include <cstring>

namespace scm {

constexpr int kTcThreads = 352;
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kProducerWarp = 8;
constexpr int kMmaWarp = 9;                // MMA warps 9 and 10 take alternate units
constexpr int kBM = 128;
constexpr int kBK = 64;                    // 64 x 16-bit = one 128-byte swizzle row
constexpr int kSlots = 12;                 // stages in flight at most
constexpr int kPlanes = 3;                 // slice operand planes: -Im, Re, Im
constexpr int kMaxSmem = 232448;           // 227 KB opt-in per block
constexpr int kTcMaxTailParts = 4;         // unit ranges per tile of the last partial wave
constexpr int kTmemCols = 512;             // the whole tensor memory of the SM
constexpr int kUnitMaxSteps = 21;          // K steps a unit word can hold
constexpr int kEpiBatch = 3;               // chunks whose tensor-memory loads share one wait

struct TcParams {
    const double *q;
    const uint2 *list;          // [0].x = units; [1 + i] = {slice t, unit word}, t ascending
    long long n_pix;
    int nx, ny, nz;
    int Nxp, Nyp;               // padded x (multiple of 16) and y (multiple of 16)
    int nkb_a, nkb_b;           // 64-element K blocks of the phase operand (2 Nyp) and of a slice row (Nyp)
    uint32_t ring_bytes;        // slice-stage ring (multiple of 1024)
    int split, bf16;
    int num_m_tiles;
    // Work units: tiles [0, whole) whole, then each of the remaining tiles cut
    // into `parts` ranges of its unit list (units whole + (tiles - whole) x
    // parts).  The field sum cuts only the last partial wave (their partial
    // fields go to Apart and a finishing kernel adds them); store mode cuts
    // every tile (units are independent there).
    int whole, parts, num_units;
    float2 *Apart;              // [part][(tile - whole) * 128 + m]
    uint32_t idesc;             // without the N field (set per unit)
    uint32_t acc_cols;          // tensor-memory columns of one accumulator buffer
    double voxel;
    float str_re, str_im;
    float2 *A;
    float *I;
    int *err;
    // store mode (the uniform-q detector's y-contraction): rows m are detector
    // rows v with q_y(v) = q[3 v + 1]; G is written as 16-bit planes
    // [-Im | Re | Im] of H at rows (3 (v / h_Rg) + plane) h_Jg + (v % h_Rg) h_Jp + j
    uint16_t *Ht;
    int h_Jp, h_Jg, h_Rg, h_Kx, h_bf16;
};

// Unit word: first chunk c_lo | chunks nch << 5 | shift << 10 | K-step mask << 11.
// nch >= 1, so a word is never 0.
__host__ __device__ inline int unit_c_lo(uint32_t w) { return (int)(w & 31u); }
__host__ __device__ inline int unit_nch(uint32_t w) { return (int)((w >> 5) & 31u); }
__host__ __device__ inline int unit_shift(uint32_t w) { return (int)((w >> 10) & 1u); }
__host__ __device__ inline uint32_t unit_kmask(uint32_t w) { return w >> 11; }

// Tensor memory holds two accumulator buffers of 256 columns (a unit of nch
// chunks fills 16 nch of them: [Re G | Im G]).  Shared memory: the phase
// operand (and its low half), the stage ring, the reduction buffer and the
// barriers.
constexpr int kAccCols = 16 * kTcMaxChunks;
static int tc_nkb(int K) { return (K + kBK - 1) / kBK; }
static size_t tc_fixed_bytes() { return 1024 /*align*/ + kBM * sizeof(float2) + 512 /*barriers*/; }
static size_t tc_a_bytes(int Nyp) { return (size_t)tc_nkb(2 * Nyp) * kBM * 128; }
// Bytes of the slice-stage ring beside the phase operand(s), or 0 when two
// stages as wide as the grid do not fit.
static size_t tc_ring_bytes(int Nxp, int Nyp, bool split) {
    const size_t used = tc_fixed_bytes() + (split ? 2 : 1) * tc_a_bytes(Nyp);
    if (used >= (size_t)kMaxSmem) return 0;
    const size_t r = ((size_t)kMaxSmem - used) / 1024 * 1024;
    const size_t widest = (size_t)kPlanes * (Nxp < 8 * kTcMaxChunks ? Nxp : 8 * kTcMaxChunks) * 128;
    return r >= 2 * widest ? r : 0;
}

bool tc_grid_ok(int Nxp, int Nyp, bool split) {
    return Nxp >= 16 && Nxp % 16 == 0 && Nxp <= 8 * kGeomChunks && Nyp >= 16 && Nyp % 16 == 0 &&
           Nyp / 16 <= kUnitMaxSteps && tc_ring_bytes(Nxp, Nyp, split) > 0;
}

// The work units of slice t from the recorded y range of each of its 8-column
// chunks (cy: the geometry buffer's chunk part, [y_lo | y_hi] x [nz][kGeomChunks]).
// The occupied chunks are cut evenly into the fewest units of at most
// max_chunks chunks; each unit drops empty chunks at its ends and covers the
// union of its chunks' y ranges with K steps of 16 y, shifted by 8 y when
// that takes fewer steps (allowed from y >= 8 on, so no step starts below 0).
// Writes at most kMaxUnitsPerSlice words; returns their number.
__host__ __device__ inline int plan_units(const int *cy, int nz, int t, int nc8, int max_chunks, bool allow_shift,
                                          uint32_t *w) {
    const int *lo = cy + (size_t)t * kGeomChunks;
    const int *hi = cy + (size_t)kGeomChunks * nz + (size_t)t * kGeomChunks;
    int a = -1, b = -1;
    for (int c = 0; c < nc8; ++c)
        if (lo[c] < hi[c]) {
            if (a < 0) a = c;
            b = c + 1;
        }
    if (a < 0) return 0;
    const int n = b - a;
    const int parts = (n + max_chunks - 1) / max_chunks;
    int cnt = 0;
    for (int p = 0; p < parts; ++p) {
        int pa = a + p * n / parts, pb = a + (p + 1) * n / parts;
        while (pa < pb && lo[pa] >= hi[pa]) ++pa;
        while (pb > pa && lo[pb - 1] >= hi[pb - 1]) --pb;
        if (pa >= pb) continue;
        int ylo = lo[pa], yhi = hi[pa];
        for (int c = pa + 1; c < pb; ++c) {
            if (lo[c] >= hi[c]) continue;
            ylo = lo[c] < ylo ? lo[c] : ylo;
            yhi = hi[c] > yhi ? hi[c] : yhi;
        }
        int k0 = ylo >> 4, k1 = (yhi + 15) >> 4, sh = 0;
        if (allow_shift && ylo >= 8) {
            const int j0 = (ylo - 8) >> 4, j1 = (yhi - 8 + 15) >> 4;
            if (j1 - j0 < k1 - k0) {
                k0 = j0;
                k1 = j1;
                sh = 1;
            }
        }
        uint32_t mask = 0;
        for (int k = k0; k < k1 && k < kUnitMaxSteps; ++k) mask |= 1u << k;
        w[cnt++] = (uint32_t)pa | ((uint32_t)(pb - pa) << 5) | ((uint32_t)sh << 10) | (mask << 11);
    }
    return cnt;
}

// Lists the work units of every slice, in slice order: list[1 + i] =
// {t, unit word}, list[0].x = their number.  One block of 256 threads, 256
// slices per pass.
__global__ void __launch_bounds__(256) pack_units_kernel(const int *cy, int nz, int nc8, int max_chunks,
                                                         int allow_shift, uint2 *list) {
    __shared__ int s_warp[8];
    __shared__ int s_base;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int t0 = 0; t0 < nz; t0 += 256) {
        const int t = t0 + (int)threadIdx.x;
        uint32_t w[kMaxUnitsPerSlice];
        const int n = t < nz ? plan_units(cy, nz, t, nc8, max_chunks, allow_shift != 0, w) : 0;
        int x = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[wid] = x;
        __syncthreads();
        int off = s_base + x - n;
        for (int k = 0; k < wid; ++k) off += s_warp[k];
        for (int i = 0; i < n; ++i) list[1 + off + i] = make_uint2((uint32_t)t, w[i]);
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = s_base;
            for (int k = 0; k < 8; ++k) tot += s_warp[k];
            s_base = tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) list[0] = make_uint2((uint32_t)s_base, 0u);
}

// Tile, part (-1: whole tile) and unit range [i_lo, i_hi) of work unit u.
struct TcUnit {
    int mt, part, i_lo, i_hi;
};
__device__ __forceinline__ TcUnit unit_info(const TcParams &P, int u, int n_units) {
    TcUnit w;
    if (u < P.whole) {
        w.mt = u;
        w.part = -1;
        w.i_lo = 0;
        w.i_hi = n_units;
    } else {
        const int v = u - P.whole;
        w.mt = P.whole + v / P.parts;
        w.part = v % P.parts;
        w.i_lo = (int)((long long)w.part * n_units / P.parts);
        w.i_hi = (int)((long long)(w.part + 1) * n_units / P.parts);
    }
    return w;
}

// Placement of a stage of `sz` bytes in the ring: a stage never wraps, it
// starts over at offset 0 when it does not fit before the end.
__device__ __forceinline__ uint32_t ring_start(uint32_t head_off, uint32_t sz, uint32_t ring) {
    return head_off + sz > ring ? 0u : head_off;
}

// Phase operand P[m, k] of one pixel tile (and its low part when split),
// K-major with the 128-byte swizzle: [Pr | Pi] over k = y and Nyp + y.
// Built by the kEpiThreads epilogue threads; thread `tid` always serves pixel
// row m = tid % 128; each group of 8 consecutive y takes one reduced sincos
// and FP32 complex products with the rotations e^{-i q_y k dy}, k = 1..4 (a
// few ulp, far below the 16-bit operands' resolution).
__device__ __forceinline__ void build_phase(const TcParams &P, double qy, bool valid, uint8_t *sA_hi,
                                           uint8_t *sA_lo, int tid) {
    const int m = tid % kBM;
    const int ny8 = P.Nyp >> 3;
    const float qh = (float)qy, ql = (float)(qy - (double)qh);
    const float yoff = 0.5f * (float)(P.ny - 1), vox = (float)P.voxel;
    // rotations by 1..3 and 4 voxels: each group of 8 phases is two levels deep
    const float2 s1 = expmi_fs(qh, ql, vox);
    const float2 s2 = cmul(s1, s1), s3 = cmul(s2, s1), s4 = cmul(s2, s2);
#pragma unroll 2
    for (int y8 = tid / kBM; y8 < ny8; y8 += kEpiThreads / kBM) {
        const float2 p0 = expmi_fs(qh, ql, ((float)(8 * y8) - yoff) * vox);
        const float2 p4 = cmul(p0, s4);
        const float2 phs[8] = {p0, cmul(p0, s1), cmul(p0, s2), cmul(p0, s3),
                               p4, cmul(p4, s1), cmul(p4, s2), cmul(p4, s3)};
        uint32_t re_hi[4], im_hi[4], re_lo[4], im_lo[4];
#pragma unroll
        for (int e = 0; e < 8; e += 2) {
            const int y = 8 * y8 + e;
            const bool in0 = valid && y < P.ny, in1 = valid && y + 1 < P.ny;
            split_pair(in0 ? phs[e].x : 0.f, in1 ? phs[e + 1].x : 0.f, P.bf16, &re_hi[e >> 1], &re_lo[e >> 1]);
            split_pair(in0 ? phs[e].y : 0.f, in1 ? phs[e + 1].y : 0.f, P.bf16, &im_hi[e >> 1], &im_lo[e >> 1]);
        }
        const uint32_t o_re = a_chunk_offset(m, 8 * y8);
        const uint32_t o_im = a_chunk_offset(m, P.Nyp + 8 * y8);
        *reinterpret_cast<uint4 *>(sA_hi + o_re) = make_uint4(re_hi[0], re_hi[1], re_hi[2], re_hi[3]);
        *reinterpret_cast<uint4 *>(sA_hi + o_im) = make_uint4(im_hi[0], im_hi[1], im_hi[2], im_hi[3]);
        if (P.split) {
            *reinterpret_cast<uint4 *>(sA_lo + o_re) = make_uint4(re_lo[0], re_lo[1], re_lo[2], re_lo[3]);
            *reinterpret_cast<uint4 *>(sA_lo + o_im) = make_uint4(im_lo[0], im_lo[1], im_lo[2], im_lo[3]);
        }
    }
}

template <bool kStoreH>
__global__ void __launch_bounds__(kTcThreads, 1)
    msft_tc_kernel(const __grid_constant__ TcMaps maps, const TcParams P) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sA_hi = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t a_bytes = (uint32_t)P.nkb_a * (uint32_t)(kBM * 128);
    uint8_t *sA_lo = sA_hi + a_bytes;
    uint8_t *ring = sA_hi + (P.split ? 2u : 1u) * a_bytes;
    const uint32_t R = P.ring_bytes;
    float2 *red = reinterpret_cast<float2 *>(ring + R);
    uint64_t *bars = reinterpret_cast<uint64_t *>(red + kBM);
    uint64_t *full = bars;
    uint64_t *empty = bars + kSlots;
    uint64_t *tfull = bars + 2 * kSlots;
    uint64_t *tempty = tfull + 2;
    uint64_t *drain = tempty + 2;
    uint64_t *a_full = drain + 1;
    uint64_t *never = a_full + 1;              // no thread arrives here (the failure-path test waits on it)
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(never + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kSlots; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&empty[s]), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(smem_u32(&tfull[b]), 1);
            mbar_init(smem_u32(&tempty[b]), kEpiWarps);
        }
        mbar_init(smem_u32(drain), 2);
        mbar_init(smem_u32(a_full), kEpiThreads);
        mbar_init(smem_u32(never), 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == kMmaWarp) {
        tmem_alloc(smem_u32(tmem_slot), kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    uint32_t prod_it = 0, oldest = 0, mma_it = 0, acc_it = 0, epi_it = 0;

    if (warp == kProducerWarp) {
        // ---------------- TMA producer: every tile, unit and occupied K block ----------------
        // The whole warp runs the loop (uniform values); one elected lane issues.
        bool ok = true;
        unsigned long long head = 0, tail = 0;     // unwrapped ring positions
        unsigned long long ends[kSlots];            // end of each stage in flight, by slot
        uint32_t head_off = 0;                      // head modulo the ring
        const int n_list = (int)__ldg(&P.list[0].x);
        for (int u = blockIdx.x; u < P.num_units && ok; u += gridDim.x) {
            const TcUnit un = unit_info(P, u, n_list);
            uint2 nxt = un.i_lo < un.i_hi ? __ldg(&P.list[1 + un.i_lo]) : make_uint2(0u, 0u);
            for (int i = un.i_lo; i < un.i_hi && ok; ++i) {
                const int t = (int)nxt.x;
                const uint32_t w = nxt.y;
                if (i + 1 < un.i_hi) nxt = __ldg(&P.list[i + 2]);
                const int c_lo = unit_c_lo(w), nch = unit_nch(w), sh = unit_shift(w);
                const uint32_t kmask = unit_kmask(w);
                const uint32_t sz = (uint32_t)(kPlanes * 8 * nch * 128);
                const CUtensorMap *map = &maps.m[nch - 1];
                for (int kb = 0; kb < P.nkb_b; ++kb) {
                    if (((kmask >> (4 * kb)) & 0xFu) == 0) continue;
                    const uint32_t off = ring_start(head_off, sz, R);
                    const unsigned long long start = head + (off == head_off ? 0u : R - head_off);
                    // reclaim consumed stages until this one has a slot and its bytes are free
                    while (oldest < prod_it && (prod_it - oldest >= (uint32_t)kSlots || start + sz > tail + R)) {
                        const uint32_t so = oldest % kSlots;
                        if (!warp_wait(smem_u32(&empty[so]), (oldest / kSlots) & 1, abort_flag, P.err,
                                       kErrTimeoutProducer)) {
                            ok = false;
                            break;
                        }
                        tail = ends[so];
                        ++oldest;
                    }
                    if (!ok) break;
                    const uint32_t s = prod_it % kSlots;
                    ends[s] = start + sz;
                    head = start + sz;
                    head_off = off + sz;
                    if (elect_one()) {
                        const uint32_t fb = smem_u32(&full[s]);
                        mbar_arrive_expect_tx(fb, sz);
                        tma_load_3d(smem_u32(ring + off), map, fb, kb * kBK + 8 * sh, 8 * c_lo, kPlanes * t);
                    }
                    __syncwarp();
                    ++prod_it;
                }
            }
        }
    } else if (warp == kMmaWarp || warp == kMmaWarp + 1) {
        // ---------------- MMA issuers (warp-wide loops, one elected lane issues) ----------------
        // Warp kMmaWarp + r takes the units with acc_it % 2 == r, so one warp's
        // waits and bookkeeping overlap the other's MMAs; both walk every stage
        // to keep the ring placement in step with the producer.
        const uint32_t mine = (uint32_t)(warp - kMmaWarp);
        bool ok = true;
        const uint64_t ring0 = sw128_desc(smem_u32(ring));
        const uint64_t ahi0 = sw128_desc(smem_u32(sA_hi)), alo0 = sw128_desc(smem_u32(sA_lo));
        uint32_t head_off = 0;
        uint32_t tl = 0;
        const int n_list = (int)__ldg(&P.list[0].x);
        if (stall_requested(P.err) && !warp_wait(smem_u32(never), 0, abort_flag, P.err, kErrTimeoutMma)) ok = false;
        for (int u = blockIdx.x; u < P.num_units && ok; u += gridDim.x, ++tl) {
            if (!warp_wait(smem_u32(a_full), tl & 1, abort_flag, P.err, kErrTimeoutMma)) break;
            tc_fence_after();
            const TcUnit un = unit_info(P, u, n_list);
            uint2 nxt = un.i_lo < un.i_hi ? __ldg(&P.list[1 + un.i_lo]) : make_uint2(0u, 0u);
            for (int i = un.i_lo; i < un.i_hi && ok; ++i) {
                const uint32_t w = nxt.y;
                if (i + 1 < un.i_hi) nxt = __ldg(&P.list[i + 2]);
                const uint32_t nr = 8u * (uint32_t)unit_nch(w);
                const uint32_t kmask = unit_kmask(w);
                const uint32_t sz = (uint32_t)kPlanes * nr * 128u;
                const uint32_t idesc = P.idesc | (((2u * nr) >> 3) << 17);
                const uint32_t b = acc_it & 1, aph = (acc_it >> 1) & 1;
                if (b != mine) {
                    // the other warp's unit: only advance the ring and stage counters
                    for (int kb = 0; kb < P.nkb_b; ++kb) {
                        if (((kmask >> (4 * kb)) & 0xFu) == 0) continue;
                        head_off = ring_start(head_off, sz, R) + sz;
                        ++mma_it;
                    }
                    ++acc_it;
                    continue;
                }
                if (!warp_wait(smem_u32(&tempty[b]), aph ^ 1, abort_flag, P.err, kErrTimeoutMma)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem_base + b * P.acc_cols;
                bool first = true;
                for (int kb = 0; kb < P.nkb_b; ++kb) {
                    const uint32_t kbits = (kmask >> (4 * kb)) & 0xFu;
                    if (kbits == 0) continue;
                    const uint32_t off = ring_start(head_off, sz, R);
                    head_off = off + sz;
                    const uint32_t s = mma_it % kSlots, ph = (mma_it / kSlots) & 1;
                    if (!warp_wait(smem_u32(&full[s]), ph, abort_flag, P.err, kErrTimeoutMma)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // descriptors advance by encoded (>> 4) byte offsets
                    const uint64_t w2 = ring0 + (uint64_t)(off >> 4);          // rows [0, 2 nr): [-Si | Sr]
                    const uint64_t w1 = w2 + (uint64_t)((nr * 128u) >> 4);    // rows [nr, 3 nr): [Sr | Si]
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        if (!((kbits >> kk) & 1u)) continue;
                        const int k = 4 * kb + kk;          // the phase operand's K step (y = 16 k)
                        const uint64_t off_r = a_k_offset(16 * k) >> 4, off_i = a_k_offset(P.Nyp + 16 * k) >> 4;
                        const uint64_t b1 = w1 + (uint64_t)(kk * 2), b2 = w2 + (uint64_t)(kk * 2);
                        const uint32_t acc0 = first ? 0u : 1u;
                        if (elect_one()) {
                            mma_f16(d, ahi0 + off_r, b1, idesc, acc0);
                            mma_f16(d, ahi0 + off_i, b2, idesc, 1u);
                            if (P.split) {
                                mma_f16(d, alo0 + off_r, b1, idesc, 1u);
                                mma_f16(d, alo0 + off_i, b2, idesc, 1u);
                            }
                        }
                        __syncwarp();
                        first = false;
                    }
                    if (elect_one()) mma_commit(smem_u32(&empty[s]));
                    __syncwarp();
                    ++mma_it;
                }
                if (!ok) break;
                if (elect_one()) mma_commit(smem_u32(&tfull[b]));
                __syncwarp();
                ++acc_it;
            }
        }
    } else if constexpr (kStoreH) {
        // ---------------- phase operand + 16-bit stores of [Re G | Im G] ----------------
        // Each thread waits for every unit's accumulator, so it has seen the
        // completion of the previous tile's MMAs before it rewrites the phase operand.
        const int quarter = warp & 3, half = warp >> 2;
        const int m = quarter * 32 + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        const int n_list = (int)__ldg(&P.list[0].x);
        const size_t plane = (size_t)P.h_Jg * P.h_Kx;
        for (int u = blockIdx.x; u < P.num_units; u += gridDim.x) {
            const TcUnit un = unit_info(P, u, n_list);
            const long long v = (long long)un.mt * kBM + m;
            const bool valid = v < P.n_pix;
            const double qy = valid ? P.q[3 * v + 1] : 0.0;
            if (__shfl_sync(0xffffffffu, *abort_flag, 0) == 0)
                build_phase(P, qy, valid, sA_hi, sA_lo, threadIdx.x);
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(smem_u32(a_full));
            const long long g = valid ? v / P.h_Rg : 0, r = valid ? v % P.h_Rg : 0;
            uint16_t *row0 = P.Ht + ((size_t)(3 * g) * P.h_Jg + (size_t)r * P.h_Jp) * P.h_Kx;   // plane 0, slice 0
            uint2 nxt = un.i_lo < un.i_hi ? __ldg(&P.list[1 + un.i_lo]) : make_uint2(0u, 0u);
            for (int i = un.i_lo; i < un.i_hi; ++i) {
                const int t = (int)nxt.x;
                const uint32_t w = nxt.y;
                if (i + 1 < un.i_hi) nxt = __ldg(&P.list[i + 2]);
                const int c_lo = unit_c_lo(w), nch = unit_nch(w);
                const uint32_t b = epi_it & 1, ph = (epi_it >> 1) & 1;
                const bool got = mbar_wait(smem_u32(&tfull[b]), ph, abort_flag, P.err, kErrTimeoutEpilogue);
                if (!__all_sync(0xffffffffu, got)) break;
                tc_fence_after();
                const uint32_t nr = 8u * (uint32_t)nch;
#pragma unroll 1
                for (int c = c_lo + ((c_lo & 1) != half); c < c_lo + nch; c += 2) {
                    // chunks alternate between the two halves
                    const uint32_t col = b * P.acc_cols + 8u * (uint32_t)(c - c_lo);
                    float gr[8], gi[8];
                    tmem_ld8(lane_base + col, gr);
                    tmem_ld8(lane_base + col + nr, gi);
                    tmem_ld_wait8(gr, gi);
                    if (valid) {
                        uint32_t re[4], im[4], mi[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            re[e] = pack_pair(gr[2 * e], gr[2 * e + 1], P.h_bf16);
                            im[e] = pack_pair(gi[2 * e], gi[2 * e + 1], P.h_bf16);
                            mi[e] = im[e] ^ 0x80008000u;        // both formats keep the sign in the top bit
                        }
                        uint16_t *dst = row0 + (size_t)t * P.h_Kx + 8 * c;
                        *reinterpret_cast<uint4 *>(dst) = make_uint4(mi[0], mi[1], mi[2], mi[3]);
                        *reinterpret_cast<uint4 *>(dst + plane) = make_uint4(re[0], re[1], re[2], re[3]);
                        *reinterpret_cast<uint4 *>(dst + 2 * plane) = make_uint4(im[0], im[1], im[2], im[3]);
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
                ++epi_it;
            }
        }
    } else {
        // ---------------- phase operand + epilogue warps ----------------
        const int quarter = warp & 3, half = warp >> 2;
        const int m = quarter * 32 + lane;
        const uint32_t lane_base = tmem_base + ((uint32_t)(quarter * 32) << 16);
        // Every epilogue thread runs every tile iteration (after an abort the
        // waits return at once), so the named barriers below always meet.
        const int n_list = (int)__ldg(&P.list[0].x);
        // q of this thread's pixel, loaded one unit ahead
        double nq0 = 0.0, nq1 = 0.0, nq2 = 0.0;
        if (blockIdx.x < (unsigned)P.num_units) {
            const long long p0 = (long long)unit_info(P, blockIdx.x, n_list).mt * kBM + m;
            if (p0 < P.n_pix) {
                nq0 = P.q[3 * p0];
                nq1 = P.q[3 * p0 + 1];
                nq2 = P.q[3 * p0 + 2];
            }
        }
        for (int u = blockIdx.x; u < P.num_units; u += gridDim.x) {
            const TcUnit un = unit_info(P, u, n_list);
            const int mt = un.mt;
            const long long p = (long long)mt * kBM + m;
            const bool valid = p < P.n_pix;
            const double qx = nq0, qy = nq1, qz = nq2;
            if (u + (int)gridDim.x < P.num_units) {
                const long long pn = (long long)unit_info(P, u + gridDim.x, n_list).mt * kBM + m;
                if (pn < P.n_pix) {
                    nq0 = P.q[3 * pn];
                    nq1 = P.q[3 * pn + 1];
                    nq2 = P.q[3 * pn + 2];
                }
            }
            // The tensor core is done with the previous tile's phase operand:
            // this thread has seen the completion of its last unit.
            if (__shfl_sync(0xffffffffu, *abort_flag, 0) == 0)
                build_phase(P, qy, valid, sA_hi, sA_lo, threadIdx.x);
            fence_async_smem();
            tc_fence_before();
            mbar_arrive(smem_u32(a_full));

            // q split once into an FP32 pair; every coordinate below is FP32
            // (FP64 throughput is a small fraction of FP32 on this part)
            const float qxh = (float)qx, qxl = (float)(qx - (double)qxh);
            const float qyh = (float)qy, qyl = (float)(qy - (double)qyh);
            const float qzh = (float)qz, qzl = (float)(qz - (double)qzh);
            const float vf = (float)P.voxel;
            const float xoff = 0.5f * (float)(P.nx - 1), zoff = 0.5f * (float)(P.nz - 1);
            float2 W[8];                                  // e^{-i q_x k dx}, k < 8
#pragma unroll
            for (int k = 0; k < 8; ++k) W[k] = expmi_fs(qxh, qxl, (float)k * vf);
            const float2 X16 = expmi_fs(qxh, qxl, 16.f * vf);   // from one chunk of a half to its next
            const float2 Ysh = expmi_fs(qyh, qyl, 8.f * vf);    // a unit's K steps shifted by 8 y
            const float2 Zstep = expmi_fs(qzh, qzl, vf);
            float2 Z = make_float2(1.f, 0.f);
            int t_prev = -2;
            float2 acc = make_float2(0.f, 0.f);
            uint2 nxt = un.i_lo < un.i_hi ? __ldg(&P.list[1 + un.i_lo]) : make_uint2(0u, 0u);
            for (int i = un.i_lo; i < un.i_hi; ++i) {
                const int t = (int)nxt.x;
                const uint32_t w = nxt.y;
                if (i + 1 < un.i_hi) nxt = __ldg(&P.list[i + 2]);
                // e^{-i q_z z_t}: kept for more units of the same slice, advanced
                // by one slice step, re-anchored after a gap and every 16 units
                if (t != t_prev) {
                    if (t == t_prev + 1 && (i & 15) != 0)
                        Z = cmul(Z, Zstep);
                    else
                        Z = expmi_fs(qzh, qzl, ((float)t - zoff) * vf);
                }
                t_prev = t;
                const int c_lo = unit_c_lo(w), c_hi = c_lo + unit_nch(w);
                const uint32_t b = epi_it & 1, ph = (epi_it >> 1) & 1;
                // one decision per warp: the lanes below meet at __syncwarp
                const bool got = mbar_wait(smem_u32(&tfull[b]), ph, abort_flag, P.err, kErrTimeoutEpilogue);
                if (!__all_sync(0xffffffffu, got)) break;
                tc_fence_after();
                const uint32_t nr = 8u * (uint32_t)(c_hi - c_lo);
                float2 acct = make_float2(0.f, 0.f);
                // this half's chunks: c_first, c_first + 2, ... (nh of them), read
                // kEpiBatch at a time with one wait; the x anchor of each is the
                // previous one's times e^{-i q_x 16 dx}
                const int c_first = c_lo + ((c_lo & 1) != half);
                const int nh = c_first < c_hi ? (c_hi - c_first + 1) >> 1 : 0;
                if (nh > 0) {
                    float2 Ec = expmi_fs(qxh, qxl, ((float)(8 * c_first) - xoff) * vf);
                    const uint32_t col0 = b * P.acc_cols + 8u * (uint32_t)(c_first - c_lo);
                    for (int j0 = 0; j0 < nh; j0 += kEpiBatch) {
                        float gr[kEpiBatch][8], gi[kEpiBatch][8];
#pragma unroll
                        for (int q = 0; q < kEpiBatch; ++q)
                            if (j0 + q < nh) {
                                const uint32_t col = col0 + 16u * (uint32_t)(j0 + q);
                                tmem_ld8(lane_base + col, gr[q]);
                                tmem_ld8(lane_base + col + nr, gi[q]);
                            }
                        tmem_ld_wait8(gr[0], gi[0]);
#pragma unroll
                        for (int q = 1; q < kEpiBatch; ++q) tmem_ld_after_wait8(gr[q], gi[q]);
#pragma unroll
                        for (int q = 0; q < kEpiBatch; ++q) {
                            if (j0 + q < nh) {
                                float hr = 0.f, hi = 0.f;
#pragma unroll
                                for (int k = 0; k < 8; ++k) {
                                    hr = fmaf(W[k].x, gr[q][k], hr);
                                    hr = fmaf(-W[k].y, gi[q][k], hr);
                                    hi = fmaf(W[k].x, gi[q][k], hi);
                                    hi = fmaf(W[k].y, gr[q][k], hi);
                                }
                                acct.x = fmaf(Ec.x, hr, fmaf(-Ec.y, hi, acct.x));
                                acct.y = fmaf(Ec.x, hi, fmaf(Ec.y, hr, acct.y));
                                Ec = cmul(Ec, X16);
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_u32(&tempty[b]));
                if (unit_shift(w)) acct = cmul(acct, Ysh);
                acc.x = fmaf(Z.x, acct.x, fmaf(-Z.y, acct.y, acc.x));
                acc.y = fmaf(Z.x, acct.y, fmaf(Z.y, acct.x, acc.y));
                ++epi_it;
            }
            if (half == 1) red[m] = acc;
            named_bar_sync(kEpiThreads);
            if (half == 0 && valid) {
                const float2 o = red[m];
                float2 a = make_float2(acc.x + o.x, acc.y + o.y);
                a = cmul(make_float2(P.str_re, P.str_im), a);
                if (un.part < 0) {
                    P.A[p] = a;
                    P.I[p] = a.x * a.x + a.y * a.y;
                } else {
                    const long long tail = (long long)(P.num_m_tiles - P.whole) * kBM;
                    P.Apart[un.part * tail + (long long)(mt - P.whole) * kBM + m] = a;
                }
            }
            named_bar_sync(kEpiThreads);
        }
    }

    // ---- teardown: make sure no tensor-core or TMA work is in flight ----
    __syncthreads();
    if (*abort_flag) {
        if ((warp == kMmaWarp || warp == kMmaWarp + 1) && lane == 0) {
            mma_commit(smem_u32(drain));       // one arrival per MMA warp
            volatile int dummy = 0;
            mbar_wait(smem_u32(drain), 0, &dummy, P.err, kErrTimeoutDrain);
        }
        if (warp == kProducerWarp && lane == 0) {
            volatile int dummy = 0;
            for (uint32_t it = oldest; it < prod_it; ++it) {
                const uint32_t s = it % kSlots, ph = (it / kSlots) & 1;
                mbar_wait(smem_u32(&full[s]), ph, &dummy, P.err, kErrTimeoutDrain);
            }
        }
    }
    __syncthreads();
    if (warp == kMmaWarp) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// Fields of the tiles whose unit lists were cut into parts: A = the parts'
// sum in part order, I = |A|^2.
__global__ void tc_tail_sum_kernel(const float2 *__restrict__ Apart, int parts, long long tail, long long p0,
                                   long long n_pix, float2 *__restrict__ A, float *__restrict__ I) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= tail || p0 + t >= n_pix) return;
    float2 a = Apart[t];
    for (int k = 1; k < parts; ++k) {
        const float2 b = Apart[k * tail + t];
        a.x += b.x;
        a.y += b.y;
    }
    A[p0 + t] = a;
    I[p0 + t] = a.x * a.x + a.y * a.y;
}

// ---- host side ------------------------------------------------------------------

double tc_issued_flops(const int *geom, int nz, int Nxp, int Nyp, long long n_pix, bool split) {
    const long long m_tiles = (n_pix + kBM - 1) / kBM;
    const int mc = kTcMaxChunks;
    double per_tile = 0.0;
    for (int t = 0; t < nz; ++t) {
        uint32_t w[kMaxUnitsPerSlice];
        const int n = plan_units(geom + 4 * (size_t)nz, nz, t, Nxp / 8, mc, true, w);
        for (int i = 0; i < n; ++i) {
            const int nsteps = __builtin_popcount(unit_kmask(w[i]));
            // two real MMAs of 128 x (2 x 8 nch) x 16 per K step and phase product
            per_tile += 2.0 * 2.0 * kBM * (2.0 * 8.0 * unit_nch(w[i])) * 16.0 * nsteps;
        }
    }
    return per_tile * (double)m_tiles * (split ? 2.0 : 1.0);
}

// One map per unit width: map k-1 copies a box of 64 y x 8k rows x the
// three planes of one slice.
bool encode_tmap_B(TcMaps *maps, void *base, int Kp, int Nxp, int nz, bool bf16, std::string *why) {
    std::memset(maps, 0, sizeof(TcMaps));
    const int nch = Nxp / 8 < kTcMaxChunks ? Nxp / 8 : kTcMaxChunks;
    if (nch < 1 || Nxp > 8 * kGeomChunks) {
        *why = "slice width outside the tensor-core range";
        return false;
    }
    for (int k = 1; k <= nch; ++k) {
        const uint64_t dims[3] = {(uint64_t)Kp, (uint64_t)Nxp, (uint64_t)kPlanes * nz};
        const uint64_t strides[2] = {(uint64_t)Kp * 2, (uint64_t)Nxp * Kp * 2};
        const uint32_t box[3] = {(uint32_t)kBK, (uint32_t)(8 * k), (uint32_t)kPlanes};
        if (!encode_tmap_3d_16bit(&maps->m[k - 1], base, dims, strides, box, bf16, why, 128)) return false;
    }
    return true;
}

static cudaError_t launch_tc(const TcMaps &maps, const double *q, long long n_pix, int nx, int ny, int nz, int Nxp,
                             int Nyp, double voxel, double str_re, double str_im, bool split, bool bf16, int *geom,
                             float2 *A, float *I, int *err, int sm_count, cudaStream_t st, const UqStore *store,
                             float2 *tail_part) {
    if (!tc_grid_ok(Nxp, Nyp, split) || nz < 1 || nz > 512 || nx > Nxp || ny > Nyp) return cudaErrorInvalidValue;
    const size_t ring = tc_ring_bytes(Nxp, Nyp, split);
    if (ring == 0) return cudaErrorInvalidValue;
    const int max_chunks = kTcMaxChunks;
    uint2 *list = geom_units(geom, nz);
    TcParams P;
    P.q = q;
    P.list = list;
    P.n_pix = n_pix;
    P.nx = nx;
    P.ny = ny;
    P.nz = nz;
    P.Nxp = Nxp;
    P.Nyp = Nyp;
    P.nkb_a = tc_nkb(2 * Nyp);
    P.nkb_b = tc_nkb(Nyp);
    P.ring_bytes = (uint32_t)ring;
    P.split = split ? 1 : 0;
    P.bf16 = bf16 ? 1 : 0;
    P.num_m_tiles = (int)((n_pix + kBM - 1) / kBM);
    P.whole = P.num_m_tiles;
    P.parts = 1;
    P.Apart = nullptr;
    if (store) {
        // about one unit per SM (units are independent there)
        const int want = (sm_count + P.num_m_tiles - 1) / P.num_m_tiles;
        P.whole = 0;
        P.parts = want < 1 ? 1 : want > nz ? nz : want;
    } else if (tail_part) {
        // the last partial wave (every tile when there are fewer tiles than
        // SMs): cut its tiles so that wave fills the SMs
        const int rem = P.num_m_tiles > sm_count ? P.num_m_tiles % sm_count : P.num_m_tiles;
        if (rem > 0) {
            int parts = (sm_count + rem / 2) / rem;
            parts = parts < 1 ? 1 : parts > kTcMaxTailParts ? kTcMaxTailParts : parts;
            if (parts > 1) {
                P.whole = P.num_m_tiles - rem;
                P.parts = parts;
                P.Apart = tail_part;
            }
        }
    }
    P.num_units = P.whole + (P.num_m_tiles - P.whole) * P.parts;
    const uint32_t M = kBM;
    P.idesc = (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) | ((M >> 4) << 24);
    P.acc_cols = (uint32_t)kAccCols;
    P.voxel = voxel;
    P.str_re = (float)str_re;
    P.str_im = (float)str_im;
    P.A = A;
    P.I = I;
    P.err = err;
    P.Ht = store ? store->Ht : nullptr;
    P.h_Jp = store ? store->Jp : 0;
    P.h_Jg = store ? store->Rg * store->Jp : 0;
    P.h_Rg = store ? store->Rg : 1;
    P.h_Kx = store ? store->Kx : 0;
    P.h_bf16 = store && store->bf16 ? 1 : 0;
    if (store && (store->Kx < Nxp || store->Kx % 8 != 0 || store->Jp < nz)) return cudaErrorInvalidValue;
    const size_t smem = (split ? 2 : 1) * tc_a_bytes(Nyp) + ring + tc_fixed_bytes();
    // The attribute is per function and shared by every thread of the process:
    // always raise it to the largest size any launch uses, never to this
    // launch's size, so concurrent launches from other threads stay valid.
    cudaError_t e = store ? cudaFuncSetAttribute(msft_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 kMaxSmem)
                          : cudaFuncSetAttribute(msft_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 kMaxSmem);
    if (e != cudaSuccess) return e;
    // units of the uniform-q y-sum keep their K steps on the 16-y grid (its
    // epilogue stores G itself, with no room for a per-unit phase)
    pack_units_kernel<<<1, 256, 0, st>>>(geom_chunk_y(geom, nz), nz, Nxp / 8, max_chunks, store ? 0 : 1, list);
    int grid = P.num_units < sm_count ? P.num_units : sm_count;
    if (grid < 1) grid = 1;
    if (store) {
        msft_tc_kernel<true><<<grid, kTcThreads, smem, st>>>(maps, P);
    } else {
        msft_tc_kernel<false><<<grid, kTcThreads, smem, st>>>(maps, P);
        if (P.whole < P.num_m_tiles) {
            const long long tail = (long long)(P.num_m_tiles - P.whole) * kBM;
            tc_tail_sum_kernel<<<(unsigned)((tail + 255) / 256), 256, 0, st>>>(
                P.Apart, P.parts, tail, (long long)P.whole * kBM, n_pix, A, I);
        }
    }
    return cudaGetLastError();
}

size_t tc_tail_part_bytes(long long n_pix, int sm_count) {
    // at most kTcMaxTailParts parts of fewer than sm_count tiles
    const long long tiles = (n_pix + kBM - 1) / kBM;
    const long long rem = tiles > sm_count ? tiles % sm_count : tiles;
    return (size_t)(rem * kBM * kTcMaxTailParts) * sizeof(float2);
}

cudaError_t launch_msft_tc(const TcMaps &maps, const double *q, long long n_pix, int nx, int ny, int nz,
                           int Nxp, int Nyp, double voxel, double str_re, double str_im, bool split,
                           bool bf16, int *geom, float2 *A, float *I, int *err,
                           int sm_count, cudaStream_t st, float2 *tail_part) {
    return launch_tc(maps, q, n_pix, nx, ny, nz, Nxp, Nyp, voxel, str_re, str_im, split, bf16, geom, A, I, err,
                     sm_count, st, nullptr, tail_part);
}

cudaError_t launch_uq_y_tc_mma(const TcMaps &maps, const double *qrow, int det_ny, int nx, int ny, int nz, int Nxp,
                               int Nyp, double voxel, bool split, bool bf16, int *geom, const UqStore &store,
                               int *err, int sm_count, cudaStream_t st) {
    return launch_tc(maps, qrow, det_ny, nx, ny, nz, Nxp, Nyp, voxel, 1.0, 0.0, split, bf16, geom, nullptr,
                     nullptr, err, sm_count, st, &store, nullptr);
}

}  // namespace scm
