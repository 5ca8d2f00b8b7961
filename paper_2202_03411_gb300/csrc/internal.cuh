// internal.cuh -- declarations shared by the library's translation units.
// Not installed; the public surface is include/scatman.h.
#pragma once

#include <cuda_runtime.h>
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/scatman.h"

#include <nvtx3/nvToolsExt.h>

namespace scm {

constexpr double kPi = 3.14159265358979323846;

// An NVTX range around a stage of the host API (visible in Nsight timelines;
// a no-op unless a profiling tool is attached).
struct StageRange {
    explicit StageRange(const char *name) { nvtxRangePushA(name); }
    ~StageRange() { nvtxRangePop(); }
    StageRange(const StageRange &) = delete;
    StageRange &operator=(const StageRange &) = delete;
};

// Device allocation used by every buffer of the library; a test hook
// (scatman_debug_fail_allocation) can make one of them fail on the host.
cudaError_t device_malloc(void **p, size_t bytes);

// Status block of a handle on the device (kStatusBytes): the error word (int,
// byte 0) that kernels set; a test flag (int, byte 4) that makes the
// tensor-core kernels' MMA warps first wait on a barrier nothing arrives at,
// so that wait runs out and takes the abort path; and at byte 8 an optional
// shorter limit in ns for the kernels' work waits (unsigned long long; 0 =
// the default).
constexpr size_t kStatusBytes = 16;
constexpr unsigned long long kWaitLimitMaxNs = 2000000000ull;   // every bounded wait: 2 s at most

// Bits of the device error word written by kernels.
enum : int {
    kErrTimeoutProducer = 1,
    kErrTimeoutMma = 2,
    kErrTimeoutEpilogue = 4,
    kErrTimeoutDrain = 8,
    kErrBadLaunch = 16,
};

// Shape as the voxeliser kernels read it: body->lab rotation, centre, sizes
// and harmonic coefficients, everything in length units.
struct ShapeParams {
    int kind;
    int lmax;
    int soft;
    float inv_w_f;
    double inv_w;
    double r, a, b, c;
    double R0;
    double rmin, rmax;              // harmonics radius clip
    double R[9];                    // row-major body->lab rotation
    double cx, cy, cz;              // centre offset
    float Rf[9];                    // the rotation and the offsets in FP32 (fast path)
    float cxf, cyf, czf;
    float r2f, inv_af, inv_bf, inv_cf;   // r^2 and 1/a, 1/b, 1/c in FP32
    float R0f, rminf, rmaxf;             // harmonics radius scale and clip in FP32
    double alm[(SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 1)];
    float almf[(SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 1)];
    // normalised associated-Legendre recurrence coefficients, index l(l+1)/2 + m
    // (see real_sh_all): a_lm, b_lm, and the diagonal factors d_m, e_m
    double sh_a[(SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 2) / 2];
    double sh_b[(SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 2) / 2];
    double sh_d[SCATMAN_MAX_LMAX + 1];
    double sh_e[SCATMAN_MAX_LMAX + 1];
    float sh_af[(SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 2) / 2];
    float sh_bf[(SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 2) / 2];
    float sh_df[SCATMAN_MAX_LMAX + 1];
    float sh_ef[SCATMAN_MAX_LMAX + 1];
    // radii map (device copies, [ntheta][nphi])
    const double *rmap;
    const float *rmapf;
    int ntheta, nphi;
    double rm_tscale, rm_pscale;    // ntheta / pi, nphi / (2 pi)
    float rm_tscalef, rm_pscalef;
    float rm_slope;                 // max |dr/d angle| between neighbouring samples (FP32 decision margin)
    // volume map (device copies, [mx][my][mz])
    const unsigned char *vmap;
    int mx, my, mz;
    double mdx;
    float mdxf;
    const double *mdelta, *mbeta;   // per-cell index, or null
    int varn;                       // 1: voxel-resolved index (s carries (n_v^2 - 1) / nscale)
    double nscale;                  // max |n_v^2 - 1| over the map's cells
    // harmonics / radii map (and soft spheres / ellipsoids): a voxel centre with
    // |p| below band_lo is inside (soft: chi = 1), above band_hi outside
    // (chi = 0) (band_hi = 0: no band)
    float band_lo, band_hi;
};

// Soft occupancy cut of the FP32 modes: chi = 1 / (1 + e^{-t}) with
// t = (r_s - |p|) / w is taken as zero when chi < 2^-24, i.e. t < -kSoftCutT.
constexpr float kSoftCutT = 16.635532f;   // ln(2^24 - 1)
// Above this t the FP32 logistic is exactly 1.0f (e^{-t} below half an ulp of 1).
constexpr float kSoftOneT = 17.5f;

// Fills the FP32 copies and the harmonic recurrence tables of a ShapeParams
// whose double fields are set (api.cu).
void finish_shape_params(ShapeParams *sp);

// Number of geometric gradient parameters: sphere [r]; ellipsoid [a, b, c];
// harmonics [a_lm for l >= 1, R0].
#ifdef __CUDACC__
__host__ __device__
#endif
inline int n_geom_params(int kind, int lmax) {
    if (kind == SCATMAN_SPHERE) return 1;
    if (kind == SCATMAN_ELLIPSOID) return 3;
    if (kind == SCATMAN_RADIALMAP || kind == SCATMAN_VOLUMEMAP) return 0;
    return (lmax + 1) * (lmax + 1);
}

struct GridParams {
    int nx, ny, nz;
    double voxel;
    double k0;
    double delta, beta;
    float voxf;                     // voxel in FP32 (set by make_grid)
};

inline GridParams make_grid(int nx, int ny, int nz, double voxel, double k0, double delta, double beta) {
    GridParams g{nx, ny, nz, voxel, k0, delta, beta, (float)voxel};
    return g;
}

// Where the voxeliser writes s = chi*T.
enum SliceLayout { kLayoutC64 = 0, kLayoutC32 = 1, kLayoutTcF16 = 2, kLayoutTcBF16 = 3 };

// Tensor maps of the tensor-core slice operand, one per span width of 8k
// rows (k = 1 .. kTcMaxChunks): a box of 64 y x 8k rows x the three planes.
constexpr int kTcMaxChunks = 16;
struct TcMaps {
    CUtensorMap m[kTcMaxChunks];
};

// Per-slice geometry the voxeliser records for the contractions, in one
// device buffer of slice_geom_ints(nz) ints:
//   [0, 4 nz)            occupied box of every slice [x_lo | x_hi | y_lo | y_hi]
//   [4 nz, 68 nz)        occupied y range of every 8-column chunk of every slice,
//                        [y_lo | y_hi] x [nz][kGeomChunks] (tensor-core grids, nx <= 256)
//   then                 the tensor-core kernel's work-unit list (uint2, kMaxUnitsPerSlice nz + 1)
constexpr int kGeomChunks = 32;
constexpr int kMaxUnitsPerSlice = 4;
inline size_t slice_geom_ints(int nz) {
    return 4 * (size_t)nz + 2 * (size_t)kGeomChunks * nz + 2 * ((size_t)kMaxUnitsPerSlice * nz + 1);
}
inline int *geom_chunk_y(int *g, int nz) { return g + 4 * (size_t)nz; }
inline uint2 *geom_units(int *g, int nz) {
    return reinterpret_cast<uint2 *>(g + 4 * (size_t)nz + 2 * (size_t)kGeomChunks * nz);
}

struct SliceOut {
    int layout;
    int Nxp, Nyp, Kp;               // tensor-core operand: padded x and y; Kp = Nyp, the K extent of a row
    void *s;                        // C64: double2[nvox]; C32: float2[nvox]; TC: 16-bit [nz*3*Nxp][Kp]
    float *chi;                     // occupancy [z][x][y]
    int *bounds;                    // per slice [x_lo | x_hi | y_lo | y_hi] of chi != 0 (nz each), or null
    int *chunk_y;                   // per slice and 8-column chunk [y_lo | y_hi] (see above), or null
};

}  // namespace scm

struct scatman_handle {
    scatman_config cfg;
    int device = 0;
    int sm_count = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    long long n_pix = 0;
    double k0 = 0;
    int precision = 0;
    bool tensor_core = false;
    bool split = false;
    bool bf16 = false;
    bool s_bf16 = false;            // 16-bit type of the tensor-core slice operand
    bool scan_fp64 = false;
    // tensor-core operand geometry
    int Nxp = 0, Nyp = 0, Kp = 0;
    size_t b_rows = 0;
    // device buffers
    double *d_q = nullptr;          // [n_pix][3]
    int *d_bounds = nullptr;        // per-slice occupied box [x_lo | x_hi | y_lo | y_hi], 4*nz ints,
                                    // then the tensor-core kernel's occupied-slice list (nz + 1 uint2)
    float *d_chi = nullptr;         // [nvox]
    void *d_s = nullptr;            // slices in the contraction's layout
    size_t s_bytes = 0;
    void *d_A = nullptr;            // field cache (double2 or float2)
    void *d_I = nullptr;            // intensity scratch for acquire
    void *d_I2 = nullptr;           // second intensity buffer of the batched acquire (on first use)
    cudaStream_t copy_stream = nullptr;   // batched acquire: device-to-host copies
    cudaEvent_t ev_fwd[2] = {nullptr, nullptr}, ev_copy[2] = {nullptr, nullptr};
    int *d_err = nullptr;
    double *d_part = nullptr;       // backward partial sums
    size_t part_count = 0;
    void *d_S = nullptr;            // backward adjoint field (complex, nvox)
    void *d_partial = nullptr;      // CUDA-core contraction: per-split partial fields
    float2 *d_tail = nullptr;       // tensor-core contraction: partial fields of the last wave's cut tiles
    void *d_H = nullptr;            // uniform-q detector: y-contracted slices [v][z][x], or in the
                                    // tensor-core modes 16-bit planes [row group][-Im | Re | Im][Rg Jp][Kx]
    bool uniform_q = false;
    bool uniform_tc = false;        // uniform-q detector with the x/z sum on the tensor cores
    int uq_Jp = 0, uq_Kx = 0, uq_Rg = 1;   // its operand geometry: nz padded to 16, nx padded to 64,
                                           // detector rows per GEMM column group
    float2 *d_uq_qz = nullptr;      // its per-pixel q_z (float pair; marker off the Ewald sphere)
    double *d_uq_qrow = nullptr;    // q of each detector row's first pixel (q_y of the row), tensor-core modes
    CUtensorMap tmap_H;
    bool from_q_list = false;       // q given by the caller: no pixel geometry
    float2 *d_adj_part = nullptr;   // tensor-core adjoint: per-pixel-range partial fields
    size_t adj_part_count = 0;
    unsigned *d_gmax = nullptr;     // tensor-core adjoint: max |w A| (float bits)
    int adj_orders = -1;            // tensor-core adjoint: Jacobi-Anger orders N (0: one GEMM per slice; -1: not chosen yet)
    float2 *d_adj_coef = nullptr;   // order mode: a[j][n] = e^{+i q_c z_j} eps_n i^n J_n(D z_j), [nz][N]
    float2 *d_adj_ord = nullptr;    // order mode: the orders' fields S~ [N][nx][ny]
    float4 *d_adj_tab = nullptr;    // tensor-core adjoint: per-pixel constants (built at the first backward)
    uint8_t *d_adj_rtile = nullptr; // tensor-core adjoint: y-phase operand tiles (built at the first backward)
    // map shapes: device copies of the last voxelised map (grown as needed)
    double *d_rmap = nullptr;
    float *d_rmapf = nullptr;
    size_t rmap_cap = 0;
    unsigned char *d_vmap = nullptr;
    size_t vmap_cap = 0;
    double *d_mdelta = nullptr, *d_mbeta = nullptr;
    size_t mindex_cap = 0;
    double str_re = 0, str_im = 0;  // global strength factor of s: n^2 - 1, or the map's index scale
    double map_index_max = 0;       // max |delta|, |beta| over a volume map's cells
    int splits = 1;
    long long device_bytes = 0;
    scm::TcMaps tmap_B;
    bool have_tmap = false;
    // state
    bool have_shape = false;
    bool have_forward = false;
    scatman_shape shape;
    std::vector<double> alm;
    scm::ShapeParams sp;
    std::string last_error;
};

namespace scm {

// ---- host helpers shared by the .cu files --------------------------------
int set_error(scatman_handle *h, int code, const std::string &msg);
int check_cuda(scatman_handle *h, cudaError_t e, const char *what);

// Voxeliser + exclusive scan (voxelise.cu).
cudaError_t launch_voxelise(const ShapeParams &sp, const GridParams &gp, const SliceOut &out,
                            bool scan_fp64, bool fp64_mode, cudaStream_t st);
// Detector q (voxelise.cu).
cudaError_t launch_detector_q(int det_nx, int det_ny, double theta_max_deg, double k0, double *q,
                              cudaStream_t st);
// Uniform-q virtual detector (msft_uniform.cu).
cudaError_t launch_detector_q_uniform(int det_nx, int det_ny, double theta_max_deg, double k0, double *q,
                                      cudaStream_t st);
// q_z table marker (a quiet-NaN bit pattern) of a pixel off the Ewald sphere.
constexpr uint32_t kUqOffSphereBits = 0x7fc00000u;
cudaError_t launch_msft_uniform(bool fp64, const void *s, int nx, int ny, int nz, int det_nx, int det_ny,
                                double theta_max_deg, double k0, double voxel, double str_re, double str_im,
                                const float2 *qz, void *H, void *A, void *I, cudaStream_t st);
// Uniform-q detector on the tensor cores (msft_tc.cu in store mode for U1,
// msft_uniform_tc.cu for the x/z contraction).
// Operand geometry: Kx = nx padded to its K block (16, 32 or 64), Jp = nz padded
// to 16, Rg rows per group.
void uq_tc_geometry(int nx, int nz, int *Kx, int *Jp, int *Rg);
size_t uq_tc_h_bytes(int nx, int nz, int det_ny);
int uq_tc_slots(int nx, int nz, bool split);
bool encode_tmap_uq(CUtensorMap *map, void *H, int nx, int nz, int det_ny, bool bf16, std::string *why);
double uq_tc_issued_flops(int nx, int nz, int det_nx, int det_ny, bool split);
// q_z per pixel as a float pair with a marker off the Ewald sphere (once per handle).
cudaError_t launch_uq_qz_table(const double *q, long long n, double k0, float2 *tab, cudaStream_t st);
cudaError_t launch_uq_tc(const CUtensorMap &map, const float2 *qz, int nx, int nz, int det_nx, int det_ny,
                         double theta_max_deg, double k0, double voxel, double str_re, double str_im, bool split,
                         bool bf16, float2 *A, float *I, int *err, int sm_count, cudaStream_t st);
// CUDA-core contraction (msft_simt.cu).
int simt_splits(long long n_pix, int nx, int nz, int sm_count);
// bounds: the voxeliser's per-slice occupied boxes (4 nz ints), or NULL for a dense sum.
cudaError_t launch_msft_simt(bool fp64, const void *s, const double *q, long long n_pix, int nx, int ny,
                             int nz, double voxel, double str_re, double str_im, void *A, void *I,
                             void *partial, int splits, cudaStream_t st, const int *bounds);
// Real flops the CUDA-core contraction executes with box skipping (host copy of the bounds).
double simt_issued_flops(const int *bounds, int nz, int ny, long long n_pix, bool fp64);
// Tensor-core contraction (msft_tc.cu).  Whether a padded grid fits its
// tensor-memory layout (phase operand and two accumulators) and unit masks.
bool tc_grid_ok(int Nxp, int Nyp, bool split);
// geom: the slice-geometry buffer (slice_geom_ints); tail_part: scratch of
// tc_tail_part_bytes for the partial fields of the last partial wave's tiles
// (null: every tile whole).
cudaError_t launch_msft_tc(const TcMaps &maps, const double *q, long long n_pix, int nx, int ny, int nz,
                           int Nxp, int Nyp, double voxel, double str_re, double str_im, bool split,
                           bool bf16, int *geom, float2 *A, float *I, int *err,
                           int sm_count, cudaStream_t st, float2 *tail_part);
size_t tc_tail_part_bytes(long long n_pix, int sm_count);
// The same kernel in store mode, the uniform-q detector's y-contraction on the
// tensor cores: rows are detector rows v (q_y(v) = qrow[3 v + 1]) and G is
// written to the x/z operand H as 16-bit planes.
struct UqStore {
    uint16_t *Ht;
    int Jp, Rg, Kx;
    bool bf16;                  // H's 16-bit type
};
cudaError_t launch_uq_y_tc_mma(const TcMaps &maps, const double *qrow, int det_ny, int nx, int ny, int nz, int Nxp,
                               int Nyp, double voxel, bool split, bool bf16, int *geom,
                               const UqStore &store, int *err, int sm_count, cudaStream_t st);
// Real flops one contraction launch issues for the recorded slice geometry
// (a host copy of the first 4 nz + 2 kGeomChunks nz ints of the buffer).
double tc_issued_flops(const int *geom_host, int nz, int Nxp, int Nyp, long long n_pix, bool split);
bool encode_tmap_B(TcMaps *maps, void *base, int Kp, int Nxp, int nz, bool bf16, std::string *why);
// A 3D tiled tensor map over 16-bit elements with a 32-, 64- or 128-byte
// swizzle (dims innermost first; strides of dims 1 and 2 in bytes; the box's
// inner extent in bytes equals the swizzle width).
bool encode_tmap_3d_16bit(CUtensorMap *map, void *base, const uint64_t dims[3], const uint64_t strides[2],
                          const uint32_t box[3], bool bf16, std::string *why, int swizzle_bytes);
// Ideal detector (detector.cu): expected photons and Poisson counts per pixel.
cudaError_t launch_photon_counts(const void *I, bool fp64, long long n, int det_nx, int det_ny, bool uniform,
                                 double theta_max_deg, double wavelength, double voxel, double photon_density,
                                 uint64_t seed, double *lambda, long long *counts, cudaStream_t st);
// Backward (adjoint.cu).
cudaError_t launch_adjoint_field(bool fp64, const void *A, const void *dLdI, const double *q, long long n_pix,
                                 int nx, int ny, int nz, double voxel, void *S, cudaStream_t st);
int grad_param_count(const ShapeParams &sp);
cudaError_t launch_grad_voxels(bool fp64, const ShapeParams &sp, const GridParams &gp, const void *S,
                               double *partials, int n_blocks, cudaStream_t st);
int grad_voxel_blocks(bool fp64, const ShapeParams &sp, const GridParams &gp, int sm_count);
cudaError_t launch_grad_pixels(bool fp64, const void *A, const void *dLdI, long long n_pix,
                               double *partials, int n_blocks, cudaStream_t st);
int grad_pixel_blocks(long long n_pix);
// Tensor-core adjoint field (adjoint_tc.cu).
bool adjoint_tc_supported(int nx, int ny);
// nz: slices, or in order mode (orders != 0) the number N of Jacobi-Anger orders;
// S receives the slices' (or orders') fields [nz][nx][ny].
int adjoint_tc_splits(long long n_pix, int nz, int sm_count, bool orders);
cudaError_t launch_adjoint_tc(const float2 *A, const float *w, const float4 *tab, const uint8_t *rtile, long long n_pix,
                              int nx, int ny, int nz, int orders, double voxel, int splits, float2 *partial,
                              unsigned *gmax_bits, float2 *S, int *err, cudaStream_t st);
// Order mode: the slices' fields from the orders' (coef: [nz][N] complex).
cudaError_t launch_adj_orders_combine(const float2 *Sord, const float2 *coef, int N, int nz, int nx, int ny, float2 *S,
                                      cudaStream_t st);
// The adjoint's y-phase operand tiles (once per handle).
size_t adj_rtile_bytes(long long n_pix, int ny);
cudaError_t launch_adj_rtile(const float4 *tab, long long n_pix, int ny, double voxel, uint8_t *rt, cudaStream_t st);
// Per-pixel constants of the tensor-core adjoint (3 float4 per pixel), once per handle.
// orders != 0: order mode with theta = acos((q_z - qc) inv_d) in place of q_z.
cudaError_t launch_adj_pixel_table(const double *q, long long n, double voxel, int orders, double qc, double inv_d,
                                   float4 *tab, cudaStream_t st);
// Fit residual 2 (I - target) and partial sums of (I - target)^2 (adjoint.cu).
int l2_residual_blocks(long long n);
cudaError_t launch_l2_residual(bool fp64, const void *I, const float *target, long long n, void *w, double *partials,
                               int n_blocks, cudaStream_t st);

}  // namespace scm

// ---- device helpers ---------------------------------------------------------
#ifdef __CUDACC__
namespace scm {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}

// e^{-i q c} for a q held in double and a coordinate c that is a small
// multiple of the voxel: the argument q*c is formed as a float pair
// (FMA-exact product of the high part plus the low part's product) and
// reduced modulo 2 pi in two pieces (Cody-Waite), so the reduced angle is
// good to ~1e-7 rad even for |q c| of a few hundred radians.
__device__ __forceinline__ float2 expmi_fs(float qh, float ql, float cf) {
    const float kTwoPiHi = 6.28318548202514648f;
    const float kTwoPiLo = -1.7484555314695172e-07f;
    const float kInvTwoPi = 0.15915494309189535f;
    float p = qh * cf;
    float e = fmaf(qh, cf, -p);
    float lo = fmaf(ql, cf, e);
    float n = rintf(p * kInvTwoPi);
    float r = fmaf(-n, kTwoPiHi, p);
    r = r + fmaf(-n, kTwoPiLo, lo);
    float s, co;
    sincosf(r, &s, &co);
    return make_float2(co, -s);
}

__device__ __forceinline__ float2 expmi_f(double q, double c) {
    float qh = (float)q;
    float ql = (float)(q - (double)qh);
    return expmi_fs(qh, ql, (float)c);
}

__device__ __forceinline__ double2 expmi_d(double q, double c) {
    double s, co;
    sincos(q * c, &s, &co);
    return make_double2(co, -s);
}

}  // namespace scm
#endif
