/*
 * scatman.h -- C ABI of the GB300 Multi-Slice Fourier Transform library.
 *
 * The library computes the Scatman's wide-angle diffraction pattern
 * (arXiv 2202.03411, Eq. 9):
 *
 *   A(q) = (n^2 - 1) sum_j e^{-i q_z z_j} sum_{x,y} chi_j(x,y) T_j(x,y) e^{-i (q_x x + q_y y)},
 *   T_j  = exp(i k0 dz (n - 1) C_j),   C_j = sum_{j' < j} chi_{j'}   (Eq. 8, exclusive),
 *   I(q) = |A(q)|^2                                                    (Sec. 3.3, Block 11),
 *
 * with n = 1 - delta + i beta (Eq. 7), k0 = 2 pi / wavelength, chi the
 * voxel occupancy of the shape (Block 5) and q the transfer momentum of each
 * detector pixel on the Ewald sphere (Eq. 3).
 *
 * Conventions shared by every call:
 *  - Voxel arrays are [z][x][y] with y fastest.  Voxel centres sit at
 *    (index - (N-1)/2) * voxel; the beam travels along +z and enters at z
 *    index 0.  q = k_out - k_in (so q_z <= 0) and the phase is e^{-i q.r}.
 *  - Detector pixel p = v*det_nx + u; u runs along x, v along y.  The flat
 *    detector is normal to z and reaches theta_max at the edge midpoints.
 *  - All device work is queued on the handle's CUDA stream and is
 *    asynchronous unless a call says it synchronises.
 *  - Errors come back as a negative scatman_status; nothing aborts or throws
 *    across the ABI.  scatman_last_error() describes the last failure.
 *  - A handle is not thread safe; distinct handles are independent.
 *  - Pointers are borrowed for the duration of the call only, unless stated.
 */
#ifndef SCATMAN_H
#define SCATMAN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SCATMAN_API __attribute__((visibility("default")))
#else
#define SCATMAN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SCATMAN_OK = 0,
    SCATMAN_ERR_ARG = -1,         /* invalid argument or unsupported size */
    SCATMAN_ERR_OOM = -2,         /* a device or host allocation failed */
    SCATMAN_ERR_CUDA = -3,        /* a CUDA runtime/driver call failed */
    SCATMAN_ERR_TIMEOUT = -4,     /* a kernel gave up a bounded wait; results invalid */
    SCATMAN_ERR_ADMISSION = -5,   /* serving: request exceeds the memory budget */
    SCATMAN_ERR_STATE = -6,       /* call out of order (e.g. forward before voxelise) */
    SCATMAN_ERR_UNSUPPORTED = -7, /* no device of compute capability 10.3 */
    SCATMAN_ERR_CANCELLED = -8    /* serving: the request was cancelled before it was admitted */
} scatman_status;

/* Arithmetic of the Fourier contraction (Eq. 9's per-slice sum). */
typedef enum {
    SCATMAN_FP64 = 0,          /* CUDA-core FP64 direct sum; FP64 scan; I and A in double */
    SCATMAN_FP32 = 1,          /* CUDA-core FP32 direct sum; I float, A float2 */
    SCATMAN_TC_F16_SPLIT = 2,  /* tcgen05, f16 operands, phases split hi+lo, FP32 accumulate */
    SCATMAN_TC_BF16_SPLIT = 3, /* tcgen05, bf16 operands, phases split hi+lo, FP32 accumulate */
    SCATMAN_TC_F16 = 4,        /* tcgen05, f16 operands, single phase product */
    SCATMAN_TC_BF16 = 5        /* tcgen05, bf16 operands, single phase product */
} scatman_precision;

enum { SCATMAN_SPHERE = 0, SCATMAN_ELLIPSOID = 1, SCATMAN_SPHHARM = 2, SCATMAN_RADIALMAP = 3, SCATMAN_VOLUMEMAP = 4 };

/* Detector geometry. */
enum {
    SCATMAN_DETECTOR_FLAT = 0,      /* flat detector normal to z; theta_max at the edge midpoints */
    SCATMAN_DETECTOR_UNIFORM_Q = 1  /* the paper's virtual detector: pixels uniform in (q_x, q_y) up to
                                       k0 sin(theta_max); q_z on the Ewald sphere (Eq. 3); pixels with
                                       q_x^2 + q_y^2 > k0^2 carry zero */
};

/* Maximum harmonic degree accepted for SCATMAN_SPHHARM. */
#define SCATMAN_MAX_LMAX 12

/*
 * Experiment and grid (Sec. 3.1, Blocks 1-3; Listing 1 set_experiment).
 *  nx, ny, nz      voxel grid (each >= 1, nx, ny <= 4096, nz <= 512; nz <= 256
 *                  in SCATMAN_FP64; tensor-core modes need nx <= 256 and, with
 *                  split phases, ny <= 128, unsplit ny <= 256)
 *  voxel           voxel edge and slice thickness dz, same length unit as wavelength
 *  wavelength      lambda; k0 = 2 pi / lambda
 *  theta_max_deg   scattering angle at the detector's edge midpoints, (0, 90)
 *  det_nx, det_ny  detector pixels (>= 1)
 *  q_list, n_q     optional host array of n_q (q_x, q_y, q_z) triples that
 *                  replaces the flat detector (copied during scatman_create);
 *                  NULL/0 selects the detector
 *  precision       scatman_precision
 *  soft            0: binary occupancy (voxel centre inside, ties inside);
 *                  1: logistic occupancy sigmoid((r_s - |p|)/soft_width);
 *                  outside SCATMAN_FP64 a voxel whose logistic is below
 *                  2^-24 counts as empty (forward and gradient alike), so
 *                  the contraction can skip the empty part of each slice
 *  soft_width      logistic width in length units (> 0 when soft)
 *  scan_fp64       1 forces the transmission scan into FP64 (always on in
 *                  SCATMAN_FP64; switched on automatically when
 *                  k0 * voxel * nz * max(delta, beta) > 5)
 *  detector        SCATMAN_DETECTOR_FLAT (0) or SCATMAN_DETECTOR_UNIFORM_Q; the
 *                  uniform-q detector runs the separable transverse sum (q_x
 *                  depends on the pixel column only, q_y on the row only),
 *                  nz <= 128: on the CUDA cores in SCATMAN_FP32 / SCATMAN_FP64,
 *                  on the tensor cores in the four TC modes (y-sum with FP16
 *                  operands, x/z sum in the mode's type; nx <= 128 and, with
 *                  split phases, ny <= 128)
 */
typedef struct {
    int nx, ny, nz;
    double voxel;
    double wavelength;
    double theta_max_deg;
    int det_nx, det_ny;
    const double *q_list;
    long long n_q;
    int precision;
    int soft;
    double soft_width;
    int scan_fp64;
    int detector;
} scatman_config;

/*
 * Shape (Sec. 5.1-5.2, Listings 1-2; orientation as in Fig. 6).
 *  kind            SCATMAN_SPHERE (r), SCATMAN_ELLIPSOID (a, b, c; c lies on
 *                  the main axis), SCATMAN_SPHHARM (R0, lmax, alm)
 *  alm             (lmax+1)^2 real coefficients indexed l*l+l+m; alm[0] is
 *                  ignored; radius r(theta,phi) = R0 (1 + sum_{l>=1} a_lm Y_lm)
 *                  with real orthonormal harmonics (Eq. 10-11), clipped to
 *                  [0.1 R0, grid half-width - voxel]
 *  delta, beta     n = 1 - delta + i beta (Eq. 7)
 *  latitude, longitude, rotation   degrees: the main axis points to
 *                  (lat, lon) with +90 deg towards the source (-z); the body
 *                  then spins by `rotation` about that axis
 *  cx, cy, cz      centre offset from the grid centre, length units
 *  radial_map      SCATMAN_RADIALMAP (Sec. 5.2 "Shape (2/3)"): radii in length
 *                  units, row-major [map_ntheta][map_nphi], at latitudes
 *                  -pi/2 + i pi/map_ntheta and longitudes 2 pi k/map_nphi of
 *                  the body frame (latitude +pi/2 on the main axis, longitude
 *                  from body x towards body y); linear interpolation in both
 *                  angles, periodic in both; a voxel is inside when its
 *                  distance from the centre is at most the interpolated radius
 *                  (soft occupancy: the logistic of the difference)
 *  volume_map      SCATMAN_VOLUMEMAP (Sec. 5.2 "Shape (3/3)"): occupancy of
 *                  map_nx x map_ny x map_nz cells, row-major [i][j][k] along
 *                  body x, y, z, non-zero = inside; cells of edge map_dx
 *                  (length units) centred on the shape centre, turning with the
 *                  body; cell (i,j,k) covers [(i - map_nx/2) map_dx,
 *                  (i + 1 - map_nx/2) map_dx) along x and likewise; occupancy
 *                  stays binary in soft mode
 *  map_delta, map_beta  optional per-cell index of a volume map (same layout;
 *                  NULL takes the shape's delta or beta): a voxel-resolved
 *                  n = 1 - delta + i beta enters both the slice strength
 *                  (n^2 - 1) chi and the transmission scan of Eq. 8
 * Map arrays are borrowed for the scatman_voxelise call only (copied to the
 * device).  Map shapes have no gradient: scatman_backward returns
 * ERR_UNSUPPORTED for them and scatman_param_count returns 0.
 */
typedef struct {
    int kind;
    double r, a, b, c;
    double R0;
    int lmax;
    const double *alm;
    double delta, beta;
    double latitude, longitude, rotation;
    double cx, cy, cz;
    const double *radial_map;
    int map_ntheta, map_nphi;
    const unsigned char *volume_map;
    int map_nx, map_ny, map_nz;
    double map_dx;
    const double *map_delta, *map_beta;
} scatman_shape;

typedef struct scatman_handle scatman_handle;

/*
 * Creates a handle on the current CUDA device.  cuda_stream is a
 * cudaStream_t (NULL: the library creates and owns a stream).  Allocates the
 * occupancy, slice, field and reduction buffers for the given sizes and
 * computes every pixel's q (Eq. 3).  The handle owns its device buffers;
 * free them with scatman_destroy.
 * Errors: ERR_ARG (bad sizes or angles), ERR_UNSUPPORTED (device is not
 * sm_103), ERR_OOM, ERR_CUDA.  On error *out is NULL.
 */
SCATMAN_API int scatman_create(const scatman_config *cfg, void *cuda_stream, scatman_handle **out);

/*
 * Block 5 + Block 9 (Sec. 3.2), Eq. 8: renders the shape's occupancy chi on
 * the grid and runs the exclusive transmission scan along z, storing
 * s_j = chi_j T_j in the layout the selected contraction reads.  The shape
 * (including a copy of alm) is kept for scatman_backward.  Asynchronous.
 * Errors: ERR_ARG (unknown kind, non-positive size, lmax > SCATMAN_MAX_LMAX,
 * NULL alm), ERR_CUDA.
 */
SCATMAN_API int scatman_voxelise(scatman_handle *h, const scatman_shape *shape);

/*
 * Eq. 9 and Block 11: A(q) for every pixel and I = |A|^2.
 *  I_dev  caller-owned device array of n_pix elements: double in
 *         SCATMAN_FP64, float otherwise
 *  A_dev  optional caller-owned device array of n_pix complex values
 *         (interleaved re, im; double in SCATMAN_FP64, float otherwise);
 *         NULL skips it.  The handle keeps its own copy of A for backward.
 * Asynchronous.  Errors: ERR_STATE (no voxelise yet), ERR_ARG, ERR_CUDA.
 */
SCATMAN_API int scatman_forward(scatman_handle *h, void *I_dev, void *A_dev);

/*
 * End-to-end acquisition with host memory (the paper's detector.acquire,
 * Listing 1): voxelise, forward, then copy I to the caller's host array
 * (n_pix elements, same element type as scatman_forward).  Synchronises
 * the stream.  Errors as voxelise/forward, plus ERR_TIMEOUT.
 */
SCATMAN_API int scatman_acquire(scatman_handle *h, const scatman_shape *shape, void *I_host);

/*
 * scatman_acquire over n shapes, pipelined: pattern i is computed while
 * pattern i - 1 is copied to the host (a second intensity buffer and a copy
 * stream, created on the first call and owned by the handle).  I_host[i]
 * receives pattern i's intensity (n_pix elements; page-locked host memory
 * lets the copies overlap the computation).  Returns after every copy has
 * landed, with the same results as n calls of scatman_acquire.  n = 0 is a
 * no-op.  Errors as scatman_acquire; on an error the later patterns are not
 * computed and their arrays are left untouched.
 */
SCATMAN_API int scatman_acquire_batch(scatman_handle *h, const scatman_shape *shapes, int n, void *const *I_host);

/*
 * The Ideal detector (Sec. 5.2, Listing 2: "photon statistics"): turns an
 * intensity I (device array from scatman_forward on this handle, n_pix
 * elements of its element type) into the expected number of scattered photons
 * per pixel and a Poisson count.  The paper leaves the normalisation to a
 * supplement; this library reads it as
 *   lambda_p = photon_density * (k0^2 voxel^3 / (4 pi))^2 * I_p * dOmega_p,
 * photon_density in photons per squared length unit (the wavelength's),
 * dOmega_p the pixel's solid angle (flat pixel of area a at distance 1:
 * a / r^3 with r^2 = 1 + X^2 + Y^2; uniform-q pixel: d2q / (k0^2 cos theta),
 * 0 without a scattering direction).  Counts are Poisson(lambda_p) draws
 * from the counter-based generator Philox-4x32-10 keyed by `seed` and counted
 * by (pixel, draw): the same seed gives the same counts on any launch.
 *  lambda_dev  optional device array of n_pix doubles (NULL skips it)
 *  counts_dev  optional device array of n_pix 64-bit counts (NULL skips it)
 * Asynchronous.  Errors: ERR_ARG (NULL I, both outputs NULL, negative or
 * non-finite density, a handle built with q_list), ERR_CUDA.
 */
SCATMAN_API int scatman_photon_counts(scatman_handle *h, double photon_density, unsigned long long seed,
                                      const void *I_dev, double *lambda_dev, long long *counts_dev);

/*
 * Gradient of a real loss L(I) with respect to the shape parameters, given
 * dL/dI on every pixel (device array, n_pix elements, same element type as
 * I), for the shape of the last scatman_voxelise and the field of the last
 * scatman_forward (soft occupancy is required for the geometric terms).
 * Writes scatman_param_count() doubles to the host array dLdparams in the
 * order: sphere [r, delta, beta]; ellipsoid [a, b, c, delta, beta];
 * harmonics [a_lm for l >= 1 in index order, R0, delta, beta].
 * Recomputes occupancy and transmission instead of storing them.
 * Synchronises the stream.  Errors: ERR_STATE (no forward yet), ERR_CUDA,
 * ERR_TIMEOUT.
 */
SCATMAN_API int scatman_backward(scatman_handle *h, const void *dLdI_dev, double *dLdparams);

/*
 * Failure-path hooks (no counterpart in the paper; they let tests reach the
 * error paths without faulting a GPU).
 *
 * scatman_set_wait_limit: every wait of the handle's tensor-core kernels on
 * another warp's work gives up after `seconds` (default and maximum 2 s;
 * seconds <= 0 restores the default) instead of 2 s.  A kernel that gives up
 * sets its error bit, waits (with the full limit) for its own TMA copies and
 * MMAs in flight, frees its tensor memory and returns; scatman_sync then
 * reports ERR_TIMEOUT and the results of that call are invalid.  The handle
 * stays usable.  Synchronises the stream.  Errors: ERR_ARG (NaN), ERR_CUDA.
 *
 * scatman_debug_stall: with on != 0, the MMA warps of the handle's
 * tensor-core contraction and adjoint kernels first wait on a barrier that no
 * thread arrives at, so that wait runs out after the wait limit and the
 * kernel takes its abort path exactly as after a real stall (the other warps
 * stop at their next wait, in-flight TMA copies and MMAs are drained, tensor
 * memory is freed); the call then reports ERR_TIMEOUT.  on = 0 restores
 * normal operation.  Synchronises the stream.  Errors: ERR_ARG, ERR_CUDA.
 *
 * scatman_debug_fail_allocation: process-wide; with after >= 0 the device
 * allocation that follows `after` more successful ones (in any handle or
 * server of the process) fails once as if the device were out of memory
 * (the call that made it returns ERR_OOM and releases what it had
 * allocated); after < 0 disarms it.
 */
SCATMAN_API int scatman_set_wait_limit(scatman_handle *h, double seconds);
SCATMAN_API int scatman_debug_stall(scatman_handle *h, int on);
SCATMAN_API void scatman_debug_fail_allocation(long long after);

/* Number of gradient entries for the current shape (0 before voxelise). */
SCATMAN_API int scatman_param_count(const scatman_handle *h);

/* Number of detector pixels (or q points) of the handle. */
SCATMAN_API long long scatman_n_pix(const scatman_handle *h);

/* Bytes per element of I (8 in SCATMAN_FP64, 4 otherwise). */
SCATMAN_API int scatman_elem_size(const scatman_handle *h);

/* Device bytes held by the handle (buffers only). */
SCATMAN_API long long scatman_device_bytes(const scatman_handle *h);

/*
 * Waits for the handle's stream and checks the kernels' error word.
 * Returns ERR_TIMEOUT if a kernel gave up a bounded wait, ERR_CUDA on a
 * CUDA error, OK otherwise.
 */
SCATMAN_API int scatman_sync(scatman_handle *h);

/* Inspection (tests): copy chi ([z][x][y], double, n_vox), the stored slices
 * s = chi*T ([z][x][y], interleaved complex double, without the n^2-1
 * factor) or the pixels' q ([pixel][3] double) to host memory.  Synchronise. */
SCATMAN_API int scatman_get_occupancy(scatman_handle *h, double *chi_host);
SCATMAN_API int scatman_get_slices(scatman_handle *h, double *s_host);
SCATMAN_API int scatman_get_q(scatman_handle *h, double *q_host);

/*
 * Real floating-point operations of one contraction launch for the current
 * shape: *issued counts what the tensor-core kernel executes (it skips the
 * parts of each slice outside the occupied box, and counts both products of
 * a split-phase mode); *dense is 8 flop per (pixel, voxel) pair times the
 * number of products.  CUDA-core modes report the dense count for both.
 * Synchronises.  Errors: ERR_STATE before voxelise.
 */
SCATMAN_API int scatman_contraction_flops(scatman_handle *h, double *issued, double *dense);

/* Text of the last error on this handle ("" if none), owned by the handle.
 * With h == NULL: the reason the calling thread's last scatman_create failed. */
SCATMAN_API const char *scatman_last_error(const scatman_handle *h);

/* Releases every buffer and the owned stream.  Accepts NULL. */
SCATMAN_API void scatman_destroy(scatman_handle *h);


/* ------------------------------------------------------------------------
 * Serving: many concurrent shape fits (the paper's forward-fitting use,
 * Sec. 6) multiplexed onto one GPU.  A native scheduler keeps a FIFO of
 * requests and `slots` worker streams.  A request is admitted as soon as a
 * slot is free and the device bytes it needs fit under hbm_budget_bytes
 * (continuous admission: work of admitted requests overlaps on the device).
 * Each slot keeps the handle of its last geometry, so repeated requests of a
 * fit reuse their device buffers.  Every request runs the same kernels with
 * the same fixed reduction orders whatever else is in flight, so its result
 * does not depend on the mix.
 * ---------------------------------------------------------------------- */
typedef struct scatman_server scatman_server;

typedef struct {
    long long hbm_budget_bytes;   /* device bytes the server may hold (> 0) */
    int slots;                    /* requests in flight at once, 1..64 */
    int precision;                /* scatman_precision of every request */
    double soft_width;            /* requests use soft occupancy of this width (> 0) */
} scatman_server_config;

/* One fit request.  Input arrays are copied during scatman_server_submit;
 * output arrays must stay valid until scatman_server_wait returns for it. */
typedef struct {
    scatman_config geometry;      /* grid and detector; precision/soft fields ignored */
    scatman_shape shape;
    const float *target;          /* host, n_pix floats; loss = sum (I - target)^2 */
    int want_gradient;            /* 1: also dloss/dparams (scatman_backward order) */
    float *I_out;                 /* host, n_pix floats, or NULL (intensity as float in every mode) */
    double *grad_out;             /* host, param count doubles (with want_gradient) */
    double *loss_out;             /* host, 1 double, or NULL */
} scatman_request;

typedef struct {
    long long submitted, completed, failed;
    long long bytes_reserved, bytes_reserved_peak;
    int inflight, inflight_peak;
    long long cancelled;
} scatman_server_stats;

/* Creates the server on the current device.  Errors: ERR_ARG, ERR_CUDA,
 * ERR_UNSUPPORTED. */
SCATMAN_API int scatman_server_create(const scatman_server_config *cfg, scatman_server **out);

/* Queues a request; *ticket identifies it.  Returns ERR_ADMISSION if the
 * request alone needs more than the budget, ERR_ARG for invalid geometry or
 * shape, including map shapes (fit requests take sphere, ellipsoid and
 * harmonics shapes); the request is not queued then. */
SCATMAN_API int scatman_server_submit(scatman_server *srv, const scatman_request *req, long long *ticket);

/* Waits up to timeout_s seconds (< 0: forever) for a request.  Returns
 * ERR_TIMEOUT if it is still running, otherwise OK with *status set to the
 * request's own status and *latency_s to submit-to-completion time. */
SCATMAN_API int scatman_server_wait(scatman_server *srv, long long ticket, double timeout_s, int *status,
                                    double *latency_s);

/* Cancels a request that is still queued: it will not run, and
 * scatman_server_wait reports it with status ERR_CANCELLED.  Returns OK, or
 * ERR_STATE once the request has been admitted (it then runs to completion),
 * ERR_ARG for an unknown ticket. */
SCATMAN_API int scatman_server_cancel(scatman_server *srv, long long ticket);

SCATMAN_API int scatman_server_stats_get(scatman_server *srv, scatman_server_stats *out);

/* Drains queued and running requests, then frees every handle and thread. */
SCATMAN_API void scatman_server_destroy(scatman_server *srv);

/* Device bytes a handle of this configuration allocates (forward and
 * backward buffers), as the server's admission uses it.  -1 on bad input. */
SCATMAN_API long long scatman_footprint_bytes(const scatman_config *cfg);

/*
 * Forward pass that allocates no device memory (the paper has no counterpart;
 * this is a service to callers that cannot call cudaMalloc -- for example a
 * host application that has already reserved nearly all device memory for its
 * own pool, or a latency-critical loop that must not take the device-wide
 * synchronisation an allocation can cause).
 *
 * Runs voxelise + transmission scan + forward (as scatman_voxelise followed by
 * scatman_forward on a SCATMAN_FP32 handle) for one shape, on cuda_stream
 * (a cudaStream_t; NULL is the legacy default stream), asynchronously.
 *  cfg     as for scatman_create; precision must be SCATMAN_FP32
 *  I_dev   caller-owned device array of n_pix floats (output)
 *  A_dev   optional caller-owned device array of n_pix complex floats; NULL skips it
 * Working memory (q, occupancy, slices, partial fields) lives in one fixed
 * 8 MiB array inside the library, which every GPU that loads the library
 * keeps until the process exits.  Problems that need more return ERR_ARG
 * with the required size.  The array is shared by every call and keeps the
 * previous call's contents; each call overwrites everything it reads, so
 * nothing has to start at zero, but calls whose GPU work overlaps (for
 * example on two streams) race on it and give wrong results.
 * The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  Errors: ERR_ARG, ERR_UNSUPPORTED, ERR_CUDA;
 * the message is available from scatman_last_error(NULL).
 */
SCATMAN_API int scatman_forward_noalloc(const scatman_config *cfg, const scatman_shape *shape, void *cuda_stream,
                                        float *I_dev, float *A_dev);

/* Library version string. */
SCATMAN_API const char *scatman_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SCATMAN_H */
