// api.cu -- the C ABI declared in include/scatman.h: handle lifecycle,
// argument checks, buffer ownership and dispatch to the kernels.
#include <cmath>
#include <cstring>
#include <atomic>
#include <new>

#include "internal.cuh"

namespace scm {

int set_error(scatman_handle *h, int code, const std::string &msg) {
    if (h) h->last_error = msg;
    return code;
}

int check_cuda(scatman_handle *h, cudaError_t e, const char *what) {
    if (e == cudaSuccess) return SCATMAN_OK;
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return set_error(h, SCATMAN_ERR_OOM, m);
    return set_error(h, SCATMAN_ERR_CUDA, m);
}

static bool is_tc(int precision) { return precision >= SCATMAN_TC_F16_SPLIT && precision <= SCATMAN_TC_BF16; }

// cos/sin of an angle in degrees, exact at multiples of 90 degrees.
static void cos_sin_deg(double deg, double *c, double *s) {
    double q = deg / 90.0;
    if (q == std::floor(q)) {
        long k = (((long)q) % 4 + 4) % 4;
        const double cs[4] = {1, 0, -1, 0}, sn[4] = {0, 1, 0, -1};
        *c = cs[k];
        *s = sn[k];
        return;
    }
    double r = deg * kPi / 180.0;
    *c = std::cos(r);
    *s = std::sin(r);
}

// Body->lab rotation for the orientation of Fig. 6: spin about the body z
// axis by `rotation`, tilt body z by 90+latitude about y, turn by longitude
// about the lab z axis.  Written as the product of the three matrices.
static void orientation_matrix(double lat, double lon, double rot, double R[9]) {
    double c1, s1, c2, s2, c3, s3;
    cos_sin_deg(lon, &c1, &s1);
    cos_sin_deg(90.0 + lat, &c2, &s2);
    cos_sin_deg(rot, &c3, &s3);
    // Rz(lon) * Ry(90+lat)
    double M[9] = {c1 * c2, -s1, c1 * s2, s1 * c2, c1, s1 * s2, -s2, 0.0, c2};
    // (.) * Rz(rot)
    for (int i = 0; i < 3; ++i) {
        double a = M[3 * i + 0], b = M[3 * i + 1], c = M[3 * i + 2];
        R[3 * i + 0] = a * c3 + b * s3;
        R[3 * i + 1] = -a * s3 + b * c3;
        R[3 * i + 2] = c;
    }
}

static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

void finish_shape_params(ShapeParams *sp) {
    for (int k = 0; k < 9; ++k) sp->Rf[k] = (float)sp->R[k];
    sp->cxf = (float)sp->cx;
    sp->cyf = (float)sp->cy;
    sp->czf = (float)sp->cz;
    sp->r2f = (float)(sp->r * sp->r);
    sp->R0f = (float)sp->R0;
    sp->rminf = (float)sp->rmin;
    sp->rmaxf = (float)sp->rmax;
    sp->inv_af = sp->a > 0 ? (float)(1.0 / sp->a) : 0.f;
    sp->inv_bf = sp->b > 0 ? (float)(1.0 / sp->b) : 0.f;
    sp->inv_cf = sp->c > 0 ? (float)(1.0 / sp->c) : 0.f;
    const int nlm = (SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 1);
    for (int k = 0; k < nlm; ++k) sp->almf[k] = (float)sp->alm[k];
    for (int m = 0; m <= SCATMAN_MAX_LMAX; ++m) {
        sp->sh_d[m] = m > 0 ? -std::sqrt((2.0 * m + 1.0) / (2.0 * m)) : 1.0;
        sp->sh_e[m] = std::sqrt(2.0 * m + 3.0);
        sp->sh_df[m] = (float)sp->sh_d[m];
        sp->sh_ef[m] = (float)sp->sh_e[m];
        for (int l = m; l <= SCATMAN_MAX_LMAX; ++l) {
            const int i = l * (l + 1) / 2 + m;
            double a = 0.0, b = 0.0;
            if (l >= m + 2) {
                a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
                b = std::sqrt(((double)(l - 1) * (l - 1) - (double)m * m) / (4.0 * (l - 1) * (l - 1) - 1.0));
            }
            sp->sh_a[i] = a;
            sp->sh_b[i] = b;
            sp->sh_af[i] = (float)a;
            sp->sh_bf[i] = (float)b;
        }
    }
}

}  // namespace scm

namespace scm {

// Allocation-failure injection for tests: when armed with n >= 0, the
// allocation after n more successful ones fails (once), as if the device were
// out of memory.  Process-wide; -1 disarms it.
static std::atomic<long long> g_fail_countdown{-1};

cudaError_t device_malloc(void **p, size_t bytes) {
    long long c = g_fail_countdown.load();
    while (c >= 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) {
            if (c == 0) {
                *p = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(p, bytes);
}

}  // namespace scm

using namespace scm;

extern "C" {

const char *scatman_version(void) { return "scatman-gb300 0.1 (sm_103a)"; }

static thread_local std::string g_create_error;

const char *scatman_last_error(const scatman_handle *h) { return h ? h->last_error.c_str() : g_create_error.c_str(); }

long long scatman_n_pix(const scatman_handle *h) { return h ? h->n_pix : 0; }

int scatman_elem_size(const scatman_handle *h) { return h && h->precision == SCATMAN_FP64 ? 8 : 4; }

long long scatman_device_bytes(const scatman_handle *h) { return h ? h->device_bytes : 0; }

static bool is_map_kind(int kind) { return kind == SCATMAN_RADIALMAP || kind == SCATMAN_VOLUMEMAP; }

int scatman_param_count(const scatman_handle *h) {
    if (!h || !h->have_shape) return 0;
    if (is_map_kind(h->sp.kind)) return 0;      // map shapes have no gradient
    return grad_param_count(h->sp) + 2;
}

static int alloc_dev(scatman_handle *h, void **p, size_t bytes, const char *what) {
    if (bytes == 0) bytes = 16;
    cudaError_t e = scm::device_malloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        return check_cuda(h, e, what);
    }
    h->device_bytes += (long long)bytes;
    return SCATMAN_OK;
}

void scatman_destroy(scatman_handle *h) {
    if (!h) return;
    int dev_prev = -1;
    cudaGetDevice(&dev_prev);
    cudaSetDevice(h->device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    cudaFree(h->d_q);
    cudaFree(h->d_bounds);
    cudaFree(h->d_chi);
    cudaFree(h->d_s);
    cudaFree(h->d_A);
    cudaFree(h->d_I);
    if (h->copy_stream) cudaStreamSynchronize(h->copy_stream);
    cudaFree(h->d_I2);
    for (int b = 0; b < 2; ++b) {
        if (h->ev_fwd[b]) cudaEventDestroy(h->ev_fwd[b]);
        if (h->ev_copy[b]) cudaEventDestroy(h->ev_copy[b]);
    }
    if (h->copy_stream) cudaStreamDestroy(h->copy_stream);
    cudaFree(h->d_err);
    cudaFree(h->d_part);
    cudaFree(h->d_S);
    cudaFree(h->d_partial);
    cudaFree(h->d_tail);
    cudaFree(h->d_H);
    cudaFree(h->d_uq_qz);
    cudaFree(h->d_uq_qrow);
    cudaFree(h->d_adj_part);
    cudaFree(h->d_gmax);
    cudaFree(h->d_adj_tab);
    cudaFree(h->d_adj_coef);
    cudaFree(h->d_adj_ord);
    cudaFree(h->d_adj_rtile);
    cudaFree(h->d_rmap);
    cudaFree(h->d_rmapf);
    cudaFree(h->d_vmap);
    cudaFree(h->d_mdelta);
    cudaFree(h->d_mbeta);
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    if (dev_prev >= 0) cudaSetDevice(dev_prev);
    delete h;
}

// Checks shared by scatman_create and scatman_forward_noalloc: grid, lengths,
// occupancy width, and the q set (explicit list or detector).  Sets *n_pix.
static bool check_config(const scatman_config &c, long long *n_pix, std::string *why) {
    if (c.nx < 1 || c.ny < 1 || c.nz < 1 || c.nz > 512 || c.nx > 4096 || c.ny > 4096) {
        *why = "grid sizes must be >= 1, nx and ny <= 4096 and nz <= 512";
        return false;
    }
    if (!(c.voxel > 0) || !(c.wavelength > 0)) {
        *why = "voxel and wavelength must be positive";
        return false;
    }
    if (c.soft && !(c.soft_width > 0)) {
        *why = "soft occupancy needs soft_width > 0";
        return false;
    }
    if (c.q_list) {
        if (c.n_q < 1) {
            *why = "n_q must be >= 1 with q_list";
            return false;
        }
        *n_pix = c.n_q;
    } else {
        if (c.det_nx < 1 || c.det_ny < 1) {
            *why = "detector size must be >= 1";
            return false;
        }
        if (!(c.theta_max_deg > 0 && c.theta_max_deg < 90)) {
            *why = "theta_max_deg must lie in (0, 90)";
            return false;
        }
        *n_pix = (long long)c.det_nx * c.det_ny;
    }
    if (c.detector != SCATMAN_DETECTOR_FLAT && c.detector != SCATMAN_DETECTOR_UNIFORM_Q) {
        *why = "unknown detector";
        return false;
    }
    return true;
}

// Checks of a sphere, ellipsoid or harmonics shape (map shapes add their own).
static bool check_param_shape(const scatman_shape *s, std::string *why) {
    if (s->kind == SCATMAN_SPHERE && !(s->r > 0)) {
        *why = "sphere radius must be > 0";
        return false;
    }
    if (s->kind == SCATMAN_ELLIPSOID && !(s->a > 0 && s->b > 0 && s->c > 0)) {
        *why = "ellipsoid semi-axes must be > 0";
        return false;
    }
    if (s->kind == SCATMAN_SPHHARM) {
        if (!(s->R0 > 0)) {
            *why = "R0 must be > 0";
            return false;
        }
        if (s->lmax < 0 || s->lmax > SCATMAN_MAX_LMAX) {
            *why = "lmax out of range";
            return false;
        }
        if (s->lmax > 0 && !s->alm) {
            *why = "alm is NULL";
            return false;
        }
    }
    if (!std::isfinite(s->delta) || !std::isfinite(s->beta)) {
        *why = "delta and beta must be finite";
        return false;
    }
    return true;
}

int scatman_create(const scatman_config *cfg, void *cuda_stream, scatman_handle **out) {
    if (!out) return SCATMAN_ERR_ARG;
    *out = nullptr;
    if (!cfg) return SCATMAN_ERR_ARG;
    scatman_handle *h = new (std::nothrow) scatman_handle();
    if (!h) return SCATMAN_ERR_OOM;
    h->cfg = *cfg;
    h->from_q_list = cfg->q_list != nullptr;
    h->cfg.q_list = nullptr;
    g_create_error.clear();
    auto fail = [&](int code) {
        g_create_error = h->last_error;   // readable through scatman_last_error(NULL)
        scatman_destroy(h);
        return code;
    };
    const scatman_config &c = *cfg;
    {
        std::string why;
        if (!check_config(c, &h->n_pix, &why)) return fail(set_error(h, SCATMAN_ERR_ARG, why));
    }
    if (c.precision < SCATMAN_FP64 || c.precision > SCATMAN_TC_BF16)
        return fail(set_error(h, SCATMAN_ERR_ARG, "unknown precision"));
    if (c.precision == SCATMAN_FP64 && c.nz > 256)
        return fail(set_error(h, SCATMAN_ERR_ARG, "SCATMAN_FP64 supports nz <= 256"));
    h->uniform_q = c.detector == SCATMAN_DETECTOR_UNIFORM_Q && !cfg->q_list;
    if (h->uniform_q && c.nz > 128)
        return fail(set_error(h, SCATMAN_ERR_ARG, "the uniform-q detector supports nz <= 128"));
    h->precision = c.precision;
    // In the tensor-core modes the uniform-q detector runs both of its sums on
    // the tensor cores: the y sum as the flat contraction kernel in store mode
    // (FP16 slice and phase operands: |s| <= 1 and |phase| <= 1 fit its range),
    // the x/z sum in the mode's 16-bit type.
    h->uniform_tc = h->uniform_q && is_tc(c.precision);
    h->tensor_core = is_tc(c.precision);
    if (h->uniform_tc) uq_tc_geometry(c.nx, c.nz, &h->uq_Kx, &h->uq_Jp, &h->uq_Rg);
    h->split = (c.precision == SCATMAN_TC_F16_SPLIT || c.precision == SCATMAN_TC_BF16_SPLIT);
    h->bf16 = (c.precision == SCATMAN_TC_BF16_SPLIT || c.precision == SCATMAN_TC_BF16);
    h->s_bf16 = h->bf16 && !h->uniform_tc;
    h->k0 = 2.0 * kPi / c.wavelength;

    // device
    if (cudaGetDevice(&h->device) != cudaSuccess)
        return fail(set_error(h, SCATMAN_ERR_UNSUPPORTED, "no CUDA device"));
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, h->device) != cudaSuccess)
        return fail(set_error(h, SCATMAN_ERR_UNSUPPORTED, "cannot query the CUDA device"));
    if (!(prop.major == 10 && prop.minor == 3))
        return fail(set_error(h, SCATMAN_ERR_UNSUPPORTED,
                              "this library is built for sm_103a (compute capability 10.3) only"));
    h->sm_count = prop.multiProcessorCount;

    if (h->tensor_core) {
        h->Nxp = (int)round_up(c.nx, 16);
        h->Nyp = (int)round_up(c.ny, 16);
        h->Kp = h->Nyp;                       // K extent of one slice-operand row
        if (h->Nxp > (h->uniform_tc ? 128 : 256))
            return fail(set_error(h, SCATMAN_ERR_ARG, h->uniform_tc ? "the uniform-q detector's tensor-core modes support nx <= 128"
                                                                   : "tensor-core modes support nx <= 256"));
        if (!tc_grid_ok(h->Nxp, h->Nyp, h->split))
            return fail(set_error(h, SCATMAN_ERR_ARG, "ny too large for the tensor-core phase operand"));
        h->b_rows = (size_t)c.nz * 3 * h->Nxp;   // planes -Im, Re, Im of every slice
    }

    if (cuda_stream) {
        h->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
            return fail(set_error(h, SCATMAN_ERR_CUDA, "cannot create a stream"));
        h->own_stream = true;
    }

    const size_t nvox = (size_t)c.nx * c.ny * c.nz;
    const size_t npix = (size_t)h->n_pix;
    const bool f64 = (h->precision == SCATMAN_FP64);
    int rc;
    if ((rc = alloc_dev(h, (void **)&h->d_q, npix * 3 * sizeof(double), "q buffer"))) return fail(rc);
    if ((rc = alloc_dev(h, (void **)&h->d_chi, nvox * sizeof(float), "occupancy buffer"))) return fail(rc);
    // per-slice occupied boxes (every mode skips the empty parts of each
    // slice), then the tensor-core kernel's occupied-slice list
    if ((rc = alloc_dev(h, (void **)&h->d_bounds, slice_geom_ints(c.nz) * sizeof(int), "slice geometry")))
        return fail(rc);
    if (h->tensor_core) {
        h->s_bytes = h->b_rows * (size_t)h->Kp * 2;
    } else {
        h->s_bytes = nvox * (f64 ? sizeof(double2) : sizeof(float2));
    }
    if ((rc = alloc_dev(h, &h->d_s, h->s_bytes, "slice buffer"))) return fail(rc);
    const size_t cx = f64 ? sizeof(double2) : sizeof(float2);
    if ((rc = alloc_dev(h, &h->d_A, npix * cx, "field buffer"))) return fail(rc);
    if ((rc = alloc_dev(h, &h->d_I, npix * (f64 ? 8 : 4), "intensity buffer"))) return fail(rc);
    if ((rc = alloc_dev(h, (void **)&h->d_err, kStatusBytes, "status block"))) return fail(rc);
    if (h->uniform_q && (rc = alloc_dev(h, (void **)&h->d_uq_qz, npix * sizeof(float2), "q_z table")))
        return fail(rc);
    if (h->uniform_tc &&
        (rc = alloc_dev(h, (void **)&h->d_uq_qrow, (size_t)c.det_ny * 3 * sizeof(double), "detector row q")))
        return fail(rc);
    if (h->uniform_tc) {
        const size_t hb = uq_tc_h_bytes(c.nx, c.nz, c.det_ny);
        // (zeroed by each forward before the y-sum writes its occupied part)
        if ((rc = alloc_dev(h, &h->d_H, hb, "y-contracted slices"))) return fail(rc);
    } else if (h->uniform_q) {
        if ((rc = alloc_dev(h, &h->d_H, (size_t)c.det_ny * nvox / c.ny * cx, "y-contracted slices"))) return fail(rc);
    } else if (h->tensor_core) {
        const size_t tb = tc_tail_part_bytes(h->n_pix, h->sm_count);
        if (tb && (rc = alloc_dev(h, (void **)&h->d_tail, tb, "tail partial fields"))) return fail(rc);
    } else {
        h->splits = simt_splits(h->n_pix, c.nx, c.nz, h->sm_count);
        if ((rc = alloc_dev(h, &h->d_partial, (size_t)h->splits * npix * cx, "partial fields"))) return fail(rc);
    }
    if ((rc = check_cuda(h, cudaMemsetAsync(h->d_err, 0, kStatusBytes, h->stream), "memset"))) return fail(rc);
    if ((rc = check_cuda(h, cudaMemsetAsync(h->d_s, 0, h->s_bytes, h->stream), "memset"))) return fail(rc);

    if (cfg->q_list) {
        rc = check_cuda(h, cudaMemcpyAsync(h->d_q, cfg->q_list, npix * 3 * sizeof(double), cudaMemcpyHostToDevice,
                                           h->stream),
                        "q upload");
        if (rc) return fail(rc);
        if ((rc = check_cuda(h, cudaStreamSynchronize(h->stream), "q upload"))) return fail(rc);
    } else {
        rc = check_cuda(h, h->uniform_q ? launch_detector_q_uniform(c.det_nx, c.det_ny, c.theta_max_deg, h->k0,
                                                                    h->d_q, h->stream)
                                         : launch_detector_q(c.det_nx, c.det_ny, c.theta_max_deg, h->k0, h->d_q,
                                                             h->stream),
                        "detector q");
        if (rc) return fail(rc);
    }
    if (h->tensor_core) {
        std::string why;
        if (!encode_tmap_B(&h->tmap_B, h->d_s, h->Kp, h->Nxp, c.nz, h->s_bf16, &why))
            return fail(set_error(h, SCATMAN_ERR_CUDA, why));
        h->have_tmap = true;
    }
    if (h->uniform_q &&
        (rc = check_cuda(h, launch_uq_qz_table(h->d_q, h->n_pix, h->k0, h->d_uq_qz, h->stream), "q_z table")))
        return fail(rc);
    if (h->uniform_tc &&
        (rc = check_cuda(h, cudaMemcpy2DAsync(h->d_uq_qrow, 3 * sizeof(double), h->d_q,
                                              (size_t)c.det_nx * 3 * sizeof(double), 3 * sizeof(double), c.det_ny,
                                              cudaMemcpyDeviceToDevice, h->stream),
                         "detector row q")))
        return fail(rc);
    if (h->uniform_tc) {
        std::string why;
        if (!encode_tmap_uq(&h->tmap_H, h->d_H, c.nx, c.nz, c.det_ny, h->bf16, &why))
            return fail(set_error(h, SCATMAN_ERR_CUDA, why));
    }
    *out = h;
    return SCATMAN_OK;
}

// Radius band of a harmonics or radii-map shape (and, with soft occupancy in
// the FP32 modes, of a sphere or ellipsoid): every direction's surface radius
// lies in [band_lo, band_hi], so voxels clearly inside or outside skip the
// radius evaluation.  Harmonics: per degree l,
// |sum_m a_lm Y_lm| <= |a_l| sqrt((2l+1)/(4 pi)) (Cauchy-Schwarz with the
// addition theorem sum_m Y_lm^2 = (2l+1)/(4 pi)), then the clip; radii map:
// the interpolation stays within the samples' range; sphere: r; ellipsoid:
// between its smallest and largest semi-axis.  Soft occupancy widens the band
// by the logistic's reach on both sides.
static void set_radius_band(const scatman_shape *s, ShapeParams *sp, bool fp64) {
    sp->band_lo = sp->band_hi = 0.f;
    if (sp->soft && fp64) return;   // FP64 soft occupancy: the exact logistic at every voxel
    double lo = 0.0, hi = 0.0;
    if (s->kind == SCATMAN_SPHHARM) {
        double b = 0.0;
        for (int l = 1; l <= s->lmax; ++l) {
            double n2 = 0.0;
            for (int m = -l; m <= l; ++m) n2 += sp->alm[l * l + l + m] * sp->alm[l * l + l + m];
            b += std::sqrt(n2) * std::sqrt((2.0 * l + 1.0) / (4.0 * kPi));
        }
        lo = std::fmin(std::fmax(s->R0 * (1.0 - b), sp->rmin), sp->rmax);
        hi = std::fmin(std::fmax(s->R0 * (1.0 + b), sp->rmin), sp->rmax);
    } else if (s->kind == SCATMAN_RADIALMAP) {
        lo = hi = s->radial_map[0];
        for (long long k = 1; k < (long long)s->map_ntheta * s->map_nphi; ++k) {
            lo = std::fmin(lo, s->radial_map[k]);
            hi = std::fmax(hi, s->radial_map[k]);
        }
    } else if (sp->soft && s->kind == SCATMAN_SPHERE) {
        lo = hi = s->r;                 // binary spheres and ellipsoids decide cheaply without it
    } else if (sp->soft && s->kind == SCATMAN_ELLIPSOID) {
        lo = std::fmin(s->a, std::fmin(s->b, s->c));   // the radius along any direction
        hi = std::fmax(s->a, std::fmax(s->b, s->c));
    } else {
        return;
    }
    // widen by a relative 1e-6 so the FP64 rounding of the radius stays inside
    double blo = lo * (1.0 - 1e-6) - 1e-9, bhi = hi * (1.0 + 1e-6) + 1e-9;
    if (sp->soft) {
        // FP32 soft occupancy: chi is exactly 1.0f where t = (r_s - |p|) / w > kSoftOneT
        // and zero (the cut) where t < -kSoftCutT; 1e-3 w covers the FP32 rounding of t
        const double w = 1.0 / sp->inv_w;
        blo -= (double)kSoftOneT * w;
        bhi += ((double)kSoftCutT + 1e-3) * w;
    }
    sp->band_lo = (float)blo;
    sp->band_hi = (float)bhi;
    if (!(sp->band_hi > 0.f)) sp->band_lo = sp->band_hi = 0.f;
}

// Copies a map shape's arrays to the device (grown buffers owned by the handle)
// and fills the map fields of the shape parameters.
static int upload_maps(scatman_handle *h, const scatman_shape *s, ShapeParams *sp) {
    int rc;
    sp->varn = 0;
    sp->nscale = 1.0;
    h->map_index_max = 0.0;
    if (s->kind == SCATMAN_RADIALMAP) {
        const int nt = s->map_ntheta, np = s->map_nphi;
        const size_t n = (size_t)nt * np;
        if (h->rmap_cap < n) {
            cudaFree(h->d_rmap);
            cudaFree(h->d_rmapf);
            h->d_rmap = nullptr;
            h->d_rmapf = nullptr;
            h->rmap_cap = 0;
            if ((rc = alloc_dev(h, (void **)&h->d_rmap, n * sizeof(double), "radial map"))) return rc;
            if ((rc = alloc_dev(h, (void **)&h->d_rmapf, n * sizeof(float), "radial map"))) return rc;
            h->rmap_cap = n;
        }
        std::vector<float> f(n);
        double slope_t = 0.0, slope_p = 0.0;
        for (int i = 0; i < nt; ++i)
            for (int k = 0; k < np; ++k) {
                const double r = s->radial_map[(size_t)i * np + k];
                f[(size_t)i * np + k] = (float)r;
                slope_t = std::fmax(slope_t, std::fabs(s->radial_map[(size_t)((i + 1) % nt) * np + k] - r));
                slope_p = std::fmax(slope_p, std::fabs(s->radial_map[(size_t)i * np + (k + 1) % np] - r));
            }
        if ((rc = check_cuda(h, cudaMemcpyAsync(h->d_rmap, s->radial_map, n * sizeof(double), cudaMemcpyHostToDevice,
                                                 h->stream), "radial map upload")))
            return rc;
        if ((rc = check_cuda(h, cudaMemcpyAsync(h->d_rmapf, f.data(), n * sizeof(float), cudaMemcpyHostToDevice,
                                                 h->stream), "radial map upload")))
            return rc;
        // a copy from pageable host memory has left the staging vector when the call returns
        sp->rmap = h->d_rmap;
        sp->rmapf = h->d_rmapf;
        sp->ntheta = nt;
        sp->nphi = np;
        sp->rm_tscale = (double)nt / kPi;
        sp->rm_pscale = (double)np / (2.0 * kPi);
        sp->rm_tscalef = (float)sp->rm_tscale;
        sp->rm_pscalef = (float)sp->rm_pscale;
        sp->rm_slope = (float)std::fmax(slope_t * sp->rm_tscale, slope_p * sp->rm_pscale);
    }
    if (s->kind == SCATMAN_VOLUMEMAP) {
        const size_t n = (size_t)s->map_nx * s->map_ny * s->map_nz;
        if (h->vmap_cap < n) {
            cudaFree(h->d_vmap);
            h->d_vmap = nullptr;
            h->vmap_cap = 0;
            if ((rc = alloc_dev(h, (void **)&h->d_vmap, n, "volume map"))) return rc;
            h->vmap_cap = n;
        }
        if ((rc = check_cuda(h, cudaMemcpyAsync(h->d_vmap, s->volume_map, n, cudaMemcpyHostToDevice, h->stream),
                             "volume map upload")))
            return rc;
        sp->vmap = h->d_vmap;
        sp->mx = s->map_nx;
        sp->my = s->map_ny;
        sp->mz = s->map_nz;
        sp->mdx = s->map_dx;
        sp->mdxf = (float)s->map_dx;
        if (s->map_delta || s->map_beta) {
            if (h->mindex_cap < n) {
                cudaFree(h->d_mdelta);
                cudaFree(h->d_mbeta);
                h->d_mdelta = h->d_mbeta = nullptr;
                h->mindex_cap = 0;
                if ((rc = alloc_dev(h, (void **)&h->d_mdelta, n * sizeof(double), "map index"))) return rc;
                if ((rc = alloc_dev(h, (void **)&h->d_mbeta, n * sizeof(double), "map index"))) return rc;
                h->mindex_cap = n;
            }
            // per-cell values, the shape's where an array is absent; the scale
            // is the largest |n^2 - 1| over the cells
            std::vector<double> dl(n), bt(n);
            double scale = 0.0, imax = 0.0;
            for (size_t k = 0; k < n; ++k) {
                dl[k] = s->map_delta ? s->map_delta[k] : s->delta;
                bt[k] = s->map_beta ? s->map_beta[k] : s->beta;
                const double re = -2.0 * dl[k] + dl[k] * dl[k] - bt[k] * bt[k];
                const double im = 2.0 * bt[k] - 2.0 * dl[k] * bt[k];
                scale = std::fmax(scale, std::sqrt(re * re + im * im));
                imax = std::fmax(imax, std::fmax(std::fabs(dl[k]), std::fabs(bt[k])));
            }
            if ((rc = check_cuda(h, cudaMemcpyAsync(h->d_mdelta, dl.data(), n * sizeof(double), cudaMemcpyHostToDevice,
                                                     h->stream), "map index upload")))
                return rc;
            if ((rc = check_cuda(h, cudaMemcpyAsync(h->d_mbeta, bt.data(), n * sizeof(double), cudaMemcpyHostToDevice,
                                                     h->stream), "map index upload")))
                return rc;
            sp->mdelta = h->d_mdelta;
            sp->mbeta = h->d_mbeta;
            sp->varn = 1;
            sp->nscale = scale > 0.0 ? scale : 1.0;
            h->map_index_max = imax;
        }
    }
    return SCATMAN_OK;
}

int scatman_voxelise(scatman_handle *h, const scatman_shape *s) {
    const StageRange nvtx_range("scatman_voxelise");
    if (!h || !s) return SCATMAN_ERR_ARG;
    const scatman_config &c = h->cfg;
    if (s->kind < SCATMAN_SPHERE || s->kind > SCATMAN_VOLUMEMAP)
        return set_error(h, SCATMAN_ERR_ARG, "unknown shape kind");
    if (s->kind == SCATMAN_RADIALMAP) {
        if (!s->radial_map || s->map_ntheta < 1 || s->map_nphi < 1)
            return set_error(h, SCATMAN_ERR_ARG, "radial map needs data and map_ntheta, map_nphi >= 1");
        for (long long k = 0; k < (long long)s->map_ntheta * s->map_nphi; ++k)
            if (!std::isfinite(s->radial_map[k])) return set_error(h, SCATMAN_ERR_ARG, "radial map values must be finite");
    }
    if (s->kind == SCATMAN_VOLUMEMAP) {
        if (!s->volume_map || s->map_nx < 1 || s->map_ny < 1 || s->map_nz < 1 || !(s->map_dx > 0))
            return set_error(h, SCATMAN_ERR_ARG, "volume map needs data, map_nx/ny/nz >= 1 and map_dx > 0");
        const long long ncell = (long long)s->map_nx * s->map_ny * s->map_nz;
        for (const double *arr : {s->map_delta, s->map_beta})
            if (arr)
                for (long long k = 0; k < ncell; ++k)
                    if (!std::isfinite(arr[k])) return set_error(h, SCATMAN_ERR_ARG, "map index values must be finite");
    }
    {
        std::string why;
        if (!check_param_shape(s, &why)) return set_error(h, SCATMAN_ERR_ARG, why);
    }

    h->shape = *s;
    // the map arrays are borrowed for this call only
    h->shape.radial_map = nullptr;
    h->shape.volume_map = nullptr;
    h->shape.map_delta = h->shape.map_beta = nullptr;
    h->alm.assign((size_t)(s->kind == SCATMAN_SPHHARM ? (s->lmax + 1) * (s->lmax + 1) : 0), 0.0);
    if (s->kind == SCATMAN_SPHHARM && s->lmax > 0)
        std::memcpy(h->alm.data(), s->alm, sizeof(double) * h->alm.size());
    h->shape.alm = h->alm.empty() ? nullptr : h->alm.data();

    ShapeParams &sp = h->sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.kind = s->kind;
    sp.lmax = s->kind == SCATMAN_SPHHARM ? s->lmax : 0;
    sp.soft = c.soft ? 1 : 0;
    sp.inv_w = c.soft ? 1.0 / c.soft_width : 0.0;
    sp.inv_w_f = (float)sp.inv_w;
    sp.r = s->r;
    sp.a = s->a;
    sp.b = s->b;
    sp.c = s->c;
    sp.R0 = s->R0;
    int nmin = c.nx < c.ny ? c.nx : c.ny;
    if (c.nz < nmin) nmin = c.nz;
    sp.rmin = 0.1 * s->R0;
    sp.rmax = 0.5 * (nmin - 1) * c.voxel - c.voxel;
    orientation_matrix(s->latitude, s->longitude, s->rotation, sp.R);
    sp.cx = s->cx;
    sp.cy = s->cy;
    sp.cz = s->cz;
    for (size_t k = 0; k < h->alm.size(); ++k) sp.alm[k] = h->alm[k];
    finish_shape_params(&sp);
    int rc = upload_maps(h, s, &sp);
    if (rc) return rc;
    set_radius_band(s, &sp, h->precision == SCATMAN_FP64);

    const GridParams gp = make_grid(c.nx, c.ny, c.nz, c.voxel, h->k0, s->delta, s->beta);
    SliceOut so;
    so.layout = h->precision == SCATMAN_FP64 ? kLayoutC64
                : !h->tensor_core ? kLayoutC32
                : h->s_bf16 ? kLayoutTcBF16 : kLayoutTcF16;
    so.Nxp = h->Nxp;
    so.Nyp = h->Nyp;
    so.Kp = h->Kp;
    so.s = h->d_s;
    so.chi = h->d_chi;
    so.bounds = h->d_bounds;
    so.chunk_y = h->tensor_core ? geom_chunk_y(h->d_bounds, c.nz) : nullptr;
    double strength = std::fmax(std::fabs(s->delta), std::fabs(s->beta));
    if (sp.varn) strength = std::fmax(strength, h->map_index_max);
    h->scan_fp64 = c.scan_fp64 || (h->k0 * c.voxel * c.nz * strength > 5.0);
    // global strength factor of the stored slices: n^2 - 1 with n = 1 - delta + i beta,
    // or the index scale when every cell carries its own n
    if (sp.varn) {
        h->str_re = sp.nscale;
        h->str_im = 0.0;
    } else {
        h->str_re = -2.0 * s->delta + s->delta * s->delta - s->beta * s->beta;
        h->str_im = 2.0 * s->beta - 2.0 * s->delta * s->beta;
    }
    rc = check_cuda(h, launch_voxelise(sp, gp, so, h->scan_fp64, h->precision == SCATMAN_FP64, h->stream),
                    "voxelise");
    if (rc) return rc;
    h->have_shape = true;
    h->have_forward = false;
    return SCATMAN_OK;
}

int scatman_forward(scatman_handle *h, void *I_dev, void *A_dev) {
    const StageRange nvtx_range("scatman_forward");
    if (!h || !I_dev) return set_error(h, SCATMAN_ERR_ARG, "I_dev is NULL");
    if (!h->have_shape) return set_error(h, SCATMAN_ERR_STATE, "forward before voxelise");
    const scatman_config &c = h->cfg;
    const double str_re = h->str_re, str_im = h->str_im;     // set by voxelise
    cudaError_t e;
    if (h->uniform_tc) {
        // the y sum writes only occupied slices and x spans: the rest of H is zero
        e = cudaMemsetAsync(h->d_H, 0, uq_tc_h_bytes(c.nx, c.nz, c.det_ny), h->stream);
        if (e == cudaSuccess) {
            const UqStore store{(uint16_t *)h->d_H, h->uq_Jp, h->uq_Rg, h->uq_Kx, h->bf16};
            e = launch_uq_y_tc_mma(h->tmap_B, h->d_uq_qrow, c.det_ny, c.nx, c.ny, c.nz, h->Nxp, h->Nyp, c.voxel,
                                   h->split, h->s_bf16, h->d_bounds, store, h->d_err, h->sm_count, h->stream);
        }
        if (e == cudaSuccess)
            e = launch_uq_tc(h->tmap_H, h->d_uq_qz, c.nx, c.nz, c.det_nx, c.det_ny, c.theta_max_deg, h->k0, c.voxel,
                             str_re, str_im, h->split, h->bf16, (float2 *)h->d_A, (float *)I_dev, h->d_err,
                             h->sm_count, h->stream);
    } else if (h->uniform_q) {
        e = launch_msft_uniform(h->precision == SCATMAN_FP64, h->d_s, c.nx, c.ny, c.nz, c.det_nx, c.det_ny,
                                c.theta_max_deg, h->k0, c.voxel, str_re, str_im, h->d_uq_qz, h->d_H, h->d_A, I_dev,
                                h->stream);
    } else if (h->tensor_core) {
        e = launch_msft_tc(h->tmap_B, h->d_q, h->n_pix, c.nx, c.ny, c.nz, h->Nxp, h->Nyp, c.voxel, str_re,
                           str_im, h->split, h->bf16, h->d_bounds, (float2 *)h->d_A,
                           (float *)I_dev, h->d_err, h->sm_count, h->stream, h->d_tail);
    } else {
        e = launch_msft_simt(h->precision == SCATMAN_FP64, h->d_s, h->d_q, h->n_pix, c.nx, c.ny, c.nz, c.voxel,
                             str_re, str_im, h->d_A, I_dev, h->d_partial, h->splits, h->stream, h->d_bounds);
    }
    int rc = check_cuda(h, e, "forward");
    if (rc) return rc;
    if (A_dev) {
        size_t cx = h->precision == SCATMAN_FP64 ? sizeof(double2) : sizeof(float2);
        rc = check_cuda(h, cudaMemcpyAsync(A_dev, h->d_A, (size_t)h->n_pix * cx, cudaMemcpyDeviceToDevice, h->stream),
                        "field copy");
        if (rc) return rc;
    }
    h->have_forward = true;
    return SCATMAN_OK;
}

int scatman_sync(scatman_handle *h) {
    if (!h) return SCATMAN_ERR_ARG;
    int rc = check_cuda(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    if (rc) return rc;
    int err = 0;
    rc = check_cuda(h, cudaMemcpy(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word");
    if (rc) return rc;
    if (err) {
        cudaMemset(h->d_err, 0, sizeof(int));
        return set_error(h, SCATMAN_ERR_TIMEOUT,
                         "a kernel gave up a bounded wait (error bits " + std::to_string(err) + ")");
    }
    return SCATMAN_OK;
}

void scatman_debug_fail_allocation(long long after) { scm::g_fail_countdown.store(after < 0 ? -1 : after); }

int scatman_set_wait_limit(scatman_handle *h, double seconds) {
    if (!h) return SCATMAN_ERR_ARG;
    if (!std::isfinite(seconds)) return set_error(h, SCATMAN_ERR_ARG, "the wait limit must be finite");
    unsigned long long ns = 0;
    if (seconds > 0) {
        const double v = seconds * 1e9;
        ns = v < 1.0 ? 1ull : v >= (double)scm::kWaitLimitMaxNs ? 0ull : (unsigned long long)v;
    }
    int rc = check_cuda(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    if (rc) return rc;
    return check_cuda(h, cudaMemcpy(reinterpret_cast<char *>(h->d_err) + 8, &ns, sizeof(ns), cudaMemcpyHostToDevice),
                      "wait limit");
}

int scatman_debug_stall(scatman_handle *h, int on) {
    if (!h) return SCATMAN_ERR_ARG;
    int rc = check_cuda(h, cudaStreamSynchronize(h->stream), "stream synchronize");
    if (rc) return rc;
    const int v = on ? 1 : 0;
    return check_cuda(h, cudaMemcpy(reinterpret_cast<char *>(h->d_err) + 4, &v, sizeof(v), cudaMemcpyHostToDevice),
                      "stall flag");
}

int scatman_acquire(scatman_handle *h, const scatman_shape *shape, void *I_host) {
    if (!h || !shape || !I_host) return set_error(h, SCATMAN_ERR_ARG, "NULL argument");
    int rc = scatman_voxelise(h, shape);
    if (rc) return rc;
    rc = scatman_forward(h, h->d_I, nullptr);
    if (rc) return rc;
    rc = check_cuda(h, cudaMemcpyAsync(I_host, h->d_I, (size_t)h->n_pix * scatman_elem_size(h),
                                       cudaMemcpyDeviceToHost, h->stream),
                    "intensity download");
    if (rc) return rc;
    return scatman_sync(h);
}

int scatman_acquire_batch(scatman_handle *h, const scatman_shape *shapes, int n, void *const *I_host) {
    const StageRange nvtx_range("scatman_acquire_batch");
    if (!h || (n > 0 && (!shapes || !I_host))) return set_error(h, SCATMAN_ERR_ARG, "NULL argument");
    if (n < 0) return set_error(h, SCATMAN_ERR_ARG, "n must be >= 0");
    for (int i = 0; i < n; ++i)
        if (!I_host[i]) return set_error(h, SCATMAN_ERR_ARG, "NULL host array");
    const size_t bytes = (size_t)h->n_pix * scatman_elem_size(h);
    int rc;
    if (!h->copy_stream) {
        if ((rc = alloc_dev(h, &h->d_I2, bytes, "second intensity buffer"))) return rc;
        if ((rc = check_cuda(h, cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking), "copy stream")))
            return rc;
        for (int b = 0; b < 2; ++b) {
            if ((rc = check_cuda(h, cudaEventCreateWithFlags(&h->ev_fwd[b], cudaEventDisableTiming), "event")))
                return rc;
            if ((rc = check_cuda(h, cudaEventCreateWithFlags(&h->ev_copy[b], cudaEventDisableTiming), "event")))
                return rc;
        }
    }
    // Two intensity buffers: pattern i computes into buffer i % 2 on the handle's
    // stream while the copy stream downloads pattern i - 1; a buffer is reused
    // only after its previous download has finished.
    for (int i = 0; i < n; ++i) {
        const int b = i & 1;
        void *buf = b ? h->d_I2 : h->d_I;
        if (i >= 2 && (rc = check_cuda(h, cudaStreamWaitEvent(h->stream, h->ev_copy[b], 0), "stream wait")))
            return rc;
        if ((rc = scatman_voxelise(h, &shapes[i]))) return rc;
        if ((rc = scatman_forward(h, buf, nullptr))) return rc;
        if ((rc = check_cuda(h, cudaEventRecord(h->ev_fwd[b], h->stream), "event record"))) return rc;
        if ((rc = check_cuda(h, cudaStreamWaitEvent(h->copy_stream, h->ev_fwd[b], 0), "stream wait"))) return rc;
        if ((rc = check_cuda(h, cudaMemcpyAsync(I_host[i], buf, bytes, cudaMemcpyDeviceToHost, h->copy_stream),
                             "intensity download")))
            return rc;
        if ((rc = check_cuda(h, cudaEventRecord(h->ev_copy[b], h->copy_stream), "event record"))) return rc;
    }
    if ((rc = check_cuda(h, cudaStreamSynchronize(h->copy_stream), "copy stream synchronize"))) return rc;
    return scatman_sync(h);
}

int scatman_get_occupancy(scatman_handle *h, double *chi_host) {
    if (!h || !chi_host) return SCATMAN_ERR_ARG;
    if (!h->have_shape) return set_error(h, SCATMAN_ERR_STATE, "no voxelised shape");
    const scatman_config &c = h->cfg;
    size_t nvox = (size_t)c.nx * c.ny * c.nz;
    std::vector<float> tmp(nvox);
    int rc = check_cuda(h, cudaMemcpyAsync(tmp.data(), h->d_chi, nvox * sizeof(float), cudaMemcpyDeviceToHost,
                                           h->stream),
                        "occupancy download");
    if (rc) return rc;
    if ((rc = scatman_sync(h))) return rc;
    for (size_t i = 0; i < nvox; ++i) chi_host[i] = tmp[i];
    return SCATMAN_OK;
}

static float half_bits_to_float(uint16_t u, bool bf16) {
    if (bf16) {
        uint32_t w = (uint32_t)u << 16;
        float f;
        std::memcpy(&f, &w, 4);
        return f;
    }
    __half_raw r;
    r.x = u;
    return __half2float(__half(r));
}

int scatman_get_slices(scatman_handle *h, double *s_host) {
    if (!h || !s_host) return SCATMAN_ERR_ARG;
    if (!h->have_shape) return set_error(h, SCATMAN_ERR_STATE, "no voxelised shape");
    const scatman_config &c = h->cfg;
    size_t nvox = (size_t)c.nx * c.ny * c.nz;
    std::vector<unsigned char> tmp(h->s_bytes);
    int rc = check_cuda(h, cudaMemcpyAsync(tmp.data(), h->d_s, h->s_bytes, cudaMemcpyDeviceToHost, h->stream),
                        "slice download");
    if (rc) return rc;
    if ((rc = scatman_sync(h))) return rc;
    if (h->precision == SCATMAN_FP64) {
        std::memcpy(s_host, tmp.data(), nvox * sizeof(double2));
    } else if (!h->tensor_core) {
        const float *f = (const float *)tmp.data();
        for (size_t i = 0; i < 2 * nvox; ++i) s_host[i] = f[i];
    } else {
        const uint16_t *B = (const uint16_t *)tmp.data();
        for (int iz = 0; iz < c.nz; ++iz)
            for (int ix = 0; ix < c.nx; ++ix)
                for (int iy = 0; iy < c.ny; ++iy) {
                    size_t row_r = ((size_t)iz * 3 + 1) * h->Nxp + ix;     // Re plane; Im plane follows
                    size_t v = ((size_t)iz * c.nx + ix) * c.ny + iy;
                    s_host[2 * v] = half_bits_to_float(B[row_r * h->Kp + iy], h->s_bf16);
                    s_host[2 * v + 1] = half_bits_to_float(B[(row_r + h->Nxp) * h->Kp + iy], h->s_bf16);
                }
    }
    return SCATMAN_OK;
}

int scatman_contraction_flops(scatman_handle *h, double *issued, double *dense) {
    if (!h || !issued || !dense) return SCATMAN_ERR_ARG;
    if (!h->have_shape) return set_error(h, SCATMAN_ERR_STATE, "no voxelised shape");
    const scatman_config &c = h->cfg;
    const double dense_pairs = (double)h->n_pix * c.nx * c.ny * c.nz;
    if (h->uniform_tc) {
        // the x/z launch only: 8 real flops per (pixel, x, z) term, twice with split phases
        *dense = 8.0 * (double)h->n_pix * c.nx * c.nz * (h->split ? 2.0 : 1.0);
        *issued = uq_tc_issued_flops(c.nx, c.nz, c.det_nx, c.det_ny, h->split);
        return SCATMAN_OK;
    }
    std::vector<int> b((4 + 2 * (size_t)kGeomChunks) * c.nz);
    int rc = check_cuda(h, cudaMemcpyAsync(b.data(), h->d_bounds, b.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                           h->stream),
                        "slice geometry download");
    if (rc) return rc;
    if ((rc = scatman_sync(h))) return rc;
    if (!h->tensor_core) {
        *dense = 8.0 * dense_pairs;
        *issued = h->uniform_q ? *dense : simt_issued_flops(b.data(), c.nz, c.ny, h->n_pix, h->precision == SCATMAN_FP64);
        return SCATMAN_OK;
    }
    *dense = 8.0 * dense_pairs * (h->split ? 2.0 : 1.0);
    *issued = tc_issued_flops(b.data(), c.nz, h->Nxp, h->Nyp, h->n_pix, h->split);
    return SCATMAN_OK;
}

int scatman_get_q(scatman_handle *h, double *q_host) {
    if (!h || !q_host) return SCATMAN_ERR_ARG;
    int rc = check_cuda(h, cudaMemcpyAsync(q_host, h->d_q, (size_t)h->n_pix * 3 * sizeof(double),
                                           cudaMemcpyDeviceToHost, h->stream),
                        "q download");
    if (rc) return rc;
    return scatman_sync(h);
}

int scatman_photon_counts(scatman_handle *h, double photon_density, unsigned long long seed, const void *I_dev,
                          double *lambda_dev, long long *counts_dev) {
    if (!h || !I_dev || (!lambda_dev && !counts_dev)) return set_error(h, SCATMAN_ERR_ARG, "NULL argument");
    if (!(photon_density >= 0.0) || !std::isfinite(photon_density))
        return set_error(h, SCATMAN_ERR_ARG, "photon density must be finite and >= 0");
    const scatman_config &c = h->cfg;
    if (h->from_q_list) return set_error(h, SCATMAN_ERR_ARG, "photon counts need the detector's pixels (no q_list)");
    return check_cuda(h, launch_photon_counts(I_dev, h->precision == SCATMAN_FP64, h->n_pix, c.det_nx, c.det_ny,
                                              h->uniform_q, c.theta_max_deg, c.wavelength, c.voxel, photon_density,
                                              seed, lambda_dev, counts_dev, h->stream),
                      "photon counts");
}

// Bessel functions J_0(w) .. J_{N-1}(w) of the first kind, by Miller's backward
// recurrence J_{k-1} = (2k / x) J_k - J_{k+1} from far above N and |w|,
// normalised with J_0 + 2 sum_{k >= 1} J_{2k} = 1; J_k(-x) = (-1)^k J_k(x).
static void bessel_j_orders(double w, int N, double *J) {
    for (int k = 0; k < N; ++k) J[k] = 0.0;
    const double x = std::fabs(w);
    if (x == 0.0) {
        J[0] = 1.0;
        return;
    }
    const double top = std::fmax((double)N, x);
    const int m = 2 * (((int)(top + 40.0 + std::sqrt(40.0 * top))) / 2);
    std::vector<double> t((size_t)m + 2, 0.0);
    double jp = 0.0, j = 1e-300, norm = 0.0;
    t[(size_t)m] = j;
    for (int k = m; k > 0; --k) {
        const double jm = 2.0 * k / x * j - jp;
        jp = j;
        j = jm;
        t[(size_t)k - 1] = j;
        if (std::fabs(j) > 1e250) {               // rescale everything computed so far
            for (int q = k - 1; q <= m; ++q) t[(size_t)q] *= 1e-250;
            j *= 1e-250;
            jp *= 1e-250;
        }
    }
    norm = t[0];
    for (int k = 2; k <= m; k += 2) norm += 2.0 * t[(size_t)k];
    for (int k = 0; k < N; ++k) J[k] = t[(size_t)k] / norm * ((w < 0.0 && (k & 1)) ? -1.0 : 1.0);
}

// Orders N after which the Jacobi-Anger tail 2 sum_{n >= N} |J_n(w)| is below
// tol for every |w| <= wmax (|J_n(w)| <= (|w|/2)^n / n!, a geometric majorant
// once n + 1 > |w| / 2).
static int adjoint_orders_needed(double wmax, double tol) {
    const double hw = 0.5 * std::fabs(wmax);
    double t = 1.0;                                // (hw)^N / N!
    for (int N = 1; N < 512; ++N) {
        t *= hw / N;
        if (hw < N + 1 && 2.0 * t / (1.0 - hw / (N + 1)) <= tol) return N;
    }
    return 512;
}

// Chooses the tensor-core adjoint's form for the handle (once): with the q_z of
// the handle's pixels in [q_c - D, q_c + D] and |z_j| <= z_max, order mode takes
// N orders for w = D z_max; it is used when N < nz.  Builds the pixel table in
// the chosen form and, in order mode, the coefficients a[j][n].
static int plan_adjoint(scatman_handle *h) {
    const scatman_config &c = h->cfg;
    std::vector<double> qz((size_t)h->n_pix);
    int rc = check_cuda(h, cudaMemcpy2DAsync(qz.data(), sizeof(double), h->d_q + 2, 3 * sizeof(double), sizeof(double),
                                             (size_t)h->n_pix, cudaMemcpyDeviceToHost, h->stream),
                        "q_z download");
    if (rc) return rc;
    if ((rc = check_cuda(h, cudaStreamSynchronize(h->stream), "q_z download"))) return rc;
    double lo = qz[0], hi = qz[0];
    for (double v : qz) {
        lo = std::fmin(lo, v);
        hi = std::fmax(hi, v);
    }
    const double qc = 0.5 * (lo + hi), D = 0.5 * (hi - lo);
    const double zmax = 0.5 * (c.nz - 1) * c.voxel;
    const int N = D > 0.0 ? adjoint_orders_needed(D * zmax, 1e-7) : 1;
    const bool orders = N < c.nz && N <= 64;
    h->adj_orders = orders ? N : 0;
    if ((rc = alloc_dev(h, (void **)&h->d_adj_tab, (size_t)h->n_pix * 3 * sizeof(float4), "adjoint pixel table")))
        return rc;
    if ((rc = check_cuda(h, launch_adj_pixel_table(h->d_q, h->n_pix, c.voxel, orders ? 1 : 0, qc,
                                                   orders && D > 0.0 ? 1.0 / D : 0.0, h->d_adj_tab, h->stream),
                         "adjoint pixel table")))
        return rc;
    if (!orders) return SCATMAN_OK;
    // a[j][n] = e^{+i q_c z_j} eps_n i^n J_n(D z_j)
    std::vector<float2> coef((size_t)c.nz * N);
    std::vector<double> J((size_t)N);
    for (int jz = 0; jz < c.nz; ++jz) {
        const double z = (jz - 0.5 * (c.nz - 1)) * c.voxel;
        bessel_j_orders(D * z, N, J.data());
        const double pr = std::cos(qc * z), pi = std::sin(qc * z);
        for (int n = 0; n < N; ++n) {
            const double m = (n == 0 ? 1.0 : 2.0) * J[(size_t)n];
            // i^n = (1, i, -1, -i)
            double ar = 0.0, ai = 0.0;
            switch (n & 3) {
                case 0: ar = m; break;
                case 1: ai = m; break;
                case 2: ar = -m; break;
                default: ai = -m; break;
            }
            coef[(size_t)jz * N + n] = make_float2((float)(pr * ar - pi * ai), (float)(pr * ai + pi * ar));
        }
    }
    if ((rc = alloc_dev(h, (void **)&h->d_adj_coef, coef.size() * sizeof(float2), "adjoint order coefficients")))
        return rc;
    if ((rc = check_cuda(h, cudaMemcpy(h->d_adj_coef, coef.data(), coef.size() * sizeof(float2), cudaMemcpyHostToDevice),
                         "adjoint order coefficients")))
        return rc;
    return alloc_dev(h, (void **)&h->d_adj_ord, (size_t)N * c.nx * c.ny * sizeof(float2), "adjoint order fields");
}

int scatman_backward(scatman_handle *h, const void *dLdI_dev, double *dLdparams) {
    const StageRange nvtx_range("scatman_backward");
    if (!h || !dLdI_dev || !dLdparams) return set_error(h, SCATMAN_ERR_ARG, "NULL argument");
    if (!h->have_forward) return set_error(h, SCATMAN_ERR_STATE, "backward before forward");
    if (is_map_kind(h->sp.kind))
        return set_error(h, SCATMAN_ERR_UNSUPPORTED, "map shapes have no gradient (forward only)");
    const scatman_config &c = h->cfg;
    const bool f64 = h->precision == SCATMAN_FP64;
    const size_t nvox = (size_t)c.nx * c.ny * c.nz;
    int rc;
    if (!h->d_S) {
        if ((rc = alloc_dev(h, &h->d_S, nvox * (f64 ? sizeof(double2) : sizeof(float2)), "adjoint field")))
            return rc;
    }
    const GridParams gp = make_grid(c.nx, c.ny, c.nz, c.voxel, h->k0, h->shape.delta, h->shape.beta);
    const int ng = grad_param_count(h->sp);
    const int nvb = grad_voxel_blocks(f64, h->sp, gp, h->sm_count), npb = grad_pixel_blocks(h->n_pix);
    const size_t need = (size_t)nvb * (ng + 2) + (size_t)npb;
    if (h->part_count < need) {
        cudaFree(h->d_part);
        h->d_part = nullptr;
        if ((rc = alloc_dev(h, (void **)&h->d_part, need * sizeof(double), "gradient partials"))) return rc;
        h->part_count = need;
    }
    if (h->tensor_core && adjoint_tc_supported(c.nx, c.ny)) {
        // adjoint contraction on the tensor cores (per slice, or per Jacobi-Anger order)
        if (h->adj_orders < 0 && (rc = plan_adjoint(h))) return rc;
        const int N = h->adj_orders;
        const int nz_eff = N > 0 ? N : c.nz;
        int splits = adjoint_tc_splits(h->n_pix, nz_eff, h->sm_count, N > 0);
        while (N > 0 && splits > 1 && splits * N > 8 * c.nz) --splits;   // within the slice mode's partial memory
        const size_t cnt = (size_t)splits * nz_eff * c.nx * c.ny;
        if (h->adj_part_count < cnt) {
            cudaFree(h->d_adj_part);
            h->d_adj_part = nullptr;
            if ((rc = alloc_dev(h, (void **)&h->d_adj_part, cnt * sizeof(float2), "adjoint partial fields")))
                return rc;
            h->adj_part_count = cnt;
        }
        if (!h->d_gmax && (rc = alloc_dev(h, (void **)&h->d_gmax, sizeof(unsigned), "adjoint scale"))) return rc;
        if (!h->d_adj_rtile) {
            if ((rc = alloc_dev(h, (void **)&h->d_adj_rtile, adj_rtile_bytes(h->n_pix, c.ny), "adjoint y-phase tiles")))
                return rc;
            if ((rc = check_cuda(h, launch_adj_rtile(h->d_adj_tab, h->n_pix, c.ny, c.voxel, h->d_adj_rtile, h->stream),
                                 "adjoint y-phase tiles")))
                return rc;
        }
        rc = check_cuda(h, launch_adjoint_tc((const float2 *)h->d_A, (const float *)dLdI_dev, h->d_adj_tab,
                                             h->d_adj_rtile, h->n_pix, c.nx, c.ny, nz_eff, N > 0 ? 1 : 0, c.voxel,
                                             splits, h->d_adj_part, h->d_gmax,
                                             N > 0 ? h->d_adj_ord : (float2 *)h->d_S, h->d_err, h->stream),
                        "adjoint field (tensor cores)");
        if (rc) return rc;
        if (N > 0 && (rc = check_cuda(h, launch_adj_orders_combine(h->d_adj_ord, h->d_adj_coef, N, c.nz, c.nx, c.ny,
                                                                   (float2 *)h->d_S, h->stream),
                                      "adjoint slices from orders")))
            return rc;
    } else {
        rc = check_cuda(h, launch_adjoint_field(f64, h->d_A, dLdI_dev, h->d_q, h->n_pix, c.nx, c.ny, c.nz, c.voxel,
                                                h->d_S, h->stream),
                        "adjoint field");
        if (rc) return rc;
    }
    rc = check_cuda(h, launch_grad_voxels(f64, h->sp, gp, h->d_S, h->d_part, nvb, h->stream), "voxel gradient");
    if (rc) return rc;
    rc = check_cuda(h, launch_grad_pixels(f64, h->d_A, dLdI_dev, h->n_pix, h->d_part + (size_t)nvb * (ng + 2), npb,
                                          h->stream),
                    "pixel gradient");
    if (rc) return rc;
    std::vector<double> part(need);
    rc = check_cuda(h, cudaMemcpyAsync(part.data(), h->d_part, need * sizeof(double), cudaMemcpyDeviceToHost,
                                       h->stream),
                    "gradient download");
    if (rc) return rc;
    if ((rc = scatman_sync(h))) return rc;
    // fixed-order sums of the per-block partials
    std::vector<double> sums(ng + 2, 0.0);
    for (int b = 0; b < nvb; ++b)
        for (int k = 0; k < ng + 2; ++k) sums[k] += part[(size_t)b * (ng + 2) + k];
    double wI = 0.0;
    for (int b = 0; b < npb; ++b) wI += part[(size_t)nvb * (ng + 2) + b];
    // n, c = n^2 - 1 and their derivatives in delta, beta
    const double d = h->shape.delta, bb = h->shape.beta;
    const double nr = 1.0 - d, ni = bb;
    const double cr = nr * nr - ni * ni - 1.0, ci = 2.0 * nr * ni;
    const double cc = cr * cr + ci * ci;
    // dc/ddelta = -2n, dc/dbeta = 2 i n;  2 Re[(c'/c) wI]
    auto re_ratio = [&](double ar, double ai) { return (ar * cr + ai * ci) / cc; };
    const double g_delta_c = 2.0 * re_ratio(-2.0 * nr, -2.0 * ni) * wI;
    const double g_beta_c = 2.0 * re_ratio(-2.0 * ni, 2.0 * nr) * wI;
    // D = sum_v R_v s_v C_v (complex); d(n-1)/ddelta = -1, d(n-1)/dbeta = i; term 2 Re(D i k0 dz d(n-1))
    const double Dr = sums[ng], Di = sums[ng + 1];
    const double kdz = h->k0 * c.voxel;
    const double g_delta_n = 2.0 * (Di * kdz);       // Re(D * i * kdz * -1) = Di kdz
    const double g_beta_n = 2.0 * (-Dr * kdz);       // Re(D * i * kdz * i) = -Dr kdz
    for (int k = 0; k < ng; ++k) dLdparams[k] = 2.0 * sums[k];
    dLdparams[ng] = g_delta_c + g_delta_n;
    dLdparams[ng + 1] = g_beta_c + g_beta_n;
    return SCATMAN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Forward pass without device allocation.
//
// Some callers cannot call cudaMalloc: a host application that has already
// reserved nearly all device memory for its own pool, or a latency-critical
// loop that must not take the device-wide synchronisation an allocation can
// cause.  scatman_forward_noalloc serves them with the CUDA-core FP32 path,
// keeping its working memory (q, occupancy, slices, partial fields) in one
// fixed array that the library image carries, so only the caller's output
// buffers are written.
// ---------------------------------------------------------------------------
#include <mutex>

namespace scm {

constexpr size_t kNoAllocScratchBytes = (size_t)8 << 20;   // 8 MiB, held by every GPU that loads the library
constexpr int kNoAllocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];
static std::mutex g_noalloc_mu;
static void *g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once
// per device; host code only ever sees a host-side stand-in for the symbol).
static int noalloc_scratch(int dev, void **out, std::string *why) {
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        *why = "device ordinal out of range for the no-allocation scratch table";
        return SCATMAN_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            *why = std::string("cudaGetSymbolAddress of the scratch array failed: ") + cudaGetErrorString(e);
            return SCATMAN_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SCATMAN_OK;
}

}  // namespace scm

extern "C" int scatman_forward_noalloc(const scatman_config *cfg, const scatman_shape *s, void *cuda_stream,
                                       float *I_dev, float *A_dev) {
    g_create_error.clear();
    auto fail = [&](int code, const std::string &msg) {
        g_create_error = msg;
        return code;
    };
    if (!cfg || !s || !I_dev) return fail(SCATMAN_ERR_ARG, "NULL argument");
    const scatman_config &c = *cfg;
    if (c.precision != SCATMAN_FP32) return fail(SCATMAN_ERR_ARG, "the no-allocation forward runs in SCATMAN_FP32 only");
    long long n_pix = 0;
    std::string why;
    if (!check_config(c, &n_pix, &why)) return fail(SCATMAN_ERR_ARG, why);
    // the flat detector's q (or the caller's q_list) only: the uniform-q
    // detector needs its own q table and a masked field
    if (c.detector != SCATMAN_DETECTOR_FLAT && !c.q_list)
        return fail(SCATMAN_ERR_ARG, "the no-allocation forward supports the flat detector or a q_list only");
    if (s->kind < SCATMAN_SPHERE || s->kind > SCATMAN_SPHHARM) return fail(SCATMAN_ERR_ARG, "unknown shape kind");
    if (!check_param_shape(s, &why)) return fail(SCATMAN_ERR_ARG, why);

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(SCATMAN_ERR_UNSUPPORTED, "no CUDA device");
    int major = 0, minor = 0, sms = 0;
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (!(major == 10 && minor == 3))
        return fail(SCATMAN_ERR_UNSUPPORTED, "this library is built for sm_103a (compute capability 10.3) only");

    // carve the scratch: q | occupancy | slices | field (if not supplied) | partial fields
    const size_t nvox = (size_t)c.nx * c.ny * c.nz;
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    const size_t q_b = up((size_t)n_pix * 3 * sizeof(double));
    const size_t chi_b = up(nvox * sizeof(float));
    const size_t s_b = up(nvox * sizeof(float2));
    const size_t a_b = A_dev ? 0 : up((size_t)n_pix * sizeof(float2));
    const size_t fixed = q_b + chi_b + s_b + a_b;
    int splits = simt_splits(n_pix, c.nx, c.nz, sms);
    while (splits > 1 && fixed + up((size_t)splits * n_pix * sizeof(float2)) > kNoAllocScratchBytes) --splits;
    const size_t need = fixed + up((size_t)splits * n_pix * sizeof(float2));
    if (need > kNoAllocScratchBytes)
        return fail(SCATMAN_ERR_ARG, "problem needs " + std::to_string(need) + " bytes of scratch; the no-allocation "
                                     "forward holds " + std::to_string(kNoAllocScratchBytes) + " bytes");
    void *base = nullptr;
    int rc = noalloc_scratch(dev, &base, &why);
    if (rc) return fail(rc, why);
    unsigned char *b = (unsigned char *)base;
    double *d_q = (double *)b;
    float *d_chi = (float *)(b + q_b);
    float2 *d_s = (float2 *)(b + q_b + chi_b);
    float2 *d_A = A_dev ? (float2 *)A_dev : (float2 *)(b + q_b + chi_b + s_b);
    float2 *d_part = (float2 *)(b + fixed);
    cudaStream_t st = (cudaStream_t)cuda_stream;

    const double k0 = 2.0 * kPi / c.wavelength;
    cudaError_t e;
    if (c.q_list) {
        e = cudaMemcpyAsync(d_q, c.q_list, (size_t)n_pix * 3 * sizeof(double), cudaMemcpyHostToDevice, st);
    } else {
        e = launch_detector_q(c.det_nx, c.det_ny, c.theta_max_deg, k0, d_q, st);
    }
    if (e != cudaSuccess) return fail(SCATMAN_ERR_CUDA, std::string("q: ") + cudaGetErrorString(e));

    ShapeParams sp;
    std::memset(&sp, 0, sizeof(sp));
    sp.kind = s->kind;
    sp.lmax = s->kind == SCATMAN_SPHHARM ? s->lmax : 0;
    sp.soft = c.soft ? 1 : 0;
    sp.inv_w = c.soft ? 1.0 / c.soft_width : 0.0;
    sp.inv_w_f = (float)sp.inv_w;
    sp.r = s->r;
    sp.a = s->a;
    sp.b = s->b;
    sp.c = s->c;
    sp.R0 = s->R0;
    int nmin = c.nx < c.ny ? c.nx : c.ny;
    if (c.nz < nmin) nmin = c.nz;
    sp.rmin = 0.1 * s->R0;
    sp.rmax = 0.5 * (nmin - 1) * c.voxel - c.voxel;
    orientation_matrix(s->latitude, s->longitude, s->rotation, sp.R);
    sp.cx = s->cx;
    sp.cy = s->cy;
    sp.cz = s->cz;
    if (s->kind == SCATMAN_SPHHARM && s->lmax > 0)        // alm may be NULL at lmax = 0
        for (int k = 0; k < (s->lmax + 1) * (s->lmax + 1); ++k) sp.alm[k] = s->alm[k];
    finish_shape_params(&sp);
    set_radius_band(s, &sp, false);   // CUDA-core FP32 path
    const GridParams gp = make_grid(c.nx, c.ny, c.nz, c.voxel, k0, s->delta, s->beta);
    SliceOut so;
    so.layout = kLayoutC32;
    so.Nxp = so.Nyp = so.Kp = 0;
    so.s = d_s;
    so.chi = d_chi;
    so.bounds = nullptr;
    so.chunk_y = nullptr;
    const double strength = std::fmax(std::fabs(s->delta), std::fabs(s->beta));
    const bool scan_fp64 = c.scan_fp64 || (k0 * c.voxel * c.nz * strength > 5.0);
    e = launch_voxelise(sp, gp, so, scan_fp64, false, st);
    if (e != cudaSuccess) return fail(SCATMAN_ERR_CUDA, std::string("voxelise: ") + cudaGetErrorString(e));
    const double d = s->delta, bb = s->beta;
    e = launch_msft_simt(false, d_s, d_q, n_pix, c.nx, c.ny, c.nz, c.voxel, -2.0 * d + d * d - bb * bb,
                         2.0 * bb - 2.0 * d * bb, d_A, I_dev, d_part, splits, st, nullptr);
    if (e != cudaSuccess) return fail(SCATMAN_ERR_CUDA, std::string("forward: ") + cudaGetErrorString(e));
    return SCATMAN_OK;
}
