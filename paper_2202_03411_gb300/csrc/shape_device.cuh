// shape_device.cuh -- device-side shape rendering shared by the voxeliser and
// the gradient kernels, so that the backward pass recomputes exactly the
// occupancy the forward pass used.
#pragma once
#include "internal.cuh"

namespace scm {

template <typename T> struct ShTab;
template <> struct ShTab<float> {
    const float *a, *b, *d, *e, *alm;
    __device__ explicit ShTab(const ShapeParams &sp) : a(sp.sh_af), b(sp.sh_bf), d(sp.sh_df), e(sp.sh_ef), alm(sp.almf) {}
};
template <> struct ShTab<double> {
    const double *a, *b, *d, *e, *alm;
    __device__ explicit ShTab(const ShapeParams &sp) : a(sp.sh_a), b(sp.sh_b), d(sp.sh_d), e(sp.sh_e), alm(sp.alm) {}
};

// ---------------------------------------------------------------------------
// Real spherical harmonics (Eq. 10-11, real orthonormal form) evaluated with
// the fully normalised associated-Legendre recurrences:
//   Pb_0^0 = 1/sqrt(4 pi),  Pb_m^m = d_m sin(th) Pb_{m-1}^{m-1},  d_m = -sqrt((2m+1)/(2m)),
//   Pb_{m+1}^m = e_m cos(th) Pb_m^m,  e_m = sqrt(2m+3),
//   Pb_l^m = a_lm (cos(th) Pb_{l-1}^m - b_lm Pb_{l-2}^m),
//   a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)),
// and Y_l0 = Pb_l^0, Y_lm = sqrt(2) Pb_l^m cos(m phi), Y_l,-m = sqrt(2) Pb_l^m sin(m phi).
// The minus sign of d_m carries the Condon-Shortley phase.  The coefficients
// come precomputed in the shape parameters.
// f(index = l*l+l+m, Y) is called for every (l, m) with l <= L.
// ---------------------------------------------------------------------------
template <typename T, typename F>
__device__ __forceinline__ void real_sh_all(const ShTab<T> &tb, int L, T ct, T st, T cphi, T sphi, F &&f) {
    const T kInvSqrt4Pi = (T)0.28209479177387814347;
    const T kSqrt2 = (T)1.41421356237309504880;
    T pmm = kInvSqrt4Pi;
    T cm = (T)1, sm = (T)0;
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            pmm = tb.d[m] * st * pmm;
            T c2 = cm * cphi - sm * sphi;
            T s2 = sm * cphi + cm * sphi;
            cm = c2;
            sm = s2;
        }
        const T wc = m == 0 ? (T)1 : kSqrt2 * cm;
        const T ws = kSqrt2 * sm;
        T p2 = (T)0, p1 = pmm;
        const int base = m * (m + 1) / 2;
        for (int l = m; l <= L; ++l) {
            T p;
            if (l == m) {
                p = pmm;
            } else if (l == m + 1) {
                p = tb.e[m] * ct * pmm;
            } else {
                const int i = l * (l + 1) / 2 + m;
                p = tb.a[i] * (ct * p1 - tb.b[i] * p2);
            }
            if (l > m) {
                p2 = p1;
                p1 = p;
            }
            if (m == 0) {
                f(l * l + l, p);
            } else {
                f(l * l + l + m, p * wc);
                f(l * l + l - m, p * ws);
            }
        }
        (void)base;
    }
}

// Harmonics surface radius R0 (1 + sum a_lm Y_lm) along body direction p
// (not normalised), |p| = rr, before clipping.
template <typename T>
__device__ __forceinline__ T sh_radius_unclipped(const ShapeParams &sp, T px, T py, T pz, T rr) {
    const ShTab<T> tb(sp);
    T ct = (T)1, st = (T)0, cphi = (T)1, sphi = (T)0;
    if (rr > (T)0) {
        ct = pz / rr;
        T rho = sqrt(px * px + py * py);
        st = rho / rr;
        if (rho > (T)0) {
            cphi = px / rho;
            sphi = py / rho;
        }
    }
    T sum = (T)0;
    real_sh_all<T>(tb, sp.lmax, ct, st, cphi, sphi, [&](int idx, T y) {
        if (idx > 0) sum += tb.alm[idx] * y;
    });
    return (T)sp.R0 * ((T)1 + sum);
}

// The same radius clipped to [rmin, rmax].
template <typename T>
__device__ __forceinline__ T sh_radius(const ShapeParams &sp, T px, T py, T pz, T rr) {
    T r = sh_radius_unclipped<T>(sp, px, py, pz, rr);
    r = r < (T)sp.rmin ? (T)sp.rmin : r;
    r = r > (T)sp.rmax ? (T)sp.rmax : r;
    return r;
}

// Body-frame coordinates of a voxel centre, p = R^T (r - c), in double with
// explicit round-to-nearest operations (no contraction).
__device__ __forceinline__ void body_coords(const ShapeParams &sp, const GridParams &gp, int ix, int iy,
                                            int iz, double &px, double &py, double &pz) {
    double dx = (ix - 0.5 * (gp.nx - 1)) * gp.voxel - sp.cx;
    double dy = (iy - 0.5 * (gp.ny - 1)) * gp.voxel - sp.cy;
    double dz = (iz - 0.5 * (gp.nz - 1)) * gp.voxel - sp.cz;
    px = __dadd_rn(__dadd_rn(__dmul_rn(sp.R[0], dx), __dmul_rn(sp.R[3], dy)), __dmul_rn(sp.R[6], dz));
    py = __dadd_rn(__dadd_rn(__dmul_rn(sp.R[1], dx), __dmul_rn(sp.R[4], dy)), __dmul_rn(sp.R[7], dz));
    pz = __dadd_rn(__dadd_rn(__dmul_rn(sp.R[2], dx), __dmul_rn(sp.R[5], dy)), __dmul_rn(sp.R[8], dz));
}

// The FP64 binary decision: sphere |d|^2 <= r^2, ellipsoid
// (x/a)^2+(y/b)^2+(z/c)^2 <= 1, harmonics |p| <= r(theta,phi); ties inside.
static __device__ __noinline__ double occupancy_binary_fp64(const ShapeParams &sp, const GridParams &gp, int ix, int iy,
                                                     int iz) {
    double px, py, pz;
    if (sp.kind == SCATMAN_SPHERE) {
        px = (ix - 0.5 * (gp.nx - 1)) * gp.voxel - sp.cx;
        py = (iy - 0.5 * (gp.ny - 1)) * gp.voxel - sp.cy;
        pz = (iz - 0.5 * (gp.nz - 1)) * gp.voxel - sp.cz;
    } else {
        body_coords(sp, gp, ix, iy, iz, px, py, pz);
    }
    double p2 = __dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz));
    if (sp.kind == SCATMAN_SPHERE) return p2 <= __dmul_rn(sp.r, sp.r) ? 1.0 : 0.0;
    if (sp.kind == SCATMAN_ELLIPSOID) {
        double u = __ddiv_rn(px, sp.a), v = __ddiv_rn(py, sp.b), w = __ddiv_rn(pz, sp.c);
        double qf = __dadd_rn(__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)), __dmul_rn(w, w));
        return qf <= 1.0 ? 1.0 : 0.0;
    }
    double rr = sqrt(p2);
    double rs = sh_radius<double>(sp, px, py, pz, rr);
    return rr <= rs ? 1.0 : 0.0;
}

// Occupancy of one voxel.  Binary decisions are the FP64 ones above; the
// FP32 modes first evaluate the same quantity in FP32 and only fall back to
// FP64 when the margin is within a bound well above the FP32 error
// (1e-4 relative for sphere and ellipsoid, 4e-3 voxel for harmonics), so the
// decision always equals the FP64 one.  Soft occupancy is the logistic of
// the signed distance to the surface along the ray from the centre.
template <bool kFp64>
__device__ __forceinline__ double occupancy(const ShapeParams &sp, const GridParams &gp, int ix, int iy, int iz) {
    if (!sp.soft) {
        if (!kFp64) {
            const float vox = (float)gp.voxel;
            const float dx = ((float)ix - 0.5f * (float)(gp.nx - 1)) * vox - sp.cxf;
            const float dy = ((float)iy - 0.5f * (float)(gp.ny - 1)) * vox - sp.cyf;
            const float dz = ((float)iz - 0.5f * (float)(gp.nz - 1)) * vox - sp.czf;
            if (sp.kind == SCATMAN_SPHERE) {
                const float r2 = sp.r2f;
                const float m = r2 - (dx * dx + dy * dy + dz * dz);
                if (fabsf(m) > 1e-4f * r2 + 1e-6f) return m > 0.f ? 1.0 : 0.0;
            } else {
                const float px = sp.Rf[0] * dx + sp.Rf[3] * dy + sp.Rf[6] * dz;
                const float py = sp.Rf[1] * dx + sp.Rf[4] * dy + sp.Rf[7] * dz;
                const float pz = sp.Rf[2] * dx + sp.Rf[5] * dy + sp.Rf[8] * dz;
                if (sp.kind == SCATMAN_ELLIPSOID) {
                    const float u = px * sp.inv_af, v = py * sp.inv_bf, w = pz * sp.inv_cf;
                    const float m = 1.f - (u * u + v * v + w * w);
                    if (fabsf(m) > 1e-4f) return m > 0.f ? 1.0 : 0.0;
                } else {
                    const float rr = sqrtf(px * px + py * py + pz * pz);
                    const float rs = sh_radius<float>(sp, px, py, pz, rr);
                    const float m = rs - rr;
                    if (fabsf(m) > 4e-3f * vox) return m > 0.f ? 1.0 : 0.0;
                }
            }
        }
        return occupancy_binary_fp64(sp, gp, ix, iy, iz);
    }
    double px, py, pz;
    if (sp.kind == SCATMAN_SPHERE) {
        px = (ix - 0.5 * (gp.nx - 1)) * gp.voxel - sp.cx;
        py = (iy - 0.5 * (gp.ny - 1)) * gp.voxel - sp.cy;
        pz = (iz - 0.5 * (gp.nz - 1)) * gp.voxel - sp.cz;
    } else {
        body_coords(sp, gp, ix, iy, iz, px, py, pz);
    }
    double p2 = __dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz));
    double rr = sqrt(p2);
    if (kFp64) {
        double rs;
        if (sp.kind == SCATMAN_SPHERE) {
            rs = sp.r;
        } else if (sp.kind == SCATMAN_ELLIPSOID) {
            double u0 = 0, u1 = 0, u2 = 1;
            if (rr > 0) { u0 = px / rr; u1 = py / rr; u2 = pz / rr; }
            rs = 1.0 / sqrt((u0 / sp.a) * (u0 / sp.a) + (u1 / sp.b) * (u1 / sp.b) + (u2 / sp.c) * (u2 / sp.c));
        } else {
            rs = sh_radius<double>(sp, px, py, pz, rr);
        }
        return 1.0 / (1.0 + exp(-(rs - rr) * sp.inv_w));
    }
    float rf = (float)rr, rs;
    if (sp.kind == SCATMAN_SPHERE) {
        rs = (float)sp.r;
    } else if (sp.kind == SCATMAN_ELLIPSOID) {
        float u0 = 0.f, u1 = 0.f, u2 = 1.f;
        if (rf > 0.f) { u0 = (float)px / rf; u1 = (float)py / rf; u2 = (float)pz / rf; }
        const float ia = sp.inv_af, ib = sp.inv_bf, ic = sp.inv_cf;
        rs = rsqrtf(u0 * u0 * ia * ia + u1 * u1 * ib * ib + u2 * u2 * ic * ic);
    } else {
        rs = sh_radius<float>(sp, (float)px, (float)py, (float)pz, rf);
    }
    return (double)(1.0f / (1.0f + __expf(-(rs - rf) * sp.inv_w_f)));
}

}  // namespace scm
