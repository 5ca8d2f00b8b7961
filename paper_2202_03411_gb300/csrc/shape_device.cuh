// shape_device.cuh -- device-side shape rendering shared by the voxeliser and
// the gradient kernels, so that the backward pass recomputes exactly the
// occupancy the forward pass used.
#pragma once
#include "internal.cuh"

namespace scm {

// ---------------------------------------------------------------------------
// Real spherical harmonics (Eq. 10-11, real orthonormal form) evaluated with
// the fully normalised associated-Legendre recurrences:
//   Pb_0^0 = 1/sqrt(4 pi),  Pb_m^m = -sqrt((2m+1)/(2m)) sin(th) Pb_{m-1}^{m-1},
//   Pb_{m+1}^m = sqrt(2m+3) cos(th) Pb_m^m,
//   Pb_l^m = a_lm (cos(th) Pb_{l-1}^m - b_lm Pb_{l-2}^m),
//   a_lm = sqrt((4l^2-1)/(l^2-m^2)),  b_lm = sqrt(((l-1)^2-m^2)/(4(l-1)^2-1)),
// and Y_l0 = Pb_l^0, Y_lm = sqrt(2) Pb_l^m cos(m phi), Y_l,-m = sqrt(2) Pb_l^m sin(m phi).
// The minus sign on the diagonal carries the Condon-Shortley phase.
// f(index = l*l+l+m, Y) is called for every (l, m) with l <= L.
// ---------------------------------------------------------------------------
template <typename T, typename F>
__device__ __forceinline__ void real_sh_all(int L, T ct, T st, T cphi, T sphi, F &&f) {
    const T kInvSqrt4Pi = (T)0.28209479177387814347;
    const T kSqrt2 = (T)1.41421356237309504880;
    T pmm = kInvSqrt4Pi;
    T cm = (T)1, sm = (T)0;
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            pmm = -sqrt((T)(2 * m + 1) / (T)(2 * m)) * st * pmm;
            T c2 = cm * cphi - sm * sphi;
            T s2 = sm * cphi + cm * sphi;
            cm = c2;
            sm = s2;
        }
        T p2 = (T)0, p1 = pmm;
        for (int l = m; l <= L; ++l) {
            T p;
            if (l == m) {
                p = pmm;
            } else if (l == m + 1) {
                p = sqrt((T)(2 * m + 3)) * ct * pmm;
            } else {
                T a = sqrt((T)(4 * l * l - 1) / (T)(l * l - m * m));
                T b = sqrt((T)((l - 1) * (l - 1) - m * m) / (T)(4 * (l - 1) * (l - 1) - 1));
                p = a * (ct * p1 - b * p2);
            }
            if (l > m) {
                p2 = p1;
                p1 = p;
            }
            if (m == 0) {
                f(l * l + l, p);
            } else {
                f(l * l + l + m, kSqrt2 * p * cm);
                f(l * l + l - m, kSqrt2 * p * sm);
            }
        }
    }
}

// Harmonics surface radius R0 (1 + sum a_lm Y_lm) along body direction p
// (not normalised), |p| = rr, before clipping.
template <typename T>
__device__ __forceinline__ T sh_radius_unclipped(const ShapeParams &sp, T px, T py, T pz, T rr) {
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
    real_sh_all<T>(sp.lmax, ct, st, cphi, sphi, [&](int idx, T y) {
        if (idx > 0) sum += (T)sp.alm[idx] * y;
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

// Body-frame coordinates of a voxel centre, p = R^T (r - c), in double.
__device__ __forceinline__ void body_coords(const ShapeParams &sp, const GridParams &gp, int ix, int iy,
                                            int iz, double &px, double &py, double &pz) {
    double dx = (ix - 0.5 * (gp.nx - 1)) * gp.voxel - sp.cx;
    double dy = (iy - 0.5 * (gp.ny - 1)) * gp.voxel - sp.cy;
    double dz = (iz - 0.5 * (gp.nz - 1)) * gp.voxel - sp.cz;
    px = __dadd_rn(__dadd_rn(__dmul_rn(sp.R[0], dx), __dmul_rn(sp.R[3], dy)), __dmul_rn(sp.R[6], dz));
    py = __dadd_rn(__dadd_rn(__dmul_rn(sp.R[1], dx), __dmul_rn(sp.R[4], dy)), __dmul_rn(sp.R[7], dz));
    pz = __dadd_rn(__dadd_rn(__dmul_rn(sp.R[2], dx), __dmul_rn(sp.R[5], dy)), __dmul_rn(sp.R[8], dz));
}

// Occupancy of one voxel.  Binary decisions are taken in FP64 (explicit
// round-to-nearest operations, no contraction): sphere |d|^2 <= r^2,
// ellipsoid (x/a)^2+(y/b)^2+(z/c)^2 <= 1, harmonics |p| <= r(theta,phi).
// For harmonics the radius is first evaluated in FP32 and only voxels within
// 4e-3 voxel of the surface are re-evaluated in FP64.  Soft occupancy is the
// logistic of the signed distance along the ray from the centre.
template <bool kFp64>
__device__ __forceinline__ double occupancy(const ShapeParams &sp, const GridParams &gp, int ix, int iy,
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
    if (!sp.soft) {
        if (sp.kind == SCATMAN_SPHERE) return p2 <= __dmul_rn(sp.r, sp.r) ? 1.0 : 0.0;
        if (sp.kind == SCATMAN_ELLIPSOID) {
            double u = __ddiv_rn(px, sp.a), v = __ddiv_rn(py, sp.b), w = __ddiv_rn(pz, sp.c);
            double qf = __dadd_rn(__dadd_rn(__dmul_rn(u, u), __dmul_rn(v, v)), __dmul_rn(w, w));
            return qf <= 1.0 ? 1.0 : 0.0;
        }
        double rr = sqrt(p2);
        if (!kFp64) {
            float rf = (float)rr;
            float rs = sh_radius<float>(sp, (float)px, (float)py, (float)pz, rf);
            float margin = rs - rf;
            if (fabsf(margin) > 4e-3f * (float)gp.voxel) return margin > 0.f ? 1.0 : 0.0;
        }
        double rs = sh_radius<double>(sp, px, py, pz, rr);
        return rr <= rs ? 1.0 : 0.0;
    }
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
        float ia = (float)(1.0 / sp.a), ib = (float)(1.0 / sp.b), ic = (float)(1.0 / sp.c);
        rs = rsqrtf(u0 * u0 * ia * ia + u1 * u1 * ib * ib + u2 * u2 * ic * ic);
    } else {
        rs = sh_radius<float>(sp, (float)px, (float)py, (float)pz, rf);
    }
    return (double)(1.0f / (1.0f + __expf(-(rs - rf) * sp.inv_w_f)));
}

}  // namespace scm
