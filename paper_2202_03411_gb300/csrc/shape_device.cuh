// shape_device.cuh -- device-side shape rendering shared by the voxeliser and
// the gradient kernels, so that the backward pass recomputes exactly the
// occupancy the forward pass used.
#pragma once
#include "internal.cuh"

namespace scm {

template <typename T> struct ShTab;
template <> struct ShTab<float> {
    const float *a, *b, *d, *e, *alm;
    float R0, rmin, rmax;
    __device__ explicit ShTab(const ShapeParams &sp)
        : a(sp.sh_af), b(sp.sh_bf), d(sp.sh_df), e(sp.sh_ef), alm(sp.almf), R0(sp.R0f), rmin(sp.rminf),
          rmax(sp.rmaxf) {}
};
template <> struct ShTab<double> {
    const double *a, *b, *d, *e, *alm;
    double R0, rmin, rmax;
    __device__ explicit ShTab(const ShapeParams &sp)
        : a(sp.sh_a), b(sp.sh_b), d(sp.sh_d), e(sp.sh_e), alm(sp.alm), R0(sp.R0), rmin(sp.rmin), rmax(sp.rmax) {}
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
// The loops are unrolled to the largest degree with an early exit at L, so
// every table index and callback index is a compile-time constant (the
// coefficients become constant-bank operands) while the arithmetic and its
// order are those of the plain loops.
// kMaxL: compile-time bound on L (the unrolled code covers degrees up to it).
template <typename T, int kMaxL = SCATMAN_MAX_LMAX, typename F>
__device__ __forceinline__ void real_sh_all(const ShTab<T> &tb, int L, T ct, T st, T cphi, T sphi, F &&f) {
    static_assert(kMaxL >= 0 && kMaxL <= SCATMAN_MAX_LMAX, "degree bound");
    const T kInvSqrt4Pi = (T)0.28209479177387814347;
    const T kSqrt2 = (T)1.41421356237309504880;
    T pmm = kInvSqrt4Pi;
    T cm = (T)1, sm = (T)0;
#pragma unroll
    for (int m = 0; m <= kMaxL; ++m) {
        if (m > L) break;
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
#pragma unroll
        for (int l = m; l <= kMaxL; ++l) {
            if (l > L) break;
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
    }
}

// Harmonics surface radius R0 (1 + sum a_lm Y_lm) along body direction p
// (not normalised), |p| = rr, before clipping.
template <typename T, int kMaxL = SCATMAN_MAX_LMAX>
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
    real_sh_all<T, kMaxL>(tb, sp.lmax, ct, st, cphi, sphi, [&](int idx, T y) {
        if (idx > 0) sum += tb.alm[idx] * y;
    });
    return tb.R0 * ((T)1 + sum);
}

// The same radius clipped to [rmin, rmax].
template <typename T>
__device__ __forceinline__ T sh_radius(const ShapeParams &sp, T px, T py, T pz, T rr) {
    T r = sh_radius_unclipped<T>(sp, px, py, pz, rr);
    const ShTab<T> tb(sp);
    r = r < tb.rmin ? tb.rmin : r;
    r = r > tb.rmax ? tb.rmax : r;
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

// Radius of a radii map (Sec. 5.2 "Shape (2/3)") along the body direction of
// p: latitude atan2(p_z, |p_xy|), longitude atan2(p_y, p_x) in [0, 2 pi);
// samples at latitudes -pi/2 + i pi/ntheta and longitudes 2 pi k/nphi,
// linear in each angle, periodic in both.  The FP64 form keeps the oracle's
// operation order (no contraction into fused multiply-adds).
__device__ __forceinline__ double rmap_radius_d(const ShapeParams &sp, double px, double py, double pz) {
    const double rxy = sqrt(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)));
    const double lat = atan2(pz, rxy);
    double lon = atan2(py, px);
    if (lon < 0.0) lon = __dadd_rn(lon, 2.0 * kPi);
    const double ti = __dmul_rn(__dadd_rn(lat, 0.5 * kPi), sp.rm_tscale);
    const double tk = __dmul_rn(lon, sp.rm_pscale);
    const double fi = floor(ti), fk = floor(tk);
    const double f = __dadd_rn(ti, -fi), g = __dadd_rn(tk, -fk);
    const int nt = sp.ntheta, np = sp.nphi;
    int i0 = (int)fi % nt, k0 = (int)fk % np;
    if (i0 < 0) i0 += nt;
    if (k0 < 0) k0 += np;
    const int i1 = (i0 + 1) % nt, k1 = (k0 + 1) % np;
    const double r00 = sp.rmap[(size_t)i0 * np + k0], r01 = sp.rmap[(size_t)i0 * np + k1];
    const double r10 = sp.rmap[(size_t)i1 * np + k0], r11 = sp.rmap[(size_t)i1 * np + k1];
    const double omf = __dadd_rn(1.0, -f), omg = __dadd_rn(1.0, -g);
    const double t1 = __dmul_rn(__dmul_rn(omf, omg), r00);
    const double t2 = __dmul_rn(__dmul_rn(omf, g), r01);
    const double t3 = __dmul_rn(__dmul_rn(f, omg), r10);
    const double t4 = __dmul_rn(__dmul_rn(f, g), r11);
    return __dadd_rn(__dadd_rn(__dadd_rn(t1, t2), t3), t4);
}
__device__ __forceinline__ float rmap_radius_f(const ShapeParams &sp, float px, float py, float pz) {
    const float lat = atan2f(pz, sqrtf(px * px + py * py));
    float lon = atan2f(py, px);
    if (lon < 0.f) lon += 2.f * (float)kPi;
    const float ti = (lat + 0.5f * (float)kPi) * sp.rm_tscalef;
    const float tk = lon * sp.rm_pscalef;
    const float fi = floorf(ti), fk = floorf(tk);
    const float f = ti - fi, g = tk - fk;
    const int nt = sp.ntheta, np = sp.nphi;
    int i0 = (int)fi % nt, k0 = (int)fk % np;
    if (i0 < 0) i0 += nt;
    if (k0 < 0) k0 += np;
    const int i1 = (i0 + 1) % nt, k1 = (k0 + 1) % np;
    const float r00 = sp.rmapf[(size_t)i0 * np + k0], r01 = sp.rmapf[(size_t)i0 * np + k1];
    const float r10 = sp.rmapf[(size_t)i1 * np + k0], r11 = sp.rmapf[(size_t)i1 * np + k1];
    return (1.f - f) * (1.f - g) * r00 + (1.f - f) * g * r01 + f * (1.f - g) * r10 + f * g * r11;
}

// Volume-map cell (Sec. 5.2 "Shape (3/3)") holding the centre of voxel
// (ix, iy, iz): cell (i, j, k) covers [(i - mx/2) dx, (i + 1 - mx/2) dx) along
// body x and likewise; -1 outside the map.  The FP32 form decides unless a
// cell coordinate lies within its error bound of a cell face; then the FP64
// form (the oracle's operation order) decides.
__device__ __forceinline__ int vmap_cell_fp64(const ShapeParams &sp, double px, double py, double pz) {
    const double ci = floor(__dadd_rn(__ddiv_rn(px, sp.mdx), 0.5 * sp.mx));
    const double cj = floor(__dadd_rn(__ddiv_rn(py, sp.mdx), 0.5 * sp.my));
    const double ck = floor(__dadd_rn(__ddiv_rn(pz, sp.mdx), 0.5 * sp.mz));
    if (ci < 0.0 || cj < 0.0 || ck < 0.0 || ci >= sp.mx || cj >= sp.my || ck >= sp.mz) return -1;
    return ((int)ci * sp.my + (int)cj) * sp.mz + (int)ck;
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
    if (sp.kind == SCATMAN_RADIALMAP) return rr <= rmap_radius_d(sp, px, py, pz) ? 1.0 : 0.0;
    if (sp.kind == SCATMAN_VOLUMEMAP) {
        const int cell = vmap_cell_fp64(sp, px, py, pz);
        return (cell >= 0 && sp.vmap[cell] != 0) ? 1.0 : 0.0;
    }
    double rs = sh_radius<double>(sp, px, py, pz, rr);
    return rr <= rs ? 1.0 : 0.0;
}

// Coefficient tables of the harmonics, staged in shared memory for
// sh_binary_fp64_warp: a and b (kShTri each), d and e (kShDiag each), then alm.
constexpr int kShTri = (SCATMAN_MAX_LMAX + 1) * (SCATMAN_MAX_LMAX + 2) / 2;
constexpr int kShDiag = SCATMAN_MAX_LMAX + 1;
constexpr int kShTabDoubles = 2 * kShTri + 2 * kShDiag + kShDiag * kShDiag;

__device__ __forceinline__ void sh_stage_tables(const ShapeParams &sp, double *tab) {
    for (int k = threadIdx.x; k < kShTabDoubles; k += blockDim.x) {
        double v;
        if (k < kShTri) v = sp.sh_a[k];
        else if (k < 2 * kShTri) v = sp.sh_b[k - kShTri];
        else if (k < 2 * kShTri + kShDiag) v = sp.sh_d[k - 2 * kShTri];
        else if (k < 2 * kShTri + 2 * kShDiag) v = sp.sh_e[k - 2 * kShTri - kShDiag];
        else v = sp.alm[k - 2 * kShTri - 2 * kShDiag];
        tab[k] = v;
    }
}

// The FP64 binary decision of one harmonics voxel by a whole warp (call with
// all 32 lanes; every lane gets the result): the body coordinates and |p| as in
// occupancy_binary_fp64, then lane m (m <= lmax) sums the terms of orders +m
// and -m over l = m..lmax with the recurrences of real_sh_all, and the warp
// adds the lanes' sums.  GB300 runs FP64 at a small fraction of its FP32 rate,
// so the warp's instruction count, not its lane count, sets the cost of the
// near-surface decisions: splitting the orders over lanes cuts it about three-fold.
// Only the summation order differs from occupancy_binary_fp64 (both decide in
// FP64; the oracle evaluates the radius by yet another route).
static __device__ __noinline__ double sh_binary_fp64_warp(const ShapeParams &sp, const GridParams &gp, int ix, int iy,
                                                         int iz, const double *tab) {
    const double *ta = tab, *tb = tab + kShTri, *td = tab + 2 * kShTri, *te = td + kShDiag, *talm = te + kShDiag;
    double px, py, pz;
    body_coords(sp, gp, ix, iy, iz, px, py, pz);
    const double p2 = __dadd_rn(__dadd_rn(__dmul_rn(px, px), __dmul_rn(py, py)), __dmul_rn(pz, pz));
    const double rr = sqrt(p2);
    double ct = 1.0, st = 0.0, cphi = 1.0, sphi = 0.0;
    if (rr > 0.0) {
        ct = pz / rr;
        const double rho = sqrt(px * px + py * py);
        st = rho / rr;
        if (rho > 0.0) {
            cphi = px / rho;
            sphi = py / rho;
        }
    }
    const int L = sp.lmax, m = threadIdx.x & 31;
    double part = 0.0;
    if (m <= L) {
        double pmm = 0.28209479177387814347, cm = 1.0, sm = 0.0;
        for (int k = 1; k <= m; ++k) {
            pmm = td[k] * st * pmm;
            const double c2 = cm * cphi - sm * sphi, s2 = sm * cphi + cm * sphi;
            cm = c2;
            sm = s2;
        }
        const double kSqrt2 = 1.41421356237309504880;
        const double wc = m == 0 ? 1.0 : kSqrt2 * cm, ws = kSqrt2 * sm;
        double q2 = 0.0, q1 = pmm;
        for (int l = m; l <= L; ++l) {
            double p;
            if (l == m) {
                p = pmm;
            } else if (l == m + 1) {
                p = te[m] * ct * pmm;
            } else {
                const int i = l * (l + 1) / 2 + m;
                p = ta[i] * (ct * q1 - tb[i] * q2);
            }
            if (l > m) {
                q2 = q1;
                q1 = p;
            }
            if (l == 0) continue;                     // a_00 is not a coefficient
            if (m == 0)
                part += talm[l * l + l] * p;
            else
                part += talm[l * l + l + m] * (p * wc) + talm[l * l + l - m] * (p * ws);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    double rs = sp.R0 * (1.0 + part);
    rs = rs < sp.rmin ? sp.rmin : rs;
    rs = rs > sp.rmax ? sp.rmax : rs;
    return rr <= rs ? 1.0 : 0.0;
}

// Volume-map cell of voxel (ix, iy, iz) in either precision (see vmap_cell_fp64).
template <bool kFp64>
__device__ __forceinline__ int vmap_cell(const ShapeParams &sp, const GridParams &gp, int ix, int iy, int iz) {
    if (!kFp64) {
        const float vox = gp.voxf;
        const float dx = ((float)ix - 0.5f * (float)(gp.nx - 1)) * vox - sp.cxf;
        const float dy = ((float)iy - 0.5f * (float)(gp.ny - 1)) * vox - sp.cyf;
        const float dz = ((float)iz - 0.5f * (float)(gp.nz - 1)) * vox - sp.czf;
        const float px = sp.Rf[0] * dx + sp.Rf[3] * dy + sp.Rf[6] * dz;
        const float py = sp.Rf[1] * dx + sp.Rf[4] * dy + sp.Rf[7] * dz;
        const float pz = sp.Rf[2] * dx + sp.Rf[5] * dy + sp.Rf[8] * dz;
        const float ci = px / sp.mdxf + 0.5f * (float)sp.mx;
        const float cj = py / sp.mdxf + 0.5f * (float)sp.my;
        const float ck = pz / sp.mdxf + 0.5f * (float)sp.mz;
        // error bound of a cell coordinate: the rotated position to ~1e-6 of
        // its size plus the division and the offset
        const float d = fabsf(dx) + fabsf(dy) + fabsf(dz) + vox;
        const float tol = 1e-4f + 4e-6f * d / sp.mdxf + 4e-7f * (float)(sp.mx + sp.my + sp.mz);
        const float fi = ci - floorf(ci), fj = cj - floorf(cj), fk = ck - floorf(ck);
        const bool clear = fi > tol && fi < 1.f - tol && fj > tol && fj < 1.f - tol && fk > tol && fk < 1.f - tol;
        if (clear) {
            const int i = (int)floorf(ci), j = (int)floorf(cj), k = (int)floorf(ck);
            if (i < 0 || j < 0 || k < 0 || i >= sp.mx || j >= sp.my || k >= sp.mz) return -1;
            return (i * sp.my + j) * sp.mz + k;
        }
    }
    double px, py, pz;
    body_coords(sp, gp, ix, iy, iz, px, py, pz);
    return vmap_cell_fp64(sp, px, py, pz);
}

// Occupancy of one voxel.  Binary decisions are the FP64 ones above; the
// FP32 modes first evaluate the same quantity in FP32 and only fall back to
// FP64 when the margin is within a bound well above the FP32 error
// (1e-4 relative for sphere and ellipsoid, 4e-3 voxel for harmonics), so the
// decision always equals the FP64 one.  Soft occupancy is the logistic of
// the signed distance to the surface along the ray from the centre; the FP32
// modes set it to zero where the logistic is below 2^-24 (soft_zero()), the
// FP64 mode keeps the exact logistic everywhere.
// kMaps: compiled for the map kinds (radii and volume maps); the parametric
// kinds' instantiation carries none of their code.
// kDefer (FP32 modes): a binary voxel the FP32 test cannot settle returns -1
// instead of taking the FP64 path here, so the caller can batch those voxels.
// Soft occupancy cut of the FP32 modes (kSoftCutT): without the cut every voxel of the grid has chi > 0 (the logistic never
// vanishes) and the contraction cannot skip the empty part of a slice.  The
// dropped voxels change the field by at most |n^2 - 1| times their summed
// occupancy (each below 2^-24; 3e-9 to 4e-9 of the total occupancy for
// 128^3 shapes at w = 0.5 voxel), and the gradient applies the same cut, so
// it stays the derivative of the function the forward computes.
__device__ __forceinline__ bool soft_zero(float t) { return t < -kSoftCutT; }

template <bool kFp64, bool kMaps = false, bool kDefer = false,
          typename OccT = typename std::conditional<kFp64, double, float>::type>
__device__ __forceinline__ OccT occupancy(const ShapeParams &sp, const GridParams &gp, int ix, int iy, int iz) {
    if (kMaps && sp.kind == SCATMAN_VOLUMEMAP) {
        // binary in both modes: a volume map has no surface radius
        const int cell = vmap_cell<kFp64>(sp, gp, ix, iy, iz);
        return (cell >= 0 && sp.vmap[cell] != 0) ? (OccT)1 : (OccT)0;
    }
    if (!sp.soft) {
        if (!kFp64) {
            const float vox = gp.voxf;
            const float dx = ((float)ix - 0.5f * (float)(gp.nx - 1)) * vox - sp.cxf;
            const float dy = ((float)iy - 0.5f * (float)(gp.ny - 1)) * vox - sp.cyf;
            const float dz = ((float)iz - 0.5f * (float)(gp.nz - 1)) * vox - sp.czf;
            if (sp.kind == SCATMAN_SPHERE) {
                const float r2 = sp.r2f;
                const float m = r2 - (dx * dx + dy * dy + dz * dz);
                if (fabsf(m) > 1e-4f * r2 + 1e-6f) return m > 0.f ? (OccT)1 : (OccT)0;
            } else {
                const float px = sp.Rf[0] * dx + sp.Rf[3] * dy + sp.Rf[6] * dz;
                const float py = sp.Rf[1] * dx + sp.Rf[4] * dy + sp.Rf[7] * dz;
                const float pz = sp.Rf[2] * dx + sp.Rf[5] * dy + sp.Rf[8] * dz;
                if (sp.kind == SCATMAN_ELLIPSOID) {
                    const float u = px * sp.inv_af, v = py * sp.inv_bf, w = pz * sp.inv_cf;
                    const float m = 1.f - (u * u + v * v + w * w);
                    if (fabsf(m) > 1e-4f) return m > 0.f ? (OccT)1 : (OccT)0;
                } else if (kMaps && sp.kind == SCATMAN_RADIALMAP) {
                    const float rr = sqrtf(px * px + py * py + pz * pz);
                    const float rs = rmap_radius_f(sp, px, py, pz);
                    const float m = rs - rr;
                    // FP32 error bound: angles to ~2e-6 rad (worse near the
                    // centre) times the map's steepest slope, plus rounding
                    const float margin = 4e-3f * vox + 1e-6f * (fabsf(rs) + rr) +
                                         sp.rm_slope * (2e-6f + 2e-5f / fmaxf(rr, vox));
                    if (fabsf(m) > margin) return m > 0.f ? (OccT)1 : (OccT)0;
                } else {
                    const float rr = sqrtf(px * px + py * py + pz * pz);
                    const float rs = sh_radius<float>(sp, px, py, pz, rr);
                    const float m = rs - rr;
                    if (fabsf(m) > 4e-3f * vox) return m > 0.f ? (OccT)1 : (OccT)0;
                }
            }
        }
        if (kDefer && !kFp64) return (OccT)-1;
        return (OccT)occupancy_binary_fp64(sp, gp, ix, iy, iz);
    }
    if constexpr (kFp64) {
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
        double rs;
        if (sp.kind == SCATMAN_SPHERE) {
            rs = sp.r;
        } else if (sp.kind == SCATMAN_ELLIPSOID) {
            double u0 = 0, u1 = 0, u2 = 1;
            if (rr > 0) { u0 = px / rr; u1 = py / rr; u2 = pz / rr; }
            rs = 1.0 / sqrt((u0 / sp.a) * (u0 / sp.a) + (u1 / sp.b) * (u1 / sp.b) + (u2 / sp.c) * (u2 / sp.c));
        } else if (kMaps && sp.kind == SCATMAN_RADIALMAP) {
            rs = rmap_radius_d(sp, px, py, pz);
        } else {
            rs = sh_radius<double>(sp, px, py, pz, rr);
        }
        return (OccT)(1.0 / (1.0 + exp(-(rs - rr) * sp.inv_w)));
    } else {
        // FP32 modes: FP32 body coordinates, as the gradient's voxel pass forms
        // them (the logistic is smooth: their rounding moves chi by ~1e-6 at
        // most, and no FP64 arithmetic runs per voxel)
        const float vox = gp.voxf;
        const float dx = ((float)ix - 0.5f * (float)(gp.nx - 1)) * vox - sp.cxf;
        const float dy = ((float)iy - 0.5f * (float)(gp.ny - 1)) * vox - sp.cyf;
        const float dz = ((float)iz - 0.5f * (float)(gp.nz - 1)) * vox - sp.czf;
        float px = dx, py = dy, pz = dz;
        if (sp.kind != SCATMAN_SPHERE) {
            px = sp.Rf[0] * dx + sp.Rf[3] * dy + sp.Rf[6] * dz;
            py = sp.Rf[1] * dx + sp.Rf[4] * dy + sp.Rf[7] * dz;
            pz = sp.Rf[2] * dx + sp.Rf[5] * dy + sp.Rf[8] * dz;
        }
        const float rf = sqrtf(px * px + py * py + pz * pz);
        float rs;
        if (sp.kind == SCATMAN_SPHERE) {
            rs = (float)sp.r;
        } else if (sp.kind == SCATMAN_ELLIPSOID) {
            float u0 = 0.f, u1 = 0.f, u2 = 1.f;
            if (rf > 0.f) { u0 = px / rf; u1 = py / rf; u2 = pz / rf; }
            const float ia = sp.inv_af, ib = sp.inv_bf, ic = sp.inv_cf;
            rs = rsqrtf(u0 * u0 * ia * ia + u1 * u1 * ib * ib + u2 * u2 * ic * ic);
        } else if (kMaps && sp.kind == SCATMAN_RADIALMAP) {
            rs = rmap_radius_f(sp, px, py, pz);
        } else {
            rs = sh_radius<float>(sp, px, py, pz, rf);
        }
        const float t = (rs - rf) * sp.inv_w_f;
        if (soft_zero(t)) return (OccT)0;
        return (OccT)(1.0f / (1.0f + __expf(-t)));
    }
}

}  // namespace scm
