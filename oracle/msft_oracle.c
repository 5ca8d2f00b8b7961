/*
 * msft_oracle.c -- plain, slow FP64 CPU oracle of the Multi-Slice Fourier
 * Transform (MSFT) as "The Scatman" (arXiv 2202.03411) defines it.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  It shares no code,
 * header, table or constant with the CUDA library; the two only share the
 * seeded input generators (workloads/), which hold none of the arithmetic.
 *
 * Every function follows one passage of the paper and is written for a reader
 * to check against it by eye: no blocking, no fusion, no reordering beyond
 * what the equation states.  The only liberty taken is precomputing per-pixel
 * phase tables e^{-i q_x x}, e^{-i q_y y}, e^{-i q_z z} (a factorisation of
 * the same exponential, exact up to rounding).
 *
 * Conventions (readings of passages where the paper is silent or ambiguous):
 *  - q = k_out - k_in with k_in = k0 z^; the phase is e^{-i q.r}.  This is
 *    Eq. 9 rewritten: E_s carries e^{i k0 s dz} and the slice prefactor is
 *    e^{-i k_z s dz}, so the net z-phase is e^{-i (k_z - k0) z}.
 *  - Flat detector normal to z at distance D=1; theta_max is reached at the
 *    edge midpoints; pixel centres X_u = tan(theta_max) (2u+1-N)/N.
 *  - Voxel centres are (index - (N-1)/2) * voxel; the shape centre is the
 *    grid centre plus an offset.
 *  - Slice strength is linear in the occupancy chi (Eq. 2 defines the slice
 *    strength as the slice integral of rho, and rho ~ n^2-1 inside the shape);
 *    propagation uses the slice-averaged index n~ - 1 = chi (n-1) (Eq. 8).
 *  - E_0 = 1 on slice 0 and slice j sees only slices < j (Eq. 8-9): the
 *    transmission is an EXCLUSIVE product along z.
 *  - Prefactor of the proportionality in Eq. 9 is 1.
 *
 * Array layouts: voxel arrays are [z][x][y] (y fastest); q arrays are
 * [pixel][3]; detector pixel p = v*det_nx + u.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <complex.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_SPHERE 0
#define ORC_ELLIPSOID 1
#define ORC_SPHHARM 2
#define ORC_RADIALMAP 3
#define ORC_VOLUMEMAP 4

/* Shape parameters as in the paper's Listings 1-2 (Sec. 5). */
typedef struct {
    int kind;
    double r, a, b, c;          /* sphere radius; ellipsoid semi-axes (c on the main axis) */
    double R0;                  /* harmonics mean radius */
    int lmax;
    const double *alm;          /* (lmax+1)^2 coefficients, index l*l+l+m, alm[0] unused */
    double delta, beta;         /* n = 1 - delta + i beta (Eq. 7) */
    double latitude, longitude, rotation;   /* degrees (Fig. 6) */
    double cx, cy, cz;          /* centre offset from the grid centre */
    /* radii map (Sec. 5.2 "Shape (2/3)"): [n_theta][n_phi], length units */
    const double *radial_map;
    int map_ntheta, map_nphi;
    /* volume map (Sec. 5.2 "Shape (3/3)"): [mx][my][mz], non-zero = inside, cell edge map_dx */
    const unsigned char *volume_map;
    int map_nx, map_ny, map_nz;
    double map_dx;
    const double *map_delta, *map_beta;   /* optional per-cell index (NULL: the shape's) */
} orc_shape;

static const double ORC_PI = 3.14159265358979323846;

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* cos and sin of an angle in degrees, exact at multiples of 90 degrees so
 * that axis-aligned orientations give exact rotation matrices. */
static void orc_cos_sin_deg(double deg, double *c, double *s)
{
    double q = deg / 90.0;
    if (q == floor(q)) {
        long k = ((long)q % 4 + 4) % 4;
        static const double cs[4] = {1.0, 0.0, -1.0, 0.0};
        static const double sn[4] = {0.0, 1.0, 0.0, -1.0};
        *c = cs[k];
        *s = sn[k];
        return;
    }
    double rad = deg * ORC_PI / 180.0;
    *c = cos(rad);
    *s = sin(rad);
}

static void orc_matmul3(const double A[9], const double B[9], double C[9])
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += A[3 * i + k] * B[3 * k + j];
            C[3 * i + j] = acc;
        }
}

/*
 * Body-to-lab rotation (Fig. 6 caption, Sec. 5.1 "Define a shape"):
 * the main axis (body z) points along latitude/longitude, where +90 deg
 * latitude points towards the incoming beam (-z) and longitude is measured
 * from +x towards +y; afterwards the body is spun about its main axis.
 * R = Rz(longitude) * Ry(90 deg + latitude) * Rz(rotation).  Row-major.
 */
void orc_rotation(double lat, double lon, double rot, double R[9])
{
    double c1, s1, c2, s2, c3, s3;
    orc_cos_sin_deg(lon, &c1, &s1);
    orc_cos_sin_deg(90.0 + lat, &c2, &s2);
    orc_cos_sin_deg(rot, &c3, &s3);
    double Rz1[9] = {c1, -s1, 0, s1, c1, 0, 0, 0, 1};
    double Ry[9] = {c2, 0, s2, 0, 1, 0, -s2, 0, c2};
    double Rz3[9] = {c3, -s3, 0, s3, c3, 0, 0, 0, 1};
    double T[9];
    orc_matmul3(Rz1, Ry, T);
    orc_matmul3(T, Rz3, R);
}

/* Associated Legendre function P_l^m(x), m >= 0, including the
 * Condon-Shortley phase (-1)^m; Eq. 11 gives the negative-m relation.
 * Standard upward recurrence in l. */
double orc_legendre(int l, int m, double x)
{
    double pmm = 1.0;
    double sx = sqrt((1.0 - x) * (1.0 + x));
    for (int k = 1; k <= m; ++k) pmm *= -(2.0 * k - 1.0) * sx;
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pl = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pl = ((2.0 * ll - 1.0) * x * pm1 - (ll + m - 1.0) * pmm) / (ll - m);
        pmm = pm1;
        pm1 = pl;
    }
    return pl;
}

/* Real orthonormal spherical harmonic built from Eq. 10's complex Y_l^m:
 * m > 0: sqrt(2) Re Y_l^m;  m < 0: sqrt(2) Im Y_l^{|m|};  m = 0: Y_l^0.
 * theta is the polar angle from the body z axis, phi the azimuth from body x. */
double orc_real_sh(int l, int m, double theta, double phi)
{
    int am = m < 0 ? -m : m;
    double ratio = 1.0;                     /* (l-|m|)! / (l+|m|)! */
    for (int k = l - am + 1; k <= l + am; ++k) ratio /= (double)k;
    double norm = sqrt((2.0 * l + 1.0) / (4.0 * ORC_PI) * ratio);
    double p = orc_legendre(l, am, cos(theta));
    if (m == 0) return norm * p;
    if (m > 0) return sqrt(2.0) * norm * p * cos(am * phi);
    return sqrt(2.0) * norm * p * sin(am * phi);
}

static double orc_half_width(int nx, int ny, int nz, double voxel)
{
    int n = nx < ny ? nx : ny;
    if (nz < n) n = nz;
    return 0.5 * (n - 1) * voxel;
}

/* Harmonics surface radius r(theta,phi) = R0 (1 + sum_{1<=l<=L} a_lm Y_lm)
 * (Sec. 5.2 "Shape (1/3)", Eq. 10-11), clipped to [0.1 R0, hw - voxel]. */
static double orc_sh_radius(const orc_shape *sh, double theta, double phi,
                            double rmax, int *clipped)
{
    double sum = 0.0;
    for (int l = 1; l <= sh->lmax; ++l)
        for (int m = -l; m <= l; ++m)
            sum += sh->alm[l * l + l + m] * orc_real_sh(l, m, theta, phi);
    double r = sh->R0 * (1.0 + sum);
    *clipped = 0;
    if (r < 0.1 * sh->R0) { r = 0.1 * sh->R0; *clipped = 1; }
    if (r > rmax) { r = rmax; *clipped = 1; }
    return r;
}

static double orc_sigmoid(double t) { return 1.0 / (1.0 + exp(-t)); }

/*
 * Sec. 5.2 "Shape (2/3)": radius of a radii map along the body direction of p
 * (|p| = rr).  The map holds radii at latitudes lat_i = -pi/2 + i pi/Nt and
 * longitudes lon_k = 2 pi k/Np (an N x M map covers latitudes -pi/2 .. pi/2 -
 * pi/Nt, as the paper's 4x4 example), linearly interpolated in each angle.
 * Reading: the interpolation is periodic in both angles (after the last
 * latitude row comes row 0, after the last longitude column comes column 0);
 * latitude = atan2(p_z, sqrt(p_x^2 + p_y^2)) (+pi/2 on the body z axis; the
 * same angle as asin(p_z/|p|), better conditioned at the poles), longitude =
 * atan2(p_y, p_x) in [0, 2 pi).
 */
static double orc_rmap_radius(const orc_shape *sh, const double p[3], double rr)
{
    int nt = sh->map_ntheta, np = sh->map_nphi;
    (void)rr;
    double lat = atan2(p[2], sqrt(p[0] * p[0] + p[1] * p[1]));
    double lon = atan2(p[1], p[0]);
    if (lon < 0.0) lon += 2.0 * ORC_PI;
    double ti = (lat + 0.5 * ORC_PI) * ((double)nt / ORC_PI);
    double tk = lon * ((double)np / (2.0 * ORC_PI));
    double fi = floor(ti), fk = floor(tk);
    double f = ti - fi, g = tk - fk;
    int i0 = (int)fi % nt, k0 = (int)fk % np;
    if (i0 < 0) i0 += nt;
    if (k0 < 0) k0 += np;
    int i1 = (i0 + 1) % nt, k1 = (k0 + 1) % np;
    const double *R = sh->radial_map;
    double r00 = R[(size_t)i0 * np + k0], r01 = R[(size_t)i0 * np + k1];
    double r10 = R[(size_t)i1 * np + k0], r11 = R[(size_t)i1 * np + k1];
    return (1.0 - f) * (1.0 - g) * r00 + (1.0 - f) * g * r01 + f * (1.0 - g) * r10 + f * g * r11;
}

/*
 * Sec. 5.2 "Shape (3/3)": cell of a volume map that contains the body point p.
 * Cell (i, j, k) covers [(i - Mx/2) dx, (i + 1 - Mx/2) dx) along body x and
 * likewise along y and z (the map is centred on the shape centre and turns
 * with the body).  Returns -1 outside the map.
 */
static long orc_vmap_cell(const orc_shape *sh, const double p[3])
{
    double ci = floor(p[0] / sh->map_dx + 0.5 * sh->map_nx);
    double cj = floor(p[1] / sh->map_dx + 0.5 * sh->map_ny);
    double ck = floor(p[2] / sh->map_dx + 0.5 * sh->map_nz);
    if (ci < 0.0 || cj < 0.0 || ck < 0.0 || ci >= sh->map_nx || cj >= sh->map_ny || ck >= sh->map_nz) return -1;
    return ((long)ci * sh->map_ny + (long)cj) * sh->map_nz + (long)ck;
}

/* Body-frame coordinates of voxel centre (ix,iy,iz). */
static void orc_body_coords(const orc_shape *sh, const double R[9], int ix, int iy, int iz,
                            int nx, int ny, int nz, double voxel, double p[3])
{
    double d[3];
    d[0] = (ix - 0.5 * (nx - 1)) * voxel - sh->cx;
    d[1] = (iy - 0.5 * (ny - 1)) * voxel - sh->cy;
    d[2] = (iz - 0.5 * (nz - 1)) * voxel - sh->cz;
    /* p = R^T d */
    for (int i = 0; i < 3; ++i) p[i] = R[0 + i] * d[0] + R[3 + i] * d[1] + R[6 + i] * d[2];
}

/*
 * Block 5 (Sec. 3.2, "render the slice's scattering potential"): occupancy
 * chi of every voxel, [z][x][y].  Binary (soft==0): the voxel centre is
 * inside (ties count as inside) -- sphere |p|^2 <= r^2, ellipsoid
 * (x/a)^2+(y/b)^2+(z/c)^2 <= 1, harmonics |p| <= r(theta,phi).  Soft:
 * chi = sigmoid((r_s(p^) - |p|)/w) with r_s the surface radius along the
 * voxel's direction from the centre.  Returns 1 if a harmonics radius was
 * clipped.
 */
int orc_voxelise(const orc_shape *sh, int nx, int ny, int nz, double voxel,
                 int soft, double w, double *chi)
{
    double R[9];
    orc_rotation(sh->latitude, sh->longitude, sh->rotation, R);
    double rmax = orc_half_width(nx, ny, nz, voxel) - voxel;
    int any_clip = 0;
#pragma omp parallel for collapse(2) reduction(| : any_clip)
    for (int iz = 0; iz < nz; ++iz)
        for (int ix = 0; ix < nx; ++ix)
            for (int iy = 0; iy < ny; ++iy) {
                double p[3];
                orc_body_coords(sh, R, ix, iy, iz, nx, ny, nz, voxel, p);
                double rr = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
                double v;
                if (!soft) {
                    if (sh->kind == ORC_SPHERE) {
                        v = (p[0] * p[0] + p[1] * p[1] + p[2] * p[2] <= sh->r * sh->r) ? 1.0 : 0.0;
                    } else if (sh->kind == ORC_ELLIPSOID) {
                        double qf = (p[0] / sh->a) * (p[0] / sh->a) + (p[1] / sh->b) * (p[1] / sh->b)
                                    + (p[2] / sh->c) * (p[2] / sh->c);
                        v = (qf <= 1.0) ? 1.0 : 0.0;
                    } else if (sh->kind == ORC_RADIALMAP) {
                        v = (rr <= orc_rmap_radius(sh, p, rr)) ? 1.0 : 0.0;
                    } else if (sh->kind == ORC_VOLUMEMAP) {
                        long cell = orc_vmap_cell(sh, p);
                        v = (cell >= 0 && sh->volume_map[cell] != 0) ? 1.0 : 0.0;
                    } else {
                        double th = rr > 0.0 ? acos(p[2] / rr) : 0.0;
                        double ph = atan2(p[1], p[0]);
                        int cl;
                        double rs = orc_sh_radius(sh, th, ph, rmax, &cl);
                        any_clip |= cl;
                        v = (rr <= rs) ? 1.0 : 0.0;
                    }
                } else if (sh->kind == ORC_VOLUMEMAP) {
                    /* a volume map has no surface radius: its occupancy stays binary */
                    long cell = orc_vmap_cell(sh, p);
                    v = (cell >= 0 && sh->volume_map[cell] != 0) ? 1.0 : 0.0;
                } else {
                    double rs;
                    if (sh->kind == ORC_SPHERE) {
                        rs = sh->r;
                    } else if (sh->kind == ORC_ELLIPSOID) {
                        double u0 = 0.0, u1 = 0.0, u2 = 1.0;
                        if (rr > 0.0) { u0 = p[0] / rr; u1 = p[1] / rr; u2 = p[2] / rr; }
                        rs = 1.0 / sqrt((u0 / sh->a) * (u0 / sh->a) + (u1 / sh->b) * (u1 / sh->b)
                                        + (u2 / sh->c) * (u2 / sh->c));
                    } else if (sh->kind == ORC_RADIALMAP) {
                        rs = orc_rmap_radius(sh, p, rr);
                    } else {
                        double th = rr > 0.0 ? acos(p[2] / rr) : 0.0;
                        double ph = atan2(p[1], p[0]);
                        int cl;
                        rs = orc_sh_radius(sh, th, ph, rmax, &cl);
                        any_clip |= cl;
                    }
                    v = orc_sigmoid((rs - rr) / w);
                }
                chi[((size_t)iz * nx + ix) * ny + iy] = v;
            }
    return any_clip;
}

/*
 * Eq. 5-9 and Blocks 4 + 9: effective slice strength
 *   rho_j(x,y) = (n^2 - 1) chi_j(x,y) E_j(x,y) / (E_0 e^{i k0 j dz})
 * with the projection-approximation recursion of Eq. 8,
 *   E_j = E_{j-1} e^{i k0 dz n~_{j-1}},  E_0 = 1 (Block 4: plane wave),
 *   n~_{j-1} - 1 = chi_{j-1} (n - 1),  n = 1 - delta + i beta (Eq. 7).
 * Dividing out the free-space phase e^{i k0 j dz} leaves the running product
 *   T_j = prod_{j'<j} e^{i k0 dz chi_{j'} (n-1)}.
 * Output [z][x][y], real and imaginary parts in separate arrays.
 */
void orc_slices(const double *chi, int nx, int ny, int nz, double dz, double wavelength,
                double delta, double beta, double *rho_re, double *rho_im)
{
    double k0 = 2.0 * ORC_PI / wavelength;
    double complex n = 1.0 - delta + I * beta;
    double complex strength = n * n - 1.0;
#pragma omp parallel for collapse(2)
    for (int ix = 0; ix < nx; ++ix)
        for (int iy = 0; iy < ny; ++iy) {
            double complex T = 1.0;                 /* E_0 / E_0 */
            for (int iz = 0; iz < nz; ++iz) {
                size_t idx = ((size_t)iz * nx + ix) * ny + iy;
                double complex rho = strength * chi[idx] * T;
                rho_re[idx] = creal(rho);
                rho_im[idx] = cimag(rho);
                /* Block 9: propagate through slice iz for the next slice */
                T = T * cexp(I * k0 * dz * chi[idx] * (n - 1.0));
            }
        }
}

/*
 * Refractive index of every voxel for a volume map with per-cell delta and
 * beta (the paper's "arbitrary voxel representation of the refractive index",
 * Sec. 5.2): the cell's values for voxels inside the map, the shape's
 * elsewhere (where chi = 0 anyway).  [z][x][y].
 */
void orc_voxel_index(const orc_shape *sh, int nx, int ny, int nz, double voxel, double *delta_v,
                     double *beta_v)
{
    double R[9];
    orc_rotation(sh->latitude, sh->longitude, sh->rotation, R);
#pragma omp parallel for collapse(2)
    for (int iz = 0; iz < nz; ++iz)
        for (int ix = 0; ix < nx; ++ix)
            for (int iy = 0; iy < ny; ++iy) {
                double p[3];
                orc_body_coords(sh, R, ix, iy, iz, nx, ny, nz, voxel, p);
                long cell = orc_vmap_cell(sh, p);
                size_t idx = ((size_t)iz * nx + ix) * ny + iy;
                delta_v[idx] = (cell >= 0 && sh->map_delta) ? sh->map_delta[cell] : sh->delta;
                beta_v[idx] = (cell >= 0 && sh->map_beta) ? sh->map_beta[cell] : sh->beta;
            }
}

/*
 * Eq. 5-9 with a voxel-resolved index: as orc_slices, but every voxel carries
 * its own n_v = 1 - delta_v + i beta_v, both in the slice strength
 * (n_v^2 - 1) chi and in the propagation of Eq. 8,
 *   T_j = prod_{j'<j} e^{i k0 dz chi_{j'} (n_{j'} - 1)}.
 */
void orc_slices_n(const double *chi, const double *delta_v, const double *beta_v, int nx, int ny, int nz,
                  double dz, double wavelength, double *rho_re, double *rho_im)
{
    double k0 = 2.0 * ORC_PI / wavelength;
#pragma omp parallel for collapse(2)
    for (int ix = 0; ix < nx; ++ix)
        for (int iy = 0; iy < ny; ++iy) {
            double complex T = 1.0;
            for (int iz = 0; iz < nz; ++iz) {
                size_t idx = ((size_t)iz * nx + ix) * ny + iy;
                double complex n = 1.0 - delta_v[idx] + I * beta_v[idx];
                double complex rho = (n * n - 1.0) * chi[idx] * T;
                rho_re[idx] = creal(rho);
                rho_im[idx] = cimag(rho);
                T = T * cexp(I * k0 * dz * chi[idx] * (n - 1.0));
            }
        }
}

/*
 * Eq. 3 and Block 1 + 3: transfer momentum of every pixel of a flat detector
 * normal to the beam.  Pixel (u,v) sits at (X_u, Y_v, 1) with
 * X_u = tan(theta_max) (2u+1-Nx)/Nx; its scattering angle is
 * theta = atan(sqrt(X^2+Y^2)) and azimuth phi = atan2(Y,X); k_out is
 * k0 (sin th cos ph, sin th sin ph, cos th) on the Ewald sphere and
 * q = k_out - k_in, so q_z = -k0 (1 - cos theta) (Eq. 3 up to the sign
 * convention stated in the header).
 */
void orc_detector_q(int det_nx, int det_ny, double theta_max_deg, double wavelength, double *q)
{
    double k0 = 2.0 * ORC_PI / wavelength;
    double h = tan(theta_max_deg * ORC_PI / 180.0);
    for (int v = 0; v < det_ny; ++v)
        for (int u = 0; u < det_nx; ++u) {
            double X = h * (2.0 * u + 1.0 - det_nx) / det_nx;
            double Y = h * (2.0 * v + 1.0 - det_ny) / det_ny;
            double th = atan(sqrt(X * X + Y * Y));
            double ph = atan2(Y, X);
            size_t p = (size_t)v * det_nx + u;
            q[3 * p + 0] = k0 * sin(th) * cos(ph);
            q[3 * p + 1] = k0 * sin(th) * sin(ph);
            q[3 * p + 2] = k0 * (cos(th) - 1.0);
        }
}

/*
 * The paper's own virtual detector (Block 1; Block 6's per-slice DFT on a
 * uniform grid): pixel centres uniform in the transverse momentum,
 * q_x(u) = q_max (2u+1-Nx)/Nx, q_y(v) likewise, q_max = k0 sin(theta_max),
 * and q_z on the Ewald sphere from Eq. 3, q_z = k0 (cos(theta) - 1) with
 * cos(theta) = sqrt(1 - (q_x^2 + q_y^2)/k0^2).  Pixels with
 * q_x^2 + q_y^2 > k0^2 have no scattering direction: valid[p] = 0 there
 * (and q_z is set to -k0).
 */
void orc_detector_q_uniform(int det_nx, int det_ny, double theta_max_deg, double wavelength, double *q,
                            int *valid)
{
    double k0 = 2.0 * ORC_PI / wavelength;
    double qmax = k0 * sin(theta_max_deg * ORC_PI / 180.0);
    for (int v = 0; v < det_ny; ++v)
        for (int u = 0; u < det_nx; ++u) {
            size_t p = (size_t)v * det_nx + u;
            double qx = qmax * (2.0 * u + 1.0 - det_nx) / det_nx;
            double qy = qmax * (2.0 * v + 1.0 - det_ny) / det_ny;
            double s2 = (qx * qx + qy * qy) / (k0 * k0);
            q[3 * p + 0] = qx;
            q[3 * p + 1] = qy;
            if (s2 <= 1.0) {
                double cth = sqrt(1.0 - s2);
                q[3 * p + 2] = k0 * (cth - 1.0);
                valid[p] = 1;
            } else {
                q[3 * p + 2] = -k0;
                valid[p] = 0;
            }
        }
}

/*
 * Eq. 9 (Blocks 6-8, 10): the scattered field at each q,
 *   A(q) = sum_j e^{-i q_z z_j} F[rho_j](q_x, q_y),
 *   F[rho_j](q_x, q_y) = sum_{x,y} rho_j(x,y) e^{-i (q_x x + q_y y)},
 * slice by slice as the main loop does (Block 6: per-slice Fourier sum;
 * Block 7: slice phase; Block 8: accumulate).  The Fourier "transform" is
 * the direct non-uniform sum at the detector's q.
 */
void orc_msft(const double *rho_re, const double *rho_im, int nx, int ny, int nz, double voxel,
              const double *q, long n_q, double *A_re, double *A_im)
{
#pragma omp parallel
    {
        double complex *ex = malloc(sizeof(double complex) * nx);
        double complex *ey = malloc(sizeof(double complex) * ny);
#pragma omp for schedule(dynamic, 4)
        for (long p = 0; p < n_q; ++p) {
            double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
            for (int ix = 0; ix < nx; ++ix) {
                double x = (ix - 0.5 * (nx - 1)) * voxel;
                ex[ix] = cexp(-I * qx * x);
            }
            for (int iy = 0; iy < ny; ++iy) {
                double y = (iy - 0.5 * (ny - 1)) * voxel;
                ey[iy] = cexp(-I * qy * y);
            }
            double complex A = 0.0;
            for (int iz = 0; iz < nz; ++iz) {
                double z = (iz - 0.5 * (nz - 1)) * voxel;
                double complex F = 0.0;            /* Block 6 */
                for (int ix = 0; ix < nx; ++ix)
                    for (int iy = 0; iy < ny; ++iy) {
                        size_t idx = ((size_t)iz * nx + ix) * ny + iy;
                        F += (rho_re[idx] + I * rho_im[idx]) * ex[ix] * ey[iy];
                    }
                A += cexp(-I * qz * z) * F;        /* Blocks 7-8 */
            }
            A_re[p] = creal(A);
            A_im[p] = cimag(A);
        }
        free(ex);
        free(ey);
    }
}

/* Block 11: I = |A|^2. */
void orc_intensity(const double *A_re, const double *A_im, long n_q, double *I_out)
{
    for (long p = 0; p < n_q; ++p) I_out[p] = A_re[p] * A_re[p] + A_im[p] * A_im[p];
}

/*
 * Adjoint of the linear map rho -> A of Eq. 9:
 *   S(r_v) = sum_q g_q e^{+i q . r_v},  [z][x][y],
 * so that sum_q conj(A(rho)_q) g_q = sum_v conj(rho_v) S_v.  Each thread owns
 * whole slices and walks every q with the same per-q phase tables as the
 * forward sum.
 */
void orc_msft_adjoint(const double *g_re, const double *g_im, const double *q, long n_q,
                      int nx, int ny, int nz, double voxel, double *S_re, double *S_im)
{
#pragma omp parallel
    {
        double complex *ex = malloc(sizeof(double complex) * nx);
        double complex *ey = malloc(sizeof(double complex) * ny);
        double complex *acc = malloc(sizeof(double complex) * (size_t)nx * ny);
#pragma omp for schedule(dynamic, 1)
        for (int iz = 0; iz < nz; ++iz) {
            double z = (iz - 0.5 * (nz - 1)) * voxel;
            for (size_t k = 0; k < (size_t)nx * ny; ++k) acc[k] = 0.0;
            for (long p = 0; p < n_q; ++p) {
                double qx = q[3 * p], qy = q[3 * p + 1], qz = q[3 * p + 2];
                for (int ix = 0; ix < nx; ++ix) ex[ix] = cexp(I * qx * ((ix - 0.5 * (nx - 1)) * voxel));
                for (int iy = 0; iy < ny; ++iy) ey[iy] = cexp(I * qy * ((iy - 0.5 * (ny - 1)) * voxel));
                double complex gz = (g_re[p] + I * g_im[p]) * cexp(I * qz * z);
                for (int ix = 0; ix < nx; ++ix) {
                    double complex gx = gz * ex[ix];
                    for (int iy = 0; iy < ny; ++iy) acc[(size_t)ix * ny + iy] += gx * ey[iy];
                }
            }
            for (int ix = 0; ix < nx; ++ix)
                for (int iy = 0; iy < ny; ++iy) {
                    size_t idx = ((size_t)iz * nx + ix) * ny + iy;
                    S_re[idx] = creal(acc[(size_t)ix * ny + iy]);
                    S_im[idx] = cimag(acc[(size_t)ix * ny + iy]);
                }
        }
        free(ex);
        free(ey);
        free(acc);
    }
}

/* Derivative of the surface radius r_s(p^) with respect to each geometric
 * parameter, plus r_s itself.  Geometric parameters:
 *   sphere: [r]; ellipsoid: [a, b, c]; harmonics: [a_lm (l>=1), R0]. */
static double orc_radius_and_grad(const orc_shape *sh, const double p[3], double rr, double rmax,
                                  double *dr)
{
    if (sh->kind == ORC_SPHERE) {
        dr[0] = 1.0;
        return sh->r;
    }
    double u0 = 0.0, u1 = 0.0, u2 = 1.0;
    if (rr > 0.0) { u0 = p[0] / rr; u1 = p[1] / rr; u2 = p[2] / rr; }
    if (sh->kind == ORC_ELLIPSOID) {
        double s = (u0 / sh->a) * (u0 / sh->a) + (u1 / sh->b) * (u1 / sh->b) + (u2 / sh->c) * (u2 / sh->c);
        double rs = 1.0 / sqrt(s);
        /* r_s = s^{-1/2}; ds/da = -2 u0^2 / a^3 */
        double f = -0.5 * rs * rs * rs;
        dr[0] = f * (-2.0 * u0 * u0 / (sh->a * sh->a * sh->a));
        dr[1] = f * (-2.0 * u1 * u1 / (sh->b * sh->b * sh->b));
        dr[2] = f * (-2.0 * u2 * u2 / (sh->c * sh->c * sh->c));
        return rs;
    }
    double th = rr > 0.0 ? acos(p[2] / rr) : 0.0;
    double ph = atan2(p[1], p[0]);
    int nlm = (sh->lmax + 1) * (sh->lmax + 1) - 1;
    double sum = 0.0;
    for (int l = 1; l <= sh->lmax; ++l)
        for (int m = -l; m <= l; ++m) {
            double y = orc_real_sh(l, m, th, ph);
            dr[l * l + l + m - 1] = sh->R0 * y;
            sum += sh->alm[l * l + l + m] * y;
        }
    dr[nlm] = 1.0 + sum;
    double rs = sh->R0 * (1.0 + sum);
    if (rs < 0.1 * sh->R0) {
        for (int k = 0; k < nlm; ++k) dr[k] = 0.0;
        dr[nlm] = 0.1;
        rs = 0.1 * sh->R0;
    } else if (rs > rmax) {
        for (int k = 0; k <= nlm; ++k) dr[k] = 0.0;
        rs = rmax;
    }
    return rs;
}

static int orc_n_geom(const orc_shape *sh)
{
    if (sh->kind == ORC_SPHERE) return 1;
    if (sh->kind == ORC_ELLIPSOID) return 3;
    return (sh->lmax + 1) * (sh->lmax + 1);   /* (L+1)^2 - 1 coefficients + R0 */
}

int orc_n_params(const orc_shape *sh) { return orc_n_geom(sh) + 2; }

/*
 * Gradient of a real loss L(I) with respect to the shape parameters, given
 * dL/dI on every pixel, for soft occupancy (binary occupancy has no shape
 * gradient).  With A_q = c F_q, c = n^2 - 1, F_q = sum_v s_v e^{-i q.r_v},
 * s_v = chi_v T_v and T_v = exp(i k0 dz (n-1) C_v), C_v = sum_{v' before v
 * along z} chi_{v'}:
 *   dL/dtheta = sum_q w_q 2 Re(conj(A_q) dA_q/dtheta),  w = dL/dI,
 *   dA_q/dtheta = c' F_q + c sum_v (ds_v/dtheta) e^{-i q.r_v}.
 * Writing R_v = c sum_q w_q conj(A_q) e^{-i q.r_v}:
 *   dL/dtheta = 2 Re[(c'/c) sum_q w_q |A_q|^2] + 2 Re sum_v R_v ds_v/dtheta,
 *   ds_v = dchi_v T_v + s_v i k0 dz [(n-1) dC_v + C_v d(n-1)].
 * The chain rule through C_v turns the per-voxel factor into a reverse
 * (suffix) sum along z.  Parameter order: geometric parameters (sphere r;
 * ellipsoid a,b,c; harmonics a_lm for l>=1 then R0), then delta, beta.
 * A_re/A_im must be the forward field for the same shape and q.
 */
int orc_gradient(const orc_shape *sh, int nx, int ny, int nz, double voxel, double wavelength,
                 double w, const double *q, long n_q, const double *dLdI,
                 const double *A_re, const double *A_im, double *grad)
{
    size_t nv = (size_t)nx * ny * nz;
    int ng = orc_n_geom(sh);
    double k0 = 2.0 * ORC_PI / wavelength;
    double dz = voxel;
    double complex n = 1.0 - sh->delta + I * sh->beta;
    double complex c = n * n - 1.0;
    double complex dc_ddelta = -2.0 * n, dc_dbeta = 2.0 * I * n;
    double complex dn_ddelta = -1.0, dn_dbeta = I;

    double *chi = malloc(sizeof(double) * nv);
    double *g_re = malloc(sizeof(double) * n_q), *g_im = malloc(sizeof(double) * n_q);
    double *S_re = malloc(sizeof(double) * nv), *S_im = malloc(sizeof(double) * nv);
    orc_voxelise(sh, nx, ny, nz, voxel, 1, w, chi);

    /* R_v = c conj(sum_q w_q A_q e^{+i q.r_v}) */
    for (long p = 0; p < n_q; ++p) {
        g_re[p] = dLdI[p] * A_re[p];
        g_im[p] = dLdI[p] * A_im[p];
    }
    orc_msft_adjoint(g_re, g_im, q, n_q, nx, ny, nz, voxel, S_re, S_im);

    /* term from c(delta, beta) */
    double sumWI = 0.0;
    for (long p = 0; p < n_q; ++p) sumWI += dLdI[p] * (A_re[p] * A_re[p] + A_im[p] * A_im[p]);
    for (int k = 0; k < ng + 2; ++k) grad[k] = 0.0;
    grad[ng + 0] += 2.0 * creal(dc_ddelta / c * sumWI);
    grad[ng + 1] += 2.0 * creal(dc_dbeta / c * sumWI);

    double R[9];
    orc_rotation(sh->latitude, sh->longitude, sh->rotation, R);
    double rmax = orc_half_width(nx, ny, nz, voxel) - voxel;
    double *dr = malloc(sizeof(double) * (ng > 0 ? ng : 1));
    double complex g_dn_delta = 0.0, g_dn_beta = 0.0;
    double complex *Rs = malloc(sizeof(double complex) * nz);
    double *C = malloc(sizeof(double) * nz);
    double complex *T = malloc(sizeof(double complex) * nz);
    for (int ix = 0; ix < nx; ++ix)
        for (int iy = 0; iy < ny; ++iy) {
            /* forward along z: C_v (exclusive) and T_v */
            double acc = 0.0;
            for (int iz = 0; iz < nz; ++iz) {
                size_t idx = ((size_t)iz * nx + ix) * ny + iy;
                C[iz] = acc;
                T[iz] = cexp(I * k0 * dz * (n - 1.0) * acc);
                acc += chi[idx];
                Rs[iz] = c * conj(S_re[idx] + I * S_im[idx]);
            }
            /* suffix[iz] = sum_{iz' > iz} R_v' s_v' */
            double complex suffix = 0.0;
            for (int iz = nz - 1; iz >= 0; --iz) {
                size_t idx = ((size_t)iz * nx + ix) * ny + iy;
                double complex s = chi[idx] * T[iz];
                /* d(n-1) terms: sum_v R_v s_v i k0 dz C_v d(n-1) */
                g_dn_delta += Rs[iz] * s * I * k0 * dz * C[iz] * dn_ddelta;
                g_dn_beta += Rs[iz] * s * I * k0 * dz * C[iz] * dn_dbeta;
                /* dchi_v enters s_v directly and every later C_v' */
                double complex chibar = Rs[iz] * T[iz] + I * k0 * dz * (n - 1.0) * suffix;
                suffix += Rs[iz] * s;
                if (ng > 0) {
                    double p[3];
                    orc_body_coords(sh, R, ix, iy, iz, nx, ny, nz, voxel, p);
                    double rr = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
                    double rs = orc_radius_and_grad(sh, p, rr, rmax, dr);
                    double sg = orc_sigmoid((rs - rr) / w);
                    double dsig = sg * (1.0 - sg) / w;
                    for (int k = 0; k < ng; ++k)
                        grad[k] += 2.0 * creal(chibar) * dsig * dr[k];
                }
            }
        }
    free(Rs);
    free(C);
    free(T);
    grad[ng + 0] += 2.0 * creal(g_dn_delta);
    grad[ng + 1] += 2.0 * creal(g_dn_beta);
    free(dr);
    free(chi);
    free(g_re);
    free(g_im);
    free(S_re);
    free(S_im);
    return 0;
}

/* ------------------------------------------------------------------------
 * The Ideal detector (Sec. 5.2, Listing 2 and its description): a perfect
 * detector still counts photons, so the simulated pattern is turned into an
 * expected number of scattered photons per pixel and then into Poisson
 * counts.  The paper's normalisation is in its (unavailable) supplement;
 * reading:
 *   lambda_p = F (k0^2 v / (4 pi))^2 I_p dOmega_p,
 * F the incident photon density (photons per length^2), v = voxel^3 (the
 * volume element of Eq. 1's integral, which the prefactor-1 field omits),
 * I_p = |A_p|^2, dOmega_p the pixel's solid angle: a flat pixel of area
 * a = (2 tan(theta_max))^2 / (Nx Ny) at distance 1 subtends a / r^3 with
 * r^2 = 1 + X^2 + Y^2; a uniform-q pixel of d2q = (2 q_max)^2 / (Nx Ny)
 * subtends d2q / (k0^2 cos(theta)) (d2q_perp = k0^2 cos(theta) dOmega), zero
 * where the pixel has no scattering direction.
 * ------------------------------------------------------------------------ */

/* Solid angle of every detector pixel (flat: uniform_q = 0). */
void orc_pixel_solid_angle(int det_nx, int det_ny, double theta_max_deg, double wavelength, int uniform_q,
                           double *domega)
{
    double k0 = 2.0 * ORC_PI / wavelength;
    double th = theta_max_deg * ORC_PI / 180.0;
    for (int v = 0; v < det_ny; ++v)
        for (int u = 0; u < det_nx; ++u) {
            size_t p = (size_t)v * det_nx + u;
            if (!uniform_q) {
                double h = tan(th);
                double X = h * (2.0 * u + 1.0 - det_nx) / det_nx;
                double Y = h * (2.0 * v + 1.0 - det_ny) / det_ny;
                double area = (2.0 * h / det_nx) * (2.0 * h / det_ny);
                double r = sqrt(1.0 + X * X + Y * Y);
                domega[p] = area / (r * r * r);
            } else {
                double qmax = k0 * sin(th);
                double qx = qmax * (2.0 * u + 1.0 - det_nx) / det_nx;
                double qy = qmax * (2.0 * v + 1.0 - det_ny) / det_ny;
                double s2 = (qx * qx + qy * qy) / (k0 * k0);
                double d2q = (2.0 * qmax / det_nx) * (2.0 * qmax / det_ny);
                domega[p] = s2 < 1.0 ? d2q / (k0 * k0 * sqrt(1.0 - s2)) : 0.0;
            }
        }
}

/*
 * Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 32x32 -> 64-bit multiplications
 * (multipliers 0xD2511F53, 0xCD9E8D57) on a 4-word counter with a 2-word key
 * bumped by the Weyl constants 0x9E3779B9, 0xBB67AE85 between rounds.
 */
static void orc_philox4x32_10(const unsigned ctr[4], const unsigned key[2], unsigned out[4])
{
    unsigned x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    unsigned k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        unsigned long long p0 = (unsigned long long)0xD2511F53u * x0;
        unsigned long long p1 = (unsigned long long)0xCD9E8D57u * x2;
        unsigned y0 = (unsigned)(p1 >> 32) ^ x1 ^ k0;
        unsigned y1 = (unsigned)p1;
        unsigned y2 = (unsigned)(p0 >> 32) ^ x3 ^ k1;
        unsigned y3 = (unsigned)p0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

void orc_philox(unsigned c0, unsigned c1, unsigned c2, unsigned c3, unsigned k0, unsigned k1, unsigned *out)
{
    unsigned ctr[4] = {c0, c1, c2, c3}, key[2] = {k0, k1};
    orc_philox4x32_10(ctr, key, out);
}

/* Draw d (0, 1, 2, ...) of pixel p: a double in (0, 1) from 53 bits of one
 * half of Philox block (p, d / 2) under the seed's key. */
static double orc_uniform(unsigned long long seed, unsigned long long p, unsigned d)
{
    unsigned ctr[4] = {(unsigned)p, (unsigned)(p >> 32), d >> 1, 0u};
    unsigned key[2] = {(unsigned)seed, (unsigned)(seed >> 32)};
    unsigned o[4];
    orc_philox4x32_10(ctr, key, o);
    unsigned hi = (d & 1u) ? o[2] : o[0], lo = (d & 1u) ? o[3] : o[1];
    unsigned long long bits = ((unsigned long long)hi << 21) ^ (unsigned long long)(lo >> 11);
    bits &= (1ull << 53) - 1ull;
    return ((double)bits + 0.5) * (1.0 / 9007199254740992.0);   /* (bits + 1/2) 2^-53 */
}

/*
 * One Poisson(lambda) count from pixel p's stream.  lambda < 12: Knuth's
 * multiplication method (count uniforms until their product drops to
 * e^-lambda).  lambda >= 12: Hormann's transformed rejection with squeeze
 * (PTRS; W. Hormann, "The transformed rejection method for generating Poisson
 * random variables", Insurance: Mathematics and Economics 12 (1993)).
 */
static long long orc_poisson(double lambda, unsigned long long seed, unsigned long long p)
{
    if (!(lambda > 0.0)) return 0;
    unsigned d = 0;
    if (lambda < 12.0) {
        double L = exp(-lambda), prod = 1.0;
        long long k = 0;
        for (;;) {
            prod *= orc_uniform(seed, p, d++);
            if (prod <= L) return k;
            ++k;
        }
    }
    double slam = sqrt(lambda), loglam = log(lambda);
    double b = 0.931 + 2.53 * slam;
    double a = -0.059 + 0.02483 * b;
    double invalpha = 1.1239 + 1.1328 / (b - 3.4);
    double vr = 0.9277 - 3.6224 / (b - 2.0);
    for (;;) {
        double U = orc_uniform(seed, p, d++) - 0.5;
        double V = orc_uniform(seed, p, d++);
        double us = 0.5 - fabs(U);
        long long k = (long long)floor((2.0 * a / us + b) * U + lambda + 0.43);
        if (us >= 0.07 && V <= vr) return k;
        if (k < 0 || (us < 0.013 && V > us)) continue;
        if (log(V) + log(invalpha) - log(a / (us * us) + b) <= -lambda + k * loglam - lgamma(k + 1.0)) return k;
    }
}

/* Expected counts and Poisson counts of every pixel (counts may be NULL). */
void orc_photon_counts(const double *intensity, const double *domega, long n, double photon_density, double wavelength,
                       double voxel, unsigned long long seed, double *lambda, long long *counts)
{
    double k0 = 2.0 * ORC_PI / wavelength;
    double amp = k0 * k0 * voxel * voxel * voxel / (4.0 * ORC_PI);
    double scale = photon_density * amp * amp;
#pragma omp parallel for schedule(dynamic, 64)
    for (long p = 0; p < n; ++p) {
        lambda[p] = scale * intensity[p] * domega[p];
        if (counts) counts[p] = orc_poisson(lambda[p], seed, (unsigned long long)p);
    }
}
