// detector.cu -- the Ideal detector (Sec. 5.2, Listing 2: photon statistics).
//
// A perfect detector still counts photons: the pattern becomes an expected
// number of scattered photons per pixel,
//   lambda_p = F (k0^2 v / (4 pi))^2 I_p dOmega_p,
// (F the incident photon density, v = voxel^3, dOmega_p the pixel's solid
// angle: a / r^3 for a flat pixel of area a at r = sqrt(1 + X^2 + Y^2),
// d2q / (k0^2 cos theta) for a uniform-q pixel), and then a Poisson count.
// The counts come from a counter-based generator, Philox-4x32-10 (Salmon et
// al., SC'11), keyed by the seed and counted by (pixel, draw), so every pixel
// is reproducible and independent of the launch shape; the Poisson draw is
// Knuth's multiplication method below lambda = 12 and Hormann's transformed
// rejection with squeeze (PTRS, 1993) above.  All of it runs in FP64 with
// explicitly rounded operations (no fused multiply-add), so that the same
// seed gives the same counts as an FP64 host implementation of the same
// definitions.
#include "internal.cuh"

namespace scm {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t y0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t y1 = (uint32_t)p1;
        const uint32_t y2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        const uint32_t y3 = (uint32_t)p0;
        c[0] = y0;
        c[1] = y1;
        c[2] = y2;
        c[3] = y3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// Draw d of pixel p: 53 bits of one half of Philox block (p, d / 2) as a
// double in (0, 1).
__device__ __forceinline__ double uniform53(uint64_t seed, uint64_t p, uint32_t d) {
    uint32_t c[4] = {(uint32_t)p, (uint32_t)(p >> 32), d >> 1, 0u};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const uint32_t hi = (d & 1u) ? c[2] : c[0], lo = (d & 1u) ? c[3] : c[1];
    uint64_t bits = ((uint64_t)hi << 21) ^ (uint64_t)(lo >> 11);
    bits &= (1ull << 53) - 1ull;
    return __dmul_rn(__dadd_rn((double)bits, 0.5), 1.0 / 9007199254740992.0);
}

__device__ long long poisson_draw(double lambda, uint64_t seed, uint64_t p) {
    if (!(lambda > 0.0)) return 0;
    uint32_t d = 0;
    if (lambda < 12.0) {
        const double L = exp(-lambda);
        double prod = 1.0;
        long long k = 0;
        for (;;) {
            prod = __dmul_rn(prod, uniform53(seed, p, d++));
            if (prod <= L) return k;
            ++k;
        }
    }
    const double slam = sqrt(lambda), loglam = log(lambda);
    const double b = __dadd_rn(0.931, __dmul_rn(2.53, slam));
    const double a = __dadd_rn(-0.059, __dmul_rn(0.02483, b));
    const double invalpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dadd_rn(b, -3.4)));
    const double vr = __dadd_rn(0.9277, -__ddiv_rn(3.6224, __dadd_rn(b, -2.0)));
    for (;;) {
        const double U = __dadd_rn(uniform53(seed, p, d++), -0.5);
        const double V = uniform53(seed, p, d++);
        const double us = __dadd_rn(0.5, -fabs(U));
        // floor((2a/us + b) U + lambda + 0.43)
        const double t = __dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, a), us), b), U), lambda), 0.43);
        const long long k = (long long)floor(t);
        if (us >= 0.07 && V <= vr) return k;
        if (k < 0 || (us < 0.013 && V > us)) continue;
        const double lhs = __dadd_rn(__dadd_rn(log(V), log(invalpha)),
                                     -log(__dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b)));
        const double rhs = __dadd_rn(__dadd_rn(-lambda, __dmul_rn((double)k, loglam)), -lgamma(__dadd_rn((double)k, 1.0)));
        if (lhs <= rhs) return k;
    }
}

// One thread per pixel: solid angle, expected count, Poisson count.
__global__ void photon_counts_kernel(const void *I, int fp64, long long n, int det_nx, int det_ny, int uniform,
                                     double h, double qmax, double k0, double scale, uint64_t seed,
                                     double *lambda, long long *counts) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int u = (int)(p % det_nx), v = (int)(p / det_nx);
    double dom;
    if (!uniform) {
        const double X = __ddiv_rn(__dmul_rn(h, (double)(2 * u + 1 - det_nx)), (double)det_nx);
        const double Y = __ddiv_rn(__dmul_rn(h, (double)(2 * v + 1 - det_ny)), (double)det_ny);
        const double area = __dmul_rn(__ddiv_rn(__dmul_rn(2.0, h), (double)det_nx),
                                      __ddiv_rn(__dmul_rn(2.0, h), (double)det_ny));
        const double r = sqrt(__dadd_rn(__dadd_rn(1.0, __dmul_rn(X, X)), __dmul_rn(Y, Y)));
        dom = __ddiv_rn(area, __dmul_rn(__dmul_rn(r, r), r));
    } else {
        const double qx = __ddiv_rn(__dmul_rn(qmax, (double)(2 * u + 1 - det_nx)), (double)det_nx);
        const double qy = __ddiv_rn(__dmul_rn(qmax, (double)(2 * v + 1 - det_ny)), (double)det_ny);
        const double s2 = __ddiv_rn(__dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)), __dmul_rn(k0, k0));
        const double d2q = __dmul_rn(__ddiv_rn(__dmul_rn(2.0, qmax), (double)det_nx),
                                     __ddiv_rn(__dmul_rn(2.0, qmax), (double)det_ny));
        dom = s2 < 1.0 ? __ddiv_rn(d2q, __dmul_rn(__dmul_rn(k0, k0), sqrt(__dadd_rn(1.0, -s2)))) : 0.0;
    }
    const double Ip = fp64 ? static_cast<const double *>(I)[p] : (double)static_cast<const float *>(I)[p];
    const double lam = __dmul_rn(__dmul_rn(scale, Ip), dom);
    if (lambda) lambda[p] = lam;
    if (counts) counts[p] = poisson_draw(lam, seed, (uint64_t)p);
}

cudaError_t launch_photon_counts(const void *I, bool fp64, long long n, int det_nx, int det_ny, bool uniform,
                                 double theta_max_deg, double wavelength, double voxel, double photon_density,
                                 uint64_t seed, double *lambda, long long *counts, cudaStream_t st) {
    const double k0 = 2.0 * kPi / wavelength;
    const double th = theta_max_deg * kPi / 180.0;
    const double amp = k0 * k0 * voxel * voxel * voxel / (4.0 * kPi);
    const double scale = photon_density * amp * amp;
    photon_counts_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        I, fp64 ? 1 : 0, n, det_nx, det_ny, uniform ? 1 : 0, tan(th), k0 * sin(th), k0, scale, seed, lambda, counts);
    return cudaGetLastError();
}

}  // namespace scm
