// crp_sky.cuh -- directions on the sky: atan2 by one stated algorithm and the HEALPix RING
// pixelization (Gorski et al. 2005), shared by the arrival-map and lens kernels. Translation
// units including it are compiled with --fmad=false, so pixel indices are those of the FP64
// reading.
#pragma once
#include <cuda_runtime.h>

namespace crp {
namespace sky {

constexpr double kPi = 3.141592653589793;
constexpr double kHalfPi = 1.5707963267948966;
constexpr double kQuarterPi = 0.7853981633974483;
constexpr double kTanPi8 = 0.41421356237309503;

// atan2 by the stated reduction: octant, tan(pi/8) split, half-angle step, Taylor series.
__device__ __forceinline__ double atan2_stated(double y, double x) {
    if (x != x || y != y) return __longlong_as_double(0x7ff8000000000000LL);
    const double ax = fabs(x), ay = fabs(y);
    if (ax == 0.0 && ay == 0.0) return 0.0;
    const bool swap = ay > ax;
    const double a = swap ? ax / ay : ay / ax;
    double base = 0.0, b = a;
    if (a > kTanPi8) {
        b = (a - 1.0) / (a + 1.0);
        base = kQuarterPi;
    }
    const double c = b / (1.0 + sqrt(1.0 + b * b));
    const double s = c * c;
    double p = -1.0 / 27.0;
    p = p * s + 1.0 / 25.0;
    p = p * s - 1.0 / 23.0;
    p = p * s + 1.0 / 21.0;
    p = p * s - 1.0 / 19.0;
    p = p * s + 1.0 / 17.0;
    p = p * s - 1.0 / 15.0;
    p = p * s + 1.0 / 13.0;
    p = p * s - 1.0 / 11.0;
    p = p * s + 1.0 / 9.0;
    p = p * s - 1.0 / 7.0;
    p = p * s + 1.0 / 5.0;
    p = p * s - 1.0 / 3.0;
    p = p * s + 1.0;
    double r = base + 2.0 * (c * p);
    if (swap) r = kHalfPi - r;
    if (x < 0.0) r = kPi - r;
    if (y < 0.0) r = -r;
    return r;
}

// HEALPix RING pixel (Gorski et al. 2005): belt |z| <= 2/3 from the edge-line indices
// jp = floor(nside (t - 3z/4 + 1/2)), jm = floor(nside (t + 3z/4 + 1/2)); caps from the
// equal-area radius sigma = nside sqrt(3 (1 - |z|)). t = phi / (pi/2) in [0, 4).
__device__ __forceinline__ long long healpix_ring(int nside, double x, double y, double z) {
    const double r = sqrt(x * x + y * y + z * z);
    if (!(r > 0.0) || !isfinite(r)) return -1;
    const double zz = z / r;
    double phi = atan2_stated(y, x);
    if (phi < 0.0) phi = phi + 2.0 * kPi;
    double t = phi / kHalfPi;
    if (t >= 4.0) t = t - 4.0;
    const long long ns = nside;
    const double dn = (double)nside;
    const double az = fabs(zz);
    if (az <= 2.0 / 3.0) {
        const double sg = 0.75 * zz;
        const long long jp = (long long)floor(dn * (t - sg + 0.5));
        const long long jm = (long long)floor(dn * (t + sg + 0.5));
        long long i = 2 * ns - (jm - jp);
        if (i < ns) i = ns;
        if (i > 3 * ns) i = 3 * ns;
        const long long s = (i - ns + 1) & 1;
        long long j = (jp + jm + 1 - ns - s) / 2;
        const long long m = 4 * ns;
        j = ((j % m) + m) % m;
        return 2 * ns * (ns - 1) + m * (i - ns) + j;
    }
    const double tp = t - floor(t);
    const double sigma = dn * sqrt(3.0 * (1.0 - az));
    long long i = (long long)floor(tp * sigma) + (long long)floor((1.0 - tp) * sigma) + 1;
    if (i > ns) i = ns;
    long long j = (long long)floor(t * (double)i);
    if (j >= 4 * i) j = 4 * i - 1;
    if (zz > 0.0) return 2 * i * (i - 1) + j;
    return 12 * ns * ns - 2 * i * (i + 1) + j;
}

}  // namespace sky
}  // namespace crp
