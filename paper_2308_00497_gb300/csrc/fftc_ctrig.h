// Compile-time cos and sin of 2 pi m / N in double precision, for the constant twiddles
// inside composite-radix butterflies. The angle is an exact rational (m mod N over N),
// folded into [0, pi/2] by the symmetries of cos and sin, then summed as the Taylor
// series of the mathematical functions (25 terms: the remainder is below 1e-20 there).
#pragma once

#ifdef __CUDACC__
#define FFTC_HD __host__ __device__
#else
#define FFTC_HD
#endif

namespace fftc {

constexpr double kCtPi = 3.14159265358979323846264338327950288;

FFTC_HD constexpr double ct_taylor_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k < 25; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}

FFTC_HD constexpr double ct_taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k < 25; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}

// cos(2 pi m / N) and sin(2 pi m / N) for integers m, N > 0
FFTC_HD constexpr double ct_cos(long m, long N) {
    m %= N;
    if (m < 0) m += N;
    if (2 * m > N) m = N - m;          // cos(2 pi - x) = cos x; now x in [0, pi]
    if (4 * m > N) {                   // cos x = -cos(pi - x), pi - x = 2 pi (N - 2m) / (2N)
        return -ct_taylor_cos(2.0 * kCtPi * (double)(N - 2 * m) / (2.0 * (double)N));
    }
    return ct_taylor_cos(2.0 * kCtPi * (double)m / (double)N);
}

FFTC_HD constexpr double ct_sin(long m, long N) {
    m %= N;
    if (m < 0) m += N;
    double sgn = 1.0;
    if (2 * m > N) {  // sin(2 pi - x) = -sin x
        m = N - m;
        sgn = -1.0;
    }
    if (4 * m > N) {  // sin x = sin(pi - x)
        return sgn * ct_taylor_sin(2.0 * kCtPi * (double)(N - 2 * m) / (2.0 * (double)N));
    }
    return sgn * ct_taylor_sin(2.0 * kCtPi * (double)m / (double)N);
}

}  // namespace fftc
