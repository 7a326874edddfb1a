// Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt on the device, scaled
// by a prefactor theta (the Obara-Saika [00|00]^(m) = theta F_m(T)).
//
// T < BOYS_TMAX: the top order F_L is a 7th-order Taylor expansion about the
// nearest grid point T_k = k / BOYS_GRID,
//   F_L(T) = sum_j F_{L+j}(T_k) (T_k - T)^j / j!      (dF_m/dT = -F_{m+1}),
// read from a table that stores F_{m+j}(T_k) / j! so that each term is one
// fused multiply-add; e^{-T} = e^{-T_k} e^{T_k - T} with the exponential
// series to 7th order (|T_k - T| <= 1/32, so the truncation is below 1e-16
// relative); the lower orders follow from the downward recursion
//   F_m(T) = (2 T F_{m+1}(T) + e^{-T}) / (2m + 1),
// stable for all T. T >= BOYS_TMAX: F_0 = (1/2) sqrt(pi / T) (erf of sqrt(T)
// is 1 in double precision there) and the upward recursion
//   F_{m+1} = ((2m + 1) F_m - e^{-T}) / (2T),
// stable because 2T > 2m + 1 for every order used here. There e^{-T} is at
// most 3e-7 of (2m + 1) F_m (T >= 40, m <= 12), so it is needed only to about
// 1e-10 relative: e^{-T_k} from the table times a fourth-order series of
// e^{T_k - T} (truncation 2.5e-10). From T = BOYS_TEXP on it is below half an
// ulp of (2m + 1) F_m for every order up to 13 (checked against 40-digit
// quadrature) and is dropped.
// The tables are filled on the host by `boys_fill_table` (series in long double).
#pragma once
#include <cuda_runtime.h>

#define BOYS_GRID 16          // table points per unit of T
#define BOYS_TMAX 40.0
#define BOYS_NT (40 * BOYS_GRID + 1)
#define BOYS_MMAX 12          // highest order any kernel asks for
#define BOYS_NTAYLOR 8        // Taylor terms
#define BOYS_MT (BOYS_MMAX + 1)
#define BOYS_TEXP 72.0        // e^{-T} dropped from here on
#define BOYS_NE (72 * BOYS_GRID + 1)
// table layout: [BOYS_NT][BOYS_MT][BOYS_NTAYLOR] F_{m+j}(T_k)/j!, then
// [BOYS_NE] e^{-T_k} (T_k = k / BOYS_GRID up to BOYS_TEXP)
#define BOYS_EXP_OFF (BOYS_NT * BOYS_MT * BOYS_NTAYLOR)
#define BOYS_TAB_DOUBLES (BOYS_EXP_OFF + BOYS_NE)

// FP32 table for the mixed-precision quartets: [BOYS_NT][BOYS_MT][4]
// F_{m+j}(T_k)/j! then [BOYS_NT] e^{-T_k} (4 Taylor terms: truncation below
// 5e-8 relative, under single-precision rounding of the recursion)
#define BOYS_NTAYLOR_F 4
#define BOYS_TAB_FLOATS (BOYS_NT * BOYS_MT * BOYS_NTAYLOR_F + BOYS_NT)

namespace pimd {

// Host: fill the table (BOYS_TAB_DOUBLES values).
void boys_fill_table(double* tab);

__device__ __forceinline__ double exp_poly(double x)
{
    // e^x = sum_j x^j / j!, j <= 7
    double e = 1.0 / 5040.0;
    e = fma(e, x, 1.0 / 720.0);
    e = fma(e, x, 1.0 / 120.0);
    e = fma(e, x, 1.0 / 24.0);
    e = fma(e, x, 1.0 / 6.0);
    e = fma(e, x, 0.5);
    e = fma(e, x, 1.0);
    return fma(e, x, 1.0);
}

// theta e^{-T} for BOYS_TMAX <= T (the asymptotic branch), 0 from BOYS_TEXP on
__device__ __forceinline__ double boys_exp_tail(double T, const double* __restrict__ tab, double theta)
{
    if (T >= BOYS_TEXP) return 0.0;
    const int k = __double2int_rn(T * BOYS_GRID);
    const double x = k * (1.0 / BOYS_GRID) - T;
    double e = 1.0 / 24.0;
    e = fma(e, x, 1.0 / 6.0);
    e = fma(e, x, 0.5);
    e = fma(e, x, 1.0);
    e = fma(e, x, 1.0);
    return theta * __ldg(tab + BOYS_EXP_OFF + k) * e;
}

// Nearest grid index k = round(T * BOYS_GRID) and the offset x = T_k - T,
// for 0 <= T < 2^31 / BOYS_GRID: adding 1.5 * 2^52 to T * BOYS_GRID rounds it
// to an integer (the spacing of doubles there is 1), which then sits in the
// low word; three FP64 operations, no conversion instructions.
__device__ __forceinline__ int boys_grid_point(double T, double& x)
{
    constexpr double kRound = 6755399441055744.0;   // 1.5 * 2^52
    const double s = fma(T, (double)BOYS_GRID, kRound);
    const double kd = s - kRound;
    x = fma(kd, 1.0 / BOYS_GRID, -T);
    return __double2loint(s);
}

// T < BOYS_TMAX for T >= 0, decided on the high word (integer compare): the
// high words of non-negative doubles are ordered like the values, and 40.0
// has an all-zero low word
__device__ __forceinline__ bool boys_in_table(double T)
{
    static_assert(BOYS_TMAX == 40.0, "high word of BOYS_TMAX");
    return __double2hiint(T) < 0x40440000;
}

// F[m] = theta F_m(T), m = 0..L (L a compile-time order)
template <int L>
__device__ __forceinline__ void boys_eval(double T, const double* __restrict__ tab, double theta, double* F)
{
    constexpr double kHalfSqrtPi = 0.88622692545275801365;   // sqrt(pi) / 2
    if (boys_in_table(T)) {
        double x;
        const int k = boys_grid_point(T, x);
        const double* t = tab + ((size_t)k * BOYS_MT + L) * BOYS_NTAYLOR;
        double f = __ldg(t + BOYS_NTAYLOR - 1);
#pragma unroll
        for (int j = BOYS_NTAYLOR - 2; j >= 0; j--) f = fma(f, x, __ldg(t + j));
        F[L] = theta * f;
        if (L > 0) {
            const double te = theta * __ldg(tab + BOYS_NT * BOYS_MT * BOYS_NTAYLOR + k) * exp_poly(x);
            const double t2 = 2.0 * T;
#pragma unroll
            for (int m = L - 1; m >= 0; m--) F[m] = fma(t2, F[m + 1], te) * (1.0 / (2 * m + 1));
        }
    } else {
        const double rs = rsqrt(T);
        F[0] = theta * kHalfSqrtPi * rs;
        if (L > 0) {
            const double te = boys_exp_tail(T, tab, theta);
            const double h = 0.5 * rs * rs;
#pragma unroll
            for (int m = 0; m < L; m++) F[m + 1] = ((2 * m + 1) * F[m] - te) * h;
        }
    }
}

template <int L>
__device__ __forceinline__ void boys_eval(float T, const float* __restrict__ tab, float theta, float* F)
{
    constexpr float kPi = 3.14159265358979f;
    if (T < (float)BOYS_TMAX) {
        const int k = __float2int_rn(T * BOYS_GRID);
        const float x = k * (1.0f / BOYS_GRID) - T;
        const float* t = tab + ((size_t)k * BOYS_MT + L) * BOYS_NTAYLOR_F;
        float f = __ldg(t + 3);
        f = fmaf(f, x, __ldg(t + 2));
        f = fmaf(f, x, __ldg(t + 1));
        f = fmaf(f, x, __ldg(t));
        F[L] = theta * f;
        if (L > 0) {
            // e^x to third order, |x| <= 1/32
            const float ex = fmaf(fmaf(fmaf(1.0f / 6.0f, x, 0.5f), x, 1.0f), x, 1.0f);
            const float te = theta * __ldg(tab + BOYS_NT * BOYS_MT * BOYS_NTAYLOR_F + k) * ex;
            const float t2 = 2.0f * T;
#pragma unroll
            for (int m = L - 1; m >= 0; m--) F[m] = fmaf(t2, F[m + 1], te) * (1.0f / (2 * m + 1));
        }
    } else {
        const float it = 1.0f / T;
        F[0] = theta * 0.5f * sqrtf(kPi * it);
        if (L > 0) {
            const float te = theta * __expf(-T);
            const float h = 0.5f * it;
#pragma unroll
            for (int m = 0; m < L; m++) F[m + 1] = ((2 * m + 1) * F[m] - te) * h;
        }
    }
}

// runtime-order FP32 version (tape kernels of the mixed-precision quartets)
__device__ __forceinline__ void boys_eval_n(int L, float T, const float* __restrict__ tab, float theta, float* F)
{
    constexpr float kPi = 3.14159265358979f;
    if (T < (float)BOYS_TMAX) {
        const int k = __float2int_rn(T * BOYS_GRID);
        const float x = k * (1.0f / BOYS_GRID) - T;
        const float* t = tab + ((size_t)k * BOYS_MT + L) * BOYS_NTAYLOR_F;
        float f = __ldg(t + 3);
        f = fmaf(f, x, __ldg(t + 2));
        f = fmaf(f, x, __ldg(t + 1));
        f = fmaf(f, x, __ldg(t));
        F[L] = theta * f;
        if (L > 0) {
            const float ex = fmaf(fmaf(fmaf(1.0f / 6.0f, x, 0.5f), x, 1.0f), x, 1.0f);
            const float te = theta * __ldg(tab + BOYS_NT * BOYS_MT * BOYS_NTAYLOR_F + k) * ex;
            const float t2 = 2.0f * T;
            for (int m = L - 1; m >= 0; m--) F[m] = fmaf(t2, F[m + 1], te) / (float)(2 * m + 1);
        }
    } else {
        const float it = 1.0f / T;
        F[0] = theta * 0.5f * sqrtf(kPi * it);
        if (L > 0) {
            const float te = theta * __expf(-T);
            const float h = 0.5f * it;
            for (int m = 0; m < L; m++) F[m + 1] = ((2 * m + 1) * F[m] - te) * h;
        }
    }
}

// runtime-order version (one-electron integrals, tape kernels)
__device__ __forceinline__ void boys_eval_n(int L, double T, const double* __restrict__ tab, double theta, double* F)
{
    constexpr double kHalfSqrtPi = 0.88622692545275801365;   // sqrt(pi) / 2
    if (boys_in_table(T)) {
        double x;
        const int k = boys_grid_point(T, x);
        const double* t = tab + ((size_t)k * BOYS_MT + L) * BOYS_NTAYLOR;
        double f = __ldg(t + BOYS_NTAYLOR - 1);
#pragma unroll
        for (int j = BOYS_NTAYLOR - 2; j >= 0; j--) f = fma(f, x, __ldg(t + j));
        F[L] = theta * f;
        if (L > 0) {
            const double te = theta * __ldg(tab + BOYS_NT * BOYS_MT * BOYS_NTAYLOR + k) * exp_poly(x);
            const double t2 = 2.0 * T;
            for (int m = L - 1; m >= 0; m--) F[m] = fma(t2, F[m + 1], te) / (2 * m + 1);
        }
    } else {
        const double rs = rsqrt(T);
        F[0] = theta * kHalfSqrtPi * rs;
        if (L > 0) {
            const double te = boys_exp_tail(T, tab, theta);
            const double h = 0.5 * rs * rs;
            for (int m = 0; m < L; m++) F[m + 1] = ((2 * m + 1) * F[m] - te) * h;
        }
    }
}

}  // namespace pimd
