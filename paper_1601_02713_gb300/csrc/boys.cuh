// Boys function F_m(T) = int_0^1 t^{2m} exp(-T t^2) dt on the device.
//
// T < BOYS_TMAX: the top order F_L is a 7th-order Taylor expansion about the
// nearest grid point T_k = k / BOYS_GRID of a table of F_m(T_k),
//   F_L(T) = sum_j F_{L+j}(T_k) (T_k - T)^j / j!      (d F_m / dT = -F_{m+1}),
// and the lower orders follow from the downward recursion
//   F_m(T) = (2 T F_{m+1}(T) + e^{-T}) / (2m + 1),
// which is stable for all T. T >= BOYS_TMAX: F_0 = (1/2) sqrt(pi / T) (erf of
// sqrt(T) is 1 in double precision there) and the upward recursion
//   F_{m+1} = ((2m + 1) F_m - e^{-T}) / (2T),
// stable because 2T > 2m + 1 for every order used here.
// The table is filled on the host by `boys_fill_table` (series in long double).
#pragma once
#include <cuda_runtime.h>

#define BOYS_GRID 16          // table points per unit of T
#define BOYS_TMAX 40.0
#define BOYS_NT (40 * BOYS_GRID + 1)
#define BOYS_MMAX 12          // highest order any kernel asks for
#define BOYS_NTAYLOR 8        // Taylor terms (FP64)
#define BOYS_NM (BOYS_MMAX + BOYS_NTAYLOR)   // table orders per grid point

namespace pimd {

// Host: fill tab[k * BOYS_NM + m] = F_m(k / BOYS_GRID).
void boys_fill_table(double* tab);

template <int L>
__device__ __forceinline__ void boys_eval(double T, const double* __restrict__ tab, double* F)
{
    constexpr double kPi = 3.14159265358979323846;
    if (T < BOYS_TMAX) {
        const int k = __double2int_rn(T * BOYS_GRID);
        const double x = k * (1.0 / BOYS_GRID) - T;
        const double* t = tab + k * BOYS_NM + L;
        double f = __ldg(t + BOYS_NTAYLOR - 1);
#pragma unroll
        for (int j = BOYS_NTAYLOR - 2; j >= 0; j--) f = __ldg(t + j) + f * x * (1.0 / (j + 1));
        F[L] = f;
        if (L > 0) {
            const double e = exp(-T);
            const double t2 = 2.0 * T;
#pragma unroll
            for (int m = L - 1; m >= 0; m--) F[m] = (t2 * F[m + 1] + e) * (1.0 / (2 * m + 1));
        }
    } else {
        const double it = 1.0 / T;
        F[0] = 0.5 * sqrt(kPi * it);
        if (L > 0) {
            const double e = exp(-T);
            const double h = 0.5 * it;
#pragma unroll
            for (int m = 0; m < L; m++) F[m + 1] = ((2 * m + 1) * F[m] - e) * h;
        }
    }
}

// runtime-order version (1e integrals, tape kernels)
__device__ __forceinline__ void boys_eval_n(int L, double T, const double* __restrict__ tab, double* F)
{
    constexpr double kPi = 3.14159265358979323846;
    if (T < BOYS_TMAX) {
        const int k = __double2int_rn(T * BOYS_GRID);
        const double x = k * (1.0 / BOYS_GRID) - T;
        const double* t = tab + k * BOYS_NM + L;
        double f = __ldg(t + BOYS_NTAYLOR - 1);
#pragma unroll
        for (int j = BOYS_NTAYLOR - 2; j >= 0; j--) f = __ldg(t + j) + f * x * (1.0 / (j + 1));
        F[L] = f;
        if (L > 0) {
            const double e = exp(-T);
            const double t2 = 2.0 * T;
            for (int m = L - 1; m >= 0; m--) F[m] = (t2 * F[m + 1] + e) / (2 * m + 1);
        }
    } else {
        const double it = 1.0 / T;
        F[0] = 0.5 * sqrt(kPi * it);
        if (L > 0) {
            const double e = exp(-T);
            const double h = 0.5 * it;
            for (int m = 0; m < L; m++) F[m + 1] = ((2 * m + 1) * F[m] - e) * h;
        }
    }
}

}  // namespace pimd
