// k_device.cuh -- device helpers: complex FP64 arithmetic, the packed-tuple rank, the resonance
// denominator and the complex divide used by every precision form.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace npf {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
// acc += a * b
__device__ __forceinline__ void cfma(double2& acc, double2 a, double2 b)
{
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += r * b (real times complex)
__device__ __forceinline__ void rfma(double2& acc, double r, double2 b)
{
    acc.x = fma(r, b.x, acc.x);
    acc.y = fma(r, b.y, acc.y);
}

// Complex quotient c/d by R. L. Smith's scaling (CACM Algorithm 116, 1962): divide numerator
// and denominator by the larger component of d so that no intermediate overflows.
__device__ __forceinline__ double2 cdiv_smith(double2 c, double2 d)
{
    double re, im;
    if (fabs(d.x) >= fabs(d.y)) {
        const double t = d.y / d.x;
        const double s = 1.0 / (d.x + d.y * t);
        re = (c.x + c.y * t) * s;
        im = (c.y - c.x * t) * s;
    } else {
        const double t = d.x / d.y;
        const double s = 1.0 / (d.y + d.x * t);
        re = (c.x * t + c.y) * s;
        im = (c.y * t - c.x) * s;
    }
    return make_double2(re, im);
}

// Resonance denominator with the clamp of Algorithm 2 step 9 (|D| < eps -> eps + 0i).
__device__ __forceinline__ double2 clamp_denominator(double2 D, double eps)
{
    if (sqrt(D.x * D.x + D.y * D.y) < eps) return make_double2(eps, 0.0);
    return D;
}

// Lexicographic rank of a non-decreasing tuple s[0..N-1] over [0, n), by the telescoped count
// rank = sum_m ( cnt(N-m, s[m-1]) - cnt(N-m, s[m]) ),  s[-1] = 0,
// where cnt(r, v) = C(n - v + r - 1, r) is the number of non-decreasing r-tuples in [v, n).
// cnt is a table [ (r)*(n+1) + v ] for r in [0, N], v in [0, n].
__device__ __forceinline__ int64_t tuple_rank(const int* s, int N, const int64_t* __restrict__ cnt,
                                              int n)
{
    int64_t r = 0;
    int prev = 0;
    for (int m = 0; m < N; ++m) {
        const int64_t* row = cnt + (int64_t)(N - m) * (n + 1);
        r += row[prev] - row[s[m]];
        prev = s[m];
    }
    return r;
}

// Insert v into the sorted array s[0..len-1] producing the sorted array t[0..len].
__device__ __forceinline__ void sorted_insert(const int* s, int len, int v, int* t)
{
    int k = 0;
    while (k < len && s[k] <= v) { t[k] = s[k]; ++k; }
    t[k] = v;
    for (; k < len; ++k) t[k + 1] = s[k];
}

__device__ __forceinline__ void sort_small(int* s, int len)
{
    for (int a = 1; a < len; ++a) {
        int x = s[a], b = a - 1;
        while (b >= 0 && s[b] > x) { s[b + 1] = s[b]; --b; }
        s[b + 1] = x;
    }
}

}  // namespace npf
