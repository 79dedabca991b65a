// Shared device/host helpers: complex arithmetic on CUDA vector types, precision traits,
// power-of-two scaling and error plumbing.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define MS_HD __host__ __device__ __forceinline__

// ------------------------------------------------------------------ precision traits
template <typename T> struct CT;
template <> struct CT<double> { typedef double2 c; };
template <> struct CT<float> { typedef float2 c; };

MS_HD double2 mk(double a, double b) { return make_double2(a, b); }
MS_HD float2 mk(float a, float b) { return make_float2(a, b); }

MS_HD double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
MS_HD float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
MS_HD double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
MS_HD float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
MS_HD double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
MS_HD float2 cmul(float2 a, float2 b) { return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
MS_HD double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
MS_HD float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
MS_HD double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
MS_HD float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// acc += a * b  (complex fused multiply-add)
MS_HD void cfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
MS_HD void cfma(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(a.y, b.x, acc.y);
}
// acc += conj(a) * b
MS_HD void cfma_conj(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
}
MS_HD void cfma_conj(float2& acc, float2 a, float2 b) {
    acc.x = fmaf(a.x, b.x, acc.x); acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y); acc.y = fmaf(-a.y, b.x, acc.y);
}
MS_HD double2 cdiv(double2 a, double2 b) {
    double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
MS_HD double cabs2(double2 a) { return a.x * a.x + a.y * a.y; }

template <typename T> MS_HD typename CT<T>::c to_c(double2 v);
template <> MS_HD double2 to_c<double>(double2 v) { return v; }
template <> MS_HD float2 to_c<float>(double2 v) { return make_float2((float)v.x, (float)v.y); }
MS_HD double2 to_d(double2 v) { return v; }
MS_HD double2 to_d(float2 v) { return make_double2((double)v.x, (double)v.y); }

// ------------------------------------------------------------------ exact power-of-two scaling
// 2^e as a double for |e| <= 1022 built from its bit pattern (exact; 0 below the normal range).
MS_HD double pow2d(int e) {
    if (e < -1022) return 0.0;
    if (e > 1023) e = 1023;
    unsigned long long bits = (unsigned long long)(e + 1023) << 52;
#ifdef __CUDA_ARCH__
    return __longlong_as_double((long long)bits);
#else
    double d; memcpy(&d, &bits, 8); return d;
#endif
}
MS_HD float pow2f(int e) {
    if (e < -126) return 0.0f;
    if (e > 127) e = 127;
    unsigned int bits = (unsigned int)(e + 127) << 23;
#ifdef __CUDA_ARCH__
    return __int_as_float((int)bits);
#else
    float f; memcpy(&f, &bits, 4); return f;
#endif
}
template <typename T> MS_HD T pow2(int e);
template <> MS_HD double pow2<double>(int e) { return pow2d(e); }
template <> MS_HD float pow2<float>(int e) { return pow2f(e); }

// Split a complex double into an FP32 mantissa pair and a common binary exponent:
// v = m * 2^e with max(|m.x|, |m.y|) in [0.5, 1) (m = 0, e = 0 for v = 0).
MS_HD void split_exp(double2 v, float2& m, int& e) {
    double a = fmax(fabs(v.x), fabs(v.y));
    if (a == 0.0 || !(a < 1e308)) { m = make_float2(0.f, 0.f); e = 0; return; }
    frexp(a, &e);
    double s = pow2d(-e);
    m = make_float2((float)(v.x * s), (float)(v.y * s));
}
