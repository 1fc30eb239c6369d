// log2pair.cuh -- float-pair arithmetic for the exponent p log2 w - C_i - V_j of the
// per-step matrices (the step kernel and the Newton path): exact two-sum and a log2 of
// integer weights accurate to about 2^-40 from a 256-entry shared table and a short series.
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace sa {

constexpr int kLog2Tab = 32768;   // weights below this take the shared-table logarithm

// s + err = a + b exactly (Knuth's two-sum; no FMA contraction is possible here)
__device__ __forceinline__ float two_sum(float a, float b, float* err) {
    const float s = a + b;
    const float bb = s - a;
    *err = (a - (s - bb)) + (b - bb);
    return s;
}

// Shared table for log2 of a weight: entry j (the top 8 mantissa bits of m in [1, 2)) holds
// g_j = 1 / (1 + (j + 0.5)/256) rounded to 9 significant bits and -log2(g_j) as a float pair.
__device__ __forceinline__ float4 log2_tab_entry(int j) {
    const double c = 1.0 + (j + 0.5) / 256.0;
    const double g = ldexp(rint(ldexp(1.0 / c, 8)), -8);   // 9 significant bits (value in (0.5, 1))
    const double t = -log2(g);
    const float th = (float)t;
    return make_float4((float)g, th, (float)(t - (double)th), 0.0f);
}

// log2 w (0 < w < 2^15) as an unevaluated float pair, accurate to about 2^-40: with
// w = 2^e m, m g_j is exact (15 + 9 significant bits), so r = m g_j - 1 is exact and
// |r| < 2^-8; log2 w = e + (-log2 g_j) + log2(1 + r), the last from its series with the
// leading product r log2(e) split exactly.
__device__ __forceinline__ float2 log2_pair(int w, const float4* tab) {
    const unsigned bits = __float_as_uint((float)w);
    const int e = (int)(bits >> 23) - 127;
    const float4 t = tab[(bits >> 15) & 0xFFu];
    const float m = __uint_as_float((bits & 0x7FFFFFu) | 0x3F800000u);
    const float r = fmaf(m, t.x, -1.0f);
    const float l2eh = 1.4426950216293335f, l2el = 1.925963033500011e-08f;   // log2(e) as a pair
    const float ph = r * l2eh;
    const float pe = fmaf(r, l2eh, -ph);
    // ln(1 + r) / r - 1 = -r/2 + r^2/3 - r^3/4 + r^4/5 - r^5/6 (next term below 2^-48)
    const float poly = r * (-0.5f + r * (0.333333343f + r * (-0.25f + r * (0.2f + r * -0.166666672f))));
    const float small = fmaf(r, l2el, pe) + ph * poly;
    float e1, e2;
    const float s1 = two_sum((float)e, t.y, &e1);
    const float s2 = two_sum(s1, ph, &e2);
    return make_float2(s2, ((e1 + e2) + t.z) + small);
}

// log2 of a positive integer weight as a float pair (shared table + series for the int16
// range; FP64 above it)
__device__ __forceinline__ float2 wlog2(const float4* stab, int w) {
    if (w < kLog2Tab) return log2_pair(w, stab);
    const double l = log2((double)w);
    const float hi = (float)l;
    return make_float2(hi, (float)(l - (double)hi));
}

}  // namespace sa
