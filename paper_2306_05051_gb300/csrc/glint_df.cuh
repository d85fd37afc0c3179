// Double-float ("double-word") arithmetic on FP32 pairs for the per-pixel
// scalars whose rounding would otherwise flip integer decisions: the lattice
// coordinate of a texel (up to ~1e6 cells) and the chain footprint ->
// (ratio, orientation, scale) -> tetrahedron weights -> trial counts (trials
// up to f^(L-1) ~ 4e6, so a weight error of 1e-7 moves a count by ~0.4).
//
// Methods: error-free TwoSum (Knuth) and TwoProd with FMA (Dekker 1971);
// the sum / product / quotient compositions and their error bounds follow
// Joldes, Muller & Popescu, "Tight and rigorous error bounds for basic
// building blocks of double-word arithmetic", ACM TOMS 44(2), 2017.
// Relative error ~2^-44 or better for each operation.  All elementary
// operations use the _rn intrinsics so that no FMA contraction or
// reassociation changes the error-free transforms.
#pragma once
#include <cstdint>

namespace glint {

struct df {
    float hi, lo;
};

__device__ __forceinline__ df mkdf(float x) { return {x, 0.0f}; }

// exact power of two as a float (-126 <= e <= 127)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df operator-(df a) { return {-a.hi, -a.lo}; }

// Sum with absolute error ~2^-48 (|a| + |b|) (Dekker's composition): the
// chains here need accuracy relative to the operands, not to a cancelled
// result; the interpolation weights, which do need relative accuracy, are
// formed from exact residuals (see dffloor_w).
__device__ __forceinline__ df operator+(df a, df b) {
    const df s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(s.lo, a.lo), b.lo));
}
__device__ __forceinline__ df operator-(df a, df b) { return a + (-b); }

__device__ __forceinline__ df operator+(df a, float b) {
    const df s = two_sum(a.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(a.lo, s.lo));
}
__device__ __forceinline__ df operator-(df a, float b) { return a + (-b); }
__device__ __forceinline__ df operator+(float a, df b) { return b + a; }
__device__ __forceinline__ df operator-(float a, df b) { return (-b) + a; }

__device__ __forceinline__ df operator*(df a, df b) {
    const df c = two_prod(a.hi, b.hi);
    const float t = __fmaf_rn(a.lo, b.hi, __fmul_rn(a.hi, b.lo));
    return fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}

__device__ __forceinline__ df operator*(df a, float b) {
    const df c = two_prod(a.hi, b);
    return fast_two_sum(c.hi, __fmaf_rn(a.lo, b, c.lo));
}

// exact scaling by 2^e (no under/overflow in this library's ranges)
__device__ __forceinline__ df scale2(df a, int e) {
    const float s = pow2f(e);
    return {__fmul_rn(a.hi, s), __fmul_rn(a.lo, s)};
}

// Approximate reciprocal (MUFU, about 2 ulp).  Every division below uses it
// for a first quotient and then corrects with an exactly computed residual,
// so the double-float result does not depend on the reciprocal's last bits.
__device__ __forceinline__ float approx_rcp(float x) { return __fdividef(1.0f, x); }

__device__ __forceinline__ df operator/(df a, df b) {
    const float ib = approx_rcp(b.hi);
    const float q1 = __fmul_rn(a.hi, ib);
    const df r = a - b * q1;
    return fast_two_sum(q1, __fmul_rn(r.hi, ib));
}

// a / b for a float b with ib ~ 1/b
__device__ __forceinline__ df div_by(df a, float b, float ib) {
    const float q1 = __fmul_rn(a.hi, ib);
    const df p = two_prod(q1, b);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p.hi), p.lo), a.lo);
    return fast_two_sum(q1, __fmul_rn(r, ib));
}
__device__ __forceinline__ df operator/(df a, float b) { return div_by(a, b, approx_rcp(b)); }
__device__ __forceinline__ df A_over(df a, int k) { return div_by(a, (float)k, approx_rcp((float)k)); }

__device__ __forceinline__ df operator*(float a, df b) { return b * a; }
__device__ __forceinline__ df operator/(float a, df b) { return mkdf(a) / b; }

// sqrt(a), a >= 0: approximate root, then one correction with the exact residual
__device__ __forceinline__ df dfsqrt(df a) {
    if (!(a.hi > 0.0f)) return {0.0f, 0.0f};
    const float r = rsqrtf(a.hi);
    const float s = __fmul_rn(a.hi, r);
    const float e = __fadd_rn(__fmaf_rn(-s, s, a.hi), a.lo);
    return fast_two_sum(s, __fmul_rn(e, __fmul_rn(0.5f, r)));
}

// 1 / sqrt(a), a > 0: approximate value y, then y + y (1 - a y^2) / 2 with
// a y^2 evaluated in double-float
__device__ __forceinline__ df dfrsqrt(df a) {
    const float y = rsqrtf(a.hi);
    const df ay2 = a * two_prod(y, y);
    const df e = 1.0f - ay2;
    return fast_two_sum(y, __fmul_rn(__fmul_rn(y, e.hi), 0.5f));
}

// sign of a normalised double-float: -1, 0, +1
__device__ __forceinline__ int dfsign(df a) {
    if (a.hi > 0.0f) return 1;
    if (a.hi < 0.0f) return -1;
    return a.lo > 0.0f ? 1 : (a.lo < 0.0f ? -1 : 0);
}
// Order of normalised double-floats (hi = fl(hi + lo)) is lexicographic.
__device__ __forceinline__ bool dflt(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool dfle(df a, df b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }
__device__ __forceinline__ bool dflt(df a, float b) { return a.hi < b || (a.hi == b && a.lo < 0.0f); }
__device__ __forceinline__ bool dfle(df a, float b) { return a.hi < b || (a.hi == b && a.lo <= 0.0f); }
__device__ __forceinline__ df dfabs(df a) { return dfsign(a) < 0 ? -a : a; }

// floor: integer part and fraction in [0, 1); requires |a| < 2^31.  The
// integer is adjusted as an int: above 2^24 a float cannot hold odd integers.
__device__ __forceinline__ int dffloor(df a, df* frac) {
    const float f = floorf(a.hi);
    df r = fast_two_sum(__fsub_rn(a.hi, f), a.lo);   // a.hi - f is exact
    int i = (int)f;
    if (fabsf(a.hi) >= 16777216.0f) {
        // above 2^24 the low word alone can exceed 1 in magnitude
        const float g = floorf(r.hi);
        r = r - g;
        i += (int)g;
    }
    if (r.hi < 0.0f || (r.hi == 0.0f && r.lo < 0.0f)) { i -= 1; r = r + 1.0f; }
    else if (!dflt(r, 1.0f)) { i += 1; r = r - 1.0f; }
    *frac = r;
    return i;
}

// Floor with the two interpolation weights of the cell: f = a - floor(a)
// and g = 1 - f, each rounded once to FP32 (full relative precision even
// when tiny: 1 - r.hi is exact whenever r.hi >= 1/2).
__device__ __forceinline__ int dffloor_w(df a, float* f, float* g) {
    df r;
    const int i = dffloor(a, &r);
    *f = __fadd_rn(r.hi, r.lo);
    *g = __fsub_rn(__fsub_rn(1.0f, r.hi), r.lo);
    return i;
}

// Tables and constants built by the host in double precision and split
// into (hi, lo) pairs; the kernels copy them into shared memory.
struct DfTables {
    float2 atan_t[65];     // atan(k / 64), k = 0..64
    float2 log2_t[65];     // log2(1 + k / 64), k = 0..64
    float2 exp2_t[64];     // 2^(j / 64), j = 0..63
    float2 pi, half_pi, inv_pi, inv_ln2, inv_sqrt2, third, ln2;
};

__device__ __forceinline__ df ldf(float2 v) { return {v.x, v.y}; }

// log2 of a positive double-float: table of log2(1 + k/64) and a degree-6
// series of ln(1 + d), |d| <= 1/128, with the leading term in double-float.
__device__ __forceinline__ df dflog2(df x, const DfTables& T) {
    int e;
    frexpf(x.hi, &e);                       // x.hi = m 2^e, m in [0.5, 1)
    const df y = scale2(x, 1 - e);          // [1, 2)
    const int k = min(max(__float2int_rn(__fmul_rn(__fsub_rn(y.hi, 1.0f), 64.0f)), 0), 64);
    const float c = __fmaf_rn((float)k, 0.015625f, 1.0f);
    const df d = (y - c) / c;
    const float h = d.hi;
    const float tail = __fmaf_rn(-h, d.lo,
        h * h * (-0.5f + h * (0.333333343f + h * (-0.25f + h * (0.2f - h * 0.166666672f)))));
    const df ln1p = d + tail;
    return ln1p * ldf(T.inv_ln2) + ldf(T.log2_t[k]) + (float)(e - 1);
}

// exp(-x) of a double-float x >= 0 by Tang's table-driven method (ACM TOMS
// 15(2), 1989): -x log2(e) = m + j/64 + r/ln 2 with |r| <= ln(2)/128, so
// exp(-x) = 2^m 2^(j/64) exp(r); exp(r) = 1 + r + r^2/2 + ... + r^5/120 with
// the linear part in double-float (the neglected r^6/720 is below 4e-17).
// Relative error ~1e-11 over the whole range; 0 where exp(-x) < 2^-125.
__device__ __forceinline__ df dfexp_neg(df x, const DfTables& T) {
    if (!(x.hi < 86.0f)) return {0.0f, 0.0f};
    const df t = -(x * ldf(T.inv_ln2));
    const int N = __float2int_rn(__fmul_rn(t.hi, 64.0f));
    const df r = (t - __fmul_rn((float)N, 0.015625f)) * ldf(T.ln2);
    const float h = r.hi;
    const float tail = __fmul_rn(__fmul_rn(h, h),
                                 __fmaf_rn(h, __fmaf_rn(h, __fmaf_rn(h, 8.33333377e-3f, 4.16666679e-2f), 0.166666672f), 0.5f));
    const df er = (r + tail) + 1.0f;
    const int j = N & 63, m = N >> 6;
    return scale2(ldf(T.exp2_t[j]) * er, m);
}

// atan2 of double-floats: octant reduction, table of atan(k/64) and the
// series of atan(e), |e| <= 1/128, with the leading term in double-float.
__device__ __forceinline__ df dfatan2(df y, df x, const DfTables& T) {
    const bool ny = dfsign(y) < 0, nx = dfsign(x) < 0;
    const df ay = ny ? -y : y, ax = nx ? -x : x;
    const bool sw = dflt(ax, ay);
    const df num = sw ? ax : ay, den = sw ? ay : ax;
    if (den.hi == 0.0f) return {0.0f, 0.0f};
    const df t = num / den;
    const int k = min(max(__float2int_rn(__fmul_rn(t.hi, 64.0f)), 0), 64);
    const float c = __fmul_rn((float)k, 0.015625f);
    const df e = (t - c) / (t * c + 1.0f);
    const float h = e.hi, h2 = h * h;
    const float tail = h * h2 * (-0.333333343f + h2 * (0.2f - h2 * 0.142857149f));
    df th = ldf(T.atan_t[k]) + (e + tail);
    if (sw) th = ldf(T.half_pi) - th;
    if (nx) th = ldf(T.pi) - th;
    if (ny) th = -th;
    return th;
}

}  // namespace glint
