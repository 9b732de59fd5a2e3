// dfloat.cuh - double-float arithmetic: a real number held as the unevaluated sum hi + lo of two
// FP32 values (|lo| <= ulp(hi) / 2), about 48 significand bits.
//
// The operations are the error-free transformations of Dekker (Numer. Math. 18, 1971) and Knuth
// (TAOCP vol. 2, Sec. 4.2.2): two-sum, the ordered ("fast") two-sum, and the exact product error
// of one FMA.  Every step is an explicitly rounded intrinsic, so the compiler neither contracts a
// product into a later sum nor reassociates.  Additions use the short form (one two-sum of the
// high parts, the low parts added once): its error is a few u^2 (|a| + |b|) with u = 2^-24, a
// normwise bound of the kind the FFT and the stencils need.  Products drop lo * lo (below u^2).
// Everything runs on the FP32 pipe, which has 64 times the FP64 rate of this GPU.
#pragma once
#include "common.cuh"

namespace lsm {

struct __align__(8) dfloat {
    float hi, lo;
    dfloat() = default;
    __host__ __device__ constexpr dfloat(float h, float l) : hi(h), lo(l) {}
    __host__ __device__ constexpr dfloat(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
    __host__ __device__ constexpr dfloat(int v) : dfloat((double)v) {}
};
struct __align__(16) dfcplx {
    dfloat x, y;
};

template <> struct cplx_of<dfloat> { typedef dfcplx type; };
template <> struct real_of<dfcplx> { typedef dfloat type; };

__host__ __device__ inline double df_value(dfloat a) { return (double)a.hi + (double)a.lo; }

// v * 2^-e as a pair: hi = v * 2^-e rounded to FP32 (nearest even), lo = the remainder rounded to
// FP32, the same pair as hi = fl32(w), lo = fl32(w - hi) for w = v * 2^-e, but by integer operations
// on the FP64 bit pattern and one int -> float conversion (FP64 arithmetic runs at 1/64 of the FP32
// rate here).  Results below FP32's normal range give +-0 (lo is dropped below 2^-74), results
// beyond it +-inf; NaN stays NaN.
__device__ __forceinline__ dfloat df_split(double v, int e) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int E = (int)((b >> 52) & 0x7ff);
    const unsigned long long frac = b & 0xFFFFFFFFFFFFFull;
    if (E == 0x7ff) return dfloat(__uint_as_float(sign | 0x7f800000u | (frac ? 0x400000u : 0u)), 0.f);
    const int fe = E - 1023 - e + 127;    // biased FP32 exponent of the leading bit
    if (E == 0 || fe <= 0) return dfloat(__uint_as_float(sign), 0.f);
    if (fe >= 255) return dfloat(__uint_as_float(sign | 0x7f800000u), 0.f);
    const unsigned long long sig = frac | (1ull << 52);          // 53-bit significand
    const unsigned keep = (unsigned)(sig >> 29);                  // its leading 24 bits
    const unsigned rem = (unsigned)(sig & 0x1FFFFFFFull);         // the 29 below
    const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (keep & 1u))) ? 1u : 0u;
    // a carry out of the 23 stored bits moves into the exponent field, as it should
    const unsigned hb = ((unsigned)fe << 23) + (keep - 0x800000u) + up;
    if (hb >= 0x7f800000u) return dfloat(__uint_as_float(sign | 0x7f800000u), 0.f);
    // remainder rem - up 2^29 (|.| <= 2^28) in units of 2^(fe - 179)
    const int r = (int)rem - (int)(up << 29);
    float lo = 0.f;
    if (fe > 52 && r != 0) lo = __fmul_rn(__int2float_rn(r), __uint_as_float((unsigned)(fe - 52) << 23));
    return dfloat(__uint_as_float(sign | hb), sign ? -lo : lo);
}

// s + e = a + b exactly
__device__ __forceinline__ dfloat df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return dfloat(s, e);
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ dfloat df_fast_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return dfloat(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ dfloat operator-(dfloat a) { return dfloat(-a.hi, -a.lo); }
__device__ __forceinline__ dfloat operator+(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    return df_fast_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat operator-(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, -b.hi);
    return df_fast_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat operator*(dfloat a, dfloat b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast_sum(p, e);
}
__device__ __forceinline__ dfloat& operator+=(dfloat& a, dfloat b) { return a = a + b; }
__device__ __forceinline__ dfloat& operator-=(dfloat& a, dfloat b) { return a = a - b; }
__device__ __forceinline__ dfloat& operator*=(dfloat& a, dfloat b) { return a = a * b; }

// sum_i a_i b_i (N >= 1): the high products are added by a chain of two-sums; every rounding error
// (of the products, of the chain) and the hi * lo cross terms are collected in one FP32 word that
// is added once at the end.  Error below (N + 3) u^2 sum_i |a_i b_i|.
template <int N>
__device__ __forceinline__ dfloat df_dot(const dfloat (&a)[N], const dfloat (&b)[N]) {
    float s = __fmul_rn(a[0].hi, b[0].hi);
    float t = __fmaf_rn(a[0].hi, b[0].hi, -s);
    t = __fmaf_rn(a[0].hi, b[0].lo, t);
    t = __fmaf_rn(a[0].lo, b[0].hi, t);
#pragma unroll
    for (int i = 1; i < N; ++i) {
        const float p = __fmul_rn(a[i].hi, b[i].hi);
        const float ep = __fmaf_rn(a[i].hi, b[i].hi, -p);
        const dfloat q = df_two_sum(s, p);
        s = q.hi;
        t = __fadd_rn(t, __fadd_rn(q.lo, ep));
        t = __fmaf_rn(a[i].hi, b[i].lo, t);
        t = __fmaf_rn(a[i].lo, b[i].hi, t);
    }
    return df_fast_sum(s, t);
}

// Complex sums of the FFT butterflies: the two-sum of the high parts, with its error and the low
// parts added into lo, and no final renormalisation (3 of 11 operations per real sum).  lo may then
// exceed ulp(hi) / 2 by the few sums between two products; hi + lo still holds the value, every
// operation here accepts such operands, and the products (df_dot) renormalise.  The error stays a
// few u^2 (|a| + |b|), the normwise bound of the FFT.
__device__ __forceinline__ dfloat df_add_lazy(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, b.hi);
    return dfloat(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ dfloat df_sub_lazy(dfloat a, dfloat b) {
    const dfloat s = df_two_sum(a.hi, -b.hi);
    return dfloat(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, b.lo)));
}
template <> __device__ __forceinline__ dfcplx cadd<dfcplx>(dfcplx a, dfcplx b) {
    dfcplx r;
    r.x = df_add_lazy(a.x, b.x);
    r.y = df_add_lazy(a.y, b.y);
    return r;
}
template <> __device__ __forceinline__ dfcplx csub<dfcplx>(dfcplx a, dfcplx b) {
    dfcplx r;
    r.x = df_sub_lazy(a.x, b.x);
    r.y = df_sub_lazy(a.y, b.y);
    return r;
}

// complex operations of the FFTs and the Green multiply as dot products
template <> __device__ __forceinline__ dfcplx cmul<dfcplx>(dfcplx a, dfcplx b) {
    const dfloat ar[2] = {a.x, -a.y}, br[2] = {b.x, b.y};
    const dfloat ai[2] = {a.x, a.y}, bi[2] = {b.y, b.x};
    dfcplx r;
    r.x = df_dot(ar, br);
    r.y = df_dot(ai, bi);
    return r;
}
template <> __device__ __forceinline__ dfcplx cmulc<dfcplx>(dfcplx a, dfcplx b) {
    const dfloat ar[2] = {a.x, a.y}, br[2] = {b.x, b.y};
    const dfloat ai[2] = {a.y, -a.x};
    dfcplx r;
    r.x = df_dot(ar, br);
    r.y = df_dot(ai, br);
    return r;
}
// a * (re + S i im_s) with compile-time constants re, im_s (folded into dfloat pairs)
template <int S>
__device__ __forceinline__ dfcplx cmul_const(dfcplx a, double re, double im_s) {
    const dfloat cr(re), ci(S * im_s);
    const dfloat ar[2] = {a.x, -a.y}, br[2] = {cr, ci};
    const dfloat ai[2] = {a.x, a.y}, bi[2] = {ci, cr};
    dfcplx r;
    r.x = df_dot(ar, br);
    r.y = df_dot(ai, bi);
    return r;
}
// g0 qa + g1 qb + g2 qc (conj(g) for CONJ)
template <bool CONJ>
__device__ __forceinline__ dfcplx gdot3(dfcplx g0, dfcplx qa, dfcplx g1, dfcplx qb, dfcplx g2, dfcplx qc) {
    const dfloat y0 = CONJ ? -g0.y : g0.y, y1 = CONJ ? -g1.y : g1.y, y2 = CONJ ? -g2.y : g2.y;
    const dfloat gr[6] = {g0.x, -y0, g1.x, -y1, g2.x, -y2};
    const dfloat gi[6] = {g0.x, y0, g1.x, y1, g2.x, y2};
    const dfloat qr[6] = {qa.x, qa.y, qb.x, qb.y, qc.x, qc.y};
    const dfloat qi[6] = {qa.y, qa.x, qb.y, qb.x, qc.y, qc.x};
    dfcplx r;
    r.x = df_dot(gr, qr);
    r.y = df_dot(gi, qi);
    return r;
}

__device__ __forceinline__ dfloat flip_sign(dfloat v, unsigned m) { return dfloat(flip_sign(v.hi, m), flip_sign(v.lo, m)); }
__device__ __forceinline__ dfcplx flip_sign(dfcplx v, unsigned m) {
    dfcplx r;
    r.x = flip_sign(v.x, m);
    r.y = flip_sign(v.y, m);
    return r;
}

// read-only loads of the pair types (the built-in overloads stay visible)
using ::__ldg;
__device__ __forceinline__ dfloat __ldg(const dfloat* p) {
    const float2 v = ::__ldg(reinterpret_cast<const float2*>(p));
    return dfloat(v.x, v.y);
}
__device__ __forceinline__ dfcplx __ldg(const dfcplx* p) {
    const float4 v = ::__ldg(reinterpret_cast<const float4*>(p));
    dfcplx r;
    r.x = dfloat(v.x, v.y);
    r.y = dfloat(v.z, v.w);
    return r;
}

}  // namespace lsm
