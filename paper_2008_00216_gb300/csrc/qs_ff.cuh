// Float-float arithmetic for complex128 on the FP32 pipe (GB300's FP64 pipe
// runs at 1/64 of its FP32 rate).
#pragma once

#include <stdint.h>

#include "qs_device.cuh"

namespace qsgb {
namespace {

// Complex128 tiles in float-float arithmetic: each amplitude d is held as
// hi + lo with hi = float(d) and lo = float(d - hi) (about 48 significant
// bits), and every product and sum runs on the FP32 pipe with error-free
// transformations (FMA-based TwoProd, Knuth's TwoSum), accumulating the
// rounding errors of a sum of products in a second float.  Only the loads
// and stores convert to and from FP64.
struct FFC {
    float2 h, l;   // (re, im) high parts, (re, im) low parts
};
// d = hi + lo with integer operations only (the FP64 pipe is the scarce one):
// hi keeps the top 24 significant bits (truncated), lo the next 29 rounded
// to 24 (total relative error below 2^-48).  Zeros (frequent: a state
// starts sparse) map to zeros; other magnitudes whose low part would leave
// float's normal range (|d| < 2^-74, |d| >= 2^128) take the plain FP64
// conversion, in out-of-line functions (rarely taken).
__device__ __noinline__ float2 ff_split_fp64(double d) {
    const float hi = (float)d;
    return make_float2(hi, (float)(d - (double)hi));
}
__device__ __noinline__ double ff_merge_fp64(float hi, float lo) { return (double)hi + (double)lo; }
__device__ __forceinline__ void ff_split(double d, float& hi, float& lo) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(d);
    const int e = (int)((b >> 52) & 0x7FFu) - 1023;
    if ((b << 1) == 0) {  // +-0 (common: states start sparse)
        hi = lo = __uint_as_float((unsigned)(b >> 32) & 0x80000000u);
        return;
    }
    if (e < -74 || e > 127) {
        const float2 r = ff_split_fp64(d);
        hi = r.x;
        lo = r.y;
        return;
    }
    const unsigned sign = (unsigned)(b >> 63) << 31;
    const unsigned long long m = b & 0xFFFFFFFFFFFFFull;
    hi = __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(m >> 29));
    const unsigned r = (unsigned)(m & 0x1FFFFFFFu);            // r * 2^(e - 52)
    const float lm = __uint2float_rn(r) * __uint_as_float((unsigned)(e - 52 + 127) << 23);
    lo = sign ? -lm : lm;
}
// hi + lo to FP64 with integer operations: hi + lo needs at most 49
// significant bits when |lo| <= ulp(hi) (as after ffa_get), so it is
// summed exactly in 64-bit fixed point at hi's scale and normalised.
__device__ __forceinline__ double ff_merge(float hi, float lo) {
    const unsigned hb = __float_as_uint(hi), lb = __float_as_uint(lo);
    const int eh = (int)((hb >> 23) & 0xFFu), el = (int)((lb >> 23) & 0xFFu);
    if (((hb | lb) << 1) == 0) return __longlong_as_double((long long)(hb >> 31) << 63);   // +-0
    if (eh == 0 || eh == 255 || el == 255 || (el != 0 && eh - el > 60)) return ff_merge_fp64(hi, lo);
    // 53-bit fixed point: value = T * 2^(eh - 127 - 52)
    long long T = (long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;
    if (el != 0) {
        const long long L = (long long)((lb & 0x7FFFFFu) | 0x800000u);
        const int sh = 29 - (eh - el);
        const long long Ls = sh >= 0 ? (L << sh) : (L >> (-sh));
        T += ((hb ^ lb) >> 31) ? -Ls : Ls;
    }
    if (T <= 0) return ff_merge_fp64(hi, lo);   // cannot happen for |lo| <= ulp(hi)
    // normalise to a 53-bit significand: leading bit at position 52
    const int lead = 63 - __clzll(T);
    int ex = eh - 127 + (lead - 52);
    unsigned long long M = (unsigned long long)T;
    M = lead >= 52 ? (M >> (lead - 52)) : (M << (52 - lead));   // lead > 52 drops no set bits here (sum of 49 bits)
    const unsigned long long bits = ((unsigned long long)(hb >> 31) << 63) | ((unsigned long long)(ex + 1023) << 52) |
                                    (M & 0xFFFFFFFFFFFFFull);
    return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ FFC ff_from(double2 d) {
    FFC r;
    ff_split(d.x, r.h.x, r.l.x);
    ff_split(d.y, r.h.y, r.l.y);
    return r;
}
__device__ __forceinline__ double2 ff_to(const FFC& v) { return make_double2(ff_merge(v.h.x, v.l.x), ff_merge(v.h.y, v.l.y)); }
struct FFAcc {
    float sr, er, si, ei;   // running sums of high parts and of everything else
};
__device__ __forceinline__ FFAcc ffa_zero() { return FFAcc{0.f, 0.f, 0.f, 0.f}; }
// S + E += (ah + al)(bh + bl), dropping al * bl (2^-48 relative)
__device__ __forceinline__ void ffa_term(float& S, float& E, float ah, float al, float bh, float bl) {
    const float p = __fmul_rn(ah, bh);  // never contracted into the sums below
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    float s, t;
    two_sum(S, p, s, t);
    S = s;
    E += t + e;
}
__device__ __forceinline__ void ffa_cmac(FFAcc& a, const FFC& m, const FFC& v) {
    ffa_term(a.sr, a.er, m.h.x, m.l.x, v.h.x, v.l.x);
    ffa_term(a.sr, a.er, -m.h.y, -m.l.y, v.h.y, v.l.y);
    ffa_term(a.si, a.ei, m.h.x, m.l.x, v.h.y, v.l.y);
    ffa_term(a.si, a.ei, m.h.y, m.l.y, v.h.x, v.l.x);
}
__device__ __forceinline__ void ffa_add(FFAcc& a, const FFC& v) {
    float s, t;
    two_sum(a.sr, v.h.x, s, t);
    a.sr = s;
    a.er += t + v.l.x;
    two_sum(a.si, v.h.y, s, t);
    a.si = s;
    a.ei += t + v.l.y;
}
__device__ __forceinline__ FFC ffa_get(const FFAcc& a) {
    FFC r;
    r.h.x = a.sr + a.er;
    r.l.x = a.er - (r.h.x - a.sr);
    r.h.y = a.si + a.ei;
    r.l.y = a.ei - (r.h.y - a.si);
    return r;
}
__device__ __forceinline__ FFC ff_rot(const FFC& v, int code) {   // i^code v
    FFC r;
    r.h = rot_i(v.h, code);
    r.l = rot_i(v.l, code);
    return r;
}
// (ah + al)(bh + bl) + (ch + cl)(dh + dl) as a float-float (hi, lo): the two
// high products exactly (FMA-based TwoProd) and summed with TwoSum, every
// other part gathered in lo (al * bl and cl * dl dropped, 2^-48 relative)
__device__ __forceinline__ float2 ff_dot2(float ah, float al, float bh, float bl, float ch, float cl, float dh, float dl) {
    const float p = __fmul_rn(ah, bh), q = __fmul_rn(ch, dh);  // never contracted into the sums below
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    float f = fmaf(ch, dh, -q);
    f = fmaf(ch, dl, f);
    f = fmaf(cl, dh, f);
    float s, t;
    two_sum(p, q, s, t);
    const float lo = (e + f) + t;
    const float h = s + lo;
    return make_float2(h, lo - (h - s));
}
__device__ __forceinline__ FFC ff_cmul(const FFC& m, const FFC& v) {
    const float2 re = ff_dot2(m.h.x, m.l.x, v.h.x, v.l.x, -m.h.y, -m.l.y, v.h.y, v.l.y);
    const float2 im = ff_dot2(m.h.x, m.l.x, v.h.y, v.l.y, m.h.y, m.l.y, v.h.x, v.l.x);
    FFC r;
    r.h = make_float2(re.x, im.x);
    r.l = make_float2(re.y, im.y);
    return r;
}
// sum of four float-float products (ah + al)(bh + bl): the high products
// exactly (TwoProd), summed with TwoSum, every other part gathered in lo
__device__ __forceinline__ float2 ff_dot4(const float (&ah)[4], const float (&al)[4], const float (&bh)[4],
                                         const float (&bl)[4]) {
    float p[4], e = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        p[k] = __fmul_rn(ah[k], bh[k]);  // never contracted into the sums below
        float ek = fmaf(ah[k], bh[k], -p[k]);
        ek = fmaf(ah[k], bl[k], ek);
        ek = fmaf(al[k], bh[k], ek);
        e += ek;
    }
    float s = p[0], t;
#pragma unroll
    for (int k = 1; k < 4; ++k) {
        float s2;
        two_sum(s, p[k], s2, t);
        s = s2;
        e += t;
    }
    const float h = s + e;
    return make_float2(h, e - (h - s));
}
// m0 a + m1 b for complex float-float values
__device__ __forceinline__ FFC ff_cmac2(const FFC& m0, const FFC& a, const FFC& m1, const FFC& b) {
    const float reah[4] = {m0.h.x, -m0.h.y, m1.h.x, -m1.h.y}, real_[4] = {m0.l.x, -m0.l.y, m1.l.x, -m1.l.y};
    const float rebh[4] = {a.h.x, a.h.y, b.h.x, b.h.y}, rebl[4] = {a.l.x, a.l.y, b.l.x, b.l.y};
    const float imah[4] = {m0.h.x, m0.h.y, m1.h.x, m1.h.y}, imal[4] = {m0.l.x, m0.l.y, m1.l.x, m1.l.y};
    const float imbh[4] = {a.h.y, a.h.x, b.h.y, b.h.x}, imbl[4] = {a.l.y, a.l.x, b.l.y, b.l.x};
    const float2 re = ff_dot4(reah, real_, rebh, rebl), im = ff_dot4(imah, imal, imbh, imbl);
    FFC r;
    r.h = make_float2(re.x, im.x);
    r.l = make_float2(re.y, im.y);
    return r;
}
// out = i^ca a + i^cb b, a zero code (-1) dropping its term: additions only
__device__ __forceinline__ FFC ff_mulfree_sum(const FFC& a, int ca, const FFC& b, int cb) {
    FFAcc acc = ffa_zero();
    if (ca >= 0) ffa_add(acc, ff_rot(a, ca));
    if (cb >= 0) ffa_add(acc, ff_rot(b, cb));
    return ffa_get(acc);
}
__device__ __forceinline__ FFC ff_shfl_xor(const FFC& v, int mask) {
    FFC r;
    r.h.x = __shfl_xor_sync(0xffffffffu, v.h.x, mask);
    r.h.y = __shfl_xor_sync(0xffffffffu, v.h.y, mask);
    r.l.x = __shfl_xor_sync(0xffffffffu, v.l.x, mask);
    r.l.y = __shfl_xor_sync(0xffffffffu, v.l.y, mask);
    return r;
}

}  // namespace
}  // namespace qsgb
