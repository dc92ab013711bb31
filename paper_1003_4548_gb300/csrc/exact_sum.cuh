// exact_sum.cuh -- exact, order-independent sums of FP32 values and of
// products of FP32 values, on the integer pipes.
//
// An FP32 value is m 2^(e-150) with a 24-bit integer m, and a product of two
// is a 48-bit integer times a power of two; both are added exactly into a
// 128-bit two's-complement fixed-point accumulator whose unit is 2^-80 (bits
// below 2^-80 are dropped: < 1e-24 per term). Magnitudes up to 2^40 for
// values and 2^44 for products fit with room for 2^16 terms. The sums are
// therefore exact, identical for any order of the terms, and are rounded
// once, correctly, when converted to FP64; central moments are formed exactly
// as n sum(xy) - sum(x) sum(y) in 256-bit arithmetic before that rounding.
#pragma once
#include <stdint.h>

struct Exact128 {
    unsigned long long lo = 0ull, hi = 0ull;  // signed 128-bit, unit 2^-80
};

__device__ __forceinline__ void x128_add(Exact128& a, unsigned long long lo, unsigned long long hi, bool neg) {
    if (!neg) {
        const unsigned long long s = a.lo + lo;
        a.hi = a.hi + hi + (s < a.lo ? 1ull : 0ull);
        a.lo = s;
    } else {
        const unsigned long long s = a.lo - lo;
        a.hi = a.hi - hi - (a.lo < lo ? 1ull : 0ull);
        a.lo = s;
    }
}

// place an unsigned integer mant (< 2^48) times 2^sh (unit 2^-80) into 128 bits
__device__ __forceinline__ void x128_place(unsigned long long mant, int sh, unsigned long long& lo,
                                           unsigned long long& hi) {
    if (sh >= 0) {
        if (sh < 64) {
            lo = mant << sh;
            hi = sh ? (mant >> (64 - sh)) : 0ull;
        } else {
            lo = 0ull;
            hi = sh < 128 ? (mant << (sh - 64)) : 0ull;
        }
    } else {
        lo = (-sh < 64) ? (mant >> (-sh)) : 0ull;
        hi = 0ull;
    }
}

__device__ __forceinline__ void f32_parts(float x, unsigned& m, int& e, bool& neg) {
    const unsigned b = __float_as_uint(x);
    e = (int)((b >> 23) & 0xffu);
    m = b & 0x7fffffu;
    if (e) m |= 0x800000u;
    else e = 1;
    neg = (b >> 31) != 0u;
}

// a += x
__device__ __forceinline__ void x128_add_f32(Exact128& a, float x) {
    unsigned m;
    int e;
    bool neg;
    f32_parts(x, m, e, neg);
    unsigned long long lo, hi;
    x128_place((unsigned long long)m, e - 70, lo, hi);  // m 2^(e-150) = m 2^(e-70) 2^-80
    x128_add(a, lo, hi, neg);
}

// a += x y, with the parts of x and y already split
__device__ __forceinline__ void x128_add_prod(Exact128& a, unsigned mx, int ex, bool nx, unsigned my, int ey,
                                              bool ny) {
    const unsigned long long P = (unsigned long long)mx * (unsigned long long)my;
    unsigned long long lo, hi;
    x128_place(P, ex + ey - 220, lo, hi);  // P 2^(ex+ey-300) = P 2^(ex+ey-220) 2^-80
    x128_add(a, lo, hi, nx != ny);
}

__device__ __forceinline__ Exact128 x128_shfl_down(const Exact128& a, int o) {
    Exact128 r;
    r.lo = __shfl_down_sync(0xffffffffu, a.lo, o);
    r.hi = __shfl_down_sync(0xffffffffu, a.hi, o);
    return r;
}

__device__ __forceinline__ void x128_merge(Exact128& a, const Exact128& b) { x128_add(a, b.lo, b.hi, false); }

__device__ __forceinline__ void x128_warp_sum(Exact128& a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x128_merge(a, x128_shfl_down(a, o));
}

// ---- wide integers for the final, once-per-element arithmetic ------------
// little-endian 64-bit limbs, two's complement
struct Wide4 {
    unsigned long long w[4];
};

__device__ __forceinline__ Wide4 w4_from128(const Exact128& a) {
    Wide4 r;
    r.w[0] = a.lo;
    r.w[1] = a.hi;
    const unsigned long long s = (a.hi >> 63) ? ~0ull : 0ull;
    r.w[2] = s;
    r.w[3] = s;
    return r;
}

__device__ __forceinline__ bool w4_neg(const Wide4& a) { return (a.w[3] >> 63) != 0ull; }

__device__ __forceinline__ Wide4 w4_negate(const Wide4& a) {
    Wide4 r;
    unsigned long long c = 1ull;
    for (int k = 0; k < 4; ++k) {
        const unsigned long long t = ~a.w[k] + c;
        c = (c && t == 0ull) ? 1ull : 0ull;
        r.w[k] = t;
    }
    return r;
}

__device__ __forceinline__ Wide4 w4_sub(const Wide4& a, const Wide4& b) {
    Wide4 r;
    unsigned long long br = 0ull;
    for (int k = 0; k < 4; ++k) {
        const unsigned long long t = a.w[k] - b.w[k];
        const unsigned long long t2 = t - br;
        br = (a.w[k] < b.w[k] || t < br) ? 1ull : 0ull;
        r.w[k] = t2;
    }
    return r;
}

// unsigned 128 x 128 -> 256
__device__ __forceinline__ Wide4 w4_mul128(unsigned long long alo, unsigned long long ahi, unsigned long long blo,
                                           unsigned long long bhi) {
    Wide4 r = {{0ull, 0ull, 0ull, 0ull}};
    const unsigned long long a[2] = {alo, ahi}, b[2] = {blo, bhi};
    for (int i = 0; i < 2; ++i) {
        unsigned long long carry = 0ull;
        for (int j = 0; j < 2; ++j) {
            const unsigned long long plo = a[i] * b[j], phi = __umul64hi(a[i], b[j]);
            unsigned long long s = r.w[i + j] + plo;
            unsigned long long c1 = s < plo ? 1ull : 0ull;
            const unsigned long long s2 = s + carry;
            c1 += s2 < s ? 1ull : 0ull;
            r.w[i + j] = s2;
            carry = phi + c1;
        }
        r.w[i + 2] += carry;
    }
    return r;
}

// signed 128 x signed 128 -> signed 256
__device__ __forceinline__ Wide4 w4_smul(const Exact128& a, const Exact128& b) {
    Wide4 A = w4_from128(a), Bw = w4_from128(b);
    const bool na = w4_neg(A), nb = w4_neg(Bw);
    if (na) A = w4_negate(A);
    if (nb) Bw = w4_negate(Bw);
    Wide4 r = w4_mul128(A.w[0], A.w[1], Bw.w[0], Bw.w[1]);
    return (na != nb) ? w4_negate(r) : r;
}

// signed 128 times a positive 32-bit n, shifted left by 80 bits
__device__ __forceinline__ Wide4 w4_mul_n_shl80(const Exact128& a, unsigned n) {
    Wide4 A = w4_from128(a);
    const bool na = w4_neg(A);
    if (na) A = w4_negate(A);
    Wide4 p = w4_mul128(A.w[0], A.w[1], (unsigned long long)n, 0ull);  // < 2^152
    // shift left by 80 = 64 + 16
    Wide4 r;
    r.w[0] = 0ull;
    r.w[1] = p.w[0] << 16;
    r.w[2] = (p.w[1] << 16) | (p.w[0] >> 48);
    r.w[3] = (p.w[2] << 16) | (p.w[1] >> 48);
    return na ? w4_negate(r) : r;
}

// correctly rounded conversion of a signed 256-bit integer times 2^scale
__device__ __forceinline__ double w4_to_double(Wide4 a, int scale) {
    const bool neg = w4_neg(a);
    if (neg) a = w4_negate(a);
    int top = 3;
    while (top >= 0 && a.w[top] == 0ull) --top;
    if (top < 0) return 0.0;
    const int lz = __clzll(a.w[top]);
    const int msb = 64 * top + 63 - lz;  // index of the leading one
    // the leading 64 bits, with the bits below them folded into a sticky bit
    unsigned long long head, sticky = 0ull;
    const int shift = msb - 63;  // bits below the 64-bit head
    if (shift <= 0) {
        head = a.w[0] << (-shift);
    } else {
        const int ws = shift >> 6, bs = shift & 63;
        head = a.w[ws] >> bs;
        if (bs && ws + 1 <= 3) head |= a.w[ws + 1] << (64 - bs);
        for (int k = 0; k < ws; ++k) sticky |= a.w[k];
        if (bs) sticky |= a.w[ws] & ((1ull << bs) - 1ull);
    }
    if (sticky) head |= 1ull;  // below the rounding position of a double (64 > 53 bits)
    const double d = __ull2double_rn(head);
    const double r = ldexp(d, (shift > 0 ? shift : 0) + (shift < 0 ? shift : 0) + scale);
    return neg ? -r : r;
}

__device__ __forceinline__ double x128_to_double(const Exact128& a) { return w4_to_double(w4_from128(a), -80); }

// exact central moment sum_i (x_i - xbar)(y_i - ybar) / n from exact sums
__device__ __forceinline__ double x128_central(const Exact128& sxy, const Exact128& sx, const Exact128& sy,
                                               unsigned n) {
    const Wide4 a = w4_mul_n_shl80(sxy, n);  // n sum(xy), unit 2^-160
    const Wide4 b = w4_smul(sx, sy);         // sum(x) sum(y), unit 2^-160
    const double d = w4_to_double(w4_sub(a, b), -160);
    return d / ((double)n * (double)n);
}
