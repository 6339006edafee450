// Conversions between FP64 and two-float (hi + lo) values by integer bit manipulation.
//
// GB300's scalar FP64 unit issues about 0.4 additions per SM per clock (a sweep level
// of the n = 4e6 graph kept it 72 % busy), so the FP64 form of the sweeps does its
// per-level arithmetic in two-float on the FP32 pipe and converts between the FP64
// values it stores and the two-floats it adds with integer instructions only:
//
//   double_to_f2_bits(v): hi = v rounded to the nearest float (ties to even), lo = v - hi
//                    rounded to the nearest float; |v - (hi + lo)| <= 2^-48 |v|.
//   f2_to_double_bits(a): hi + lo rounded toward zero to 53 bits (at most one unit in the
//                    last place of the double from the exact sum).
//
// Magnitudes below 2^-126 (about 1.2e-38) map to zero and lo parts below that bound are
// dropped: the sweeps carry probabilities and similarities in [0, 5], where such terms
// are far below every tolerance.  Infinities and NaNs do not occur.
#pragma once

#include <stdint.h>
#include <string.h>

#include "twofloat.cuh"

namespace esim {

__host__ __device__ __forceinline__ uint32_t fbits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}
__host__ __device__ __forceinline__ float bitsf(uint32_t u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
}
__host__ __device__ __forceinline__ uint64_t dbits(double d) {
    uint64_t u;
    memcpy(&u, &d, 8);
    return u;
}
__host__ __device__ __forceinline__ double bitsd(uint64_t u) {
    double d;
    memcpy(&d, &u, 8);
    return d;
}

__host__ __device__ __forceinline__ f2 double_to_f2_bits(double v) {
    const uint64_t b = dbits(v);
    const uint32_t sign = (uint32_t)(b >> 63) << 31;
    const int e = (int)((b >> 52) & 0x7ff);
    const int ef = e - 896;  // the float exponent field of the same magnitude
    if (ef <= 0) return f2{bitsf(sign), 0.f};
    const uint64_t M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);  // 53-bit significand
    uint32_t hm = (uint32_t)(M >> 29);                           // 24 bits
    int64_t rem = (int64_t)(M & 0x1FFFFFFFull);                  // 29 bits below hi
    if (rem > (1ll << 28) || (rem == (1ll << 28) && (hm & 1u))) {
        ++hm;
        rem -= 1ll << 29;
    }
    int efh = ef;
    if (hm == (1u << 24)) {  // the rounding carried into a new binade
        hm >>= 1;
        ++efh;
    }
    const float hi = bitsf(sign | ((uint32_t)efh << 23) | (hm & 0x7FFFFFu));
    float lo = 0.f;
    const int el = e - 948;  // float exponent field of 2^(e - 1075), the unit of rem
    if (rem != 0 && el >= 1) {
        const float r = (float)(int32_t)rem;  // |rem| <= 2^28: one rounding to 24 bits
        lo = r * bitsf((uint32_t)el << 23);   // exact scaling by a power of two
        if (sign) lo = -lo;
    }
    return f2{hi, lo};
}

__host__ __device__ __forceinline__ double f2_to_double_bits(f2 a) {
    const uint32_t bh = fbits(a.hi);
    const int eh = (int)((bh >> 23) & 0xff);
    if (eh == 0) return 0.0;
    const uint64_t sh = (uint64_t)(bh >> 31);
    // hi = Mh 2^(eh - 150); as a 53-bit significand T 2^(eh - 179)
    int64_t T = (int64_t)((uint64_t)((bh & 0x7FFFFFu) | 0x800000u) << 29);
    const uint32_t bl = fbits(a.lo);
    const int el = (int)((bl >> 23) & 0xff);
    if (el != 0) {
        // lo = Ml 2^(el - 150) = Ml 2^(el - eh + 29) units of T
        const int64_t Ml = (int64_t)((bl & 0x7FFFFFu) | 0x800000u);
        const int s = el - eh + 29;
        int64_t add = 0;
        if (s >= 0) add = Ml << s;
        else if (s > -25) add = Ml >> (-s);
        if ((bl >> 31) != (uint32_t)sh) add = -add;
        T += add;
    }
    int e = eh + 896;  // double exponent field of T 2^(eh - 179) with T in [2^52, 2^53)
    if (T <= 0) return bitsd(sh << 63);  // cannot happen for |lo| <= ulp(hi)/2; kept safe
    uint64_t U = (uint64_t)T;
    if (U >= (1ull << 53)) {
        U >>= 1;
        ++e;
    } else if (U < (1ull << 52)) {
        U <<= 1;
        --e;
    }
    return bitsd((sh << 63) | ((uint64_t)e << 52) | (U & 0xFFFFFFFFFFFFFull));
}

}  // namespace esim
