// fbt_fx.h — conversion of the tile-update epilogue's 64-bit fixed-point products to FP64 with
// integer instructions (host and device).
//
// The epilogue of the emulated-FP64 tile product (ozaki.cu) recombines the exact digit-plane
// group sums into a 64-bit integer fx whose unit is 2^s, then subtracts fx 2^s from C in FP64.
// The value it subtracts is (double)fx scaled by 2^s: fx rounded once to 53 bits, to nearest with
// ties to even.  This file builds that double from fx's bits with 32/64-bit integer operations:
// the leading one found by a count of leading zeros, the 53 bits below it kept, the 11 bits
// under them deciding the rounding, the biased exponent placed above.  On this GPU the FP64
// pipe issues two lanes per clock per SM, so taking the int64-to-double conversion off it halves
// the epilogue's FP64 instructions (the subtraction from C stays FP64).
//
// Results outside the normal range (biased exponent outside 1..2046) take ldexp of the
// converted value, as the FP64 conversion does; the tile products never come near it.
#pragma once

#if defined(__CUDACC__)
#define FBT_FX_HD __host__ __device__ __forceinline__
#else
#define FBT_FX_HD inline
#endif

#include <math.h>
#include <stdint.h>
#include <string.h>

FBT_FX_HD int fbt_clz64(unsigned long long u) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)u);
#else
    return __builtin_clzll(u);
#endif
}

FBT_FX_HD double fbt_bits_to_double(unsigned long long b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double d;
    memcpy(&d, &b, sizeof d);
    return d;
#endif
}

// (neg ? -fx : fx) 2^s, rounded to the nearest double (ties to even) exactly as
// ldexp((double)(neg ? -fx : fx), s).  |fx| < 2^63.
FBT_FX_HD double fx_to_double_int(long long fx, int s, bool neg) {
    if (fx == 0) return 0.0;
    const unsigned long long neg_bit = (unsigned long long)neg << 63;
    const unsigned long long sign = ((unsigned long long)fx & 0x8000000000000000ull) ^ neg_bit;
    unsigned long long m = fx < 0 ? 0ull - (unsigned long long)fx : (unsigned long long)fx;
    const int lz = fbt_clz64(m);
    m <<= lz;                                            // leading one at bit 63
    // 53 kept bits (leading one at bit 52) plus one where the 11 dropped bits are above half, or
    // exactly half with an odd last kept bit; a carry to 2^53 moves into the exponent below
    const unsigned int lo = (unsigned int)m;
    const unsigned int inc = (((lo & 0x7FFu) + ((lo >> 11) & 1u) + 0x3FFu) >> 11);
    const unsigned long long q = (m >> 11) + inc;
    const int e = 1086 - lz + s;                         // biased exponent of the leading one
    if (e < 1 || e > 2046) {
        const double y = (double)fx;
        return ldexp(neg ? -y : y, s);
    }
    return fbt_bits_to_double(sign | ((((unsigned long long)(e - 1)) << 52) + q));
}
