// ca_fconv.h -- integer to binary32 conversions in plain integer arithmetic.
//
// The fit converts 64- and 128-bit integer numerators to binary32, rounded to
// nearest with ties to even.  The GPU's own 64-bit integer conversions issue
// on the double-precision pipe, which is narrow on this part, so these build
// the float from its bits with integer instructions instead: normalise, keep
// 24 bits, round on the bits below, and let a mantissa carry from rounding up
// move into the exponent field.  The same source compiles for the host, where
// a test checks it against the compiler's own conversions.
#pragma once
#include <cstdint>
#include <cstring>

#if defined(__CUDACC__)
#define CA_FCONV_HD __host__ __device__ __forceinline__
#else
#define CA_FCONV_HD inline
#endif

namespace ca {

CA_FCONV_HD int clz64_(uint64_t u) {   // u != 0
#if defined(__CUDA_ARCH__)
    return __clzll((long long)u);
#else
    return __builtin_clzll(u);
#endif
}

CA_FCONV_HD float f32_from_bits_(uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __uint_as_float(b);
#else
    float f;
    std::memcpy(&f, &b, sizeof(f));
    return f;
#endif
}

// Nearest binary32 (ties to even) of u.
CA_FCONV_HD float u64_to_f32(uint64_t u) {
    if (u == 0) return 0.0f;
    const int lz = clz64_(u);
    const uint64_t nrm = u << lz;                // leading one at bit 63
    uint32_t mant = (uint32_t)(nrm >> 40);       // 24 bits with the leading one
    const uint64_t rest = nrm << 24;             // the bits below, left-aligned
    const uint64_t half = 1ull << 63;
    if (rest > half || (rest == half && (mant & 1u))) ++mant;   // may reach 2^24
    const uint32_t e = (uint32_t)(63 - lz + 127);               // biased exponent
    return f32_from_bits_(((e - 1u) << 23) + mant);   // mant's leading one adds 1 << 23
}

// Nearest binary32 (ties to even) of v.
CA_FCONV_HD float i64_to_f32(int64_t v) {
    const bool neg = v < 0;
    const uint64_t m = neg ? 0ull - (uint64_t)v : (uint64_t)v;
    const float f = u64_to_f32(m);
    return neg ? -f : f;
}

// Nearest binary32 (ties to even) of the unsigned 128-bit integer hi:lo.
CA_FCONV_HD float u128_to_f32(uint64_t hi, uint64_t lo) {
    if (hi == 0) return u64_to_f32(lo);
    const int lz = clz64_(hi);
    const int sh = 64 - lz;   // bits dropped to fit 64
    uint64_t top, rest;
    if (lz == 0) { top = hi; rest = lo; }
    else { top = (hi << lz) | (lo >> sh); rest = lo << lz; }
    top |= (rest != 0) ? 1ull : 0ull;   // sticky bit, far below the rounding point
    // top has 64 significant bits: scaling its rounded value by 2^sh is exact
    const float f = u64_to_f32(top);
    return f * f32_from_bits_((uint32_t)(127 + sh) << 23);
}

// Nearest binary32 (ties to even) of num / den, den != 0, |num| and |den|
// below 2^37; +0 for num = 0.  The quotient is taken to 25 or 26 significant
// bits (the operands shifted by a power of two), estimated by a binary32
// division and corrected to the exact integer quotient with 64-bit products;
// the bits below the 24 kept and the remainder then decide the rounding.
CA_FCONV_HD float ratio_to_f32(int64_t num, int64_t den) {
    if (num == 0) return 0.0f;
    const bool neg = (num < 0) != (den < 0);
    const uint64_t a = num < 0 ? 0ull - (uint64_t)num : (uint64_t)num;
    const uint64_t b = den < 0 ? 0ull - (uint64_t)den : (uint64_t)den;
    const int sh = 25 - (clz64_(b) - clz64_(a));   // a 2^sh / b in [2^24, 2^26)
    const uint64_t n = sh >= 0 ? a << sh : a;        // below 2^63
    const uint64_t d = sh >= 0 ? b : b << -sh;
#if defined(__CUDA_ARCH__)
    uint64_t q = __float2uint_rz(__fdiv_rn(u64_to_f32(n), u64_to_f32(d)));
#else
    uint64_t q = (uint64_t)(u64_to_f32(n) / u64_to_f32(d));
#endif
    for (int i = 0; i < 64 && q * d > n; ++i) --q;        // the estimate is within a few units
    for (int i = 0; i < 64 && (q + 1) * d <= n; ++i) ++q;
    bool sticky = n - q * d != 0;
    int e2 = -sh;                                        // num / den = (q + rem / d) 2^e2
    if (q >> 25) {
        sticky = sticky || (q & 1u);
        q >>= 1;
        ++e2;
    }
    uint32_t mant = (uint32_t)(q >> 1);                  // 24 bits; q's bit 0 rounds
    if ((q & 1u) && (sticky || (mant & 1u))) ++mant;     // 2^24 at most: still exact
    const float v = (float)mant * f32_from_bits_((uint32_t)(127 + e2 + 1) << 23);
    return neg ? -v : v;
}

}  // namespace ca
