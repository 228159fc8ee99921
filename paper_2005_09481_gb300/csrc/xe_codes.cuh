// xe_codes.cuh -- encodings of 4-bit sample values as tensor-core operands (shared by the
// correlation staging kernels and the beam kernel).
#pragma once
#include <cstdint>

namespace xe {

// e4m3: sign bit 7, 4-bit exponent (bias 7) in bits 3-6, 3-bit mantissa.  Integers up to
// 16 in magnitude are exact.  f16: sign bit 15, 5-bit exponent (bias 15), 10-bit mantissa.
__host__ __device__ constexpr uint32_t encode_small_int(int v, int elem_bytes) {
    if (v == 0) return 0u;
    const uint32_t neg = v < 0 ? 1u : 0u;
    const int m = v < 0 ? -v : v;
    const int e = m >= 16 ? 4 : m >= 8 ? 3 : m >= 4 ? 2 : m >= 2 ? 1 : 0;
    const int frac = m - (1 << e);
    if (elem_bytes == 1)
        return (neg << 7) | (uint32_t(e + 7) << 3) | uint32_t(frac << (3 - e));
    return (neg << 15) | (uint32_t(e + 15) << 10) | uint32_t(frac << (10 - e));
}

__host__ __device__ constexpr int nibble_value(int nib) { return nib >= 8 ? nib - 16 : nib; }

// Four e4m3 codes packed little-endian into one word: nibble values lo..lo+3.
__host__ __device__ constexpr uint32_t pack_codes(int lo) {
    return encode_small_int(nibble_value(lo), 1) | (encode_small_int(nibble_value(lo + 1), 1) << 8) |
           (encode_small_int(nibble_value(lo + 2), 1) << 16) | (encode_small_int(nibble_value(lo + 3), 1) << 24);
}

// Four packed samples -> their eight e4m3 codes in nibble order: lo = {im0, re0, im1, re1},
// hi = {im2, re2, im3, re3} (byte k of v: high nibble re_k, low nibble im_k).  The word's own
// nibbles, with bit 3 cleared, are the byte-permute selectors into the code tables (the
// selector uses the low 16 bits, i.e. samples 0 and 1, hence the shift for samples 2 and 3);
// the sign masks come from sign-replicate selectors on v (re signs, bit 7 of each byte) and
// v << 4 (im signs, bit 3).
__device__ __forceinline__ void e4m3_of_bytes_nibble_order(uint32_t v, uint32_t &lo, uint32_t &hi) {
    constexpr uint32_t P0 = pack_codes(0), P1 = pack_codes(4), N0 = pack_codes(8), N1 = pack_codes(12);
    const uint32_t m = v & 0x77777777u;
    const uint32_t v4 = v << 4;
    uint32_t ml, mh;
    asm("prmt.b32 %0, %1, %2, 0x9D8C;" : "=r"(ml) : "r"(v), "r"(v4));
    asm("prmt.b32 %0, %1, %2, 0xBFAE;" : "=r"(mh) : "r"(v), "r"(v4));
    lo = (__byte_perm(P0, P1, m) & ~ml) | (__byte_perm(N0, N1, m) & ml);
    const uint32_t m2 = m >> 16;
    hi = (__byte_perm(P0, P1, m2) & ~mh) | (__byte_perm(N0, N1, m2) & mh);
}

// Four packed samples -> the e4m3 codes of their real parts (re) and imaginary parts (im),
// byte k each: the nibble-order codes above, de-interleaved by two byte permutes.
__device__ __forceinline__ void e4m3_of_bytes(uint32_t v, uint32_t &re, uint32_t &im) {
    uint32_t lo, hi;
    e4m3_of_bytes_nibble_order(v, lo, hi);
    re = __byte_perm(lo, hi, 0x7531);
    im = __byte_perm(lo, hi, 0x6420);
}

}  // namespace xe
