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

// Four two's-complement nibbles (one in the low 4 bits of each byte) -> four e4m3 codes.
// A byte permute looks each nibble up in the 16-entry code table (held in four words:
// values 0..3, 4..7, -8..-5, -4..-1): the low 3 bits select within the non-negative or the
// negative half, bit 3 chooses the half.
__device__ __forceinline__ uint32_t e4m3_of_nibbles(uint32_t x) {
    constexpr uint32_t P0 = pack_codes(0), P1 = pack_codes(4), N0 = pack_codes(8), N1 = pack_codes(12);
    const uint32_t y = x & 0x07070707u;
    const uint32_t z = y | (y >> 4);
    const uint32_t sel = __byte_perm(z, 0, 0x0020);
    const uint32_t pos = __byte_perm(P0, P1, sel);
    const uint32_t neg = __byte_perm(N0, N1, sel);
    const uint32_t m = ((x >> 3) & 0x01010101u) * 0xFFu;
    return (pos & ~m) | (neg & m);
}

// Byte k of the result = 0xFF if bit 7 of byte k of a is set, else 0 (the byte permute's
// sign-replicate selectors 8..11; the __byte_perm intrinsic uses 3-bit selectors only).
__device__ __forceinline__ uint32_t byte_sign_mask(uint32_t a) {
    uint32_t d;
    asm("prmt.b32 %0, %1, 0, 0xBA98;" : "=r"(d) : "r"(a));
    return d;
}

// Four packed samples (byte k: high nibble re, low nibble im, two's complement) -> the e4m3
// codes of their real parts (re) and imaginary parts (im), byte k each.  The same table
// lookup as e4m3_of_nibbles, with the sign masks taken directly from the nibbles' top bits:
// the re sign is bit 7 of each byte, the im sign bit 3 (bit 7 after a 4-bit shift).
__device__ __forceinline__ void e4m3_of_bytes(uint32_t v, uint32_t &re, uint32_t &im) {
    constexpr uint32_t P0 = pack_codes(0), P1 = pack_codes(4), N0 = pack_codes(8), N1 = pack_codes(12);
    const uint32_t yi = v & 0x07070707u;
    const uint32_t si = __byte_perm(yi | (yi >> 4), 0, 0x0020);
    const uint32_t mi = byte_sign_mask(v << 4);
    im = (__byte_perm(P0, P1, si) & ~mi) | (__byte_perm(N0, N1, si) & mi);
    const uint32_t yr = (v >> 4) & 0x07070707u;
    const uint32_t sr = __byte_perm(yr | (yr >> 4), 0, 0x0020);
    const uint32_t mr = byte_sign_mask(v);
    re = (__byte_perm(P0, P1, sr) & ~mr) | (__byte_perm(N0, N1, sr) & mr);
}

}  // namespace xe
