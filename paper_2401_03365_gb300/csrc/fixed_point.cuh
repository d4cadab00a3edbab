// Rounding of a float times a power of two to a 64-bit integer, for the exact
// fixed-point sums of the adjoint's buckets.  Host-and-device code: the same
// function runs in the kernels and in a host test against the exact rounding.
#pragma once

#include <stdint.h>
#include <string.h>

#if defined(__CUDACC__)
#define MLS_FX_FN __host__ __device__ __forceinline__
#else
#define MLS_FX_FN inline
#endif

namespace mls {

MLS_FX_FN uint32_t fx_float_bits(float v) {
#if defined(__CUDA_ARCH__)
    return __float_as_uint(v);
#else
    uint32_t b;
    memcpy(&b, &v, sizeof b);
    return b;
#endif
}

// v 2^s rounded to the nearest integer, ties to even, for |v| 2^s < 2^62: the
// same integer as converting the (exact) product v 2^s to a 64-bit integer,
// computed from the float's bits with integer instructions (on the GPU that
// conversion runs on the FP64 pipe).  v = mant 2^e2 with a 24-bit (or, for
// subnormals, smaller) integer mant; the result is mant shifted by e2 + s,
// rounded on the bits shifted out.
MLS_FX_FN long long to_fixed(float v, int s) {
    const uint32_t bits = fx_float_bits(v);
    const uint32_t ex = (bits >> 23) & 0xffu, frac = bits & 0x7fffffu;
    const uint32_t mant = ex ? (frac | 0x800000u) : frac;
    const int sh = (ex ? (int)ex - 150 : -149) + s;
    long long q;
    if (sh >= 0) {
        q = (long long)mant << sh;
    } else if (sh > -25) {
        const int r = -sh;
        const uint32_t t = mant >> r, rem = mant & ((1u << r) - 1u), half = 1u << (r - 1);
        q = (long long)(t + ((rem > half || (rem == half && (t & 1u))) ? 1u : 0u));
    } else {
        q = 0;      // below one half
    }
    return (bits >> 31) ? -q : q;
}

}  // namespace mls
