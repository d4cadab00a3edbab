// The grid's sort key: the index of a level-0 cell along the 3-D Hilbert
// curve.  Host-and-device code: the kernels use it, and a host test checks
// the properties the grid relies on (a bijection; the top 3 l bits name the
// level-l cell, so every cell of every level is a run of consecutive keys;
// consecutive keys are face-adjacent cells).
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define MLS_HB_FN __host__ __device__ __forceinline__
#else
#define MLS_HB_FN inline
#endif

namespace mls {

// Bit b of the low 21 bits of v moved to bit 3 b.
MLS_HB_FN uint64_t hb_spread3(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | (x << 32)) & 0x1f00000000ffffull;
    x = (x | (x << 16)) & 0x1f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

// Index of the cell (x, y, z) (each coordinate below 2^bits, bits <= 21)
// along the Hilbert curve of `bits` levels, by Skilling's transform
// ("Programming the Hilbert curve", AIP Conf. Proc. 707, 2004): the
// coordinates are turned in place into the transposed index (undo the
// curve's rotations and reflections from the top bit down, then Gray-decode),
// whose bits, interleaved with the first coordinate most significant in every
// triple, give the index.
MLS_HB_FN uint64_t hilbert3(uint32_t x, uint32_t y, uint32_t z, int bits) {
    uint32_t X[3] = {x, y, z};
    for (uint32_t Q = 1u << (bits - 1); Q > 1; Q >>= 1) {
        const uint32_t P = Q - 1;
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;                              // reflect
            } else {
                const uint32_t t = (X[0] ^ X[i]) & P;   // swap the low bits of X[0] and X[i]
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    uint32_t t = 0;
    for (uint32_t Q = 1u << (bits - 1); Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    return hb_spread3(X[2] ^ t) | (hb_spread3(X[1] ^ t) << 1) | (hb_spread3(X[0] ^ t) << 2);
}

}  // namespace mls
