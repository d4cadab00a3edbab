// Host check of mls::hilbert3, the grid's sort key, for the properties the
// grid relies on: on every grid of 1..6 bits per axis it is a bijection onto
// 0 .. 8^bits - 1, the top 3 l bits of a cell's key depend only on its
// level-l cell (so each cell of each level is one run of consecutive keys),
// and consecutive keys are face-adjacent cells; on the 21-bit grid the
// level property holds on random cells, and the index of a cell's level-l
// cell on the coarse curve of 21 - l levels is the cell's key shifted down
// by 3 l (what a build that sorts only the levels from l up computes).
// Prints "failures N".
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "hilbert.cuh"

static uint64_t state = 0x2545f4914f6cdd1dull;
static uint64_t next_u64() {       // splitmix64
    uint64_t z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

int main() {
    long failures = 0;
    for (int bits = 1; bits <= 6; ++bits) {
        const uint32_t N = 1u << bits;
        const uint64_t cells = (uint64_t)N * N * N;
        std::vector<int> seen(cells, 0);
        std::vector<uint32_t> at(3 * cells);
        for (uint32_t x = 0; x < N; ++x)
            for (uint32_t y = 0; y < N; ++y)
                for (uint32_t z = 0; z < N; ++z) {
                    const uint64_t h = mls::hilbert3(x, y, z, bits);
                    if (h >= cells || seen[h]++) {
                        ++failures;
                        continue;
                    }
                    at[3 * h] = x;
                    at[3 * h + 1] = y;
                    at[3 * h + 2] = z;
                    for (int l = 1; l < bits; ++l) {
                        const uint32_t m = ~((1u << l) - 1u);
                        if ((h >> (3 * l)) != (mls::hilbert3(x & m, y & m, z & m, bits) >> (3 * l))) ++failures;
                    }
                }
        for (uint64_t h = 0; h + 1 < cells; ++h) {
            const int d = abs((int)at[3 * h] - (int)at[3 * h + 3]) + abs((int)at[3 * h + 1] - (int)at[3 * h + 4]) +
                          abs((int)at[3 * h + 2] - (int)at[3 * h + 5]);
            if (d != 1) ++failures;
        }
    }
    for (int it = 0; it < 200000; ++it) {
        const uint64_t r = next_u64();
        const uint32_t x = r & 0x1fffff, y = (r >> 21) & 0x1fffff, z = (r >> 42) & 0x1fffff;
        const int l = 1 + (int)((next_u64() >> 7) % 20);
        const uint32_t m = ~((1u << l) - 1u);
        const uint64_t full = mls::hilbert3(x, y, z, 21);
        if ((full >> (3 * l)) != (mls::hilbert3(x & m, y & m, z & m, 21) >> (3 * l))) ++failures;
        if ((full >> (3 * l)) != mls::hilbert3(x >> l, y >> l, z >> l, 21 - l)) ++failures;
    }
    printf("failures %ld\n", failures);
    return failures != 0;
}
