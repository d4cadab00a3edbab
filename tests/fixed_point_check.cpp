// Host check of mls::to_fixed (the adjoint's bucket-sum rounding) against the
// exact rounding of v 2^s to the nearest integer, ties to even, computed in
// long double (64-bit significand: every product v 2^s with |v 2^s| < 2^62 is
// exact there, and llrintl rounds it in the default rounding mode).
// Usage: fixed_point_check <random cases> ; prints "cases N mismatches M".
#include <algorithm>
#include <cfenv>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "fixed_point.cuh"

static uint64_t state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64() {       // splitmix64
    uint64_t z = (state += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static long long exact(float v, int s) { return llrintl(ldexpl((long double)v, s)); }

int main(int argc, char **argv) {
    std::fesetround(FE_TONEAREST);
    const long n = argc > 1 ? atol(argv[1]) : 1000000;
    long cases = 0, bad = 0;
    auto check = [&](float v, int s) {
        if (!std::isfinite(v) || fabsl(ldexpl((long double)v, s)) >= 0x1p62L) return;
        ++cases;
        const long long a = mls::to_fixed(v, s), b = exact(v, s);
        if (a != b) {
            if (bad < 5) printf("mismatch v=%a s=%d got %lld want %lld\n", v, s, a, b);
            ++bad;
        }
    };
    for (long it = 0; it < n; ++it) {
        const uint64_t r = next_u64();
        uint32_t bits = (uint32_t)r;
        float v;
        memcpy(&v, &bits, sizeof v);
        // scales as the bucket sum chooses them: s = 61 - E - lc for the
        // bucket's largest exponent E >= that of v, lc in [0, 7]
        int E = v == 0.f ? -126 : std::max(ilogbf(fabsf(v)), -126);
        const int lc = (int)((r >> 32) & 7), extra = (int)((r >> 35) % 48);
        check(v, 61 - E - lc - extra);
    }
    // exact ties m + 1/2 at every shift, and their neighbours
    for (int rbits = 1; rbits < 25; ++rbits)
        for (uint32_t m = 0x800000u; m < 0x800000u + 2048u; ++m) {
            const float v = ldexpf((float)m, -23);
            check(v, 23 - rbits);
            check(-v, 23 - rbits);
        }
    // subnormals and zeros
    for (uint32_t b = 0; b < 4096; ++b) {
        float v;
        memcpy(&v, &b, sizeof v);
        check(v, 149);
        check(v, 160);
        check(-v, 150);
    }
    printf("cases %ld mismatches %ld\n", cases, bad);
    return bad != 0;
}
