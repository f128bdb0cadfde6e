// Host-only check of rept::fast_mod (the division-free x mod m used for the colour hash) and of
// rept::mod_equals (the divisibility test behind the colour comparison) against the % operator, for edge values and 20 million pseudo-random (x, m) pairs.  Exit code 0 = all equal.
#include <cstdio>
#include <cstdint>
#include "rept_common.cuh"

static uint64_t xs(uint64_t& s) { s ^= s << 13; s ^= s >> 7; s ^= s << 17; return s; }  // xorshift64

int main() {
    const uint32_t ms[] = {2u, 3u, 5u, 7u, 10u, 20u, 64u, 100u, 1000u, 65537u, 2147483647u, 4294967295u, 4294967294u};
    const uint64_t xs_edge[] = {0ull, 1ull, 2ull, ~0ull, ~0ull - 1, 1ull << 63, (1ull << 63) - 1, 0xFFFFFFFFull,
                                0x100000000ull, 0x9E3779B97F4A7C15ull};
    long bad = 0;
    for (uint32_t m : ms) {
        const rept::FastMod f = rept::make_fastmod(m);
        for (uint64_t x : xs_edge) {
            for (int64_t dlt = -2; dlt <= 2; ++dlt) {
                uint64_t y = x + (uint64_t)dlt;
                if (rept::fast_mod(y, f) != y % m) ++bad;
                uint64_t z = (x / m) * m + (uint64_t)dlt;  // around multiples of m
                if (rept::fast_mod(z, f) != z % m) ++bad;
            }
        }
    }
    uint64_t s = 88172645463325252ull;
    for (long i = 0; i < 20000000; ++i) {
        uint64_t x = xs(s);
        uint32_t m = (uint32_t)(xs(s) >> (i % 31));
        if (m < 2) m = 2;
        const rept::FastMod f = rept::make_fastmod(m);
        if (rept::fast_mod(x, f) != x % m) ++bad;
    }
    // mod_equals(x, j) == (x % m == j) for j around the true remainder and beyond m
    s = 2463534242ull;
    for (long i = 0; i < 5000000; ++i) {
        uint64_t x = xs(s);
        if (i % 7 == 0) x >>= (i % 64);
        uint32_t m = (uint32_t)(xs(s) >> (i % 31));
        if (m < 2) m = 2;
        const rept::FastMod f = rept::make_fastmod(m);
        const uint32_t r = (uint32_t)(x % m);
        const uint32_t js[4] = {r, r + 1u, r ? r - 1u : m - 1u, (uint32_t)(xs(s) % m)};
        for (uint32_t j : js)
            if (rept::mod_equals(x, j, f) != (r == j)) ++bad;
        if (rept::mod_equals(x, m, f)) ++bad;
    }
    for (uint32_t m : ms) {
        const rept::FastMod f = rept::make_fastmod(m);
        for (uint64_t x : xs_edge)
            for (uint32_t j = 0; j < 3 && j < m; ++j)
                if (rept::mod_equals(x, j, f) != (x % m == j)) ++bad;
    }
    const rept::FastMod one = rept::make_fastmod(1);
    if (!rept::mod_equals(12345, 0, one) || rept::mod_equals(12345, 1, one)) ++bad;
    if (rept::fast_mod(12345, one) != 0) ++bad;
    std::printf("mismatches: %ld\n", bad);
    return bad != 0;
}
