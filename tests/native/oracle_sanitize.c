/* Host check of the CPU oracle under AddressSanitizer and UndefinedBehaviorSanitizer: random small
 * graphs (each edge kept with probability q, shuffled stream order, a self-loop mixed in) through
 * every oracle routine, with the streaming counts checked against the static enumeration.  Exit
 * code 0 = every check held and the sanitizers reported nothing (they abort on the first report). */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

int orc_rept_stream(const uint32_t*, const uint32_t*, uint64_t, uint32_t, uint32_t, uint32_t, uint64_t,
                    uint64_t*, uint64_t*, uint64_t*, uint64_t*, uint64_t*, uint64_t*, uint64_t*);
int orc_rept_stream_parallel(const uint32_t*, const uint32_t*, uint64_t, uint32_t, uint32_t, uint32_t, uint64_t,
                             uint64_t*, uint64_t*, uint64_t*, int);
void orc_estimates(uint32_t, uint32_t, const uint64_t*, const uint64_t*, const uint64_t*, const uint64_t*,
                   const uint64_t*, uint32_t, double*, double*);
int orc_semitriangles(const uint32_t*, const uint32_t*, uint64_t, uint32_t, uint32_t, uint32_t, uint64_t,
                      uint64_t*, uint64_t*, uint64_t*, uint64_t*, uint64_t*, uint64_t*, uint64_t*, uint64_t*);
int orc_mascot_stream(const uint32_t*, const uint32_t*, uint64_t, uint32_t, uint32_t, uint32_t, uint64_t,
                      uint64_t*, uint64_t*, uint64_t*, uint64_t*);
int orc_mascot_semitriangles(const uint32_t*, const uint32_t*, uint64_t, uint32_t, uint32_t, uint32_t, uint64_t,
                             uint64_t*, uint64_t*, uint64_t*);

static uint64_t rng = 0x1234567ull;
static uint32_t next32(void) {  /* xorshift64* */
    rng ^= rng >> 12; rng ^= rng << 25; rng ^= rng >> 27;
    return (uint32_t)((rng * 0x2545F4914F6CDD1Dull) >> 32);
}

static int same(const uint64_t* a, const uint64_t* b, size_t k) { return memcmp(a, b, k * sizeof(uint64_t)) == 0; }

int main(void) {
    int bad = 0;
    const uint32_t cases[][2] = {{1, 1}, {3, 2}, {2, 4}, {3, 7}, {4, 8}};
    for (uint32_t n = 12; n <= 60; n += 16) {
        uint32_t cap = n * (n - 1) / 2 + 1, T = 0;
        uint32_t* src = malloc(cap * sizeof(uint32_t));
        uint32_t* dst = malloc(cap * sizeof(uint32_t));
        for (uint32_t a = 0; a < n; ++a)
            for (uint32_t b = a + 1; b < n; ++b)
                if (next32() % 100 < 45) { src[T] = (next32() & 1) ? a : b; dst[T] = src[T] == a ? b : a; ++T; }
        src[T] = dst[T] = n / 2; ++T;  /* a self-loop */
        for (uint32_t t = T - 1; t > 0; --t) {
            uint32_t j = next32() % (t + 1), x = src[t], y = dst[t];
            src[t] = src[j]; dst[t] = dst[j]; src[j] = x; dst[j] = y;
        }
        for (size_t k = 0; k < sizeof cases / sizeof cases[0]; ++k) {
            uint32_t m = cases[k][0], c = cases[k][1];
            uint64_t* tau = calloc(c, 8); uint64_t* eta = calloc(c, 8); uint64_t* tau2 = calloc(c, 8);
            uint64_t* l1 = calloc(n, 8); uint64_t* l2 = calloc(n, 8); uint64_t* el = calloc(n, 8);
            uint64_t* p1 = calloc(n, 8); uint64_t* p2 = calloc(n, 8);
            uint64_t* lp = calloc((size_t)c * n, 8); uint64_t* lp2 = calloc((size_t)c * n, 8);
            uint64_t* s1 = calloc(n, 8); uint64_t* s2 = calloc(n, 8); uint64_t* tl = calloc(n, 8); uint64_t* etl = calloc(n, 8);
            uint64_t skipped = 0, tri = 0, et = 0;
            double g = 0, *loc = calloc(n, sizeof(double));
            if (orc_rept_stream(src, dst, T, n, m, c, 9, tau, eta, l1, l2, el, lp, &skipped)) bad++;
            if (skipped != 1) bad++;
            if (orc_semitriangles(src, dst, T, n, m, c, 9, tau2, s1, s2, lp2, &tri, tl, &et, etl)) bad++;
            if (!same(tau, tau2, c) || !same(l1, s1, n) || !same(l2, s2, n) || !same(lp, lp2, (size_t)c * n)) bad++;
            if (orc_rept_stream_parallel(src, dst, T, n, m, c, 9, tau2, p1, p2, 3)) bad++;
            if (!same(tau, tau2, c) || !same(l1, p1, n) || !same(l2, p2, n)) bad++;
            orc_estimates(m, c, tau, eta, l1, l2, el, n, &g, loc);
            if (!(g >= 0.0)) bad++;
            if (orc_mascot_stream(src, dst, T, n, m, c, 9, tau, l1, lp, &skipped)) bad++;
            if (orc_mascot_semitriangles(src, dst, T, n, m, c, 9, tau2, s1, lp2)) bad++;
            if (!same(tau, tau2, c) || !same(l1, s1, n) || !same(lp, lp2, (size_t)c * n)) bad++;
            free(tau); free(eta); free(tau2); free(l1); free(l2); free(el); free(p1); free(p2); free(lp); free(lp2);
            free(s1); free(s2); free(tl); free(etl); free(loc);
        }
        free(src); free(dst);
    }
    printf("oracle sanitize failures: %d\n", bad);
    return bad != 0;
}
