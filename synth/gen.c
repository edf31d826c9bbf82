/*
 * Seeded synthetic ring hypergraphs: the inputs that stand in for the
 * paper's benchmark flow networks (Section 8, "Instances"; the networks the
 * paper extracts from its set B are not available).
 *
 * This module only draws random structure.  It holds none of the flow
 * method's arithmetic and is shared, as input data, by the CPU oracle and by
 * the CUDA path.
 *
 * Random numbers: xoshiro256** (Blackman and Vigna, "Scrambled linear
 * pseudorandom number generators", 2018) seeded through SplitMix64 (Steele,
 * Lea and Flood, 2014), both written from their published definitions.
 * All arithmetic that shapes the output is integer or correctly rounded
 * IEEE (+, *, /, sqrt), and the file is compiled with -ffp-contract=off, so
 * x86-64 and aarch64 hosts produce the same hypergraph for the same seed.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; i++) r->s[i] = splitmix64_next(&x);
}

static uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

/* uniform integer in [0, range) by the multiply-high map of 32 random bits */
static uint32_t rng_below(rng_t *r, uint32_t range) {
    uint64_t x = rng_next(r) >> 32;
    return (uint32_t)((x * (uint64_t)range) >> 32);
}

/* uniform double in [0, 1) with 53 random bits */
static double rng_unit(rng_t *r) {
    return (double)(rng_next(r) >> 11) * (1.0 / 9007199254740992.0);
}

/* distinct sub-streams for sizes, pins, net weights, vertex weights, moves */
enum { STREAM_SIZES = 1, STREAM_PINS = 2, STREAM_NETW = 3, STREAM_NODEW = 4, STREAM_PART = 5 };

static void stream_seed(rng_t *r, uint64_t seed, uint64_t stream) {
    rng_seed(r, seed * 0x100000001b3ULL + stream * 0x9e3779b97f4a7c15ULL);
}

/*
 * Net sizes.  dist 0: 2 + Geometric(1/2) counted as failures before the first
 * success (support 0, 1, ...), truncated so that size <= cap.  dist 1:
 * 2 + Zipf(2.5) on support k >= 1 with P(k) proportional to k^-2.5, truncated
 * to size <= cap (the distribution is renormalised over 1..cap-2).
 * Returns the total number of pins, or -1 on bad arguments.
 */
int64_t synth_net_sizes(int32_t m, int32_t dist, int32_t cap, uint64_t seed, int32_t *sizes) {
    if (m < 0 || cap < 2 || (dist != 0 && dist != 1)) return -1;
    rng_t r;
    stream_seed(&r, seed, STREAM_SIZES);
    int64_t total = 0;
    if (dist == 0) {
        for (int32_t e = 0; e < m; e++) {
            int32_t g;
            for (;;) {
                uint64_t x = rng_next(&r);
                g = x ? __builtin_ctzll(x) : 64;
                if (2 + g <= cap) break;
            }
            sizes[e] = 2 + g;
            total += sizes[e];
        }
        return total;
    }
    int32_t kmax = cap - 2;
    if (kmax < 1) {
        for (int32_t e = 0; e < m; e++) { sizes[e] = 2; total += 2; }
        return total;
    }
    double *cdf = (double *)malloc(sizeof(double) * (size_t)kmax);
    if (!cdf) return -1;
    double acc = 0.0;
    for (int32_t k = 1; k <= kmax; k++) {
        double kd = (double)k;
        acc += 1.0 / (kd * kd * sqrt(kd));
        cdf[k - 1] = acc;
    }
    for (int32_t e = 0; e < m; e++) {
        double u = rng_unit(&r) * acc;
        int32_t lo = 0, hi = kmax - 1;          /* smallest k with cdf[k-1] > u */
        while (lo < hi) {
            int32_t mid = lo + (hi - lo) / 2;
            if (cdf[mid] > u) hi = mid; else lo = mid + 1;
        }
        sizes[e] = 2 + (lo + 1);
        total += sizes[e];
    }
    free(cdf);
    return total;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/*
 * Pins on a ring of n positions.  Net e draws sizes[e] distinct positions
 * without replacement (Floyd's sampling) from the window
 * [c - w/2, c + w/2) mod n around a uniform centre c, with
 * w = min(n, max(window, 2 * sizes[e])); sizes above w are clipped to w.
 * Pins of a net are stored in ascending vertex order.  net_off must hold
 * m+1 entries and pins the total returned by synth_net_sizes.
 * Net weights are uniform in [wlo, whi]; vertex weights uniform in
 * [clo, chi] (clo == chi == 1 gives unit weights).
 * Returns the number of pins written, or -1 on bad arguments.
 */
int64_t synth_ring_pins(int32_t n, int32_t m, const int32_t *sizes, int32_t window,
                        int32_t wlo, int32_t whi, int32_t clo, int32_t chi, uint64_t seed,
                        uint32_t *net_off, int32_t *pins, int32_t *net_w, int32_t *node_w) {
    if (n <= 0 || m < 0 || window <= 0 || wlo < 1 || whi < wlo || clo < 1 || chi < clo) return -1;
    rng_t rp, rw, rc;
    stream_seed(&rp, seed, STREAM_PINS);
    stream_seed(&rw, seed, STREAM_NETW);
    stream_seed(&rc, seed, STREAM_NODEW);
    int32_t wmax = window;
    for (int32_t e = 0; e < m; e++) if (2 * sizes[e] > wmax) wmax = 2 * sizes[e];
    if (wmax > n) wmax = n;
    uint32_t *mark = (uint32_t *)calloc((size_t)wmax, sizeof(uint32_t));
    if (!mark) return -1;
    uint32_t stamp = 0;
    int64_t off = 0;
    for (int32_t e = 0; e < m; e++) {
        int32_t w = window;
        if (2 * sizes[e] > w) w = 2 * sizes[e];
        if (w > n) w = n;
        int32_t sz = sizes[e] < w ? sizes[e] : w;
        int32_t c = (int32_t)rng_below(&rp, (uint32_t)n);
        int64_t base = (int64_t)c - w / 2;
        stamp++;
        if (off + sz > (int64_t)0xFFFFFFFFu) { free(mark); return -1; }
        net_off[e] = (uint32_t)off;
        int32_t cnt = 0;
        for (int32_t j = w - sz; j < w; j++) {       /* Floyd: sz distinct offsets in [0, w) */
            int32_t t = (int32_t)rng_below(&rp, (uint32_t)(j + 1));
            int32_t pick = (mark[t] == stamp) ? j : t;
            mark[pick] = stamp;
            int64_t pos = (base + pick) % n;
            if (pos < 0) pos += n;
            pins[off + cnt++] = (int32_t)pos;
        }
        qsort(pins + off, (size_t)sz, sizeof(int32_t), cmp_i32);
        off += sz;
        net_w[e] = wlo + (int32_t)rng_below(&rw, (uint32_t)(whi - wlo + 1));
    }
    net_off[m] = (uint32_t)off;
    for (int32_t v = 0; v < n; v++)
        node_w[v] = clo + (int32_t)rng_below(&rc, (uint32_t)(chi - clo + 1));
    free(mark);
    return off;
}

/*
 * k-way partition of the ring into k contiguous arcs (block of v is
 * floor(v * k / n)); then every vertex, with probability frac_ppm / 10^6,
 * moves to block b-1 or b+1 (mod k), each with probability 1/2.
 */
int32_t synth_kway_partition(int32_t n, int32_t k, int32_t frac_ppm, uint64_t seed, int32_t *part) {
    if (n <= 0 || k < 1 || frac_ppm < 0 || frac_ppm > 1000000) return -1;
    rng_t r;
    stream_seed(&r, seed, STREAM_PART);
    int32_t moved = 0;
    for (int32_t v = 0; v < n; v++) {
        int32_t b = (int32_t)(((int64_t)v * k) / n);
        uint32_t x = rng_below(&r, 1000000u);
        uint32_t dir = rng_below(&r, 2u);
        if (k > 1 && x < (uint32_t)frac_ppm) {
            b = dir ? (b + 1) % k : (b + k - 1) % k;
            moved++;
        }
        part[v] = b;
    }
    return moved;
}
