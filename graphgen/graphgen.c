/*
 * graphgen.c -- seeded synthetic graph inputs.
 *
 * This module produces INPUTS only: directed edge tuples (src[e], dst[e]) and
 * BFS roots.  It holds none of the BFS, directory, sieve or codec arithmetic;
 * both the CPU oracle and the CUDA library consume its output.
 *
 * Kronecker generator (the synthetic graphs of the paper's experiments, Sec. VII-A):
 *   N = 2^scale vertices, M = edgefactor * N tuples.  Each tuple picks, for each
 *   of `scale` bit levels (most significant first), one quadrant of the 2x2
 *   initiator with probabilities A=0.57, B=0.19, C=0.19, D=0.05
 *   (A: row bit 0 / col bit 0, B: 0/1, C: 1/0, D: 1/1).  No initiator noise.
 *   Vertex labels are then mapped through a seeded bijection of [0, N).
 * Erdos-Renyi control: both endpoints uniform in [0, N), then the same bijection.
 *
 * Randomness is counter based: SplitMix64 (Steele, Lea and Flood, "Fast
 * splittable pseudorandom number generators", OOPSLA 2014) evaluated at a
 * counter, so each tuple depends only on (seed, tuple index) and the output is
 * identical for any thread count and on any little- or big-endian host.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>
#include <unistd.h>

#define GOLDEN_GAMMA 0x9E3779B97F4A7C15ULL

/* k-th output (k = 0, 1, ...) of a SplitMix64 stream started at `seed`. */
uint64_t graphgen_splitmix64(uint64_t seed, uint64_t k)
{
    uint64_t z = seed + (k + 1u) * GOLDEN_GAMMA;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Quadrant thresholds on a uniform 32-bit draw r:
 * r < T_A -> A, r < T_AB -> B, r < T_ABC -> C, else D.
 * T = round(p * 2^32) for the cumulative probabilities 0.57, 0.76, 0.95. */
#define T_A   2448131359u
#define T_AB  3264175145u
#define T_ABC 4080218931u

/* Seeded bijection of [0, 2^bits): four rounds of (odd multiply, xorshift,
 * add), each step invertible modulo 2^bits. */
typedef struct { uint64_t mul[4], add[4], mask; int shift; } perm_t;

static void perm_init(perm_t *p, int bits, uint64_t seed)
{
    p->mask = (bits >= 64) ? ~0ULL : ((1ULL << bits) - 1ULL);
    p->shift = (bits + 1) / 2;
    if (p->shift < 1) p->shift = 1;
    for (int r = 0; r < 4; ++r) {
        p->mul[r] = graphgen_splitmix64(seed, 2u * r) | 1ULL;
        p->add[r] = graphgen_splitmix64(seed, 2u * r + 1u);
    }
}

static inline uint64_t perm_apply(const perm_t *p, uint64_t x)
{
    for (int r = 0; r < 4; ++r) {
        x = (x * p->mul[r]) & p->mask;
        x ^= x >> p->shift;
        x = (x + p->add[r]) & p->mask;
    }
    return x;
}

/* Public form of the label bijection (for tests of the bijection itself). */
int64_t graphgen_permute(int scale, uint64_t seed, int64_t x)
{
    perm_t p;
    perm_init(&p, scale, seed);
    return (int64_t)perm_apply(&p, (uint64_t)x);
}

typedef struct {
    int kind;              /* 0 Kronecker, 1 Erdos-Renyi */
    int scale;
    uint64_t seed;
    int64_t e0, e1;
    int32_t *src, *dst;
    const perm_t *perm;
} job_t;

static void *gen_range(void *arg)
{
    const job_t *J = (const job_t *)arg;
    const int scale = J->scale;
    const uint64_t words = (uint64_t)(scale + 1) / 2u;   /* two 32-bit draws per 64-bit word */
    const uint64_t mask = (1ULL << scale) - 1ULL;
    for (int64_t e = J->e0; e < J->e1; ++e) {
        uint64_t u = 0, v = 0;
        if (J->kind == 0) {
            uint64_t d = 0;
            for (int l = 0; l < scale; ++l) {
                if ((l & 1) == 0) d = graphgen_splitmix64(J->seed, (uint64_t)e * words + (uint64_t)(l / 2));
                uint32_t r = (l & 1) ? (uint32_t)(d & 0xFFFFFFFFu) : (uint32_t)(d >> 32);
                uint64_t ub, vb;
                if (r < T_A)        { ub = 0; vb = 0; }
                else if (r < T_AB)  { ub = 0; vb = 1; }
                else if (r < T_ABC) { ub = 1; vb = 0; }
                else                { ub = 1; vb = 1; }
                u = (u << 1) | ub;
                v = (v << 1) | vb;
            }
        } else {
            u = graphgen_splitmix64(J->seed, 2u * (uint64_t)e) & mask;
            v = graphgen_splitmix64(J->seed, 2u * (uint64_t)e + 1u) & mask;
        }
        J->src[e] = (int32_t)perm_apply(J->perm, u);
        J->dst[e] = (int32_t)perm_apply(J->perm, v);
    }
    return NULL;
}

/*
 * Generate M tuples into src[0..M), dst[0..M).
 *   kind: 0 Kronecker, 1 Erdos-Renyi; scale in [1, 31];
 *   seed: tuple stream seed; perm_seed: label bijection seed;
 *   threads: 0 = one per online core.
 * Returns 0 on success, -1 on a bad argument.
 */
int graphgen_edges(int kind, int scale, int64_t m, uint64_t seed, uint64_t perm_seed,
                   int32_t *src, int32_t *dst, int threads)
{
    if (scale < 1 || scale > 31 || m < 0 || !src || !dst || (kind != 0 && kind != 1)) return -1;
    perm_t perm;
    perm_init(&perm, scale, perm_seed);
    if (threads <= 0) {
        long c = sysconf(_SC_NPROCESSORS_ONLN);
        threads = c > 0 ? (int)c : 1;
    }
    if (threads > 256) threads = 256;
    if ((int64_t)threads > m) threads = m > 0 ? (int)m : 1;
    pthread_t tid[256];
    int running[256];
    job_t jobs[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t].kind = kind; jobs[t].scale = scale; jobs[t].seed = seed;
        jobs[t].e0 = m * t / threads; jobs[t].e1 = m * (t + 1) / threads;
        jobs[t].src = src; jobs[t].dst = dst; jobs[t].perm = &perm;
        running[t] = 0;
    }
    for (int t = 1; t < threads; ++t) {
        if (pthread_create(&tid[t], NULL, gen_range, &jobs[t]) == 0) running[t] = 1;
        else gen_range(&jobs[t]);       /* no thread available: do the range here */
    }
    gen_range(&jobs[0]);
    for (int t = 1; t < threads; ++t)
        if (running[t]) pthread_join(tid[t], NULL);
    return 0;
}

/*
 * Pick up to `count` distinct roots, each with at least one neighbour other
 * than itself (in either direction), by drawing SplitMix64(seed, k) mod n for
 * k = 0, 1, ... and keeping eligible, not yet chosen vertices.  Stops after
 * 64*n + 1024 draws.  Returns the number of roots written.
 */
int64_t graphgen_pick_roots(int64_t n, int64_t m, const int32_t *src, const int32_t *dst,
                            int64_t count, uint64_t seed, int32_t *roots)
{
    if (n <= 0 || count <= 0) return 0;
    uint8_t *ok = (uint8_t *)calloc((size_t)n, 1);
    uint8_t *taken = (uint8_t *)calloc((size_t)n, 1);
    if (!ok || !taken) { free(ok); free(taken); return -1; }
    for (int64_t e = 0; e < m; ++e) {
        int32_t a = src[e], b = dst[e];
        if (a != b && a >= 0 && b >= 0 && a < n && b < n) { ok[a] = 1; ok[b] = 1; }
    }
    int64_t got = 0;
    const uint64_t limit = 64u * (uint64_t)n + 1024u;
    for (uint64_t k = 0; k < limit && got < count; ++k) {
        int64_t v = (int64_t)(graphgen_splitmix64(seed, k) % (uint64_t)n);
        if (ok[v] && !taken[v]) { taken[v] = 1; roots[got++] = (int32_t)v; }
    }
    free(ok); free(taken);
    return got;
}
