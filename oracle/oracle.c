/*
 * oracle.c -- plain, slow, single-threaded CPU reference for the compressed
 * and sieved level-synchronous BFS.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the bench's
 * CPU-baseline leg may load this code.  It shares no code, header, table or
 * helper with the CUDA library, and neither side includes the other.
 *
 * What each function follows:
 *   oracle_csr            -- the adjacency the search runs on (Sec. VII-A): one
 *                            directed entry per tuple and, when symmetrising,
 *                            the reverse entry too (a self-loop gives two).
 *   oracle_bfs_levels     -- BFS as defined in Sec. II: hop distance from the
 *                            source; unreachable vertices get -1.
 *   oracle_bfs_sample     -- the same search stopped after a budget of scanned
 *                            entries (a bounded sample for timing).
 *   oracle_parents        -- deterministic parent: the smallest (or, for the
 *                            paper's (select,max) semiring of Sec. III-A, the
 *                            largest) neighbour on the previous level.
 *   oracle_directory      -- directory vector V_{i,j} of Eq. 4: bit k set iff
 *                            column k of block A_{i,j} holds a nonzero.
 *   oracle_wah_encode/_decode -- word-aligned hybrid code of Sec. IV, Table 3:
 *                            literal / fill / active words over (w-1)-bit groups.
 *   oracle_plwah_encode/_decode -- position-list WAH, the alternative bitmap
 *                            code Sec. IV names beside WAH (Deliege and
 *                            Pedersen): a fill word also carries the one odd
 *                            bit of the group that follows its run.
 *   oracle_bbc_encode/_decode -- byte-aligned bitmap code, the other bitmap
 *                            code Sec. IV names (Antoshenkov): runs of gap
 *                            bytes and map bytes behind one-byte headers.
 *   oracle_adaptive_encode/_decode -- a sieved slice sent as the smallest of
 *                            its WAH stream, its sparse vector (Sec. II,
 *                            Table 2; Sec. V-A) and its raw bitmap (Alg. 1).
 *   oracle_dynamic_sieve_stats -- the pairs and entries a dynamic cross
 *                            directory (Sec. V-B's synchronous update) drops,
 *                            level by level, by definition.
 *   oracle_dist_bfs       -- Algorithms 1, 2 and 3 (BIT, WAH, DIR-WAH) on a
 *                            simulated p x p grid: the frontier exchange
 *                            (raw, compressed, or sieved by f_j (.) V_{i,j}
 *                            and compressed), the per-block products of the
 *                            (select, min) semiring, their fold over a
 *                            block-row and the visited mask, recording every
 *                            exchanged buffer -- the column streams and, for
 *                            DIR-WAH, the compressed row buffers of the fold.
 *
 * Bitmaps are held one byte per bit (0 or 1) so every step reads as its
 * definition.  Vertex ranges: range b of a p-way split of n vertices is
 * [b*nb, min(n, (b+1)*nb)) with nb = ceil(n/p) (Eq. 1-2).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ CSR -- */

/* Count the directed entries first: returns the number of entries the CSR
 * will hold (m, or 2m when symmetrising). */
int64_t oracle_csr_size(int64_t m, int symmetrize) { return symmetrize ? 2 * m : m; }

/* Build CSR by source vertex.  Entries keep tuple order inside each row.
 * row_ptr has n+1 entries; col has oracle_csr_size(m, symmetrize) entries.
 * Returns 0, or -1 if a tuple names a vertex outside [0, n). */
int oracle_csr(int64_t n, int64_t m, const int32_t *src, const int32_t *dst, int symmetrize,
               int64_t *row_ptr, int32_t *col)
{
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return -1;
    for (int64_t v = 0; v <= n; ++v) row_ptr[v] = 0;
    for (int64_t e = 0; e < m; ++e) {
        row_ptr[src[e] + 1] += 1;
        if (symmetrize) row_ptr[dst[e] + 1] += 1;
    }
    for (int64_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    int64_t *fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!fill) return -2;
    for (int64_t v = 0; v < n; ++v) fill[v] = row_ptr[v];
    for (int64_t e = 0; e < m; ++e) {
        col[fill[src[e]]++] = dst[e];
        if (symmetrize) col[fill[dst[e]]++] = src[e];
    }
    free(fill);
    return 0;
}

/* ------------------------------------------------------------------ BFS -- */

/* level[v] = hop distance from root following CSR entries u -> v, or -1.
 * Returns the number of reached vertices, or -1 for a bad root. */
int64_t oracle_bfs_levels(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t root,
                          int32_t *level)
{
    if (root < 0 || root >= n) return -1;
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!queue) return -2;
    int64_t head = 0, tail = 0;
    level[root] = 0;
    queue[tail++] = root;
    while (head < tail) {
        int32_t u = queue[head++];
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (level[v] < 0) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
    }
    free(queue);
    return tail;
}

/* A bounded sample of oracle_bfs_levels for timing: the same queue BFS, which
 * stops dequeuing once `budget` adjacency entries have been scanned (the vertex
 * being scanned is finished).  Vertices dequeue in level order, so every level
 * it assigns is the final one; unassigned vertices keep -1.  Returns the
 * entries scanned, or -1 for a bad root. */
int64_t oracle_bfs_sample(int64_t n, const int64_t *row_ptr, const int32_t *col, int32_t root,
                          int64_t budget, int32_t *level)
{
    if (root < 0 || root >= n) return -1;
    for (int64_t v = 0; v < n; ++v) level[v] = -1;
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!queue) return -2;
    int64_t head = 0, tail = 0, scanned = 0;
    level[root] = 0;
    queue[tail++] = root;
    while (head < tail && scanned < budget) {
        int32_t u = queue[head++];
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (level[v] < 0) {
                level[v] = level[u] + 1;
                queue[tail++] = v;
            }
        }
        scanned += row_ptr[u + 1] - row_ptr[u];
    }
    free(queue);
    return scanned;
}

/* Parent of every reached v != root: the smallest (use_max = 0) or largest
 * (use_max = 1) u with an entry u -> v and level[u] = level[v] - 1.
 * parent[root] = root; unreached vertices get -1. */
void oracle_parents(int64_t n, const int64_t *row_ptr, const int32_t *col, const int32_t *level,
                    int32_t root, int use_max, int32_t *parent)
{
    for (int64_t v = 0; v < n; ++v) parent[v] = -1;
    for (int64_t u = 0; u < n; ++u) {
        if (level[u] < 0) continue;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int32_t v = col[e];
            if (v == root || level[v] != level[u] + 1) continue;
            if (parent[v] < 0 || (!use_max && u < parent[v]) || (use_max && u > parent[v]))
                parent[v] = (int32_t)u;
        }
    }
    if (root >= 0 && root < n) parent[root] = root;
}

/* ------------------------------------------------------------ partition -- */

static int64_t range_size(int64_t n, int p) { return (n + p - 1) / p; }

static int64_t range_begin(int64_t n, int p, int b)
{
    int64_t x = (int64_t)b * range_size(n, p);
    return x < n ? x : n;
}

static int64_t range_end(int64_t n, int p, int b) { return range_begin(n, p, b + 1); }

int64_t oracle_range_begin(int64_t n, int p, int b) { return range_begin(n, p, b); }
int64_t oracle_range_len(int64_t n, int p, int b) { return range_end(n, p, b) - range_begin(n, p, b); }

/* ------------------------------------------------------------ directory -- */

/* Eq. 4: V_{i,j}[k] = 1 iff column k of A_{i,j} has a nonzero, i.e. the
 * source u = begin(j) + k has at least one entry u -> v with v in range i.
 * V receives range_len(j) bytes. */
void oracle_directory(int64_t n, int p, const int64_t *row_ptr, const int32_t *col, int i, int j,
                      uint8_t *V)
{
    const int64_t jb = range_begin(n, p, j), je = range_end(n, p, j);
    const int64_t ib = range_begin(n, p, i), ie = range_end(n, p, i);
    for (int64_t u = jb; u < je; ++u) {
        uint8_t bit = 0;
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (col[e] >= ib && col[e] < ie) { bit = 1; break; }
        V[u - jb] = bit;
    }
}

/* Cross directory (Eq. 5) of every processor at once: D[i*n + u] = V_{i,j}[u - begin(j)]
 * for the source range j holding u.  Built in one pass over the entries (every
 * entry u -> v marks column u of the block in block-row range(v)); the same
 * definition as oracle_directory, reached a different way.  D has p*n bytes. */
void oracle_cross_directory(int64_t n, int p, const int64_t *row_ptr, const int32_t *col, uint8_t *D)
{
    const int64_t nb = range_size(n, p);
    memset(D, 0, (size_t)n * (size_t)p);
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            D[(size_t)(col[e] / nb) * (size_t)n + (size_t)u] = 1;
}

/* ------------------------------------------------------------------ WAH -- */

/*
 * Word-aligned hybrid code with w-bit words (Sec. IV, Table 3).
 *   The bitmap is cut into groups of g = w-1 bits; the first bit of a group
 *   is the most significant of its g payload bits.
 *   Literal word: top bit 0, the g payload bits.
 *   Fill word:    top bit 1; with fill_bit, bit w-2 holds the fill value and
 *                 bits 0..w-3 the run length in groups; without it (the
 *                 paper's 4-bit example, whose fill words carry no value
 *                 bit) only zero runs are fills and bits 0..w-2 hold the
 *                 run length.
 *                 An all-zero group (or, with fill_bit, an all-one group) is
 *                 always written as a fill; adjacent equal fills merge up to
 *                 the largest length the count field holds.
 *   Active word:  present iff nbits mod g != 0; holds the r = nbits mod g
 *                 trailing bits right-aligned, first bit highest.
 * Returns the number of words written to out (at most nbits/g + 1).
 */
int64_t oracle_wah_encode(const uint8_t *bits, int64_t nbits, int w, int fill_bit, uint64_t *out)
{
    const int g = w - 1;
    const uint64_t top = 1ULL << (w - 1);
    const uint64_t ones = (g >= 64) ? ~0ULL : ((1ULL << g) - 1ULL);
    const int count_bits = fill_bit ? w - 2 : w - 1;
    const uint64_t max_count = (1ULL << count_bits) - 1ULL;
    const int64_t full = nbits / g;
    const int64_t r = nbits % g;
    int64_t nw = 0;
    int last_fill = -1;     /* fill value of out[nw-1] if it is a fill word, else -1 */
    for (int64_t k = 0; k < full; ++k) {
        uint64_t x = 0;
        for (int b = 0; b < g; ++b) x = (x << 1) | (uint64_t)(bits[k * g + b] & 1);
        int fill_value = -1;
        if (x == 0) fill_value = 0;
        else if (fill_bit && x == ones) fill_value = 1;
        if (fill_value < 0) {
            out[nw++] = x;
            last_fill = -1;
            continue;
        }
        if (last_fill == fill_value && (out[nw - 1] & max_count) < max_count) {
            out[nw - 1] += 1;
        } else {
            uint64_t word = top | 1ULL;
            if (fill_bit && fill_value) word |= 1ULL << (w - 2);
            out[nw++] = word;
            last_fill = fill_value;
        }
    }
    if (r > 0) {
        uint64_t x = 0;
        for (int64_t b = 0; b < r; ++b) x = (x << 1) | (uint64_t)(bits[full * g + b] & 1);
        out[nw++] = x;
    }
    return nw;
}

/* Inverse of oracle_wah_encode.  Accepts any well-formed stream (canonical
 * or not).  Returns 0, or -1 if the stream is malformed: a fill of length 0,
 * a literal with the top bit set, groups beyond nbits, a missing or oversized
 * active word, or trailing words. */
int oracle_wah_decode(const uint64_t *words, int64_t nwords, int64_t nbits, int w, int fill_bit,
                      uint8_t *bits)
{
    const int g = w - 1;
    const uint64_t top = 1ULL << (w - 1);
    const int count_bits = fill_bit ? w - 2 : w - 1;
    const uint64_t count_mask = (1ULL << count_bits) - 1ULL;
    const int64_t full = nbits / g;
    const int64_t r = nbits % g;
    int64_t pos = 0;     /* groups written */
    int64_t k = 0;       /* words read */
    while (pos < full) {
        if (k >= nwords) return -1;
        uint64_t word = words[k++];
        if (w < 64 && (word >> w) != 0) return -1;
        if (word & top) {
            uint64_t len = word & count_mask;
            int value = fill_bit ? (int)((word >> (w - 2)) & 1ULL) : 0;
            if (len == 0 || (int64_t)len > full - pos) return -1;
            for (uint64_t q = 0; q < len; ++q, ++pos)
                for (int b = 0; b < g; ++b) bits[pos * g + b] = (uint8_t)value;
        } else {
            for (int b = 0; b < g; ++b) bits[pos * g + b] = (uint8_t)((word >> (g - 1 - b)) & 1ULL);
            ++pos;
        }
    }
    if (r > 0) {
        if (k >= nwords) return -1;
        uint64_t word = words[k++];
        if ((word >> r) != 0) return -1;
        for (int64_t b = 0; b < r; ++b) bits[full * g + b] = (uint8_t)((word >> (r - 1 - b)) & 1ULL);
    }
    return k == nwords ? 0 : -1;
}

/* ---------------------------------------------------------------- PLWAH -- */

/*
 * Position-list word-aligned hybrid code, 32-bit words over 31-bit groups
 * (bit order and active word as in WAH: first bit of a group most
 * significant; the nbits mod 31 trailing bits right-aligned in a last word,
 * first bit highest).  Word kinds:
 *   literal: bit 31 = 0, bits 30..0 = the 31 bits of one group;
 *   fill:    bit 31 = 1, bit 30 = the fill value v, bits 29..25 = a position
 *            q (0: none), bits 24..0 = the run length in groups (>= 1).  A
 *            position q > 0 stands for one more group right after the run:
 *            all bits equal to v except bit q of the group (q = 1 is the
 *            group's first bit).
 * Encoding rule: an all-0 or all-1 group is a fill group; a run of equal fill
 * groups is one fill word (a run longer than 2^25 - 1 groups continues in a
 * new word); a literal group that directly follows a run and differs from
 * the run's value in exactly one bit is not written -- its bit goes into the
 * position of the run's last word; every other literal group is a literal
 * word.  Returns the number of words written (at most nbits/31 + 1).
 */
int64_t oracle_plwah_encode(const uint8_t *bits, int64_t nbits, uint32_t *out)
{
    const uint32_t ones = 0x7fffffffu;
    const uint32_t max_count = (1u << 25) - 1u;
    const int64_t full = nbits / 31;
    const int64_t r = nbits % 31;
    int64_t nw = 0;
    int run_value = -1;     /* value of the run the previous group belongs to, else -1 */
    for (int64_t k = 0; k < full; ++k) {
        uint32_t x = 0;
        for (int b = 0; b < 31; ++b) x = (x << 1) | (uint32_t)(bits[k * 31 + b] & 1);
        const int value = (x == 0) ? 0 : (x == ones ? 1 : -1);
        if (value < 0) {
            /* a literal: folded into the run before it if one bit differs */
            const uint32_t diff = x ^ (run_value == 1 ? ones : 0u);
            if (run_value >= 0 && (diff & (diff - 1u)) == 0u) {
                int q = 1;          /* the odd bit's place in the group, first bit = 1 */
                while (!((diff >> (31 - q)) & 1u)) ++q;
                out[nw - 1] |= (uint32_t)q << 25;
            } else {
                out[nw++] = x;
            }
            run_value = -1;
            continue;
        }
        if (run_value == value && (out[nw - 1] & max_count) < max_count) {
            out[nw - 1] += 1u;
        } else {
            out[nw++] = 0x80000000u | ((uint32_t)value << 30) | 1u;
        }
        run_value = value;
    }
    if (r > 0) {
        uint32_t x = 0;
        for (int64_t b = 0; b < r; ++b) x = (x << 1) | (uint32_t)(bits[full * 31 + b] & 1);
        out[nw++] = x;
    }
    return nw;
}

/* Inverse of oracle_plwah_encode (any well-formed stream, canonical or not).
 * Returns 0, or -1 if the stream is malformed: a fill of length 0, groups
 * beyond nbits (a position group included), a missing or oversized active
 * word, or trailing words. */
int oracle_plwah_decode(const uint32_t *words, int64_t nwords, int64_t nbits, uint8_t *bits)
{
    const int64_t full = nbits / 31;
    const int64_t r = nbits % 31;
    int64_t pos = 0;     /* groups written */
    int64_t k = 0;       /* words read */
    while (pos < full) {
        if (k >= nwords) return -1;
        const uint32_t word = words[k++];
        if (word & 0x80000000u) {
            const int64_t len = (int64_t)(word & ((1u << 25) - 1u));
            const int value = (int)((word >> 30) & 1u);
            const int q = (int)((word >> 25) & 31u);
            if (len == 0 || len + (q ? 1 : 0) > full - pos) return -1;
            for (int64_t g = 0; g < len; ++g, ++pos)
                for (int b = 0; b < 31; ++b) bits[pos * 31 + b] = (uint8_t)value;
            if (q) {
                for (int b = 0; b < 31; ++b) bits[pos * 31 + b] = (uint8_t)(b == q - 1 ? !value : value);
                ++pos;
            }
        } else {
            for (int b = 0; b < 31; ++b) bits[pos * 31 + b] = (uint8_t)((word >> (30 - b)) & 1u);
            ++pos;
        }
    }
    if (r > 0) {
        if (k >= nwords) return -1;
        const uint32_t word = words[k++];
        if ((word >> r) != 0) return -1;
        for (int64_t b = 0; b < r; ++b) bits[full * 31 + b] = (uint8_t)((word >> (r - 1 - b)) & 1u);
    }
    return k == nwords ? 0 : -1;
}

/* ------------------------------------------------------------------ BBC -- */

/*
 * Byte-aligned bitmap code (BBC, Antoshenkov), the other bitmap code Sec. IV
 * names beside WAH; the paper does not define it, so this is the reading the
 * build uses (four kinds of run, as BBC has).  The bitmap is cut into bytes:
 * byte k holds bits 8k .. 8k+7, the first of them the most significant; the
 * bits past nbits in the last byte are 0.  A gap byte of value b is 0x00
 * (b = 0) or 0xFF (b = 1); every other byte is a map byte.  A map byte is odd
 * for b when it differs from the gap byte of value b in exactly one bit, its
 * odd position (0 = the byte's first, most significant bit).
 *
 * The stream is a sequence of runs.  A run is a fill of F >= 0 gap bytes of
 * value b followed either by a tail of T = 0 .. 15 map bytes, stored as they
 * are, or by one odd byte, stored as its position in the header:
 *   1 b F F T T T T            F <= 3, tail          (then the T bytes)
 *   0 1 b F F P P P            F <= 3, odd byte at P
 *   0 0 1 b T T T T            F >= 4, tail          (then F, then the T bytes)
 *   0 0 0 1 b P P P            F >= 4, odd byte at P (then F)
 * (header bits from the most significant); F >= 4 follows the header as a
 * base-128 counter, least significant group first, bit 7 set on every byte
 * but the last.  Headers 0x00 .. 0x0F are not used.
 *
 * Encoding, left to right: a unit is a maximal run of equal gap bytes (its
 * fill; F = 0 and b = 0 when the unit starts with map bytes, which happens
 * only at byte 0) and the maximal run of map bytes after it (length L >= 0).
 * The unit's first run carries the fill and the first min(L, 15) map bytes;
 * the other map bytes follow in runs with F = 0, 15 at a time.  A run whose
 * tail would be one byte that is also the unit's last map byte is an odd-byte
 * run when that byte is odd for the run's b (for F = 0: b = 0 if the byte is
 * odd for 0, else b = 1 if it is odd for 1).  Returns the bytes written (at
 * most nbytes + nbytes / 15 + 11 for nbytes = ceil(nbits / 8)).
 */
static int bbc_gap(uint8_t x) { return x == 0x00 ? 0 : (x == 0xFF ? 1 : -1); }

/* Position of the odd bit of x for fill value b, or -1. */
static int bbc_odd(uint8_t x, int b)
{
    const unsigned d = (unsigned)(x ^ (b ? 0xFFu : 0x00u));
    if (d == 0 || (d & (d - 1u)) != 0) return -1;
    int pos = 0;
    while (!((d >> (7 - pos)) & 1u)) ++pos;
    return pos;
}

static int64_t bbc_counter(uint8_t *out, int64_t at, int64_t f)
{
    do {
        uint8_t g = (uint8_t)(f & 0x7F);
        f >>= 7;
        if (f) g |= 0x80;
        out[at++] = g;
    } while (f);
    return at;
}

int64_t oracle_bbc_encode(const uint8_t *bits, int64_t nbits, uint8_t *out)
{
    const int64_t nbytes = (nbits + 7) / 8;
    uint8_t *by = (uint8_t *)calloc((size_t)(nbytes > 0 ? nbytes : 1), 1);
    if (!by) return -1;
    for (int64_t i = 0; i < nbits; ++i)
        if (bits[i] & 1) by[i / 8] |= (uint8_t)(0x80u >> (i % 8));
    int64_t at = 0, k = 0;
    while (k < nbytes) {
        /* the unit: its fill, then its map bytes */
        int b = 0;
        int64_t f = 0;
        if (bbc_gap(by[k]) >= 0) {
            b = bbc_gap(by[k]);
            while (k + f < nbytes && bbc_gap(by[k + f]) == b) ++f;
        }
        const int64_t m0 = k + f;
        int64_t l = 0;
        while (m0 + l < nbytes && bbc_gap(by[m0 + l]) < 0) ++l;
        /* its runs: the first carries the fill */
        int64_t done = 0;
        int first = 1;
        do {
            const int64_t fill = first ? f : 0;
            int rb = first ? b : 0;
            const int64_t t = (l - done < 15) ? l - done : 15;
            int pos = -1;
            if (t == 1 && done + 1 == l) {
                pos = bbc_odd(by[m0 + done], rb);
                if (pos < 0 && fill == 0) { rb = 1; pos = bbc_odd(by[m0 + done], 1); }
                if (pos < 0) rb = first ? b : 0;
            }
            if (pos >= 0) {
                if (fill <= 3) out[at++] = (uint8_t)(0x40 | (rb << 5) | ((int)fill << 3) | pos);
                else { out[at++] = (uint8_t)(0x10 | (rb << 3) | pos); at = bbc_counter(out, at, fill); }
            } else {
                if (fill <= 3) out[at++] = (uint8_t)(0x80 | (rb << 6) | ((int)fill << 4) | (int)t);
                else { out[at++] = (uint8_t)(0x20 | (rb << 4) | (int)t); at = bbc_counter(out, at, fill); }
                for (int64_t q = 0; q < t; ++q) out[at++] = by[m0 + done + q];
            }
            done += t;
            first = 0;
        } while (done < l);
        k = m0 + l;
    }
    free(by);
    return at;
}

/* Inverse of oracle_bbc_encode (any well-formed stream).  Returns 0, or -1 if
 * the stream is malformed: an unused header, a cut counter or tail, a counter
 * above 2^56, bytes past nbits, padding bits set, or trailing bytes. */
int oracle_bbc_decode(const uint8_t *in, int64_t nin, int64_t nbits, uint8_t *bits)
{
    const int64_t nbytes = (nbits + 7) / 8;
    uint8_t *by = (uint8_t *)calloc((size_t)(nbytes > 0 ? nbytes : 1), 1);
    if (!by) return -1;
    int64_t k = 0, at = 0;
    int rc = 0;
    while (at < nin) {
        const uint8_t h = in[at++];
        int b, odd = -1;
        int64_t f, t = 0;
        if (h & 0x80) { b = (h >> 6) & 1; f = (h >> 4) & 3; t = h & 15; }
        else if (h & 0x40) { b = (h >> 5) & 1; f = (h >> 3) & 3; odd = h & 7; }
        else if (h & 0x20) { b = (h >> 4) & 1; f = -1; t = h & 15; }
        else if (h & 0x10) { b = (h >> 3) & 1; f = -1; odd = h & 7; }
        else { rc = -1; break; }
        if (f < 0) {                      /* a counter follows */
            f = 0;
            int shift = 0, more = 1;
            while (more) {
                if (at >= nin || shift > 49) { rc = -1; break; }
                const uint8_t g = in[at++];
                f |= (int64_t)(g & 0x7F) << shift;
                shift += 7;
                more = g & 0x80;
            }
            if (rc) break;
        }
        const int64_t tail = odd >= 0 ? 1 : t;
        if (f > nbytes - k || tail > nbytes - k - f) { rc = -1; break; }
        for (int64_t q = 0; q < f; ++q) by[k++] = b ? 0xFF : 0x00;
        if (odd >= 0) {
            by[k++] = (uint8_t)((b ? 0xFFu : 0x00u) ^ (0x80u >> odd));
        } else {
            if (t > nin - at) { rc = -1; break; }
            for (int64_t q = 0; q < t; ++q) by[k++] = in[at++];
        }
    }
    if (rc == 0 && k != nbytes) rc = -1;
    if (rc == 0 && (nbits % 8) && (by[nbytes - 1] & (0xFFu >> (nbits % 8)))) rc = -1;
    if (rc == 0)
        for (int64_t i = 0; i < nbits; ++i) bits[i] = (uint8_t)((by[i / 8] >> (7 - i % 8)) & 1u);
    free(by);
    return rc;
}

/* ------------------------------------------------------ adaptive format -- */

/*
 * Level-adaptive format of one exchanged slice of nbits bits: the smallest,
 * in bytes, of three encodings, the lower number on a tie:
 *   0  its WAH stream (w-bit words, Sec. IV), w/8 bytes a word;
 *   1  its sparse vector (Sec. II represents a sparse frontier as the list of
 *      its vertices, Table 2; Sec. V-A notes that a sieved slice is very
 *      sparse): the offsets of its set bits inside the slice in increasing
 *      order, 4 bytes each (a slice is a range of fewer than 2^31 vertices);
 *   2  its raw bitmap (the BIT exchange of Alg. 1): ceil(nbits/32) 32-bit
 *      words, bit b = bit b%32 of word b/32.
 * Every element goes to out as one uint64 value; returns their count and
 * sets *format.  out must hold max(nbits/(w-1) + 1, nbits, ceil(nbits/32)).
 */
int64_t oracle_adaptive_encode(const uint8_t *bits, int64_t nbits, int w, int *format, uint64_t *out)
{
    int64_t ones = 0;
    for (int64_t b = 0; b < nbits; ++b) ones += bits[b] & 1;
    const int64_t raw_words = (nbits + 31) / 32;
    const int64_t wah_words = oracle_wah_encode(bits, nbits, w, 1, out);
    const int64_t wah_bytes = wah_words * (w / 8), list_bytes = 4 * ones, raw_bytes = 4 * raw_words;
    if (wah_bytes <= list_bytes && wah_bytes <= raw_bytes) {
        *format = 0;
        return wah_words;
    }
    if (list_bytes <= raw_bytes) {
        *format = 1;
        int64_t k = 0;
        for (int64_t b = 0; b < nbits; ++b)
            if (bits[b] & 1) out[k++] = (uint64_t)b;
        return k;
    }
    *format = 2;
    for (int64_t x = 0; x < raw_words; ++x) {
        uint64_t word = 0;
        for (int q = 0; q < 32 && x * 32 + q < nbits; ++q) word |= (uint64_t)(bits[x * 32 + q] & 1) << q;
        out[x] = word;
    }
    return raw_words;
}

/* Inverse of oracle_adaptive_encode for any of the three formats.  Returns 0,
 * or -1 if the elements are malformed: a bad WAH stream; a sparse vector that
 * is not strictly increasing or names an offset >= nbits; a raw bitmap of the
 * wrong length or with bits set past nbits; an unknown format. */
int oracle_adaptive_decode(int format, const uint64_t *in, int64_t count, int64_t nbits, int w, uint8_t *bits)
{
    for (int64_t b = 0; b < nbits; ++b) bits[b] = 0;
    if (format == 0) return oracle_wah_decode(in, count, nbits, w, 1, bits);
    if (format == 1) {
        for (int64_t k = 0; k < count; ++k) {
            if (in[k] >= (uint64_t)nbits || (k > 0 && in[k] <= in[k - 1])) return -1;
            bits[in[k]] = 1;
        }
        return 0;
    }
    if (format == 2) {
        if (count != (nbits + 31) / 32) return -1;
        for (int64_t x = 0; x < count; ++x) {
            if (in[x] >> 32) return -1;
            for (int q = 0; q < 32; ++q) {
                const int64_t b = x * 32 + q;
                const int v = (int)((in[x] >> q) & 1u);
                if (b >= nbits) {
                    if (v) return -1;
                } else {
                    bits[b] = (uint8_t)v;
                }
            }
        }
        return 0;
    }
    return -1;
}

/* ------------------------------------------- Algorithms 1-3 on a p x p grid -- */

/*
 * Distributed BFS on a simulated p x p grid (Eq. 1-3), one processor P_i per
 * vertex range i (the paper's indices shifted to start at 0).  mode 0 = BIT
 * (Alg. 1), 1 = WAH (Alg. 2), 2 = DIR-WAH (Alg. 3).  Every level computes:
 *   the exchange of the frontier f (the frontier of level k):
 *     BIT:     every P_i receives the raw bitmap of every range j;
 *     WAH:     every range j is WAH-compressed once (Sec. IV, Table 3), every
 *              P_i receives the p streams and decompresses them;
 *     DIR-WAH: the slice of range j bound for P_i is sieved by the cross
 *              directory first, f_j (.) V_{i,j} (Eq. 4-5, Sec. V), then
 *              compressed; P_i decompresses the stream it receives from
 *              every range j;
 *   the product of every block, t_{i,j} = A_{i,j} (x) f_{i,j} over the
 *     (select, min) semiring (or (select, max), use_max): t_{i,j}[v] is the
 *     smallest (largest) source u of range j that P_i received with an entry
 *     u -> v, for v in range i;
 *   the fold of block-row i, t_i = (+)_j t_{i,j} (the same semiring);
 *   the visited mask and update, t_i = t_i (.) not(pi_i), pi_i = pi_i + t_i,
 *     and the next frontier f_i = t_i, whose vertices get level k + 1 and
 *     parent t_i[v].
 * The exchange before level 0 carries f = {root}.
 *
 * Column trace (optional, trace_counts != NULL; modes 1 and 2): the
 * compressed frontier slices of the exchange that feeds level k,
 *   WAH:     one stream per source range j, slot s = j        (p slots)
 *   DIR-WAH: the stream of f_j (.) V_{i,j}, slot s = i*p + j   (p*p slots)
 * trace_counts[k * slots + s] = word count; the words are appended to
 * trace_words in (k, s) order (trace_cap words available).
 *
 * Row trace (optional, row_counts != NULL; mode 2): the row buffer of every
 * block in the level-k fold when the fold is itself a compressed exchange
 * (the 2D partitioning the paper names in Sec. VIII): the WAH stream of the
 * vertices block (i,j) reached, sieved by the visited set of range i before
 * the level, support(t_{i,j}) (.) not(pi_i), slot s = i*p + j, counted and
 * appended like the column trace (row_cap words available).  The oracle
 * decompresses every row buffer and checks that their OR over j is the next
 * frontier of range i.
 *
 * Outputs level[] and parent[] (length n).  Returns the number of levels
 * traced (the number of exchanges), -1 on a bad argument, -2 if a trace does
 * not fit, -3 on a decode failure (cannot happen for encoder output), -4 if
 * the OR of the row buffers differs from the next frontier (cannot happen).
 */
int64_t oracle_dist_bfs(int64_t n, int p, const int64_t *row_ptr, const int32_t *col, int32_t root,
                        int mode, int w, int use_max, int32_t *level, int32_t *parent,
                        uint64_t *trace_words, int64_t trace_cap, int64_t *trace_counts,
                        int64_t max_levels, uint64_t *row_words, int64_t row_cap, int64_t *row_counts)
{
    if (n <= 0 || p <= 0 || p > n || root < 0 || root >= n || mode < 0 || mode > 3) return -1;
    /* mode 3: DIR-WAH with a dynamic cross directory (the reading of Sec. V-B's
     * synchronous update): V_{i,j}(u) is cleared once every entry of u into
     * range i leads to a visited vertex; traced and sieved like mode 2 */
    const int dynamic = (mode == 3);
    if (dynamic) mode = 2;
    const int64_t nb = range_size(n, p);
    const int rows = (mode == 2 && row_counts != NULL);
    uint8_t *f = (uint8_t *)calloc((size_t)n, 1);        /* current frontier, all ranges */
    uint8_t *pi = (uint8_t *)calloc((size_t)n, 1);       /* visited */
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);   /* semiring value, -1 = zero */
    int32_t *tij = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nb + 1));  /* one block's product */
    uint8_t *recv = (uint8_t *)calloc((size_t)n * (size_t)p, 1);   /* f_{i,j} as received by P_i */
    uint8_t *slice = (uint8_t *)malloc((size_t)nb + 1);
    uint8_t *dec = (uint8_t *)malloc((size_t)nb + 1);
    uint8_t *fold = (uint8_t *)calloc((size_t)n, 1);     /* OR of the decoded row buffers */
    uint64_t *words = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nb + 2));
    uint8_t *D = (mode == 2) ? (uint8_t *)malloc((size_t)n * (size_t)p) : NULL;
    if (!f || !pi || !t || !tij || !recv || !slice || !dec || !fold || !words || (mode == 2 && !D)) {
        free(f); free(pi); free(t); free(tij); free(recv); free(slice); free(dec); free(fold); free(words);
        free(D);
        return -1;
    }
    /* the cross directories of every processor (Eq. 5), static for the graph */
    if (mode == 2) oracle_cross_directory(n, p, row_ptr, col, D);
    /* dynamic: cnt[i*n + u] = entries u -> v with v in range i not yet visited;
     * the update walks the entries into every newly visited vertex (in_ptr/in_src) */
    int64_t *cnt = NULL, *in_ptr = NULL;
    int32_t *in_src = NULL;
    if (dynamic) {
        const int64_t m = row_ptr[n];
        cnt = (int64_t *)calloc((size_t)n * (size_t)p, sizeof(int64_t));
        in_ptr = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
        in_src = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
        int64_t *fillp = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
        if (!cnt || !in_ptr || !in_src || !fillp) {
            free(cnt); free(in_ptr); free(in_src); free(fillp);
            free(f); free(pi); free(t); free(tij); free(recv); free(slice); free(dec); free(fold); free(words); free(D);
            return -1;
        }
        for (int64_t u = 0; u < n; ++u)
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                cnt[(size_t)(col[e] / nb) * (size_t)n + (size_t)u] += 1;
                in_ptr[col[e] + 1] += 1;
            }
        for (int64_t v = 0; v < n; ++v) in_ptr[v + 1] += in_ptr[v];
        for (int64_t v = 0; v < n; ++v) fillp[v] = in_ptr[v];
        for (int64_t u = 0; u < n; ++u)
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) in_src[fillp[col[e]]++] = (int32_t)u;
        free(fillp);
    }
    /* recv[i*n + u] = bit u of the frontier as P_i holds it after the exchange */
    for (int64_t v = 0; v < n; ++v) { level[v] = -1; parent[v] = -1; }
    level[root] = 0; parent[root] = root;
    f[root] = 1; pi[root] = 1;
    if (dynamic) {                         /* the root is visited before the first exchange */
        for (int64_t e = in_ptr[root]; e < in_ptr[root + 1]; ++e) {
            int64_t *c = &cnt[(size_t)(root / nb) * (size_t)n + (size_t)in_src[e]];
            if (--*c == 0) D[(size_t)(root / nb) * (size_t)n + (size_t)in_src[e]] = 0;
        }
    }
    const int64_t slots = (mode == 2) ? (int64_t)p * p : (mode == 1 ? p : 0);
    int64_t k = 0, used = 0, row_used = 0, rc = 0;
    for (;;) {
        /* ---- exchange of f (the frontier of level k) ---- */
        int64_t fsize = 0;
        for (int64_t v = 0; v < n; ++v) fsize += f[v];
        if (fsize == 0) break;
        for (int i = 0; i < p; ++i) {
            for (int j = 0; j < p; ++j) {
                const int64_t jb = range_begin(n, p, j), jl = range_end(n, p, j) - jb;
                uint8_t *dst = recv + (size_t)i * (size_t)n + (size_t)jb;
                if (mode == 0) {                                   /* BIT: raw bitmap */
                    memcpy(dst, f + jb, (size_t)jl);
                    continue;
                }
                if (mode == 1 && i > 0) {                          /* WAH: one stream per j, */
                    memcpy(dst, recv + (size_t)jb, (size_t)jl);    /* everyone gets the same */
                    continue;
                }
                if (mode == 2) {                                   /* sieve: f_j (.) V_{i,j} */
                    const uint8_t *Vij = D + (size_t)i * (size_t)n + (size_t)jb;
                    for (int64_t q = 0; q < jl; ++q) slice[q] = (uint8_t)(f[jb + q] & Vij[q]);
                } else {
                    for (int64_t q = 0; q < jl; ++q) slice[q] = f[jb + q];
                }
                int64_t nw = oracle_wah_encode(slice, jl, w, 1, words);
                if (trace_counts && k < max_levels) {
                    const int64_t s = (mode == 2) ? (int64_t)i * p + j : j;
                    trace_counts[k * slots + s] = nw;
                    if (used + nw > trace_cap) { rc = -2; goto done; }
                    memcpy(trace_words + used, words, sizeof(uint64_t) * (size_t)nw);
                    used += nw;
                }
                if (oracle_wah_decode(words, nw, jl, w, 1, dec) != 0) { rc = -3; goto done; }
                memcpy(dst, dec, (size_t)jl);
            }
        }
        /* ---- t_i = (+)_j t_{i,j}, t_{i,j} = A_{i,j} (x) f_{i,j} over (select, min|max) ---- */
        for (int64_t v = 0; v < n; ++v) { t[v] = -1; fold[v] = 0; }
        for (int i = 0; i < p; ++i) {
            const int64_t ib = range_begin(n, p, i), ie = range_end(n, p, i);
            const uint8_t *fi = recv + (size_t)i * (size_t)n;
            for (int j = 0; j < p; ++j) {
                const int64_t jb = range_begin(n, p, j), je = range_end(n, p, j);
                for (int64_t v = ib; v < ie; ++v) tij[v - ib] = -1;
                for (int64_t u = jb; u < je; ++u) {
                    if (!fi[u]) continue;
                    for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                        const int32_t v = col[e];
                        if (v < ib || v >= ie) continue;
                        int32_t *x = &tij[v - ib];
                        if (*x < 0 || (!use_max && u < *x) || (use_max && u > *x)) *x = (int32_t)u;
                    }
                }
                if (rows && k < max_levels) {
                    /* row buffer of block (i,j): what it reached, sieved by not(pi_i) */
                    for (int64_t v = ib; v < ie; ++v) slice[v - ib] = (uint8_t)(tij[v - ib] >= 0 && !pi[v]);
                    const int64_t nw = oracle_wah_encode(slice, ie - ib, w, 1, words);
                    row_counts[k * slots + (int64_t)i * p + j] = nw;
                    if (row_used + nw > row_cap) { rc = -2; goto done; }
                    memcpy(row_words + row_used, words, sizeof(uint64_t) * (size_t)nw);
                    row_used += nw;
                    if (oracle_wah_decode(words, nw, ie - ib, w, 1, dec) != 0) { rc = -3; goto done; }
                    for (int64_t v = ib; v < ie; ++v) fold[v] |= dec[v - ib];
                }
                /* the fold: t_i = t_i (+) t_{i,j} */
                for (int64_t v = ib; v < ie; ++v) {
                    const int32_t x = tij[v - ib];
                    if (x < 0) continue;
                    if (t[v] < 0 || (!use_max && x < t[v]) || (use_max && x > t[v])) t[v] = x;
                }
            }
        }
        /* ---- t = t (.) not(pi); pi = pi + t; f = t ---- */
        for (int64_t v = 0; v < n; ++v) {
            if (pi[v]) t[v] = -1;
            f[v] = (uint8_t)(t[v] >= 0);
            if (f[v]) { pi[v] = 1; level[v] = (int32_t)(k + 1); parent[v] = t[v]; }
        }
        /* ---- dynamic directory: every entry u -> v into a newly visited v ---- */
        if (dynamic)
            for (int64_t v = 0; v < n; ++v) {
                if (!f[v]) continue;
                for (int64_t e = in_ptr[v]; e < in_ptr[v + 1]; ++e) {
                    const size_t x = (size_t)(v / nb) * (size_t)n + (size_t)in_src[e];
                    if (--cnt[x] == 0) D[x] = 0;
                }
            }
        if (rows && k < max_levels)
            for (int64_t v = 0; v < n; ++v)
                if (fold[v] != f[v]) { rc = -4; goto done; }
        ++k;
    }
    rc = k;
done:
    free(f); free(pi); free(t); free(tij); free(recv); free(slice); free(dec); free(fold); free(words); free(D);
    free(cnt); free(in_ptr); free(in_src);
    return rc;
}

/*
 * What a dynamic cross directory would drop, by definition, level by level of
 * the search from root on a p x p grid.  With F_k the frontier of level k and
 * pi_k the vertices visited when it is exchanged (levels <= k):
 *   out[5k+0]  pairs (u, i), u in F_k, that the static directory sends
 *              (u has an entry into range i: V_{i,range(u)}(u) = 1);
 *   out[5k+1]  pairs a dynamic directory sends (u has an entry into range i
 *              leading to a vertex not in pi_k);
 *   out[5k+2]  entries the static pairs make the expansion read;
 *   out[5k+3]  entries of the dropped pairs (all of them lead to visited
 *              vertices: the work the dynamic directory saves);
 *   out[5k+4]  entries into the vertices of F_k, which the update of the
 *              dynamic directory walks when F_k becomes visited.
 * Returns the number of levels written (at most max_levels), -1 on bad input.
 */
int64_t oracle_dynamic_sieve_stats(int64_t n, int p, const int64_t *row_ptr, const int32_t *col, int32_t root,
                                   int64_t max_levels, int64_t *out)
{
    if (n <= 0 || p <= 0 || p > n || root < 0 || root >= n) return -1;
    const int64_t nb = range_size(n, p);
    int32_t *level = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *in_deg = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *to_range = (int64_t *)calloc((size_t)p, sizeof(int64_t));
    int64_t *fresh_in_range = (int64_t *)calloc((size_t)p, sizeof(int64_t));
    if (!level || !in_deg || !to_range || !fresh_in_range) {
        free(level); free(in_deg); free(to_range); free(fresh_in_range);
        return -1;
    }
    oracle_bfs_levels(n, row_ptr, col, root, level);
    for (int64_t u = 0; u < n; ++u)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) in_deg[col[e]] += 1;
    int64_t depth = 0;
    for (int64_t v = 0; v < n; ++v) if (level[v] + 1 > depth) depth = level[v] + 1;
    if (depth > max_levels) depth = max_levels;
    for (int64_t k = 0; k < depth; ++k) {
        int64_t *o = out + 5 * k;
        for (int q = 0; q < 5; ++q) o[q] = 0;
        for (int64_t u = 0; u < n; ++u) {
            if (level[u] != k) continue;
            o[4] += in_deg[u];
            for (int i = 0; i < p; ++i) { to_range[i] = 0; fresh_in_range[i] = 0; }
            for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                const int32_t v = col[e];
                const int i = (int)(v / nb);
                to_range[i] += 1;
                if (level[v] < 0 || level[v] > k) fresh_in_range[i] += 1;     /* not in pi_k */
            }
            for (int i = 0; i < p; ++i) {
                if (!to_range[i]) continue;
                o[0] += 1;
                o[2] += to_range[i];
                if (fresh_in_range[i]) o[1] += 1;
                else o[3] += to_range[i];
            }
        }
    }
    free(level); free(in_deg); free(to_range); free(fresh_in_range);
    return depth;
}
