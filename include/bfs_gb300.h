/*
 * bfs_gb300.h -- C ABI of the compressed and sieved level-synchronous BFS on
 * one GB300 (sm_103a).
 *
 * The method (Lv, Tan, Chen, Sun, "Compression and Sieve: Reducing
 * Communication in Parallel Breadth First Search on Distributed Memory
 * Systems"): BFS as a boolean sparse matrix-vector product per level
 * (Sec. III-A, Alg. 1); the adjacency matrix split into a p x p grid of blocks
 * A_{i,j} (Eq. 1-3); the frontier exchanged between block-rows compressed
 * with the word-aligned hybrid code (Sec. IV, Table 3, Alg. 2) after being
 * sieved by the cross directory V_{i,j} (Eq. 4-5, Sec. V-B, Alg. 3).  On one
 * GPU the p x p processor grid is a virtual grid of blocks in HBM and every
 * exchanged message is a per-block buffer in HBM.  Beside the paper's three
 * algorithms: the hybrid top-down / bottom-up levels it names as future work
 * (Sec. VIII, IX; bfs_graph_set_direction), bit-parallel batches of up to 64
 * roots and a continuous-batching server (bfs_run_batch, bfs_server_*), the
 * row exchange of the 2D partition (Sec. VIII; bfs_graph_set_row_exchange),
 * the level-adaptive exchange format (Sec. II, Table 2;
 * bfs_graph_set_exchange_format), the dynamic cross directory (Sec. V-B;
 * bfs_graph_set_dynamic_directory), and the PLWAH and BBC codes it names
 * beside WAH (Sec. IV; bfs_plwah_*, bfs_bbc_*).
 *
 * Conventions for every entry point:
 *   - Errors are returned as a bfs_status; nothing throws across the ABI and
 *     outputs are unspecified when the status is not BFS_OK.  A one-line
 *     description of the last error of the calling thread is available from
 *     bfs_last_error().
 *   - `cuda_stream` is a cudaStream_t (NULL = the legacy default stream).  Work
 *     is ordered on that stream; entry points that must report a result to the
 *     host (a status from the device, a size) synchronise that stream and say so.
 *   - Device pointers are CUDA device allocations of the current device.  Where
 *     an argument says "host or device", the library asks the CUDA runtime which
 *     it is and copies host data itself.
 *   - Vertex ids are int32 in [0, n), 1 <= n <= 2^31 - 1.
 *   - Every wait inside the library is bounded; no call blocks forever.
 *
 * Citations name the paper's sections, equations, algorithms and tables.
 */
#ifndef BFS_GB300_H
#define BFS_GB300_H

#include <stdint.h>

#if defined(__GNUC__)
#define BFS_API __attribute__((visibility("default")))
#else
#define BFS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bfs_graph *bfs_graph_t;
typedef struct bfs_server *bfs_server_t;

typedef enum {
    BFS_OK = 0,
    BFS_ERR_INVALID_ARG = 1,    /* an argument is out of range or inconsistent */
    BFS_ERR_OUT_OF_MEMORY = 2,  /* a device or host allocation failed */
    BFS_ERR_CUDA = 3,           /* a CUDA runtime call failed (see bfs_last_error) */
    BFS_ERR_TIMEOUT = 4,        /* a bounded wait ran out */
    BFS_ERR_CORRUPT = 5,        /* a compressed stream is malformed */
    BFS_ERR_BUSY = 6,           /* the object is in use by another call */
    BFS_ERR_NOT_FOUND = 7       /* an id or ticket is unknown */
} bfs_status;

/* Frontier exchange of each level (the three algorithms of Table 5). */
enum {
    BFS_MODE_PLAIN = 0,          /* BIT, Alg. 1: raw bitmap frontier */
    BFS_MODE_COMPRESS = 1,       /* WAH, Alg. 2: one WAH stream per source range */
    BFS_MODE_COMPRESS_SIEVE = 2  /* DIR-WAH, Alg. 3: one WAH stream per (source range j,
                                    block-row i) holding f_j sieved by V_{i,j} */
};

typedef struct {
    int32_t grid_r;          /* virtual grid rows p (destination ranges); 1 <= p <= min(n, 1024) */
    int32_t grid_c;          /* virtual grid columns; must equal grid_r (square grid, Eq. 1-2) */
    int32_t mode;            /* BFS_MODE_* */
    int32_t wah_word_bits;   /* 32 (31-bit groups, Table 3) or 64 (63-bit groups) */
    int32_t autotune;        /* 1: the first bfs_run_batch on the graph runs bfs_batch_autotune
                                on its own roots and keeps the fastest launch shape */
    int32_t debug_checks;    /* 1: bfs_run checks its outputs before returning (bfs_check_search,
                                plus: the reached vertices are those the search visited) and
                                reports BFS_ERR_CORRUPT.  The device-side bounds and stream checks
                                of the kernels (a sieved vertex without a column, a malformed
                                row buffer, a full piece list) run in every mode. */
    int32_t row_exchange;    /* 1: compressed row exchange of the fold in COMPRESS_SIEVE mode
                                (see bfs_graph_set_row_exchange) */
} bfs_options;

/* Fill `opt` with the defaults: 1 x 1 grid, BFS_MODE_COMPRESS_SIEVE, 32-bit words,
 * row exchange on. */
BFS_API void bfs_options_default(bfs_options *opt);

/* Human-readable name of a status ("BFS_OK", ...). Never NULL. */
BFS_API const char *bfs_status_string(bfs_status s);

/* Copy the calling thread's last error message (NUL-terminated, truncated to
 * `len` bytes) into `buf`.  Returns the status of that error. */
BFS_API bfs_status bfs_last_error(char *buf, int64_t len);

/*
 * Build a graph from n_edges directed tuples (src[e], dst[e]) (Sec. VII-A:
 * the tuples of the generated edge list, multi-edges and self-loops kept).
 * With `symmetrize` != 0 every tuple also adds the reverse entry dst -> src
 * (a self-loop therefore adds two entries), giving the undirected graph the
 * paper searches.  src/dst may be host or device pointers; they are copied and
 * the caller keeps ownership.  The build lays the entries out on the device as
 * the p x p grid of blocks A_{i,j} (block-row i = destination range i, block
 * column j = source range j; range b = [b*ceil(n/p), min(n, (b+1)*ceil(n/p)))),
 * each block stored column-compressed over its nonempty source columns with
 * the directory vector V_{i,j} of Eq. 4 as the column index.  The graph owns
 * all of its device memory.  Synchronises `cuda_stream`.
 * Errors: BFS_ERR_INVALID_ARG for n outside [1, 2^31-1], n_edges < 0, an id
 * outside [0, n), a bad option; BFS_ERR_OUT_OF_MEMORY; BFS_ERR_CUDA.
 */
BFS_API bfs_status bfs_graph_create_edges(int64_t n_vertices, int64_t n_edges, const int32_t *src,
                                  const int32_t *dst, int32_t symmetrize, const bfs_options *opt,
                                  void *cuda_stream, bfs_graph_t *out);

/*
 * Build a graph from a CSR adjacency: row_ptr[n+1] (int64, row_ptr[0] = 0,
 * nondecreasing) and col[row_ptr[n]] (int32), entry u -> col[e] for e in
 * [row_ptr[u], row_ptr[u+1]).  No symmetrisation.  Host or device pointers,
 * copied.  Same layout, ownership and errors as bfs_graph_create_edges.
 */
BFS_API bfs_status bfs_graph_create_csr(int64_t n_vertices, const int64_t *row_ptr, const int32_t *col,
                                const bfs_options *opt, void *cuda_stream, bfs_graph_t *out);

/* Free the graph and all of its device memory.  NULL is accepted. */
BFS_API bfs_status bfs_graph_destroy(bfs_graph_t g);

/* Device bytes held by the graph (layout plus per-search workspace). */
BFS_API bfs_status bfs_graph_footprint(bfs_graph_t g, int64_t *bytes);

typedef struct {
    int64_t n_vertices;
    int64_t n_entries;       /* directed adjacency entries */
    int32_t p;               /* grid is p x p */
    int32_t mode;
    int32_t wah_word_bits;
    int32_t row_exchange;
    int64_t range_size;      /* ceil(n / p) */
    int64_t nonempty_columns;/* sum over blocks of |V_{i,j}| (set directory bits) */
    int32_t exchange_format; /* BFS_FORMAT_* */
    int32_t direction;       /* BFS_DIRECTION_* */
    int32_t dynamic_directory; /* 1: the sieve reads the search's dynamic cross directory */
    int32_t reserved;
} bfs_graph_info_t;

BFS_API bfs_status bfs_graph_info(bfs_graph_t g, bfs_graph_info_t *info);

/* Switch the exchange mode and WAH word width of later searches (the layout
 * serves all three algorithms of Table 5).  Not safe while a search on `g`
 * is running. */
BFS_API bfs_status bfs_graph_set_mode(bfs_graph_t g, int32_t mode, int32_t wah_word_bits);

/*
 * The row exchange of the 2D partition: the fold of block-row i, which the
 * paper names as the combination of its method with 2D partitioning (Sec.
 * VIII), made a compressed and sieved exchange like the column exchange of
 * Alg. 3.  On a level with the row exchange every block (i,j) records the
 * vertices of range i it reached, t_{i,j} = support(A_{i,j} (x) f_{i,j}), in a
 * bitmap of its own; the partial is sieved by not(pi_i) -- vertices visited
 * before the level are dropped -- and WAH-encoded (Sec. IV, Table 3, the
 * graph's word width) into the row buffer of slot i*p + j; the fold
 * OR-decodes the p buffers of block-row i into t_i.  Row buffers are unique
 * (they depend on the graph, the frontier and pi only) and can be traced
 * (bfs_run_stats.row_trace_*).  The result never changes t_i.
 *   enabled: 1 (the default) or 0 (the partials are ORed into t directly,
 *   as one undivided next bitmap).
 * Applies to top-down levels of COMPRESS_SIEVE searches (bfs_run); PLAIN and
 * COMPRESS searches (Alg. 1, 2), bottom-up levels and the batched and served
 * searches fold without buffers.  The first search with it allocates the
 * partials (p*p directory-sized bitmaps) and the row buffers (p*p worst-case
 * WAH streams), kept with the graph and counted by bfs_graph_footprint.  Not
 * safe while a search on `g` is running.
 */
BFS_API bfs_status bfs_graph_set_row_exchange(bfs_graph_t g, int32_t enabled);

/* Format of the exchanged column slices (bfs_graph_set_exchange_format). */
enum {
    BFS_FORMAT_WAH = 0,          /* every slice a WAH stream (Sec. IV; Alg. 2, 3) */
    BFS_FORMAT_ADAPTIVE = 1      /* per slice and level the smallest of its WAH stream, sparse vector
                                    and raw bitmap */
};

/*
 * The level-adaptive exchange format.  Sec. II sets the bitmap against the
 * sparse vector as the two ways to hold a frontier (Table 2: which is smaller
 * depends on the frontier's density) and Sec. V-A notes that a sieved slice is
 * very sparse; Alg. 1 sends the raw bitmap.  With BFS_FORMAT_ADAPTIVE every
 * exchanged slice of the column exchange (COMPRESS and COMPRESS_SIEVE) goes,
 * level by level, as the smallest in bytes of
 *   0  its WAH stream (32-bit words, as with BFS_FORMAT_WAH),
 *   1  its sparse vector: the offsets of its set bits within the slice, in
 *      increasing order, one uint32 each,
 *   2  its raw bitmap: ceil(bits/32) uint32 words, bit b = bit b%32 of word b/32,
 * the lower number on a tie.  The choice is made on the device from the
 * slice's WAH size and set-bit count; the expansion (and the bottom-up stream
 * decode) reads all three.  The exchange trace then holds each slot's
 * elements and, in bfs_run_stats.trace_formats, its format.  Needs 32-bit WAH
 * words (bfs_run returns BFS_ERR_INVALID_ARG with 64-bit words).  The row
 * buffers of the fold stay WAH.  Not safe while a search on `g` is running.
 */
BFS_API bfs_status bfs_graph_set_exchange_format(bfs_graph_t g, int32_t format);

/*
 * The dynamic cross directory.  Sec. V-B has both sides of the exchange keep
 * the directories up to date as the search goes on; Alg. 3 sieves every level
 * with the static V_{i,j} of Eq. 4.  With the dynamic directory on, a search
 * sieves with its own directories D_{i,j}, where D_{i,j}(u) = 1 while column
 * u of block A_{i,j} still holds an entry into a vertex that is not visited:
 * once every entry of u into range i leads to a visited vertex, u can reach
 * nothing more in block-row i and is no longer sent there.  The sieve of
 * level k sends f_j (.) D_{i,j} with the visited set of levels 0..k, the
 * state that updating D after every visit leaves.  A bit matters only at the
 * exchange that sends its vertex and never comes back once cleared, so the
 * library evaluates, just before each exchange, the bits of the frontier's
 * vertices from their definition (a scan of the column that stops at the
 * first unvisited destination) in a copy of the directories taken at the
 * search's start.  Levels and parents never change; the exchanged streams
 * carry fewer vertices (bfs_level_stats.exchanged_vertices), and the scans
 * cost time before each exchange (bfs_level_stats.ms_directory_update).
 *   enabled: 1, or 0 (the default: the static directory of Alg. 3).
 * Applies to COMPRESS_SIEVE searches (bfs_run), directed or undirected
 * graphs, top-down and bottom-up levels, with or without the row exchange
 * and either exchange format; PLAIN and COMPRESS searches have no sieve, and
 * the batched and served searches keep the static directory.  The first
 * search with it allocates the copy (p*p directory bitmaps), kept with the
 * graph and counted by bfs_graph_footprint.  Not safe while a search on `g`
 * is running.
 */
BFS_API bfs_status bfs_graph_set_dynamic_directory(bfs_graph_t g, int32_t enabled);

/* Direction of each level (bfs_graph_set_direction). */
enum {
    BFS_DIRECTION_TOP_DOWN = 0,   /* every level top-down: Alg. 1-3 as printed */
    BFS_DIRECTION_HYBRID = 1,     /* top-down or bottom-up, chosen per level */
    BFS_DIRECTION_BOTTOM_UP = 2   /* every level bottom-up (a test setting) */
};

/*
 * The hybrid top-down / bottom-up traversal of Beamer et al., which the paper
 * names in Sec. VIII and IX as the next method to combine with compression and
 * sieve.  The algorithms of Table 5 expand top-down: every frontier vertex u
 * scans its columns.  A bottom-up level instead lets every unvisited vertex v
 * of block-row i scan its own neighbours range by range (j = 0, 1, ..., p-1:
 * the column of v in block (j, i)), testing each neighbour u against the
 * frontier that the exchange delivered for block (i, j): the stream of slot
 * (i, j) (f_j sieved by V_{i,j} in COMPRESS_SIEVE mode, f_j in COMPRESS mode)
 * decoded, or the raw slice f_j in PLAIN mode.  All streams of a level are
 * decoded into one n-bit bitmap, ORed over the block-rows; it holds at u the
 * bit of slot (i, j) itself, since u has a neighbour in range i
 * (V_{i,j}(u) = 1).  The first range
 * holding a frontier neighbour gives v its parent, the smallest such
 * neighbour, which is the smallest neighbour on the previous level: levels and
 * parents are identical to the top-down search, and so is every exchanged
 * stream (the exchange of a level does not depend on its direction).
 *   policy: BFS_DIRECTION_*.  HYBRID switches top-down -> bottom-up when the
 *     frontier grew and its degree sum m_f exceeds m_u / alpha (m_u: degree
 *     sum of the unvisited vertices), and bottom-up -> top-down when the
 *     frontier shrank below n / beta vertices (Beamer et al.'s rule; they
 *     use alpha = 14, beta = 24).
 *   alpha, beta: 1 .. 1,000,000; used by HYBRID only.
 * Bottom-up needs the in-neighbours of v, which are its out-neighbours only
 * when the graph is undirected: a graph created with symmetrize = 0 (every
 * CSR graph included) returns BFS_ERR_INVALID_ARG for any policy other than
 * TOP_DOWN.  The first such call computes every vertex's degree and a copy of
 * the adjacency laid out for bottom-up scans: v's columns in blocks (0, i),
 * (1, i), ... back to back (4 + 8 bytes per vertex and 4 bytes per entry, kept
 * with the graph and counted by bfs_graph_footprint; ordered on the legacy
 * default stream and synchronised).  Applies to bfs_run; the batched and
 * served searches (bfs_run_batch, bfs_server_*) stay top-down.  Not safe
 * while a search on `g` is running.
 */
BFS_API bfs_status bfs_graph_set_direction(bfs_graph_t g, int32_t policy, int32_t alpha, int32_t beta);

/*
 * Copy the directory vector V_{i,j} (Eq. 4: bit k set iff source column
 * begin(j)+k of block A_{i,j} has an entry) into `out_words` (device,
 * ceil(range_len(j)/32) uint32 words, bit k = bit k%32 of word k/32).
 * Ordered on `cuda_stream`.
 */
BFS_API bfs_status bfs_graph_directory(bfs_graph_t g, int32_t i, int32_t j, uint32_t *out_words,
                               void *cuda_stream);

/* Per-level counters of one search (Table 6 phase labels for the timers). */
typedef struct {
    int64_t frontier_vertices;   /* |f_k| of the frontier exchanged for level k */
    int64_t exchanged_vertices;  /* set bits carried by the exchange (after the sieve);
                                    PLAIN/COMPRESS: p * |f_k| */
    int64_t column_hits;         /* (vertex, block) pairs with a nonempty column, the
                                    work items of the expansion (bottom-up: the columns
                                    of unvisited vertices read) */
    int64_t raw_bytes;           /* bytes of the raw bitmap exchange: p slices of each range */
    int64_t wah_bytes;           /* bytes of the compressed streams (0 in PLAIN mode) */
    int64_t edges_scanned;       /* adjacency entries read by the expansion */
    int64_t row_wah_bytes;       /* bytes of the row buffers of the fold (0 when the row exchange is
                                    off and on bottom-up levels) */
    float ms_compress_sieve;     /* sieve + compress + decompress kernels */
    float ms_communication;      /* exchange: size scan (and packing when traced) */
    float ms_traversing;         /* expansion (the local SpMV) */
    float ms_reducing;           /* mask, visited update, level writeback, frontier count */
    int32_t bottom_up;           /* 1: the level ran bottom-up (bfs_graph_set_direction) */
    float ms_row_compress;       /* row exchange: sieve by not(pi) + compress of the partials */
    float ms_row_fold;           /* row exchange: decompress + OR of the row buffers (the fold) */
    float ms_directory_update;   /* dynamic cross directory: the frontier's bits evaluated before
                                    the exchange (bfs_graph_set_dynamic_directory; 0 without it) */
    int64_t compress_chunks;     /* chunks of 1024 groups the column sieve + compress read (each:
                                    the chunk's frontier and directory bits) */
    int64_t row_compress_chunks; /* chunks the row sieve + compress read (partial and visited bits) */
} bfs_level_stats;

typedef struct {
    int32_t capacity_levels;     /* entries of `levels` (and rows of trace_counts) */
    int32_t n_levels;            /* out: exchanges performed (= BFS depth + 1 when reached set > 1) */
    int32_t timing;              /* 1: fill the ms_* fields with CUDA-event times */
    int32_t reserved;
    bfs_level_stats *levels;     /* host array of capacity_levels entries, or NULL */
    /* Optional exchange trace (device pointers, or NULL): for each exchange k,
     * the streams of all slots packed back to back in slot order (slot = i*p + j
     * in COMPRESS_SIEVE mode, j in COMPRESS mode) -- the receive buffer g' of
     * Alg. 3 -- with each 32-bit WAH word as one uint32 and each 64-bit word as
     * two uint32 (low half first). trace_counts[k*slots + s] = words in slot s. */
    uint32_t *trace_words;
    int64_t trace_capacity;      /* uint32 elements available in trace_words */
    int64_t *trace_counts;       /* device, capacity_levels * slots entries */
    int64_t trace_used;          /* out: uint32 elements written */
    uint8_t *trace_formats;      /* device, capacity_levels * slots entries, or NULL: the format of
                                    every traced slot (BFS_FORMAT_ADAPTIVE's 0 / 1 / 2; 0 otherwise) */
    /* Optional row-buffer trace (device pointers, or NULL; COMPRESS_SIEVE with the
     * row exchange on): for each level k, the row buffers of the fold packed in
     * slot order (slot = i*p + j: the WAH stream of the vertices of range i that
     * block (i,j) reached, sieved by not(pi_i)), words as in trace_words;
     * row_trace_counts[k*p*p + s] = words in slot s (0 on bottom-up levels). */
    uint32_t *row_trace_words;
    int64_t row_trace_capacity;  /* uint32 elements available in row_trace_words */
    int64_t *row_trace_counts;   /* device, capacity_levels * p * p entries */
    int64_t row_trace_used;      /* out: uint32 elements written */
} bfs_run_stats;

/*
 * One breadth-first search from `root` (Alg. 1, 2 or 3 per the graph's mode).
 * Outputs, length n: level[v] = hop distance from root (root 0, unreached -1);
 * parent[v] = the smallest neighbour u of v with level[u] = level[v] - 1
 * (root: root; unreached: -1).  parent/level may both be device pointers (the
 * search stays on the device and is ordered on `cuda_stream`) or both host
 * pointers (results are copied back before returning).  With `stats` NULL the
 * level loop runs on the device as one CUDA-graph launch (a conditional node
 * repeats the level while the frontier is not empty; the graph is built on the
 * first call for the graph's mode and output buffers and reused), and the call
 * synchronises the stream once at the end; with `stats` the host steps through
 * the levels and synchronises once per level to read the counters.
 * Errors: BFS_ERR_INVALID_ARG (root out of range, trace too small),
 * BFS_ERR_BUSY (another search on this graph is running), BFS_ERR_CORRUPT
 * (debug checks found a broken invariant), BFS_ERR_CUDA.
 */
BFS_API bfs_status bfs_run(bfs_graph_t g, int32_t root, int32_t *parent, int32_t *level,
                   bfs_run_stats *stats, void *cuda_stream);

/*
 * Check the outputs of a search from `root` (the definition of level[] and
 * parent[] in Sec. II and the output specification of Alg. 1): level[root] = 0
 * and parent[root] = root; an unreached vertex has level -1 and parent -1; a
 * reached vertex v != root has level > 0 and a parent in [0, n) whose level is
 * level[v] - 1.  (Whether parent -> v is an entry of the graph is not checked.)
 * parent/level: device, length n.  Synchronises `cuda_stream`.  Allocates a
 * few bytes of scratch.  Errors: BFS_ERR_CORRUPT with the number of failing
 * vertices and the smallest one in bfs_last_error(); BFS_ERR_INVALID_ARG.
 */
BFS_API bfs_status bfs_check_search(bfs_graph_t g, int32_t root, const int32_t *parent, const int32_t *level,
                                    void *cuda_stream);

/* Counters of one batched search. */
typedef struct {
    int32_t n_levels;            /* levels performed (the deepest search's depth + 1) */
    int32_t reserved;
    int64_t edges_scanned;       /* adjacency entries read, all levels */
} bfs_batch_stats;

/*
 * Up to 64 breadth-first searches at once, bit-parallel: every vertex holds a
 * 64-bit lane word per state (frontier, visited, next; bit r = search r), and
 * one level is the boolean SpMV of Sec. III-A applied to all lanes, sieved by
 * the directories V_{i,j} (Eq. 4) like the single search.  The whole batch is
 * one CUDA-graph launch (a conditional WHILE node iterates the level body on
 * the device).
 *   roots: n_roots (1..64) vertex ids, host or device; duplicates allowed.
 *   levels: device, [n_roots][n] int32; levels[r][v] = hop distance of v from
 *     roots[r], or -1.
 *   parents: device [n_roots][n] or NULL; parents[r][v] = the smallest
 *     neighbour u of v with levels[r][u] = levels[r][v] - 1 (roots[r] for the
 *     root, -1 if unreached).  Computing parents adds one reduction per newly
 *     reached (vertex, search) pair per candidate edge and is markedly slower.
 *   stats: NULL or filled after the batch.
 * Synchronises `cuda_stream` before returning.  The first call on a graph
 * builds and instantiates the CUDA graph.
 * Errors: BFS_ERR_INVALID_ARG (n_roots, a root out of range, host output
 * pointers), BFS_ERR_BUSY, BFS_ERR_CUDA.
 */
BFS_API bfs_status bfs_run_batch(bfs_graph_t g, const int32_t *roots, int32_t n_roots, int32_t *levels,
                                 int32_t *parents, bfs_batch_stats *stats, void *cuda_stream);

/*
 * Autotune the launch shape of the batched expansion on `g`: time the batch
 * for every candidate (threads per CTA in {128, 256, 512, 1024} x CTAs per SM
 * in {1, 2, 4, 8, 16}, at most 2048 threads per SM) on the given roots and
 * keep the fastest for later bfs_run_batch calls.  `levels` is a device
 * [n_roots][n] scratch output.  best_threads / best_ctas_per_sm may be NULL.
 */
BFS_API bfs_status bfs_batch_autotune(bfs_graph_t g, const int32_t *roots, int32_t n_roots, int32_t *levels,
                                      int32_t *best_threads, int32_t *best_ctas_per_sm, void *cuda_stream);

/*
 * Query server with continuous batching (no counterpart in the paper, which
 * runs one search at a time): graphs stay resident with up to 64 lanes of the
 * batched search each; a server thread runs one level of every running lane
 * per iteration, each graph on its own stream (their work overlaps on the
 * GPU), admits queued queries into free lanes at every iteration boundary and
 * retires lanes whose frontier emptied.  Every result is the level and
 * parent vectors of a single search from the query's root, the same as
 * bfs_run alone.
 * Graphs are admitted against `hbm_budget_bytes` by footprint (layout + lane
 * state + level and parent rows; the lane count is halved until it fits);
 * results not yet collected count against the budget and hold back new
 * admissions.
 * All waits are bounded.  Thread-safe.
 */
typedef struct {
    int64_t submitted, completed, rejected, queued;
    int64_t iterations;          /* level iterations run, all graphs */
    int32_t peak_lanes;          /* most lanes running at once, all graphs */
    int32_t graphs;
    int64_t hbm_used_bytes;      /* resident graphs + results awaiting collection */
    double p50_us, p99_us, max_us;   /* latency submit -> result ready */
} bfs_server_stats_t;

/* max_lanes in [1, 64] per graph. */
BFS_API bfs_status bfs_server_create(int64_t hbm_budget_bytes, int32_t max_lanes, bfs_server_t *out);
/* Make `g` resident; the server holds it (BFS_ERR_BUSY for other calls on it)
 * until bfs_server_destroy.  BFS_ERR_OUT_OF_MEMORY if it does not fit. */
BFS_API bfs_status bfs_server_add_graph(bfs_server_t s, bfs_graph_t g, int32_t *graph_id);
/* Queue a query; BFS_ERR_BUSY when the queue is full (the rejection is counted
 * in bfs_server_stats_t.rejected), BFS_ERR_NOT_FOUND for an unknown graph,
 * BFS_ERR_INVALID_ARG for a root outside the graph. */
BFS_API bfs_status bfs_server_submit(bfs_server_t s, int32_t graph_id, int32_t root, int64_t *ticket);
/* Flags of bfs_server_submit_ex. */
enum {
    BFS_QUERY_PARENTS = 1        /* also compute the query's parent vector (one more reduction per
                                    newly reached vertex and candidate edge in its lane) */
};
/* bfs_server_submit with flags (0 or BFS_QUERY_PARENTS); bfs_server_submit is flags = 0. */
BFS_API bfs_status bfs_server_submit_ex(bfs_server_t s, int32_t graph_id, int32_t root, int32_t flags,
                                        int64_t *ticket);
/* Queued (not yet admitted) queries accepted before bfs_server_submit returns
 * BFS_ERR_BUSY: 1 .. 1,048,576 (the default). */
BFS_API bfs_status bfs_server_set_queue_limit(bfs_server_t s, int64_t limit);
BFS_API bfs_status bfs_server_poll(bfs_server_t s, int64_t ticket, int32_t *done);
/* Wait at most timeout_us for the query (BFS_ERR_TIMEOUT otherwise; the query
 * stays valid and can be waited for again), copy its level vector (n int32) to
 * `level` and, for a query submitted with BFS_QUERY_PARENTS, its parent vector
 * (n int32: the smallest neighbour one level closer to the root, the root
 * itself for the root, -1 if unreached) to `parent` (each host or device, or
 * NULL), and release it.  A non-NULL `parent` for a query submitted without
 * the flag is BFS_ERR_INVALID_ARG (the query is kept). */
BFS_API bfs_status bfs_server_wait(bfs_server_t s, int64_t ticket, int64_t timeout_us, int32_t *level,
                                   int32_t *parent);
BFS_API bfs_status bfs_server_stats(bfs_server_t s, bfs_server_stats_t *stats);
/* Stop the server thread, drop uncollected results, release the graphs. */
BFS_API bfs_status bfs_server_destroy(bfs_server_t s);

/*
 * Failure injection for tests of the error paths (no counterpart in the
 * paper): the k-th device allocation the library makes from now on (k >= 1;
 * allocations of graphs, search workspaces, batches, server lanes and codec
 * scratch) fails as if the device were out of memory, and the call that made
 * it returns BFS_ERR_OUT_OF_MEMORY after releasing what it had allocated.
 * k = 0 disarms.  Process-wide; not for production use.
 */
BFS_API bfs_status bfs_debug_fail_allocation(int64_t k);

/*
 * WAH-encode one bitmap (Sec. IV, Table 3) on the device.
 *   bits: device, bit b of the bitmap = bit b%32 of bits[b/32], nbits >= 0
 *         bits; the array must hold ceil(nbits/32) + 2 words (the encoder
 *         reads up to two words past the end and ignores them).
 *   word_bits: 32 or 64.  Words are (word_bits-1)-bit groups, first bit of a
 *         group most significant; literal top bit 0; fill top bit 1, next bit
 *         the fill value, the rest the run length in groups; an all-0 or all-1
 *         group is always a fill and equal fills merge; an active word holds the
 *         nbits mod (word_bits-1) trailing bits right-aligned, first bit highest.
 *   words: device output, capacity_words words of word_bits bits; at most
 *         floor(nbits/(word_bits-1)) + 1 are written.
 *   nwords: device int64, receives the word count.
 * Uses scratch memory allocated on `cuda_stream` (stream-ordered allocator).
 * Errors: BFS_ERR_INVALID_ARG (bad width, capacity below the bound above).
 */
BFS_API bfs_status bfs_wah_encode(const uint32_t *bits, int64_t nbits, int32_t word_bits, void *words,
                          int64_t capacity_words, int64_t *nwords, void *cuda_stream);

/*
 * Decode a WAH stream (the inverse of bfs_wah_encode; accepts non-canonical
 * but well-formed streams) into `bits` (device, ceil(nbits/32) words, bits past
 * nbits in the last word are cleared).  Synchronises `cuda_stream` to report
 * the result.  Errors: BFS_ERR_CORRUPT if the stream is malformed (a fill of
 * length 0, groups past nbits, a missing or oversized active word, trailing
 * words); `bits` is then unspecified.  BFS_ERR_INVALID_ARG for a bad width.
 */
BFS_API bfs_status bfs_wah_decode(const void *words, int64_t nwords, int64_t nbits, int32_t word_bits,
                          uint32_t *bits, void *cuda_stream);

/*
 * bfs_wah_decode without any allocation.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory during a
 * call -- a serving process that has reserved the whole HBM budget for
 * resident graphs (where a cudaMalloc in the middle of a request fails), or a
 * latency-critical thread that must not pay for cudaFree, which waits for the
 * whole device.  It calls no cudaMalloc, cudaFree or allocating library code.
 * Same arguments, output and errors as bfs_wah_decode, with one limit:
 *   nbits <= 8,388,608; larger requests return BFS_ERR_INVALID_ARG.
 * Its scratch (an error word and a staging copy of the bitmap, about 1 MiB) is
 * one array in the library's static device memory, held by every device that
 * loads the library until the process exits.  The first call on a device
 * looks the array's address up (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  Every call on a
 * device shares the array and clears the part it uses before decoding, so
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race on it: order them.  Synchronises `cuda_stream`.
 */
BFS_API bfs_status bfs_wah_decode_static(const void *words, int64_t nwords, int64_t nbits, int32_t word_bits,
                                         uint32_t *bits, void *cuda_stream);

/*
 * PLWAH, the position-list word-aligned hybrid code that Sec. IV names beside
 * WAH as an alternative bitmap code (Deliege and Pedersen), for one bitmap on
 * the device.  32-bit words over 31-bit groups, bit order and active word as
 * in 32-bit WAH (bfs_wah_encode):
 *   literal: bit 31 = 0, bits 30..0 = one group;
 *   fill:    bit 31 = 1, bit 30 = the fill value v, bits 29..25 = a position q
 *            (0: none), bits 24..0 = the run length in groups (>= 1); q > 0
 *            stands for one more group right after the run, equal to v in
 *            every bit but its q-th (q = 1: the group's first bit).
 * An all-0 or all-1 group is a fill group and equal fill groups form one run;
 * a literal group right after a run that differs from the run's value in one
 * bit is carried by the run's position and not written.  The exchange of the
 * search keeps WAH; this code is offered beside it, for callers that ship
 * bitmaps themselves and for comparing the two codes on the same frontiers.
 *   bits: device, as for bfs_wah_encode (ceil(nbits/32) + 2 words readable).
 *   nbits: 0 .. 1,040,187,361 (31 x (2^25 - 1): every run fits the 25-bit
 *         length); larger requests return BFS_ERR_INVALID_ARG.
 *   words: device output, capacity_words >= floor(nbits/31) + 1.
 *   nwords: device int64, receives the word count.
 * Allocates scratch (cudaMalloc) and synchronises `cuda_stream`.
 */
BFS_API bfs_status bfs_plwah_encode(const uint32_t *bits, int64_t nbits, uint32_t *words, int64_t capacity_words,
                                   int64_t *nwords, void *cuda_stream);

/*
 * Decode a PLWAH stream (the inverse of bfs_plwah_encode; accepts well-formed
 * non-canonical streams) into `bits` (device, ceil(nbits/32) words, bits past
 * nbits in the last word cleared).  Allocates scratch and synchronises
 * `cuda_stream`.  Errors: BFS_ERR_CORRUPT for a malformed stream (a fill of
 * length 0, groups -- a position's group included -- past nbits, a missing
 * or oversized active word, trailing words); BFS_ERR_INVALID_ARG for nbits
 * above the limit of bfs_plwah_encode or bad pointers.
 */
BFS_API bfs_status bfs_plwah_decode(const uint32_t *words, int64_t nwords, int64_t nbits, uint32_t *bits,
                                   void *cuda_stream);

/*
 * BBC, the byte-aligned bitmap code (Antoshenkov) that Sec. IV names beside
 * WAH and PLWAH, for one bitmap on the device.  The paper does not define it;
 * this is the reading used here (four kinds of run, as BBC has):
 *   the bitmap is cut into bytes, byte k = bits 8k .. 8k+7 with bit 8k the
 *   most significant (bits past nbits are 0); a gap byte of value b is 0x00
 *   (b = 0) or 0xFF (b = 1), every other byte a map byte; a map byte is odd
 *   for b when it differs from the gap byte of value b in exactly one bit, at
 *   position P (0 = the most significant bit);
 *   a run is a fill of F >= 0 gap bytes of value b followed by a tail of
 *   T = 0 .. 15 map bytes (stored as they are) or by one odd byte (stored as
 *   P in the header); its header byte, most significant bit first:
 *     1 b F F T T T T    F <= 3, tail
 *     0 1 b F F P P P    F <= 3, odd byte
 *     0 0 1 b T T T T    F >= 4, tail       (F follows as a counter)
 *     0 0 0 1 b P P P    F >= 4, odd byte   (F follows as a counter)
 *   the counter is base 128, least significant group first, bit 7 set on
 *   every byte but the last; headers 0x00 .. 0x0F are not used;
 *   encoding: a unit is a maximal run of equal gap bytes and the maximal run
 *   of map bytes after it (a unit opening with map bytes, only at byte 0, has
 *   F = 0, b = 0); its first run carries the fill and up to 15 map bytes, the
 *   rest follow in runs with F = 0, 15 bytes each; a final one-byte tail that
 *   is odd for the run's b (for F = 0: b = 0, else b = 1) is an odd-byte run.
 * The exchange of the search keeps WAH; this code is offered beside it, to
 * compare the codes on the same frontiers (as the paper weighs WAH against
 * other codes).
 *   bits: device, ceil(nbits/32) uint32 words (bit b = bit b%32 of word b/32).
 *   nbits: 0 .. 2^31 - 1.
 *   bytes: device output, capacity_bytes >= n + n/15 + 11 for n = ceil(nbits/8).
 *   nbytes: device int64, receives the stream's length.
 * Allocates scratch (cudaMalloc) and synchronises `cuda_stream`.
 */
BFS_API bfs_status bfs_bbc_encode(const uint32_t *bits, int64_t nbits, uint8_t *bytes, int64_t capacity_bytes,
                                  int64_t *nbytes, void *cuda_stream);

/*
 * Decode a BBC stream (the inverse of bfs_bbc_encode; any well-formed stream,
 * canonical or not) into `bits` (device, ceil(nbits/32) words, written whole:
 * bits past nbits are 0).  Allocates scratch and synchronises `cuda_stream`.
 * Errors: BFS_ERR_CORRUPT for a malformed stream (an unused header, a counter
 * cut short or above 2^56, a record past the stream, bytes past nbits or too
 * few, padding bits set); BFS_ERR_INVALID_ARG for nbits outside the range or
 * bad pointers.
 */
BFS_API bfs_status bfs_bbc_decode(const uint8_t *bytes, int64_t nbytes, int64_t nbits, uint32_t *bits,
                                  void *cuda_stream);

/* ------------------------------------------------------------ diagnostics -- */

/* bfs_measure_scatter_reads -- the rate of scattered 4-byte reads of this GPU,
 * the bound of the expansion's visited test when it goes through L1/L2 (one
 * read at a random address per adjacency entry).  The paper has no counterpart:
 * it is a measurement the library offers so that a caller can set the
 * expansion's entry rate against the rate the memory system serves.
 *   region_bytes   size of the region read (>= 4096 and <= 1 GiB; the
 *                  expansion reads its visited bitmap slice: n/p/8 bytes)
 *   iterations     reads per thread (>= 1, rounded up to a multiple of 4; 4096
 *                  is enough for a stable rate)
 *   reads_per_s    out: reads per second (one 1024-thread CTA per SM, every
 *                  thread reading `iterations` words at pseudo-random addresses
 *                  -- four xorshift32 sequences, masked into a power-of-two
 *                  region -- with four reads in flight)
 *   cuda_stream    stream for the launches (NULL: legacy default stream)
 * The region is allocated and freed by the call.  Synchronises `cuda_stream`.
 * Errors: BFS_ERR_INVALID_ARG (NULL output, sizes outside the ranges),
 * BFS_ERR_OUT_OF_MEMORY, BFS_ERR_CUDA. */
BFS_API bfs_status bfs_measure_scatter_reads(int64_t region_bytes, int32_t iterations, double *reads_per_s,
                                             void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* BFS_GB300_H */
