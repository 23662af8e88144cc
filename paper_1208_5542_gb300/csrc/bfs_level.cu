// bfs_level.cu -- one level of the level-synchronous BFS (Alg. 1, 2, 3) on the
// virtual p x p block grid, and the bfs_run entry point.
//
// Per level k (f = frontier of level k, pi = visited, t = next frontier):
//   PLAIN (BIT, Alg. 1):   every block (i,j) reads the raw slice f_j and keeps
//                          the vertices whose column of A_{i,j} is nonempty
//                          (the directory test of its column index).
//   COMPRESS (WAH, Alg. 2): f_j is WAH-encoded once per source range j; every
//                          block-row i decodes stream j and tests its directory.
//   COMPRESS_SIEVE (DIR-WAH, Alg. 3): for every (j, i) the slice f_j is sieved
//                          by V_{i,j} and WAH-encoded; block (i,j) decodes its
//                          stream -- every decoded vertex has a nonempty
//                          column, so only its rank is looked up.
//   expansion:             for every decoded (u, block) item, every entry
//                          u -> v of its column: if v is not in pi, set t[v]
//                          and lower parent[v] to u (the (select, min) semiring).
//   reduce:                t = t & ~pi; pi |= t; level[v] = k + 1 for v in t;
//                          |t| counted on the device; f <- t.
// The exchange itself (Alg. 2, 3) is the identity on one GPU: the receive buffer
// g' is the send buffer in HBM; its sizes are scanned for the statistics and
// packed into the caller's trace when one is requested.
//
// The expansion is row-affine: a block (i,j) only ever writes destinations of
// range i, so a persistent CTA settles on one block-row at a time and keeps
// that row's visited bits pi_i and its own partial next bits t_i in shared
// memory (when a range fits); its warps take the row's units one at a time.
// Visited tests and next-bit updates are then on-chip; the partial t_i of
// every CTA is OR-folded into t when the CTA leaves the row (the fold of the
// 2D partition, done through L2).
//
// Bottom-up levels (the hybrid traversal the paper names in Sec. VIII and IX,
// when enabled): the exchange is the same, its streams are decoded into a
// bitmap, and every unvisited vertex v of range i scans its columns in blocks
// (j, i), j = 0 .. p-1, for a neighbour in the frontier delivered to block
// (i, j); the first range with one gives v the smallest of them as its
// parent.  The device picks each level's direction (level_next), and the
// kernels of the other direction return at once.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "wah.cuh"

namespace bfsgb {

int64_t parallel_encode_chunks(int64_t max_nbits, int wah_bits);
bfs_status launch_wah_encode_parallel(const EncodeArgs& a, int wah_bits, void* sums, void* bases, int64_t cps,
                                      void* flags, unsigned long long* setbits, int grid, cudaStream_t st);
size_t parallel_encode_sum_bytes();
size_t parallel_encode_base_bytes();

namespace {

constexpr int kNT = 256;            // threads of the small kernels
constexpr int kXT = 1024;           // threads of the expansion CTAs
constexpr int kXW = kXT / 32;       // warps of the expansion CTAs
constexpr uint32_t kCoop = 64;      // columns of at least this many entries take the whole warp
constexpr uint32_t kHub = 2048;     // columns longer than this are cut into pieces
constexpr uint32_t kPiece = 2048;   // entries per piece
#ifndef BFS_GUIDE
#define BFS_GUIDE 1
#endif
constexpr int64_t kGuide = BFS_GUIDE;  // a grab takes 1/(kGuide * warps) of the units left in the row
constexpr int64_t kSmemLimit = 227 * 1024;

// Per-level values that the device keeps from level to level, so that one
// level is the same launch sequence every time (and a CUDA graph can repeat it).
struct LevelCtl {
    int64_t frontier;      // vertices of the current frontier
    int64_t visited;       // vertices visited so far
    int32_t level;         // current level k
    int32_t plain_batch;   // PLAIN units per hand-out
    int32_t dedup;         // read the parent before updating it
    int32_t go;            // 1 while another level follows
    int64_t m_f;           // degree sum of the frontier
    int64_t m_u;           // degree sum of the unvisited vertices
    int32_t bu;            // 1: this level runs bottom-up
    int32_t policy;        // BFS_DIRECTION_*
    int32_t alpha, beta;   // thresholds of the hybrid
};

struct LevelArgs {
    // layout
    const uint32_t* dir;
    const uint32_t* rank;
    int64_t dir_stride;
    const uint32_t* cp;
    const int64_t* cp_base;
    const int64_t* ir_base;
    const int32_t* ir;
    int p;
    int64_t nb, n;
    // state
    const uint32_t* f;
    const uint32_t* pi;
    uint32_t* t;
    int32_t* parent;
    // exchange
    const void* xbuf;
    int64_t slot_cap;
    const int64_t* xcount;
    int64_t* chunk_base;
    int64_t chunks_per_slot;
    int64_t* slot_unit_base;            // p*p + 1: WAH units of slot s are [base[s], base[s+1])
    const uint8_t* fmt;                 // per-slot format of the level-adaptive exchange, or nullptr (WAH)
    // work distribution (per level)
    unsigned long long* row_next;       // p
    unsigned long long* row_piece_count;// p
    unsigned long long* row_piece_next; // p
    const int64_t* row_piece_base;      // p
    const int64_t* row_piece_cap;       // p
    Item* pieces;
    unsigned long long* ctr;
    int mode;
    int64_t plain_upb;                  // PLAIN units per block
    int64_t win_words;                  // words of the shared-memory row window (0: none)
    // compressed row exchange (the fold of the 2D partition): per block (i,j)
    // the destinations it reached, t_{i,j}, as a bitmap of range i; the
    // encoder turns t_{i,j} & ~pi_i into the row buffer of slot i*p + j
    int row_exchange;
    uint32_t* tblk;                     // p*p partial bitmaps, dir_stride words each
    const void* rowbuf;                 // row buffers: p*p slots of row_cap words
    int64_t row_cap;
    const int64_t* row_count;           // words in each row buffer
    const int64_t* row_first;           // per (slot, chunk): first word and its first group
    const int64_t* col_first;           // the same for the column slots (bottom-up levels)
    int64_t row_cps;                    // encoder chunks per slot
    int64_t row_bcps;                   // fold chunks per range
    int sweep;                          // all CTAs start at row 0 (rows in turn)
    const LevelCtl* ctl;                // this level's values
    // bottom-up levels
    uint32_t* gbits;                    // decoded streams (n bits, OR over the block-rows)
    int range_aligned;                  // 1: ranges start at word boundaries (n_b a multiple of 32)
    int64_t g_words;                    // its uint32 words (a multiple of 4)
    const int64_t* bu_ptr;              // bottom-up rows: offsets (n + 1)
    const int32_t* bu_adj;              // bottom-up rows: neighbour ids
};

__device__ __forceinline__ int64_t range_begin(const LevelArgs& a, int64_t b) {
    const int64_t x = b * a.nb;
    return x < a.n ? x : a.n;
}

// -------------------------------------------------------------- visiting --
// Visit entry u -> v: if v was not visited before this level, lower parent[v]
// to u and set v's next bit.  The parent update is a reduction whose result
// is not used (fire-and-forget at L2).  With a row window, the visited test
// and the next bit live in shared memory; without, the visited word is read
// through the read-only path (pi does not change during the expansion) and
// the next bit is a reduction at L2.
template <bool WIN, bool DEDUP, bool ROWX>
struct Visitor {
    const uint32_t* s_pi;
    uint32_t* s_t;
    int64_t rb;     // first vertex of the row
    uint32_t* tb;   // row exchange: the partial bitmap of the visiting block (i,j), or nullptr
    uint32_t jb;    // row exchange: first vertex of the block's source range j
    // The visited word of v (loads of several entries are issued before
    // their visits, so that their latencies overlap).
    __device__ __forceinline__ uint32_t probe(const LevelArgs& a, int32_t v) const {
        if (WIN) return s_pi[(uint32_t)(v - rb) >> 5];
        return __ldg(a.pi + ((uint32_t)v >> 5));
    }
    __device__ __forceinline__ bool fresh(int32_t v, uint32_t piw) const {
        const uint32_t b = WIN ? (uint32_t)(v - rb) : (uint32_t)v;
        return !(piw & (1u << (b & 31u)));
    }
    // The parent recorded so far for a fresh v (possibly an older value: the
    // parent only decreases during a level, from -1 = the largest unsigned).
    __device__ __forceinline__ uint32_t seen(const LevelArgs& a, int32_t v) const {
        return __ldcg(reinterpret_cast<const unsigned int*>(a.parent) + v);
    }
    // The word of v's bit in the visiting block's partial t_{i,j} (row exchange).
    __device__ __forceinline__ uint32_t seen_t(int32_t v) const {
        const uint32_t vl = (uint32_t)(v - rb);
        return __ldcg(tb + (vl >> 5));
    }
    // After the visited word piw of v was probed: v <- -1 if v was visited
    // before the level (nothing to do), else pv <- the parent read first
    // (DEDUP) or -1, and tw <- the partial's word read first (DEDUP with the
    // row exchange) or 0.
    __device__ __forceinline__ void stage(const LevelArgs& a, int32_t& v, uint32_t& piw, uint32_t& tw) const {
        tw = 0u;
        if (v < 0 || !fresh(v, piw)) {
            v = -1;
            return;
        }
        piw = DEDUP ? seen(a, v) : 0xffffffffu;
        if (DEDUP && ROWX) tw = seen_t(v);
    }
    // Visit of a fresh v from u, given an earlier read pv of its parent: when
    // pv <= u the visit changes nothing (pv != -1 means v already has a
    // visitor in this level, which set the next bit); otherwise lower the
    // parent, and the visitor that read -1 sets the next bit.  The visitor of
    // the first update read -1, so the bit is always set.
    __device__ __forceinline__ void mark(const LevelArgs& a, int32_t v, int32_t u, uint32_t pv, uint32_t tw) const {
        if (ROWX) {
            // Row exchange: every block that reaches v records it in its own
            // partial t_{i,j}.  The bit is already there when the word read
            // first has it, or when the parent read first lies in [jb, u]: a
            // visitor of the same source range lowered it and records v in
            // the same partial.  The parent is lowered when pv > u.
            const uint32_t vl = (uint32_t)(v - rb);
            const bool have = ((tw >> (vl & 31u)) & 1u) || (pv <= (uint32_t)u && pv >= jb);
            if (pv > (uint32_t)u) atomicMin(reinterpret_cast<unsigned int*>(a.parent) + v, (unsigned int)u);
            if (!have) atomicOr(tb + (vl >> 5), 1u << (vl & 31u));
            return;
        }
        if (pv <= (uint32_t)u) return;
        atomicMin(reinterpret_cast<unsigned int*>(a.parent) + v, (unsigned int)u);
        if (pv != 0xffffffffu) return;
        if (WIN) {
            const uint32_t vl = (uint32_t)(v - rb);
            atomicOr(s_t + (vl >> 5), 1u << (vl & 31u));
        } else {
            atomicOr(a.t + ((uint32_t)v >> 5), 1u << ((uint32_t)v & 31u));
        }
    }
};

// Entries per lane whose loads are in flight together.  The entries are read
// once per search: their loads are marked streaming (evict first), so that
// they do not push the visited, parent and next-bit lines out of L2 (-21% DRAM
// bytes at the growing level of a scale-24 search).
constexpr int kIlp = 4;
#ifndef BFS_PIECE_ILP
#define BFS_PIECE_ILP 8
#endif
constexpr int kPieceIlp = BFS_PIECE_ILP;   // the piece kernel: long columns only, more entries in flight

// All 32 lanes expand one column: ILP x 32 consecutive entries per step.
template <bool WIN, bool DEDUP, bool ROWX, int ILP = kIlp>
__device__ __forceinline__ void warp_column(const LevelArgs& a, const Visitor<WIN, DEDUP, ROWX>& vis, int32_t u, int64_t beg,
                                            uint32_t len) {
    const int32_t* col = a.ir + beg;
    for (uint32_t e = lane_id(); e < len; e += 32 * ILP) {
        int32_t v[ILP];
        uint32_t w[ILP], t[ILP];
#pragma unroll
        for (int k = 0; k < ILP; ++k) v[k] = (e + 32 * k < len) ? __ldcs(col + e + 32 * k) : -1;
#pragma unroll
        for (int k = 0; k < ILP; ++k) w[k] = (v[k] >= 0) ? vis.probe(a, v[k]) : 0u;
#pragma unroll
        for (int k = 0; k < ILP; ++k) vis.stage(a, v[k], w[k], t[k]);
#pragma unroll
        for (int k = 0; k < ILP; ++k)
            if (v[k] >= 0) vis.mark(a, v[k], u, w[k], t[k]);
    }
}

// Expand one item per lane (u, offset of its column in ir, length; length 0 =
// none).  Columns longer than kHub go to the row's piece list; columns of at
// least kCoop entries are expanded by the whole warp one after the other; the
// short ones share the warp through a load-balanced search over their entry
// counts, 32 consecutive entries of the concatenated columns per step.
template <bool WIN, bool DEDUP, bool ROWX>
__device__ __forceinline__ void warp_expand(const LevelArgs& a, const Visitor<WIN, DEDUP, ROWX>& vis, int row, int32_t u,
                                            int64_t beg, uint32_t len, unsigned long long& edges,
                                            unsigned long long& hits) {
    const uint32_t lane = lane_id();
    hits += (len > 0);
    edges += len;
    if (__any_sync(0xffffffffu, len > kHub)) {
        if (len > kHub) {
            const uint32_t np = (len + kPiece - 1) / kPiece;
            const unsigned long long base = atomicAdd(a.row_piece_count + row, (unsigned long long)np);
            if (base + np <= (unsigned long long)a.row_piece_cap[row]) {
                Item* dst = a.pieces + a.row_piece_base[row] + base;
                for (uint32_t k = 0; k < np; ++k) {
                    Item it;
                    it.u = u;
                    it.len = (len - k * kPiece < kPiece) ? len - k * kPiece : kPiece;
                    it.begin = beg + (int64_t)k * kPiece;
                    dst[k] = it;
                }
            } else {
                atomicOr(a.ctr + C_ERROR, 8ull);        // piece list overflow (cannot happen by the bound)
            }
            len = 0;
        }
    }
    uint32_t coop = __ballot_sync(0xffffffffu, len >= kCoop);
    while (coop) {
        const int src = __ffs(coop) - 1;
        coop &= coop - 1;
        warp_column<WIN, DEDUP, ROWX>(a, vis, __shfl_sync(0xffffffffu, u, src), __shfl_sync(0xffffffffu, beg, src),
                         __shfl_sync(0xffffffffu, len, src));
    }
    if (len >= kCoop) len = 0;
    const uint32_t incl = warp_incl_sum(len);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - len;
    for (uint32_t e0 = 0; e0 < total; e0 += 32 * kIlp) {
        int32_t v[kIlp], ou[kIlp];
        uint32_t w[kIlp], t[kIlp];
#pragma unroll
        for (int k = 0; k < kIlp; ++k) {
            const uint32_t e = e0 + 32 * k + lane;
            int lo = 0, hi = 31;                   // owner: first lane whose inclusive count exceeds e
#pragma unroll
            for (int step = 0; step < 5; ++step) {
                const int mid = (lo + hi) >> 1;
                const uint32_t im = __shfl_sync(0xffffffffu, incl, mid);
                if (im > e) hi = mid; else lo = mid + 1;
            }
            const int64_t ob = __shfl_sync(0xffffffffu, beg, lo);
            const uint32_t oe = __shfl_sync(0xffffffffu, excl, lo);
            ou[k] = __shfl_sync(0xffffffffu, u, lo);
            v[k] = (e < total) ? __ldcs(a.ir + ob + (int64_t)(e - oe)) : -1;
        }
#pragma unroll
        for (int k = 0; k < kIlp; ++k) w[k] = (v[k] >= 0) ? vis.probe(a, v[k]) : 0u;
#pragma unroll
        for (int k = 0; k < kIlp; ++k) vis.stage(a, v[k], w[k], t[k]);
#pragma unroll
        for (int k = 0; k < kIlp; ++k)
            if (v[k] >= 0) vis.mark(a, v[k], ou[k], w[k], t[k]);
    }
}

// Column of source u_local in block b: (offset into ir, length); 0 if empty.
struct BlockView {
    const uint32_t* dir;
    const uint32_t* rank;
    const uint32_t* cp;
    int64_t ir0;
};

__device__ __forceinline__ BlockView block_view(const LevelArgs& a, int64_t b) {
    BlockView bv;
    bv.dir = a.dir + b * a.dir_stride;
    bv.rank = a.rank + b * a.dir_stride;
    bv.cp = a.cp + __ldg(a.cp_base + b);
    bv.ir0 = __ldg(a.ir_base + b);
    return bv;
}

__device__ __forceinline__ void column_of(const LevelArgs& a, const BlockView& bv, int64_t ul, bool test_dir,
                                          int64_t* begin, uint32_t* len) {
    const uint32_t dw = __ldg(bv.dir + (ul >> 5));
    const uint32_t rk = __ldg(bv.rank + (ul >> 5));
    const uint32_t bit = 1u << (ul & 31);
    if (!(dw & bit)) {                  // empty column: nothing to expand
        *begin = 0;
        *len = 0;
        if (!test_dir) atomicOr(a.ctr + C_ERROR, 4ull);   // a sieved vertex must have a column
        return;
    }
    const uint32_t c = rk + __popc(dw & (bit - 1u));
    const uint32_t c0 = __ldg(bv.cp + c), c1 = __ldg(bv.cp + c + 1);
    *begin = bv.ir0 + c0;
    *len = c1 - c0;
}

// Bring the L2 lines of a short column's entries on chip ahead of their use
// (long columns are read by the whole warp, coalesced).
__device__ __forceinline__ void prefetch_column(const LevelArgs& a, int64_t begin, uint32_t len) {
    if (len == 0 || len >= kCoop) return;
    const int32_t* p0 = a.ir + begin;
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p0));
    const int32_t* p1 = p0 + (len - 1);
    if ((reinterpret_cast<uintptr_t>(p0) >> 7) != (reinterpret_cast<uintptr_t>(p1) >> 7))
        asm volatile("prefetch.global.L2 [%0];" ::"l"(p1));
}

__device__ __forceinline__ void flush_counts(const LevelArgs& a, unsigned long long edges, unsigned long long hits,
                                             unsigned long long items) {
    edges = warp_sum(edges);
    hits = warp_sum(hits);
    items = warp_sum(items);
    if (lane_id() == 0) {
        if (edges) atomicAdd(a.ctr + C_EDGES, edges);
        if (hits) atomicAdd(a.ctr + C_HITS, hits);
        if (items) atomicAdd(a.ctr + C_ITEMS, items);
    }
}

// Lane of the last of the 32 lanes whose exclusive count is <= q (the counts
// are nondecreasing over the lanes); every lane must call it.
__device__ __forceinline__ int owner_lane(uint32_t excl, uint64_t q) {
    int lo = 0, hi = 31;
#pragma unroll
    for (int step = 0; step < 5; ++step) {
        const int mid = (lo + hi + 1) >> 1;
        const uint32_t em = __shfl_sync(0xffffffffu, excl, mid);
        if ((uint64_t)em <= q) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------ row window --
// Leave the current row: fold the CTA's partial next bits into t (OR through
// L2).  With the row exchange the visits record their blocks' partials in HBM
// instead and the window holds no next bits.
__device__ void window_leave(const LevelArgs& a, uint32_t* s_t, int row) {
    if (a.row_exchange) return;
    const int64_t rb = range_begin(a, row);
    for (int64_t w = threadIdx.x; w < a.win_words; w += kXT) {
        const uint32_t x = s_t[w];
        if (!x) continue;
        const int64_t pos = rb + 32 * w;
        const int64_t gw = pos >> 5;
        const uint32_t sh = (uint32_t)(pos & 31);
        atomicOr(a.t + gw, x << sh);
        if (sh && (x >> (32 - sh))) atomicOr(a.t + gw + 1, x >> (32 - sh));
    }
}

// Enter a row: load pi_i into the window and clear the partial next bits.
__device__ void window_enter(const LevelArgs& a, uint32_t* s_pi, uint32_t* s_t, int row) {
    const int64_t rb = range_begin(a, row);
    for (int64_t w = threadIdx.x; w < a.win_words; w += kXT) {
        const int64_t pos = rb + 32 * w;
        s_pi[w] = (pos < a.n) ? bits32_at_cg(a.pi, (uint64_t)pos) : 0xffffffffu;
        s_t[w] = 0u;
    }
}

// Row-affine persistent loop.  The CTA settles on a block-row with units
// left; its warps take the row's units one at a time (warp-granular, no block
// barrier per unit; `batch` units per hand-out) until the row is drained, then
// the CTA folds its partial next bits into t, picks the next row with units
// left and loads that row's visited bits.  Every row is tried at most once
// per CTA.
template <bool WIN, typename Units, typename Work>
__device__ __forceinline__ void row_affine(const LevelArgs& a, unsigned long long* counters, int64_t batch,
                                           Units units_in_row, Work do_unit, uint32_t* s_pi, uint32_t* s_t,
                                           int* s_row) {
    const int p = a.p;
    int tried = 0;
    int start = a.sweep ? 0 : blockIdx.x % p;
    auto pick = [&](int from) -> int {          // thread 0: next row with units, or -1
        while (tried < p) {
            const int r = from;
            from = (from + 1 == p) ? 0 : from + 1;
            ++tried;
            if ((int64_t)*reinterpret_cast<volatile unsigned long long*>(counters + r) < units_in_row(r)) return r;
        }
        return -1;
    };
    if (threadIdx.x == 0) s_row[0] = pick(start);
    __syncthreads();
    int row = s_row[0];
    if (WIN && row >= 0) window_enter(a, s_pi, s_t, row);
    __syncthreads();
    while (row >= 0) {
        const int64_t nu = units_in_row(row);
        for (;;) {
            // guided hand-out: a share of what is left (at least `batch`), so
            // that early grabs are large and the last ones small
            int64_t x = 0, b = batch;
            if (lane_id() == 0) {
                const int64_t cur = (int64_t)*reinterpret_cast<volatile unsigned long long*>(counters + row);
                if (cur < nu) {
                    const int64_t g = (uint32_t)(nu - cur) / (uint32_t)(kGuide * gridDim.x * kXW);   // units of a row < 2^31
                    b = g > batch ? g : batch;
                    x = (int64_t)atomicAdd(counters + row, (unsigned long long)b);
                } else {
                    x = nu;
                }
            }
            x = __shfl_sync(0xffffffffu, x, 0);
            b = __shfl_sync(0xffffffffu, b, 0);
            if (x >= nu) break;
            const int64_t xe = (x + b < nu) ? x + b : nu;
            for (; x < xe; ++x) do_unit(row, x);
        }
        __syncthreads();
        if (WIN) window_leave(a, s_t, row);
        if (threadIdx.x == 0) s_row[0] = pick(row + 1 == p ? 0 : row + 1);
        __syncthreads();
        row = s_row[0];
        if (WIN && row >= 0) window_enter(a, s_pi, s_t, row);
        __syncthreads();
    }
}

// ---------------------------------------------------------------- kernels --
// Expansion of the WAH units (COMPRESS, COMPRESS_SIEVE).  Unit = 32 words of
// one stream, decoded by one warp: a warp scan of run lengths from the
// chunk's group base places every word, a scan of item counts numbers the
// decoded vertices, and the warp expands them 32 at a time.
template <typename W, bool WIN, bool DEDUP, bool ROWX>
__global__ void __launch_bounds__(kXT, 1) expand_wah(LevelArgs a) {
    if (a.ctl->dedup != (DEDUP ? 1 : 0) || a.ctl->bu) return;   // another variant expands this level
    using T = Wah<W>;
    constexpr int GB = T::GB;
    extern __shared__ uint32_t s_win[];                   // s_pi | s_t (WIN only)
    __shared__ int s_row[2];
    uint32_t* s_pi = s_win;
    uint32_t* s_t = s_win + a.win_words;
    const int p = a.p;
    unsigned long long edges = 0, hits = 0, nitems = 0;
    auto units_in_row = [&](int r) -> int64_t {
        return a.slot_unit_base[(int64_t)(r + 1) * p] - a.slot_unit_base[(int64_t)r * p];
    };
    // the slot of the previous unit: a grab hands out consecutive units, so the
    // next one is mostly in the same slot or a few slots on
    int last_slot = -1;
    auto do_unit = [&](int row, int64_t x) {
        // unit -> (slot, chunk): the slot s of the row with base[s] <= g < base[s+1]
        const int r0 = row * p;
        const int64_t g = a.slot_unit_base[r0] + x;
        int sl;
        if (last_slot >= r0 && last_slot < r0 + p && a.slot_unit_base[last_slot] <= g) {
            sl = last_slot;
            while (sl + 1 < r0 + p && a.slot_unit_base[sl + 1] <= g) ++sl;
        } else {
            int lo = r0, hi = r0 + p - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.slot_unit_base[mid] <= g) lo = mid; else hi = mid - 1;
            }
            sl = lo;
        }
        last_slot = sl;
        const int64_t s = sl, k = g - a.slot_unit_base[sl];
        const int64_t j = sl - r0;
        const int64_t stream = (a.mode == BFS_MODE_COMPRESS_SIEVE) ? s : j;
        const int64_t jb = range_begin(a, j), jl = range_begin(a, j + 1) - jb;
        const int64_t G = (uint32_t)jl / (uint32_t)GB;                 // a range is below 2^31 vertices
        const int r = (int)((uint32_t)jl - (uint32_t)G * (uint32_t)GB);
        const W* in = static_cast<const W*>(a.xbuf) + stream * a.slot_cap;
        const int64_t count = a.xcount[stream];
        const int64_t xw = k * 32 + lane_id();
        const W y = (xw < count) ? in[xw] : W(0);
        // per lane: its element's vertices as (first vertex, bits in group
        // order; a 1-fill is a run, marked by an empty bit pattern)
        uint32_t c = 0;
        W wbits = W(0);
        int64_t wbase = 0;
        const int fm = a.fmt ? (int)a.fmt[stream] : FMT_WAH;
        if (fm == FMT_WAH) {
            // groups of a slot fit in 32 bits (n < 2^31)
            const uint32_t glen = (xw < count) ? (uint32_t)word_groups<W>(y) : 0u;
            const uint32_t gincl = warp_incl_sum(glen);
            const int64_t gs = a.chunk_base[stream * a.chunks_per_slot + k] + (int64_t)(gincl - glen);
            if (xw < count) {
                if (gs < G) {
                    wbase = gs * GB;
                    if (is_fill<W>(y)) c = (y & T::VAL) ? (uint32_t)(glen * GB) : 0u;
                    else { wbits = T::from_payload(y); c = (uint32_t)T::popc(wbits); }
                } else if (r > 0) {
                    wbase = G * GB;
                    wbits = T::from_active(y, r);                     // the active word
                    c = (uint32_t)T::popc(wbits);
                }
            }
        } else if (xw < count) {
            const uint32_t e = (uint32_t)y;
            if (fm == FMT_LIST) {                                     // one vertex offset
                wbase = e;
                c = 1;
            } else {                                                  // 32 bits of the raw slice
                wbase = xw * 32;
                wbits = (W)e;
                c = (uint32_t)__popc(e);
            }
        }
        const uint32_t cincl = warp_incl_sum(c);
        const uint32_t cexcl = cincl - c;
        const uint32_t items = __shfl_sync(0xffffffffu, cincl, 31);
        nitems += c;
        const BlockView bv = block_view(a, s);
        const Visitor<WIN, DEDUP, ROWX> vis{s_pi, s_t, range_begin(a, row), ROWX ? a.tblk + s * a.dir_stride : nullptr,
                                            (uint32_t)jb};
        // items q0 .. q0+31, one per lane: decode, look up the column and
        // prefetch its entries; the next batch's lookups and prefetches are
        // issued before this batch is expanded
        auto item = [&](uint32_t q0, int32_t& u, int64_t& begin, uint32_t& len) {
            const uint32_t q = q0 + lane_id();
            const int o = owner_lane(cexcl, q < items ? q : items - 1);
            const W ob = __shfl_sync(0xffffffffu, wbits, o);
            const int64_t obase = __shfl_sync(0xffffffffu, wbase, o);
            const uint32_t oex = __shfl_sync(0xffffffffu, cexcl, o);
            u = 0;
            begin = 0;
            len = 0;
            if (q < items) {
                const int kk = (int)(q - oex);
                const int64_t ul = obase + (ob ? T::select(ob, kk) : kk);   // empty pattern: a 1-fill
                column_of(a, bv, ul, a.mode != BFS_MODE_COMPRESS_SIEVE, &begin, &len);
                u = (int32_t)(jb + ul);
                prefetch_column(a, begin, len);
            }
        };
        int32_t u;
        int64_t begin;
        uint32_t len;
        item(0, u, begin, len);
        for (uint32_t q0 = 0; q0 < items; q0 += 32) {
            int32_t un = 0;
            int64_t bn = 0;
            uint32_t ln = 0;
            if (q0 + 32 < items) item(q0 + 32, un, bn, ln);
            warp_expand<WIN, DEDUP, ROWX>(a, vis, row, u, begin, len, edges, hits);
            u = un;
            begin = bn;
            len = ln;
        }
    };
    row_affine<WIN>(a, a.row_next, 2, units_in_row, do_unit, s_pi, s_t, s_row);
    flush_counts(a, edges, hits, nitems);
}

// Expansion of the PLAIN units.  Unit = (block (row, j), 32 raw frontier words
// of range j), one warp: lane l keeps word l's bits whose column is nonempty
// (word-wise AND with V_{i,j}, the block's column index) and the warp expands
// them 32 at a time.
template <bool WIN, bool DEDUP>
__global__ void __launch_bounds__(kXT, 1) expand_plain(LevelArgs a) {
    if (a.ctl->dedup != (DEDUP ? 1 : 0) || a.ctl->bu) return;   // another variant expands this level
    extern __shared__ uint32_t s_win[];
    __shared__ int s_row[2];
    uint32_t* s_pi = s_win;
    uint32_t* s_t = s_win + a.win_words;
    const int p = a.p;
    unsigned long long edges = 0, hits = 0, nitems = 0;
    const int64_t per_row = (int64_t)p * a.plain_upb;
    auto units_in_row = [&](int) -> int64_t { return per_row; };
    auto do_unit = [&](int row, int64_t x) {
        const uint32_t xu = (uint32_t)x, upb = (uint32_t)a.plain_upb;   // p * upb units per row fit in 32 bits
        const int64_t j = xu / upb, c = xu - (uint32_t)j * upb;
        const int64_t b = (int64_t)row * p + j;
        const int64_t jb = range_begin(a, j), jl = range_begin(a, j + 1) - jb;
        const int64_t w = c * 32 + lane_id();
        uint32_t bits = 0;
        if (w * 32 < jl) {
            bits = bits32_at_cg(a.f, (uint64_t)(jb + w * 32));
            const int64_t left = jl - w * 32;
            if (left < 32) bits &= (1u << left) - 1u;
            if (bits) bits &= __ldg(a.dir + b * a.dir_stride + w);
        }
        const uint32_t cnt = __popc(bits);
        const uint32_t cincl = warp_incl_sum(cnt);
        const uint32_t cexcl = cincl - cnt;
        const uint32_t items = __shfl_sync(0xffffffffu, cincl, 31);
        if (items == 0) return;
        nitems += cnt;
        const BlockView bv = block_view(a, b);
        const Visitor<WIN, DEDUP, false> vis{s_pi, s_t, range_begin(a, row), nullptr, (uint32_t)jb};
        auto item = [&](uint32_t q0, int32_t& u, int64_t& begin, uint32_t& len) {
            const uint32_t q = q0 + lane_id();
            const int o = owner_lane(cexcl, q < items ? q : items - 1);
            const uint32_t ob = __shfl_sync(0xffffffffu, bits, o);
            const uint32_t oex = __shfl_sync(0xffffffffu, cexcl, o);
            u = 0;
            begin = 0;
            len = 0;
            if (q < items) {
                const int64_t ul = (c * 32 + o) * 32 + select32(ob, (int)(q - oex));
                column_of(a, bv, ul, false, &begin, &len);
                u = (int32_t)(jb + ul);
                prefetch_column(a, begin, len);
            }
        };
        int32_t u;
        int64_t begin;
        uint32_t len;
        item(0, u, begin, len);
        for (uint32_t q0 = 0; q0 < items; q0 += 32) {
            int32_t un = 0;
            int64_t bn = 0;
            uint32_t ln = 0;
            if (q0 + 32 < items) item(q0 + 32, un, bn, ln);
            warp_expand<WIN, DEDUP, false>(a, vis, row, u, begin, len, edges, hits);
            u = un;
            begin = bn;
            len = ln;
        }
    };
    row_affine<WIN>(a, a.row_next, a.ctl->plain_batch, units_in_row, do_unit, s_pi, s_t, s_row);
    flush_counts(a, edges, hits, nitems);
}

// Pieces of long columns, row by row: one warp per piece.
template <bool WIN, bool DEDUP, bool ROWX>
__global__ void __launch_bounds__(kXT, 1) expand_pieces(LevelArgs a) {
    if (a.ctl->dedup != (DEDUP ? 1 : 0) || a.ctl->bu) return;   // another variant expands this level
    extern __shared__ uint32_t s_win[];
    __shared__ int s_row[2];
    uint32_t* s_pi = s_win;
    uint32_t* s_t = s_win + a.win_words;
    auto units_in_row = [&](int r) -> int64_t {
        return (int64_t)min(a.row_piece_count[r], (unsigned long long)a.row_piece_cap[r]);
    };
    auto do_unit = [&](int row, int64_t x) {
        const Item it = a.pieces[a.row_piece_base[row] + x];
        const uint32_t j = (uint32_t)it.u / (uint32_t)a.nb;               // the piece's source range
        const Visitor<WIN, DEDUP, ROWX> vis{s_pi, s_t, range_begin(a, row),
                                            ROWX ? a.tblk + ((int64_t)row * a.p + j) * a.dir_stride : nullptr,
                                            (uint32_t)range_begin(a, j)};
        warp_column<WIN, DEDUP, ROWX, kPieceIlp>(a, vis, it.u, it.begin, it.len);
    };
    row_affine<WIN>(a, a.row_piece_next, 1, units_in_row, do_unit, s_pi, s_t, s_row);
}

// ------------------------------------------------------------------ fold --
// OR the bits of v (bit q at image bit pos + q; at most 63 bits) into a
// shared-memory image of bitmap words.
template <typename W>
__device__ __forceinline__ void img_or(uint32_t* img, uint32_t pos, W v) {
    if (!v) return;
    const uint32_t w = pos >> 5, sh = pos & 31u;
    if constexpr (sizeof(W) == 4) {
        atomicOr(img + w, v << sh);
        if (sh && (v >> (32 - sh))) atomicOr(img + w + 1, v >> (32 - sh));
    } else {
        const unsigned long long x = v;
        const uint32_t w0 = (uint32_t)(x << sh);
        const uint32_t w1 = sh ? (uint32_t)(x >> (32 - sh)) : (uint32_t)(x >> 32);
        const uint32_t w2 = sh ? (uint32_t)(x >> (64 - sh)) : 0u;
        if (w0) atomicOr(img + w, w0);
        if (w1) atomicOr(img + w + 1, w1);
        if (w2) atomicOr(img + w + 2, w2);
    }
}

// Set the image bits [b0, b1), by the whole warp.
__device__ __forceinline__ void img_fill(uint32_t* img, uint32_t b0, uint32_t b1) {
    if (b1 <= b0) return;
    const uint32_t w0 = b0 >> 5, w1 = (b1 - 1) >> 5;
    for (uint32_t w = w0 + lane_id(); w <= w1; w += 32) {
        uint32_t mask = 0xffffffffu;
        if (w == w0) mask &= 0xffffffffu << (b0 & 31u);
        if (w == w1) mask &= 0xffffffffu >> (31u - ((b1 - 1) & 31u));
        atomicOr(img + w, mask);
    }
}

constexpr int kFT = 512;            // threads of the fold CTAs
constexpr int kFoldIlp = 4;         // word tiles whose loads a fold warp issues together

// Chunk-wise OR-decode of exchanged slots.  One CTA per (range b, chunk c of
// kEncChunkGroups groups of the range): its warps take the p slots that carry
// range b in turn, start at the word the encoder recorded for the chunk and
// decode the words covering the chunk's groups (and the active word, in the
// chunk that holds the range's last bits) into a shared-memory image of the
// destination's words; the image is then stored, the words shared with a
// neighbouring chunk or range ORed.  The destination is clear before.
//   ROWS = true: the fold of the compressed row exchange on a top-down level --
//     t_i is the OR over j of the row buffers (i, j), each the WAH stream of
//     t_{i,j} & ~pi_i; nothing else writes t on such a level.
//   ROWS = false: the column slots of a bottom-up level decoded into the one
//     bitmap the bottom-up scan reads -- the OR over the block-rows i of slots
//     (i, j) (COMPRESS_SIEVE) or slot j (COMPRESS); a raw slot of the adaptive
//     format is ORed word by word, vector slots are left to decode_streams.
// Malformed streams set C_ERROR (16).
template <typename W, bool ROWS>
__global__ void __launch_bounds__(kFT) fold_slots(LevelArgs a) {
    if (ROWS ? a.ctl->bu : !a.ctl->bu) return;
    using T = Wah<W>;
    constexpr int GB = T::GB;
    constexpr int64_t CG = kEncChunkGroups;
    constexpr int64_t CBITS = CG * GB;
    constexpr int IW = (int)(CBITS / 32) + 2;
    constexpr int NW = kFT / 32;
    __shared__ uint32_t img[IW];
    __shared__ int s_err;
    const int p = a.p;
    const int lane = (int)lane_id(), warp = (int)(threadIdx.x >> 5);
    const int64_t items = (int64_t)p * a.row_bcps;
    const bool sieve = a.mode == BFS_MODE_COMPRESS_SIEVE;
    const int nsrc = (ROWS || sieve) ? p : 1;                      // slots carrying one range
    const void* buf = ROWS ? a.rowbuf : a.xbuf;
    const int64_t cap = ROWS ? a.row_cap : a.slot_cap;
    const int64_t* counts = ROWS ? a.row_count : a.xcount;
    const int64_t* first = ROWS ? a.row_first : a.col_first;
    uint32_t* dst = ROWS ? a.t : a.gbits;
    for (int64_t q = blockIdx.x; q < items; q += gridDim.x) {
        const int b = (int)(q / a.row_bcps);
        const int64_t c = q - (int64_t)b * a.row_bcps;
        const int64_t ib = range_begin(a, b), nbits = range_begin(a, b + 1) - ib;
        const int64_t b0 = c * CBITS;
        if (b0 >= nbits) continue;
        const int64_t b1 = (b0 + CBITS < nbits) ? b0 + CBITS : nbits;
        const int64_t G = nbits / GB;
        const int r = (int)(nbits - G * GB);
        const int64_t nch = (G + CG - 1) / CG;
        const int64_t g_lo = c * CG, g_hi = (g_lo + CG < G) ? g_lo + CG : G;
        const uint32_t al = (uint32_t)((ib + b0) & 31);
        const int nimg = (int)((al + (b1 - b0) + 31) >> 5);
        for (int k = threadIdx.x; k < nimg; k += kFT) img[k] = 0u;
        if (threadIdx.x == 0) s_err = 0;
        __syncthreads();
        for (int x_src = warp; x_src < nsrc; x_src += NW) {
            const int64_t s = ROWS ? (int64_t)b * p + x_src : (sieve ? (int64_t)x_src * p + b : (int64_t)b);
            const int64_t count = counts[s];
            if (!ROWS && a.fmt) {
                const int fm = (int)a.fmt[s];
                if (fm == FMT_LIST) continue;                   // decode_streams ORs the offsets
                if (fm == FMT_RAW) {                            // the slice's raw words of this chunk
                    const uint32_t* in = static_cast<const uint32_t*>(a.xbuf) + s * a.slot_cap;
                    const int64_t w0 = b0 >> 5, w1 = (b1 + 31) >> 5;
                    for (int64_t w = w0 + lane; w < w1 && w < count; w += 32) {
                        const uint32_t x = in[w];
                        if (x) img_or<uint32_t>(img, al + (uint32_t)(32 * w - b0), x);
                    }
                    continue;
                }
            }
            const W* in = static_cast<const W*>(buf) + s * cap;
            if (c < nch) {
                int64_t x0 = first[2 * (s * a.row_cps + c)];
                int64_t gpos = first[2 * (s * a.row_cps + c) + 1];
                // a run length is at most the slot's G groups: clamped to G + 1,
                // 32 of them sum within 32 bits (a longer fill is malformed and
                // still clipped to the chunk)
                const uint32_t lcap = (uint32_t)(G + 1);
                while (gpos < g_hi) {
                    if (x0 >= count) {                         // the words end before the groups do
                        if (lane == 0) s_err = 1;
                        break;
                    }
                    W y[kFoldIlp];                              // kFoldIlp tiles of 32 words in flight
#pragma unroll
                    for (int k = 0; k < kFoldIlp; ++k) {
                        const int64_t x = x0 + 32 * k + lane;
                        y[k] = (x < count) ? in[x] : W(0);
                    }
#pragma unroll
                    for (int k = 0; k < kFoldIlp; ++k) {
                        if (gpos >= g_hi || x0 >= count) break;   // warp-uniform
                        const int64_t x = x0 + lane;
                        const bool valid = x < count;
                        const bool fill = valid && is_fill<W>(y[k]);
                        uint32_t len = valid ? 1u : 0u, incl;
                        if (__any_sync(0xffffffffu, fill)) {
                            if (fill) {
                                const uint64_t l = word_groups<W>(y[k]);
                                len = l < lcap ? (uint32_t)l : lcap;
                            }
                            incl = warp_incl_sum(len);
                        } else {
                            // literals only: one group each; the lanes past the words are a suffix
                            const uint32_t nvalid = (count - x0 < 32) ? (uint32_t)(count - x0) : 32u;
                            incl = valid ? (uint32_t)lane + 1u : nvalid;
                        }
                        const int64_t gs = gpos + (int64_t)(incl - len);
                        bool one = false;
                        if (valid && gs < g_hi && gs + (int64_t)len > g_lo) {
                            if (!fill) img_or<W>(img, al + (uint32_t)((gs - g_lo) * GB), T::from_payload(y[k]));
                            else one = (y[k] & T::VAL) != W(0);
                        }
                        uint32_t m = __ballot_sync(0xffffffffu, one);
                        while (m) {                             // 1-fills, by the whole warp
                            const int o = __ffs(m) - 1;
                            m &= m - 1;
                            int64_t f0 = __shfl_sync(0xffffffffu, gs, o);
                            int64_t f1 = f0 + (int64_t)__shfl_sync(0xffffffffu, len, o);
                            if (f0 < g_lo) f0 = g_lo;
                            if (f1 > g_hi) f1 = g_hi;
                            img_fill(img, al + (uint32_t)((f0 - g_lo) * GB), al + (uint32_t)((f1 - g_lo) * GB));
                        }
                        x0 += 32;
                        gpos += (int64_t)__shfl_sync(0xffffffffu, incl, 31);
                    }
                }
            }
            // the active word holds the range's last r bits
            if (r > 0 && lane == 0 && G * GB >= b0 && G * GB < b1) {
                const W y = (count > 0) ? in[count - 1] : W(0);
                if (count <= 0 || (y >> r) != W(0)) s_err = 1;
                else img_or<W>(img, al + (uint32_t)(G * GB - b0), T::from_active(y, r));
            }
        }
        __syncthreads();
        const int64_t gw0 = (ib + b0) >> 5;
        // a word inside the chunk (or the bitmap's last, partial word) is this
        // CTA's alone: stored; a word shared with a neighbouring range is ORed.
        // With word-aligned ranges every word of the decoded bitmap is some
        // chunk's alone and is stored even when zero (no clearing pass)
        const bool store_zero = !ROWS && a.range_aligned;
        for (int k = threadIdx.x; k < nimg; k += kFT) {
            const uint32_t x = img[k];
            const int64_t wlo = (gw0 + k) * 32;
            const bool own = wlo >= ib + b0 && (wlo + 32 <= ib + b1 || ib + b1 >= a.n);
            if (own) {
                if (x || store_zero) dst[gw0 + k] = x;
            } else if (x) {
                atomicOr(dst + gw0 + k, x);
            }
        }
        if (threadIdx.x == 0 && s_err) atomicOr(a.ctr + C_ERROR, 16ull);
        __syncthreads();
    }
}

// ----------------------------------------------------- dynamic directory --
// The dynamic cross directory (Sec. V-B): D_{i,j}(u) = 1 while column u of
// block (i,j) still holds an entry into a vertex that is not visited; the
// sieve of exchange k sends f_j (.) D_{i,j}.  A bit matters only at the
// exchange that sends u (u is in one frontier only), and a cleared bit stays
// clear (the visited set only grows), so the bits of the frontier's vertices
// are evaluated from their definition just before the exchange: D starts as a
// copy of V each search, and every (u, i) with f_j(u) = D_{i,j}(u) = 1 whose
// column reaches only visited vertices is cleared.  pi holds the vertices
// visited up to this level, which is the state the synchronous update of
// every earlier visit leaves (the entries into the visited vertices have all
// been counted).  PLAIN-style units: (block (i,j), 32 words of range j), one
// warp; each item (u, i) is decided by its lane (the column's first kDynLane
// entries) and, for the rest of a long column, by the whole warp, stopping at
// the first unvisited destination.
constexpr uint32_t kDynStep = 8;      // entries a lane tests together
constexpr uint32_t kDynLane = 64;     // entries a lane tests before the warp takes over

__global__ void __launch_bounds__(kNT) dyn_sieve(LevelArgs a, uint32_t* __restrict__ ddir,
                                                 const uint8_t* __restrict__ fsum) {
    const int p = a.p;
    const int64_t units = (int64_t)p * p * a.plain_upb;
    const int64_t gw0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t gstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = (int)lane_id();
    for (int64_t x = gw0; x < units; x += gstride) {
        const int64_t b = x / a.plain_upb, c = x - b * a.plain_upb;
        const int j = (int)(b % p);
        const int64_t jb = range_begin(a, j), jl = range_begin(a, j + 1) - jb;
        if (c * 1024 >= jl) continue;
        const int64_t g0 = jb + c * 1024;               // the unit's first global bit
        if (!fsum[g0 >> 10] && !fsum[(g0 + 1023) >> 10]) continue;   // no frontier bit (warp-uniform)
        const int64_t w = c * 32 + lane;
        uint32_t bits = 0;
        if (w * 32 < jl) {
            bits = bits32_at_cg(a.f, (uint64_t)(jb + w * 32));
            const int64_t left = jl - w * 32;
            if (left < 32) bits &= (1u << left) - 1u;
            if (bits) bits &= ddir[b * a.dir_stride + w];
        }
        const uint32_t cnt = __popc(bits);
        const uint32_t cincl = warp_incl_sum(cnt);
        const uint32_t cexcl = cincl - cnt;
        const uint32_t items = __shfl_sync(0xffffffffu, cincl, 31);
        if (items == 0) continue;
        const BlockView bv = block_view(a, b);
        // the column of item q0 + lane (none past the items); the next round's
        // lookups are issued before this round's scan, so that they overlap
        auto lookup = [&](uint32_t q0, int64_t& ul, int64_t& begin, uint32_t& len) {
            const uint32_t q = q0 + lane;
            const int o = owner_lane(cexcl, q < items ? q : items - 1);
            const uint32_t ob = __shfl_sync(0xffffffffu, bits, o);
            const uint32_t oex = __shfl_sync(0xffffffffu, cexcl, o);
            ul = -1;
            begin = 0;
            len = 0;
            if (q < items) {
                ul = (c * 32 + o) * 32 + select32(ob, (int)(q - oex));
                column_of(a, bv, ul, false, &begin, &len);
                prefetch_column(a, begin, len);
            }
        };
        int64_t ul, begin;
        uint32_t len;
        lookup(0, ul, begin, len);
        for (uint32_t q0 = 0; q0 < items; q0 += 32) {
            int64_t ul_n = -1, begin_n = 0;
            uint32_t len_n = 0;
            if (q0 + 32 < items) lookup(q0 + 32, ul_n, begin_n, len_n);
            uint32_t e = 0;
            bool alive = ul < 0;
            // the lane scans its column kDynStep entries at a time (their loads
            // in flight together) up to kDynLane entries
            while (!alive && e < len && e < kDynLane) {
                int32_t v[kDynStep];
#pragma unroll
                for (uint32_t k = 0; k < kDynStep; ++k) v[k] = (e + k < len) ? __ldg(a.ir + begin + e + k) : -1;
#pragma unroll
                for (uint32_t k = 0; k < kDynStep; ++k)
                    if (v[k] >= 0 && !((__ldg(a.pi + ((uint32_t)v[k] >> 5)) >> ((uint32_t)v[k] & 31u)) & 1u))
                        alive = true;
                e += kDynStep;
            }
            // the rest of the long columns whose first kDynLane entries are all
            // visited: the whole warp, 32 entries a step, until an unvisited one
            uint32_t m = __ballot_sync(0xffffffffu, !alive && e < len);
            while (m) {
                const int l = __ffs(m) - 1;
                m &= m - 1;
                const int64_t lb = __shfl_sync(0xffffffffu, begin, l);
                const uint32_t ll = __shfl_sync(0xffffffffu, len, l);
                bool found = false;
                for (uint32_t e0 = kDynLane; e0 < ll && !found; e0 += 32) {
                    bool un = false;
                    if (e0 + lane < ll) {
                        const uint32_t v = (uint32_t)__ldg(a.ir + lb + e0 + lane);
                        un = !((__ldg(a.pi + (v >> 5)) >> (v & 31u)) & 1u);
                    }
                    found = __any_sync(0xffffffffu, un);
                }
                if (lane == l) alive = found;
            }
            if (!alive)
                atomicAnd(ddir + b * a.dir_stride + (ul >> 5), ~(1u << ((uint32_t)ul & 31u)));
            ul = ul_n;
            begin = begin_n;
            len = len_n;
        }
    }
}

// ------------------------------------------------------------- bottom-up --
// OR the group bits `bits` (bit q = bitmap bit bit0 + q) into a bitmap.
template <typename W>
__device__ __forceinline__ void or_bits(uint32_t* dst, int64_t bit0, W bits) {
    if (!bits) return;
    const int64_t w = bit0 >> 5;
    const uint32_t sh = (uint32_t)(bit0 & 31);
    if constexpr (sizeof(W) == 4) {
        atomicOr(dst + w, bits << sh);
        if (sh) {
            const uint32_t hi = bits >> (32 - sh);
            if (hi) atomicOr(dst + w + 1, hi);
        }
    } else {
        const unsigned long long x = bits;
        const uint32_t w0 = (uint32_t)(x << sh);
        const uint32_t w1 = sh ? (uint32_t)(x >> (32 - sh)) : (uint32_t)(x >> 32);
        const uint32_t w2 = sh ? (uint32_t)(x >> (64 - sh)) : 0u;
        if (w0) atomicOr(dst + w, w0);
        if (w1) atomicOr(dst + w + 1, w1);
        if (w2) atomicOr(dst + w + 2, w2);
    }
}

// Zero the decoded bitmap (bottom-up levels only).
__global__ void __launch_bounds__(kNT) clear_gbits(LevelArgs a) {
    if (!a.ctl->bu) return;
    const int64_t quads = a.g_words / 4;
    uint4* q = reinterpret_cast<uint4*>(a.gbits);
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < quads; x += (int64_t)gridDim.x * blockDim.x)
        q[x] = make_uint4(0u, 0u, 0u, 0u);
}

// The exchanged streams decoded into one n-bit bitmap (bottom-up levels only):
// bit q of the stream of slot (i, j) lands on vertex begin(j) + q, ORed over
// the block-rows i.  A block (i, j) only ever tests vertices u of range j with
// a neighbour in range i, whose bit its own stream carries (V_{i,j}(u) = 1):
// the OR holds exactly that bit, and one bitmap serves every block-row.  One
// warp per 32-word unit of the decoder's plan (COMPRESS: the plan of row 0,
// whose blocks hold the p streams once), each word placed by a scan of run
// lengths from its chunk's group base; literal groups and the active word are
// ORed in, 1-fill runs set by the whole warp, 0-fills left as cleared.
template <typename W>
__global__ void __launch_bounds__(kNT) decode_streams(LevelArgs a) {
    if (!a.ctl->bu) return;
    using T = Wah<W>;
    constexpr int GB = T::GB;
    const int p = a.p;
    const bool sieve = a.mode == BFS_MODE_COMPRESS_SIEVE;
    const int nblk = sieve ? p * p : p;
    const int64_t total = a.slot_unit_base[nblk];
    // every warp takes a contiguous share of the units: the slot of the next
    // unit is the current one or a few on (one search per warp)
    const int64_t gw = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t u0 = total * gw / nw, u1 = total * (gw + 1) / nw;
    int sl = -1;
    for (int64_t g = u0; g < u1; ++g) {
        if (sl < 0) {
            int lo = 0, hi = nblk - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (a.slot_unit_base[mid] <= g) lo = mid; else hi = mid - 1;
            }
            sl = lo;
        } else {
            while (sl + 1 < nblk && a.slot_unit_base[sl + 1] <= g) ++sl;
        }
        const int64_t s = sl, k = g - a.slot_unit_base[sl];
        const int64_t j = sieve ? s % p : s;
        const int64_t jb = range_begin(a, j), jl = range_begin(a, j + 1) - jb;
        const int64_t G = (uint32_t)jl / (uint32_t)GB;
        const int r = (int)((uint32_t)jl - (uint32_t)G * (uint32_t)GB);
        const W* in = static_cast<const W*>(a.xbuf) + s * a.slot_cap;
        const int64_t count = a.xcount[s];
        const int64_t xw = k * 32 + lane_id();
        const W y = (xw < count) ? in[xw] : W(0);
        uint32_t* dst = a.gbits;
        const int fm = a.fmt ? (int)a.fmt[s] : FMT_WAH;
        if (fm != FMT_LIST) continue;            // fold_slots decodes the WAH and raw slots
        if (xw < count) or_bits<uint32_t>(dst, jb + (int64_t)(uint32_t)y, 1u);   // a vertex offset
        continue;
        const uint32_t glen = (xw < count) ? (uint32_t)word_groups<W>(y) : 0u;
        const uint32_t gincl = warp_incl_sum(glen);
        const int64_t gs = a.chunk_base[s * a.chunks_per_slot + k] + (int64_t)(gincl - glen);
        bool one = false;
        if (xw < count) {
            if (gs < G) {
                if (!is_fill<W>(y)) or_bits<W>(dst, jb + gs * GB, T::from_payload(y));
                else one = (y & T::VAL) != W(0);
            } else if (r > 0) {
                or_bits<W>(dst, jb + G * GB, T::from_active(y, r));
            }
        }
        uint32_t m = __ballot_sync(0xffffffffu, one);
        while (m) {
            const int o = __ffs(m) - 1;
            m &= m - 1;
            const int64_t g0 = __shfl_sync(0xffffffffu, gs, o);
            int64_t g1 = g0 + __shfl_sync(0xffffffffu, (int64_t)glen, o);
            if (g1 > G) g1 = G;
            const int64_t b0 = jb + g0 * GB, b1 = jb + g1 * GB;   // bits [b0, b1)
            if (b1 <= b0) continue;
            const int64_t w0 = b0 >> 5, w1 = (b1 - 1) >> 5;
            for (int64_t w = w0 + lane_id(); w <= w1; w += 32) {
                uint32_t mask = 0xffffffffu;
                if (w == w0) mask &= 0xffffffffu << (b0 & 31);
                if (w == w1) mask &= 0xffffffffu >> (31 - ((b1 - 1) & 31));
                atomicOr(dst + w, mask);
            }
        }
    }
}

// One bottom-up level: every unvisited vertex v of range i scans its columns
// in blocks (j, i) -- its neighbours in range j, the graph being undirected --
// for j = 0, 1, ..., testing each neighbour u against the frontier delivered
// to block (i, j) (the decoded slot, or the raw slice f_j in PLAIN mode).  The
// smallest frontier neighbour of the first range that has one is v's parent:
// the ranges are ordered intervals of ids, so it is the smallest neighbour of
// v on the previous level, and it is the smallest frontier neighbour seen
// once the scan has passed the end of its range.  v's columns are read from
// the bottom-up rows (stored back to back, range by range).  One warp per
// visited word (32 vertices): a row of at most kBuLane entries is scanned by
// its own lane (kIlp entries and their frontier words in flight), a longer
// one by the whole warp (kIlp x 32 entries per step); the warp's next bits
// are one store (t is clear and no other kernel writes it this level).
constexpr int64_t kBuLane = 32;

__device__ __forceinline__ uint32_t warp_min(uint32_t x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, d);
        x = y < x ? y : x;
    }
    return x;
}

struct BuFrontier {
    const uint32_t* g;        // the decoded streams, or the raw frontier (PLAIN)
    uint32_t nb;
    // the range of u and whether the frontier delivered to block (i, range) holds u
    __device__ __forceinline__ uint32_t test(uint32_t u, uint32_t& j) const {
        j = u / nb;
        return (__ldg(g + (u >> 5)) >> (u & 31u)) & 1u;
    }
};

__global__ void __launch_bounds__(kNT) expand_bottom_up(LevelArgs a) {
    if (!a.ctl->bu) return;
    const int64_t words = (a.n + 31) >> 5;
    const int64_t gw0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t gstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t nb = (uint32_t)a.nb;                                // n < 2^31
    const uint32_t NONE = 0xffffffffu;
    unsigned long long edges = 0, cols = 0;
    for (int64_t w = gw0; w < words; w += gstride) {
        const uint32_t piw = __ldg(a.pi + w);
        if (piw == 0xffffffffu) continue;
        const int64_t v = w * 32 + lane_id();
        const bool mine = v < a.n && !((piw >> lane_id()) & 1u);
        int64_t e0 = 0, e1 = 0;
        if (mine) {
            e0 = __ldg(a.bu_ptr + v);
            e1 = __ldg(a.bu_ptr + v + 1);
        }
        const BuFrontier fr{a.mode != BFS_MODE_PLAIN ? a.gbits : a.f, nb};
        uint32_t best = NONE;
        if (mine && e1 - e0 <= kBuLane) {
            uint32_t cur = NONE;                                        // range of the entries so far
            for (int64_t e = e0; e < e1; e += kIlp) {
                const int cnt = (e1 - e < kIlp) ? (int)(e1 - e) : kIlp;
                uint32_t u[kIlp], j[kIlp], hit[kIlp];
#pragma unroll
                for (int k = 0; k < kIlp; ++k) u[k] = (k < cnt) ? (uint32_t)__ldg(a.bu_adj + e + k) : 0u;
#pragma unroll
                for (int k = 0; k < kIlp; ++k) hit[k] = (k < cnt) ? fr.test(u[k], j[k]) : 0u;
                bool stop = false;
#pragma unroll
                for (int k = 0; k < kIlp; ++k) {
                    if (k >= cnt || stop) continue;
                    if (j[k] != cur) {                                  // a new range
                        if (best != NONE) { stop = true; continue; }
                        cur = j[k];
                        ++cols;
                    }
                    ++edges;
                    if (hit[k] && u[k] < best) best = u[k];
                }
                if (stop) break;
            }
        }
        // long rows, one after the other, by the whole warp
        uint32_t lm = __ballot_sync(0xffffffffu, mine && e1 - e0 > kBuLane);
        while (lm) {
            const int o = __ffs(lm) - 1;
            lm &= lm - 1;
            const int64_t b0 = __shfl_sync(0xffffffffu, e0, o), b1 = __shfl_sync(0xffffffffu, e1, o);
            uint32_t wb = NONE, wend = NONE;                            // best so far and the end of its range
            uint32_t jlast = NONE;                                      // range of the last entry scanned
            for (int64_t e = b0; e < b1; e += kIlp * 32) {
                uint32_t u[kIlp], j[kIlp], hit[kIlp];
#pragma unroll
                for (int k = 0; k < kIlp; ++k) {
                    const int64_t x = e + k * 32 + lane_id();
                    u[k] = (x < b1) ? (uint32_t)__ldg(a.bu_adj + x) : NONE;
                }
#pragma unroll
                for (int k = 0; k < kIlp; ++k) {
                    hit[k] = 0u;
                    j[k] = NONE;
                    if (u[k] != NONE) hit[k] = fr.test(u[k], j[k]);
                }
                uint32_t cand = NONE;
                bool past = false;
#pragma unroll
                for (int k = 0; k < kIlp; ++k) {
                    if (hit[k] && u[k] < cand) cand = u[k];
                    // entries (in row order) that open a range
                    uint32_t jp = __shfl_up_sync(0xffffffffu, j[k], 1);
                    if (lane_id() == 0) jp = jlast;
                    const uint32_t opens = __ballot_sync(0xffffffffu, u[k] != NONE && j[k] != jp);
                    const uint32_t valid = __ballot_sync(0xffffffffu, u[k] != NONE);
                    if (lane_id() == (uint32_t)o) { cols += __popc(opens); edges += __popc(valid); }
                    const uint32_t jl = __shfl_sync(0xffffffffu, j[k], 31);
                    if (jl != NONE) jlast = jl;
                }
                cand = warp_min(cand);
                if (cand < wb) {
                    wb = cand;
                    wend = (uint32_t)range_begin(a, cand / nb + 1);
                }
#pragma unroll
                for (int k = 0; k < kIlp; ++k) past |= u[k] != NONE && u[k] >= wend;
                if (wb != NONE && __any_sync(0xffffffffu, past)) break;   // the best's range is complete
            }
            if (lane_id() == (uint32_t)o) best = wb;
        }
        const bool found = best != NONE;
        if (found) a.parent[v] = (int32_t)best;
        const uint32_t m = __ballot_sync(0xffffffffu, found);
        if (lane_id() == 0 && m) a.t[w] = m;
    }
    flush_counts(a, edges, cols, 0ull);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.ctr[C_BOTTOM_UP] = 1ull;
}

// ---------------------------------------------------------------- reduce --
// x = t & ~pi; pi |= x; level of the new vertices; |x|; the next frontier f = x
// and t cleared for the next level; frontier summary of x.
__global__ void __launch_bounds__(kNT) reduce_level(uint32_t* __restrict__ t, uint32_t* __restrict__ pi,
                                                    uint32_t* __restrict__ f, uint8_t* __restrict__ fsum,
                                                    int64_t words, int64_t n, int32_t* __restrict__ level,
                                                    const LevelCtl* __restrict__ ctl, unsigned long long* ctr,
                                                    const uint32_t* __restrict__ deg) {
    const int32_t next_level = ctl->level + 1;
    const int64_t nwarps = (words + 31) / 32;
    const int64_t gw0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t gstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gw = gw0; gw < nwarps; gw += gstride) {
        const int64_t w = gw * 32 + lane_id();
        uint32_t x = 0;
        unsigned long long dsum = 0;
        if (w < words) {
            const uint32_t pw = pi[w];
            x = t[w] & ~pw;
            if (x) pi[w] = pw | x;
            f[w] = x;
            t[w] = 0u;
        }
        const uint32_t any = __ballot_sync(0xffffffffu, x != 0u);
        // the levels (and degrees) of the fresh vertices, one word at a time
        // by the whole warp: lane l takes bit l (coalesced stores and loads)
        for (uint32_t m = any; m;) {
            const int k = __ffs(m) - 1;
            m &= m - 1;
            const uint32_t xk = __shfl_sync(0xffffffffu, x, k);
            const int64_t v = (gw * 32 + k) * 32 + lane_id();
            if (((xk >> lane_id()) & 1u) && v < n) {
                level[v] = next_level;
                if (deg) dsum += __ldg(deg + v);
            }
        }
        const int cnt = warp_sum(__popc(x));
        if (deg) dsum = warp_sum(dsum);
        if (lane_id() == 0) {
            fsum[gw] = any ? 1 : 0;
            if (cnt) atomicAdd(ctr + C_NEXT_COUNT, (unsigned long long)cnt);
            if (dsum) atomicAdd(ctr + C_NEXT_DEGREE, dsum);
        }
    }
}

// One thread: the values of the next level, and whether it runs (the
// frontier is not empty, no invariant failed, fewer than max_levels levels).
// In a CUDA graph the decision drives the conditional WHILE node.
// In the graph-launched loop (use_handle) it also clears the per-level
// counters and the row hand-out counters (lvl, nlvl of them) for the next
// level, in place of memset nodes; the stepwise loop reads them first and
// clears them itself.
__global__ void level_next(LevelCtl* c, unsigned long long* ctr, int64_t n, int win, int32_t max_levels,
                           cudaGraphConditionalHandle handle, int use_handle, unsigned long long* lvl, int nlvl) {
    const int64_t f = (int64_t)ctr[C_NEXT_COUNT];
    const int64_t prev = c->frontier;
    const int64_t mf = (int64_t)ctr[C_NEXT_DEGREE];
    c->m_u -= mf;
    c->m_f = mf;
    // direction of the next level (Beamer et al.): bottom-up once the growing
    // frontier's edges outweigh 1/alpha of the unvisited vertices' edges; back
    // to top-down once the shrinking frontier is below n / beta vertices
    if (c->policy == BFS_DIRECTION_BOTTOM_UP) {
        c->bu = 1;
    } else if (c->policy == BFS_DIRECTION_HYBRID) {
        if (!c->bu) c->bu = (f > prev && mf * (int64_t)c->alpha > c->m_u) ? 1 : 0;
        else c->bu = (f < prev && f * (int64_t)c->beta < n) ? 0 : 1;
    } else {
        c->bu = 0;
    }
    c->frontier = f;
    c->visited += f;
    c->level += 1;
    // PLAIN scans every raw word of every block: many units per hand-out on
    // sparse levels (few items each), few on dense ones (balance)
    c->plain_batch = (f * 64 < n) ? 32 : 2;
    // While few vertices are visited, most entries lead to fresh vertices,
    // each reached from many frontier vertices: reading the parent first turns
    // most of those visits into one L2 read instead of two atomics.  With a
    // window the next bit is a shared-memory atomic: not worth it.
    c->dedup = (!win && c->visited * 16 < n) ? 1 : 0;
    const int go = (f > 0 && ctr[C_ERROR] == 0 && c->level < max_levels) ? 1 : 0;
    c->go = go;
    if (use_handle) {
        for (int k = 0; k < C_ERROR; ++k) ctr[k] = 0ull;          // the error flag and trace cursors stay
        for (int k = C_WAH_WORDS; k < C_NUM; ++k) ctr[k] = 0ull;
        for (int k = 0; k < nlvl; ++k) lvl[k] = 0ull;
        cudaGraphSetConditional(handle, go ? 1u : 0u);
    }
}

__global__ void level_first(LevelCtl* c, int64_t n, int win, int policy, int alpha, int beta,
                            const uint32_t* deg, int32_t root, int64_t entries) {
    c->frontier = 1;
    c->visited = 1;
    c->level = 0;
    c->plain_batch = (64 < n) ? 32 : 2;
    c->dedup = (!win && 16 < n) ? 1 : 0;
    c->go = 1;
    c->policy = policy;
    c->alpha = alpha;
    c->beta = beta;
    c->bu = (policy == BFS_DIRECTION_BOTTOM_UP) ? 1 : 0;
    c->m_f = deg ? (int64_t)deg[root] : 0;
    c->m_u = entries - c->m_f;
}

// A search starts from nothing visited -- or, with bottom-up levels, from the
// vertices without entries marked visited (iso): no level reaches them, and
// the bottom-up scans skip them.
__global__ void init_search(int32_t* __restrict__ level, int32_t* __restrict__ parent, int64_t n,
                            uint32_t* __restrict__ pi, uint32_t* __restrict__ fa, uint32_t* __restrict__ fb,
                            int64_t words, uint8_t* __restrict__ fsum, int64_t fsum_len,
                            const uint32_t* __restrict__ iso) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        level[v] = -1;
        parent[v] = -1;
    }
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words; w += stride) {
        pi[w] = iso ? iso[w] : 0u;
        fa[w] = 0u;
        fb[w] = 0u;
    }
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < fsum_len; q += stride) fsum[q] = 0;
}

__global__ void set_root(int32_t* level, int32_t* parent, uint32_t* pi, uint32_t* fa, uint8_t* fsum, int32_t root) {
    level[root] = 0;
    parent[root] = root;
    pi[root >> 5] |= 1u << (root & 31);
    fa[root >> 5] |= 1u << (root & 31);
    fsum[root >> 10] = 1;
}

// Pack the streams of this exchange into a trace (the receive buffer g'):
// ctr[cursor] is the trace's fill, kept from level to level.
__global__ void __launch_bounds__(kNT) trace_offsets(const int64_t* __restrict__ counts, int nslots, int u32_per_word,
                                                     int64_t* __restrict__ slot_off, int64_t* __restrict__ trace_counts,
                                                     unsigned long long* ctr, int cursor, int64_t capacity,
                                                     const uint8_t* fmt, uint8_t* trace_fmt) {
    __shared__ unsigned long long red[kNT / 32 + 1];
    const unsigned long long used = ctr[cursor];
    unsigned long long carry = 0;
    for (int s0 = 0; s0 < nslots; s0 += kNT) {
        const int s = s0 + threadIdx.x;
        const unsigned long long c = (s < nslots) ? (unsigned long long)counts[s] * u32_per_word : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan<kNT>(c, 0ull, OpSum(), red, &tot);
        if (s < nslots) {
            slot_off[s] = (int64_t)(used + carry + ex);
            trace_counts[s] = counts[s];
            if (trace_fmt) trace_fmt[s] = fmt ? fmt[s] : (uint8_t)FMT_WAH;
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (used + carry > (unsigned long long)capacity) {
            ctr[C_ERROR] |= 2ull;                 // trace overflow
            ctr[cursor] = (unsigned long long)capacity + 1;
        } else {
            ctr[cursor] = used + carry;
        }
    }
}

__global__ void trace_copy(const uint32_t* __restrict__ xbuf, int64_t slot_cap_u32, const int64_t* __restrict__ counts,
                           int nslots, int u32_per_word, const int64_t* __restrict__ slot_off,
                           uint32_t* __restrict__ trace, int64_t capacity) {
    for (int s = blockIdx.y; s < nslots; s += gridDim.y) {
        const int64_t c = counts[s] * u32_per_word;
        const int64_t off = slot_off[s];
        if (off + c > capacity) continue;
        for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < c; x += (int64_t)gridDim.x * blockDim.x)
            trace[off + x] = xbuf[(int64_t)s * slot_cap_u32 + x];
    }
}

// The output checks of bfs_check_search: root level 0 and its own parent;
// an unreached vertex -1 / -1; a reached one a parent in [0, n) one level
// closer to the root.  out[0] counts failures, out[1] keeps the smallest
// failing vertex, out[2] counts the reached vertices.
__global__ void __launch_bounds__(kNT) verify_search(const int32_t* __restrict__ parent,
                                                     const int32_t* __restrict__ level, int64_t n, int32_t root,
                                                     unsigned long long* out) {
    unsigned long long bad = 0, reached = 0, first = ~0ull;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t lv = level[v], pv = parent[v];
        bool ok;
        if (v == root) ok = lv == 0 && pv == root;
        else if (lv < 0) ok = lv == -1 && pv == -1;
        else ok = lv > 0 && pv >= 0 && (int64_t)pv < n && level[pv] == lv - 1;
        reached += lv >= 0;
        if (!ok) {
            ++bad;
            if ((unsigned long long)v < first) first = (unsigned long long)v;
        }
    }
    bad = warp_sum(bad);
    reached = warp_sum(reached);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const unsigned long long y = __shfl_xor_sync(0xffffffffu, first, d);
        first = y < first ? y : first;
    }
    if (lane_id() == 0) {
        if (bad) atomicAdd(out, bad);
        if (first != ~0ull) atomicMin(out + 1, first);
        if (reached) atomicAdd(out + 2, reached);
    }
}

__global__ void visited_count(const LevelCtl* c, unsigned long long* out) { out[3] = (unsigned long long)c->visited; }

int sm_count() {
    static int cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached = v > 0 ? v : 1;
    }
    return cached;
}

int64_t l2_bytes() {
    static int64_t cached = 0;
    if (!cached) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev);
        cached = v > 0 ? v : (64ll << 20);
    }
    return cached;
}

// Dynamic shared memory of the expansion kernels: the row window (pi_i and
// the partial t_i), when it fits next to the static arrays.
size_t window_bytes(int64_t win_words) { return (size_t)(2 * win_words * sizeof(uint32_t)); }

template <typename K>
bfs_status allow_smem(K kernel, size_t dyn) {
    BFS_CUDA_TRY(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    return BFS_OK;
}

// The expansion of a level: with the row window one kernel; without, the two
// variants (with and without reading the parent first), of which the level's
// device-side choice runs and the other returns at once.
template <typename W, bool ROWX>
void launch_expand_wah(const LevelArgs& a, bool win, int grid, size_t dyn, cudaStream_t s) {
    if (win) {
        expand_wah<W, true, false, ROWX><<<grid, kXT, dyn, s>>>(a);
    } else {
        expand_wah<W, false, true, ROWX><<<grid, kXT, 0, s>>>(a);
        expand_wah<W, false, false, ROWX><<<grid, kXT, 0, s>>>(a);
    }
}

template <bool ROWX>
void launch_expand_pieces(const LevelArgs& a, bool win, int grid, size_t dyn, cudaStream_t s) {
    if (win) {
        expand_pieces<true, false, ROWX><<<grid, kXT, dyn, s>>>(a);
    } else {
        expand_pieces<false, true, ROWX><<<grid, kXT, 0, s>>>(a);
        expand_pieces<false, false, ROWX><<<grid, kXT, 0, s>>>(a);
    }
}

}  // namespace

// ------------------------------------------------------------- workspace --
bfs_status ensure_workspace_once(bfs_graph* g);

// All of the search workspace or none of it: a failed allocation releases the rest.
bfs_status ensure_workspace(bfs_graph* g, cudaStream_t st) {
    (void)st;
    if (g->W.bm_words) return BFS_OK;
    const bfs_status rc = ensure_workspace_once(g);
    if (rc != BFS_OK) free_workspace(g);
    return rc;
}

bfs_status ensure_workspace_once(bfs_graph* g) {
    Workspace& W = g->W;
    const Layout& L = g->L;
    const int p = L.p;
    const int64_t p2 = (int64_t)p * p;
    W.bm_words = ((L.n + 31) / 32 + 4 + 3) / 4 * 4;
    W.fsum_len = ((W.bm_words + 31) / 32 + 64 + 3) / 4 * 4;   // whole 32-bit words
    const int64_t cap32 = L.nb / 31 + 2, cap64 = L.nb / 63 + 2;
    W.slot_cap = cap32;
    W.chunk_words = 32;
    W.chunks_per_slot = (cap32 + 31) / 32;
    const int64_t xbytes = p2 * std::max<int64_t>(4 * cap32, 8 * cap64);
    BFS_TRY(W.pi.alloc(4 * W.bm_words));
    BFS_TRY(W.fa.alloc(4 * W.bm_words));
    BFS_TRY(W.fb.alloc(4 * W.bm_words));
    BFS_TRY(W.fsum.alloc(W.fsum_len));
    BFS_TRY(W.xbuf.alloc(xbytes));
    BFS_TRY(W.xcount.alloc(sizeof(int64_t) * p2));
    BFS_TRY(W.chunk_base.alloc(sizeof(int64_t) * p2 * W.chunks_per_slot));
    BFS_TRY(W.units.alloc(sizeof(int64_t) * (p2 + 1)));              // slot unit bases
    BFS_TRY(W.xfmt.alloc((size_t)p2));
    W.enc_cps = parallel_encode_chunks(L.nb, 32);                       // 31-bit groups: the most chunks
    BFS_TRY(W.enc_sums.alloc(parallel_encode_sum_bytes() * p2 * W.enc_cps));
    BFS_TRY(W.enc_bases.alloc(parallel_encode_base_bytes() * p2 * W.enc_cps));
    BFS_TRY(W.enc_flags.alloc(p2 * W.enc_cps));
    BFS_TRY(W.enc_done.alloc(sizeof(unsigned int)));
    BFS_TRY(W.ctl.alloc(sizeof(LevelCtl)));
    BFS_CUDA_TRY(cudaMemset(W.enc_done.ptr, 0, sizeof(unsigned int)));
    BFS_TRY(W.counters.alloc(sizeof(unsigned long long) * C_NUM));
    // pieces: per row, sum over long columns of ceil(len/kPiece) <= nnz_row/kPiece + nnz_row/kHub
    std::vector<int64_t> meta(2 * (size_t)p);
    int64_t total = 0;
    for (int i = 0; i < p; ++i) {
        int64_t nnz_row = 0;
        for (int j = 0; j < p; ++j) nnz_row += L.nnz_b[(int64_t)i * p + j];
        const int64_t cap = nnz_row / kPiece + nnz_row / kHub + 4;
        meta[i] = total;
        meta[p + i] = cap;
        total += cap;
    }
    W.piece_cap = total;
    BFS_TRY(W.pieces.alloc(sizeof(Item) * (total > 0 ? total : 1)));
    // per-level scratch: row_next[p], row_piece_count[p], row_piece_next[p]; row piece bases and caps
    BFS_TRY(W.level_scratch.alloc(sizeof(unsigned long long) * (3 * p + 1)));
    BFS_TRY(W.row_meta.alloc(sizeof(int64_t) * 2 * p));
    BFS_CUDA_TRY(cudaMemcpy(W.row_meta.ptr, meta.data(), sizeof(int64_t) * 2 * p, cudaMemcpyHostToDevice));
    if (!W.h_counters) {
        void* h = nullptr;
        BFS_CUDA_TRY(cudaMallocHost(&h, sizeof(uint64_t) * C_NUM));
        W.h_counters = static_cast<uint64_t*>(h);
    }
    if (!W.events) {
        for (auto& e : W.ev) BFS_CUDA_TRY(cudaEventCreate(&e));
        W.events = true;
    }
    // the row window of the expansion: pi_i and t_i of one range, if they fit
    const int64_t win = (L.nb + 31) / 32;
    const size_t static_bytes = 4096;
    W.win_words = (window_bytes(win) + static_bytes <= (size_t)kSmemLimit) ? win : 0;
    if (W.win_words) {
        const size_t dyn = window_bytes(W.win_words);
        BFS_TRY(allow_smem(expand_wah<uint32_t, true, false, false>, dyn));
        BFS_TRY(allow_smem(expand_wah<unsigned long long, true, false, false>, dyn));
        BFS_TRY(allow_smem(expand_wah<uint32_t, true, false, true>, dyn));
        BFS_TRY(allow_smem(expand_wah<unsigned long long, true, false, true>, dyn));
        BFS_TRY(allow_smem(expand_pieces<true, false, true>, dyn));
        BFS_TRY(allow_smem(expand_plain<true, false>, dyn));
        BFS_TRY(allow_smem(expand_pieces<true, false, false>, dyn));
    }
    return BFS_OK;
}

void free_workspace(bfs_graph* g) {
    Workspace& W = g->W;
    W.pi.release(); W.fa.release(); W.fb.release(); W.fsum.release(); W.xbuf.release();
    W.xcount.release(); W.chunk_base.release(); W.units.release(); W.counters.release(); W.pieces.release();
    W.level_scratch.release(); W.row_meta.release();
    W.tblk.release(); W.rowbuf.release(); W.rowcount.release(); W.rowfirst.release(); W.rowlive.release();
    W.tblk_dirty = false;
    W.enc_sums.release(); W.enc_bases.release(); W.enc_flags.release(); W.enc_done.release(); W.ctl.release();
    W.gbits.release();
    W.colfirst.release();
    W.xfmt.release();
    W.ddir.release();
    for (auto& c : W.sgraph) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        if (c.graph) cudaGraphDestroy(c.graph);
        c = SearchGraph();
    }
    W.sgraph_next = 0;
    W.tmp_parent.release(); W.tmp_level.release();
    if (W.h_counters) cudaFreeHost(W.h_counters);
    W.h_counters = nullptr;
    if (W.events) for (auto& e : W.ev) cudaEventDestroy(e);
    W.events = false;
    W.bm_words = 0;
}

namespace {

struct BusyGuard {
    bfs_graph* g;
    bool ok;
    explicit BusyGuard(bfs_graph* gg) : g(gg) {
        int expect = 0;
        ok = g->busy.compare_exchange_strong(expect, 1);
    }
    ~BusyGuard() { if (ok) g->busy.store(0); }
};

float elapsed(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) { cudaGetLastError(); return 0.f; }
    return ms;
}

// Run the output checks on device outputs; with ctl, the reached count must
// also equal the vertices the search visited.
bfs_status check_outputs(int64_t n, int32_t root, const int32_t* parent, const int32_t* level, const LevelCtl* ctl,
                         cudaStream_t st) {
    DevBuf out;
    BFS_TRY(out.alloc(4 * sizeof(unsigned long long)));
    unsigned long long init[4] = {0ull, ~0ull, 0ull, 0ull};
    BFS_CUDA_TRY(cudaMemcpyAsync(out.ptr, init, sizeof(init), cudaMemcpyHostToDevice, st));
    verify_search<<<(int)std::min<int64_t>((n + kNT - 1) / kNT, (int64_t)sm_count() * 8), kNT, 0, st>>>(
        parent, level, n, root, out.as<unsigned long long>());
    if (ctl) visited_count<<<1, 1, 0, st>>>(ctl, out.as<unsigned long long>());
    BFS_CUDA_TRY(cudaGetLastError());
    unsigned long long h[4];
    BFS_CUDA_TRY(cudaMemcpyAsync(h, out.ptr, sizeof(h), cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h[0])
        return set_error(BFS_ERR_CORRUPT, "%llu vertices fail the level/parent checks (first: vertex %llu)", h[0], h[1]);
    if (ctl && h[2] != h[3])
        return set_error(BFS_ERR_CORRUPT, "%llu vertices reached but %llu visited by the search", h[2], h[3]);
    return BFS_OK;
}

bfs_status run_search(bfs_graph* g, int32_t root, int32_t* parent, int32_t* level, bfs_run_stats* stats,
                      cudaStream_t st) {
    Layout& L = g->L;
    Workspace& W = g->W;
    BFS_TRY(ensure_workspace(g, st));
    const int mode = g->mode;
    const int wbits = g->wah_bits;
    const int p = L.p;
    const int64_t p2 = (int64_t)p * p;
    const int64_t slot_cap = (wbits == 32) ? L.nb / 31 + 2 : L.nb / 63 + 2;
    const int nslots = (mode == BFS_MODE_COMPRESS_SIEVE) ? (int)p2 : (mode == BFS_MODE_COMPRESS ? p : 0);
    const bool timing = stats && stats->timing;
    const bool tracing = stats && stats->trace_words && stats->trace_counts && nslots > 0;
    unsigned long long* ctr = W.counters.as<unsigned long long>();
    const bool win = W.win_words > 0;
    const int xgrid = sm_count();                  // persistent: one 1024-thread CTA per SM
    // the compressed row exchange of the fold belongs to DIR-WAH (COMPRESS_SIEVE)
    const bool rowx = g->row_exchange && mode == BFS_MODE_COMPRESS_SIEVE;
    if (rowx && !W.tblk.ptr) {
        // allocated once (all or none): captured level loops keep the addresses
        const int64_t cap32 = L.nb / 31 + 2, cap64 = L.nb / 63 + 2;
        W.row_cap = cap32;
        bfs_status rc = W.rowbuf.alloc((size_t)p2 * std::max<int64_t>(4 * cap32, 8 * cap64));
        if (rc == BFS_OK) rc = W.rowcount.alloc(sizeof(int64_t) * (size_t)p2);
        if (rc == BFS_OK) rc = W.rowfirst.alloc(sizeof(int64_t) * 2 * (size_t)(p2 * W.enc_cps));
        if (rc == BFS_OK) rc = W.rowlive.alloc((size_t)p2);
        if (rc == BFS_OK) rc = W.tblk.alloc(sizeof(uint32_t) * (size_t)(p2 * L.dir_stride));
        if (rc != BFS_OK) {
            W.tblk.release(); W.rowbuf.release(); W.rowcount.release(); W.rowfirst.release(); W.rowlive.release();
            return rc;
        }
        BFS_CUDA_TRY(cudaMemsetAsync(W.tblk.ptr, 0, W.tblk.bytes, st));
        W.tblk_dirty = false;
    }
    if (rowx && W.tblk_dirty) {          // an earlier search stopped between marking and encoding
        BFS_CUDA_TRY(cudaMemsetAsync(W.tblk.ptr, 0, W.tblk.bytes, st));
        W.tblk_dirty = false;
    }
    const int64_t row_cap = (wbits == 32) ? L.nb / 31 + 2 : L.nb / 63 + 2;
    const bool adaptive = g->adaptive && mode != BFS_MODE_PLAIN;
    if (adaptive && wbits != 32)
        return set_error(BFS_ERR_INVALID_ARG, "the level-adaptive exchange format needs 32-bit WAH words");
    const bool row_tracing = stats && rowx && stats->row_trace_words && stats->row_trace_counts;
    // the dynamic cross directory belongs to the sieve (COMPRESS_SIEVE)
    const bool dynamic = g->dynamic_dir && mode == BFS_MODE_COMPRESS_SIEVE;
    if (dynamic && !W.ddir.ptr) {
        // allocated once: captured level loops keep the address
        BFS_TRY(W.ddir.alloc(sizeof(uint32_t) * (size_t)(p2 * L.dir_stride)));
    }
    const size_t dyn = win ? window_bytes(W.win_words) : 0;
    // bottom-up levels: degrees (direction choice) and the decoded streams
    const bool bu_kernels = g->direction != BFS_DIRECTION_TOP_DOWN;
    if (bu_kernels) BFS_TRY(ensure_degrees(g, st));
    const int64_t g_words = (W.bm_words + 3) / 4 * 4;
    if (bu_kernels && (!W.gbits.ptr || !W.colfirst.ptr)) {
        // allocated once (both or neither): captured level loops keep the addresses
        bfs_status rc = W.gbits.alloc(sizeof(uint32_t) * (size_t)g_words);
        if (rc == BFS_OK) rc = W.colfirst.alloc(sizeof(int64_t) * 2 * (size_t)(p2 * W.enc_cps));
        if (rc != BFS_OK) { W.gbits.release(); W.colfirst.release(); return rc; }
    }
    DevBuf slot_off;
    if (tracing || row_tracing) BFS_TRY(slot_off.alloc(sizeof(int64_t) * (size_t)std::max<int64_t>(nslots, p2)));
    if (stats) { stats->n_levels = 0; stats->trace_used = 0; stats->row_trace_used = 0; }

    init_search<<<sm_count() * 4, kNT, 0, st>>>(level, parent, L.n, W.pi.as<uint32_t>(), W.fa.as<uint32_t>(),
                                                W.fb.as<uint32_t>(), W.bm_words, W.fsum.as<uint8_t>(), W.fsum_len,
                                                bu_kernels ? L.iso.as<uint32_t>() : nullptr);
    BFS_CUDA_TRY(cudaGetLastError());
    set_root<<<1, 1, 0, st>>>(level, parent, W.pi.as<uint32_t>(), W.fa.as<uint32_t>(), W.fsum.as<uint8_t>(), root);
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * C_NUM, st));

    LevelArgs a;
    memset(&a, 0, sizeof(a));
    a.dir = L.dir.as<uint32_t>();
    a.rank = L.rank.as<uint32_t>();
    a.dir_stride = L.dir_stride;
    a.cp = L.cp.as<uint32_t>();
    a.cp_base = L.cp_base_d.as<int64_t>();
    a.ir_base = L.ir_base_d.as<int64_t>();
    a.ir = L.ir.as<int32_t>();
    a.p = p;
    a.nb = L.nb;
    a.n = L.n;
    a.pi = W.pi.as<uint32_t>();
    a.parent = parent;
    a.xbuf = W.xbuf.ptr;
    a.slot_cap = slot_cap;
    a.xcount = W.xcount.as<int64_t>();
    a.chunk_base = W.chunk_base.as<int64_t>();
    a.chunks_per_slot = W.chunks_per_slot;
    a.slot_unit_base = W.units.as<int64_t>();
    unsigned long long* lvl = W.level_scratch.as<unsigned long long>();
    BFS_CUDA_TRY(cudaMemsetAsync(lvl, 0, sizeof(unsigned long long) * (3 * p + 1), st));   // the first level's
    a.row_next = lvl;
    a.row_piece_count = lvl + p;
    a.row_piece_next = lvl + 2 * p;
    a.row_piece_base = W.row_meta.as<int64_t>();
    a.row_piece_cap = W.row_meta.as<int64_t>() + p;
    a.pieces = W.pieces.as<Item>();
    a.ctr = ctr;
    a.mode = mode;
    a.plain_upb = (L.nb + 1023) / 1024;               // 32 raw words per PLAIN unit
    a.win_words = W.win_words;
    a.row_exchange = rowx ? 1 : 0;
    // Without a window the visited test, the next bit and the parent update
    // go through L2.  When the parent array does not fit in half of L2, all
    // CTAs take the block-rows in turn, so that only one row's slice of it
    // (and of pi and t) is being updated at a time.
    a.sweep = (!win && 4 * L.n > l2_bytes() / 2) ? 1 : 0;
    a.tblk = W.tblk.as<uint32_t>();
    a.rowbuf = W.rowbuf.ptr;
    a.row_cap = row_cap;
    a.row_count = W.rowcount.as<int64_t>();
    a.row_first = W.rowfirst.as<int64_t>();
    a.row_cps = W.enc_cps;
    a.row_bcps = (L.nb + (int64_t)kEncChunkGroups * (wbits - 1) - 1) / ((int64_t)kEncChunkGroups * (wbits - 1));
    a.gbits = W.gbits.as<uint32_t>();
    a.range_aligned = (L.nb % 32 == 0) ? 1 : 0;
    a.g_words = g_words;
    a.bu_ptr = L.bu_ptr.as<int64_t>();
    a.bu_adj = L.bu_adj.as<int32_t>();

    EncodeArgs ea;
    memset(&ea, 0, sizeof(ea));
    ea.dir = (mode == BFS_MODE_COMPRESS_SIEVE) ? (dynamic ? W.ddir.as<uint32_t>() : L.dir.as<uint32_t>()) : nullptr;
    ea.dir_stride = L.dir_stride;
    ea.p = p;
    ea.nb = L.nb;
    ea.n = L.n;
    ea.sieve = (mode == BFS_MODE_COMPRESS_SIEVE);
    ea.nslots = nslots;
    ea.fsum = W.fsum.as<uint8_t>();
    ea.out = W.xbuf.ptr;
    ea.slot_cap = slot_cap;
    ea.counts = W.xcount.as<int64_t>();
    ea.unit_base = W.chunk_base.as<int64_t>();      // the decoder's unit bases, written by the encoder
    ea.unit_stride = W.chunks_per_slot;
    ea.wah_words = ctr + C_WAH_WORDS;
    ea.plan_base = W.units.as<int64_t>();            // the unit plan, laid out by the encoder's scan
    ea.plan_units = ctr + C_UNITS;
    ea.plan_done = W.enc_done.as<unsigned int>();
    ea.frontier_words = W.bm_words;
    if (rowx) ea.slot_bits = W.rowlive.as<uint8_t>();    // the row encoder skips blocks that expanded nothing
    ea.adaptive = adaptive ? 1 : 0;
    ea.fmt = W.xfmt.as<uint8_t>();
    if (bu_kernels) ea.chunk_first = W.colfirst.as<int64_t>();   // the bottom-up decode starts chunk by chunk
    a.col_first = W.colfirst.as<int64_t>();
    a.fmt = adaptive ? W.xfmt.as<uint8_t>() : nullptr;

    // the row encoder: slot s = i*p + j is the partial t_{i,j} (the directory
    // operand, consumed and cleared) sieved by not(pi_i) (the frontier operand
    // at range i, complemented)
    EncodeArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.frontier = W.pi.as<uint32_t>();
    ra.frontier_words = W.bm_words;
    ra.invert_frontier = 1;
    ra.dir = W.tblk.as<uint32_t>();
    ra.dir_clear = W.tblk.as<uint32_t>();
    ra.dir_stride = L.dir_stride;
    ra.p = p;
    ra.nb = L.nb;
    ra.n = L.n;
    ra.sieve = 1;
    ra.row_slots = 1;
    ra.nslots = (int)p2;
    ra.out = W.rowbuf.ptr;
    ra.slot_cap = row_cap;
    ra.counts = W.rowcount.as<int64_t>();
    ra.wah_words = ctr + C_ROW_WORDS;
    ra.chunk_first = W.rowfirst.as<int64_t>();
    ra.slot_live = W.rowlive.as<uint8_t>();      // t_{i,j} = 0 when stream (i,j) carried no vertex

    uint32_t* f = W.fa.as<uint32_t>();       // frontier of the level (reduce_level writes the next one here)
    uint32_t* t = W.fb.as<uint32_t>();       // next bits (cleared by reduce_level)
    LevelCtl* ctl = W.ctl.as<LevelCtl>();
    a.f = f;
    a.t = t;
    a.ctl = ctl;
    ea.frontier = f;
    ra.skip = &ctl->bu;                      // bottom-up levels have no row exchange
    const int32_t max_levels = (int32_t)std::min<int64_t>(L.n + 1, INT32_MAX);
    const uint32_t* deg = bu_kernels ? L.deg.as<uint32_t>() : nullptr;

    if (dynamic)                     // the search's directories start as V
        BFS_CUDA_TRY(cudaMemcpyAsync(W.ddir.ptr, L.dir.ptr, W.ddir.bytes, cudaMemcpyDeviceToDevice, st));
    level_first<<<1, 1, 0, st>>>(ctl, L.n, win ? 1 : 0, g->direction, g->alpha, g->beta, deg, root, L.nnz);
    BFS_CUDA_TRY(cudaGetLastError());

    // One level: the same launch sequence every time.  `host` adds the
    // statistics, the trace and the phase events (and k is known on the host).
    auto level_body = [&](cudaStream_t s, bool host, int32_t k, cudaGraphConditionalHandle handle) -> bfs_status {
        // per-level counters (the error flag and the trace cursor persist): the
        // stepwise loop clears them here, the graph-launched loop's level_next
        // at the end of the level before (and the search's setup for the first)
        if (host) {
            BFS_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * C_ERROR, s));
            BFS_CUDA_TRY(cudaMemsetAsync(ctr + C_WAH_WORDS, 0, sizeof(unsigned long long) * (C_NUM - C_WAH_WORDS), s));
            BFS_CUDA_TRY(cudaMemsetAsync(lvl, 0, sizeof(unsigned long long) * (3 * p + 1), s));
        }
        if (host && timing) cudaEventRecord(W.ev[7], s);
        if (dynamic) {                  // the frontier's bits of the dynamic directory
            dyn_sieve<<<sm_count() * 8, kNT, 0, s>>>(a, W.ddir.as<uint32_t>(), W.fsum.as<uint8_t>());
            BFS_CUDA_TRY(cudaGetLastError());
        }
        if (host && timing) cudaEventRecord(W.ev[0], s);
        if (mode == BFS_MODE_PLAIN) {
            if (host && timing) { cudaEventRecord(W.ev[1], s); cudaEventRecord(W.ev[2], s); }
            if (win) {
                expand_plain<true, false><<<xgrid, kXT, dyn, s>>>(a);
            } else {
                expand_plain<false, true><<<xgrid, kXT, 0, s>>>(a);
                expand_plain<false, false><<<xgrid, kXT, 0, s>>>(a);
            }
            BFS_CUDA_TRY(cudaGetLastError());
        } else {
            // the exchanged-vertex and chunk counts are statistics: only the stepwise loop asks for them
            EncodeArgs eh = ea;
            eh.live_chunks = host ? ctr + C_ENC_CHUNKS : nullptr;
            BFS_TRY(launch_wah_encode_parallel(eh, wbits, W.enc_sums.ptr, W.enc_bases.ptr, W.enc_cps,
                                               W.enc_flags.ptr, host ? ctr + C_EXCHANGED : nullptr, sm_count() * 6, s));
            if (bu_kernels) {           // a bottom-up level reads the streams as bitmaps
                if (!a.range_aligned) clear_gbits<<<sm_count() * 4, kNT, 0, s>>>(a);   // shared boundary words
                const int64_t fitems = (int64_t)p * a.row_bcps;
                const int fgrid = (int)std::min<int64_t>(std::max<int64_t>(fitems, 1), (int64_t)sm_count() * 4);
                if (wbits == 32) fold_slots<uint32_t, false><<<fgrid, kFT, 0, s>>>(a);
                else fold_slots<unsigned long long, false><<<fgrid, kFT, 0, s>>>(a);
                if (adaptive) decode_streams<uint32_t><<<sm_count() * 8, kNT, 0, s>>>(a);   // vector slots
                BFS_CUDA_TRY(cudaGetLastError());
            }
            if (host && timing) cudaEventRecord(W.ev[1], s);
            if (host && tracing && k < stats->capacity_levels) {
                const int u32pw = wbits / 32;
                trace_offsets<<<1, kNT, 0, s>>>(W.xcount.as<int64_t>(), nslots, u32pw, slot_off.as<int64_t>(),
                                                stats->trace_counts + (int64_t)k * nslots, ctr, C_TRACE_USED,
                                                stats->trace_capacity, a.fmt,
                                                stats->trace_formats ? stats->trace_formats + (int64_t)k * nslots
                                                                     : nullptr);
                dim3 tg(8, std::min(nslots, 65535));
                trace_copy<<<tg, kNT, 0, s>>>(W.xbuf.as<uint32_t>(), slot_cap * u32pw, W.xcount.as<int64_t>(), nslots,
                                              u32pw, slot_off.as<int64_t>(), stats->trace_words, stats->trace_capacity);
                BFS_CUDA_TRY(cudaGetLastError());
            }
            if (host && timing) cudaEventRecord(W.ev[2], s);
            if (wbits == 32) {
                if (rowx) launch_expand_wah<uint32_t, true>(a, win, xgrid, dyn, s);
                else launch_expand_wah<uint32_t, false>(a, win, xgrid, dyn, s);
            } else {
                if (rowx) launch_expand_wah<unsigned long long, true>(a, win, xgrid, dyn, s);
                else launch_expand_wah<unsigned long long, false>(a, win, xgrid, dyn, s);
            }
            BFS_CUDA_TRY(cudaGetLastError());
        }
        if (rowx) launch_expand_pieces<true>(a, win, xgrid, dyn, s);
        else launch_expand_pieces<false>(a, win, xgrid, dyn, s);
        BFS_CUDA_TRY(cudaGetLastError());
        if (bu_kernels) {
            expand_bottom_up<<<sm_count() * 8, kNT, 0, s>>>(a);
            BFS_CUDA_TRY(cudaGetLastError());
        }
        if (host && timing) cudaEventRecord(W.ev[3], s);
        if (rowx) {
            // the row exchange: every block's partial, sieved by not(pi_i), WAH-encoded
            // into its row buffer; the fold OR-decodes the buffers of each block-row into t
            EncodeArgs rh = ra;
            rh.live_chunks = host ? ctr + C_ROW_CHUNKS : nullptr;
            BFS_TRY(launch_wah_encode_parallel(rh, wbits, W.enc_sums.ptr, W.enc_bases.ptr, W.enc_cps, W.enc_flags.ptr,
                                               nullptr, sm_count() * 6, s));
            if (host && timing) cudaEventRecord(W.ev[5], s);
            if (host && row_tracing && k < stats->capacity_levels) {
                const int u32pw = wbits / 32;
                trace_offsets<<<1, kNT, 0, s>>>(W.rowcount.as<int64_t>(), (int)p2, u32pw, slot_off.as<int64_t>(),
                                                stats->row_trace_counts + (int64_t)k * p2, ctr, C_ROW_TRACE_USED,
                                                stats->row_trace_capacity, nullptr, nullptr);
                dim3 tg(8, (unsigned)std::min<int64_t>(p2, 65535));
                trace_copy<<<tg, kNT, 0, s>>>(static_cast<const uint32_t*>(W.rowbuf.ptr), row_cap * u32pw,
                                              W.rowcount.as<int64_t>(), (int)p2, u32pw, slot_off.as<int64_t>(),
                                              stats->row_trace_words, stats->row_trace_capacity);
                BFS_CUDA_TRY(cudaGetLastError());
            }
            const int64_t fitems = (int64_t)p * a.row_bcps;
            const int fgrid = (int)std::min<int64_t>(std::max<int64_t>(fitems, 1), (int64_t)sm_count() * 4);
            if (wbits == 32) fold_slots<uint32_t, true><<<fgrid, kFT, 0, s>>>(a);
            else fold_slots<unsigned long long, true><<<fgrid, kFT, 0, s>>>(a);
            BFS_CUDA_TRY(cudaGetLastError());
            if (host && timing) cudaEventRecord(W.ev[6], s);
        } else if (host && timing) {
            cudaEventRecord(W.ev[5], s);
            cudaEventRecord(W.ev[6], s);
        }
        reduce_level<<<std::min<int64_t>((W.bm_words + 255) / 256 + 1, sm_count() * 16), kNT, 0, s>>>(
            t, W.pi.as<uint32_t>(), f, W.fsum.as<uint8_t>(), W.bm_words, L.n, level, ctl, ctr, deg);
        BFS_CUDA_TRY(cudaGetLastError());
        if (host && timing) cudaEventRecord(W.ev[4], s);
        level_next<<<1, 1, 0, s>>>(ctl, ctr, L.n, win ? 1 : 0, max_levels, handle, host ? 0 : 1, lvl, 3 * p + 1);
        BFS_CUDA_TRY(cudaGetLastError());
        return BFS_OK;
    };

    if (!stats) {
        // The whole level loop as one CUDA-graph launch: a conditional WHILE
        // node repeats the level while level_next says so.  No host round
        // trip per level; the graph is built once per configuration and output
        // buffers and reused.
        SearchGraph* sg = nullptr;
        for (auto& c : W.sgraph)
            if (c.exec && c.mode == mode && c.wbits == wbits && c.rowx == (int)rowx &&
                c.bottom_up == (int)bu_kernels && c.adaptive == (int)adaptive && c.dynamic == (int)dynamic &&
                c.parent == parent &&
                c.level == level)
                sg = &c;
        if (!sg) {
            SearchGraph& c = W.sgraph[W.sgraph_next];
            W.sgraph_next = (W.sgraph_next + 1) % (int)(sizeof(W.sgraph) / sizeof(W.sgraph[0]));
            if (c.exec) { cudaGraphExecDestroy(c.exec); c.exec = nullptr; }
            if (c.graph) { cudaGraphDestroy(c.graph); c.graph = nullptr; }
            cudaGraph_t graph = nullptr;
            BFS_CUDA_TRY(cudaGraphCreate(&graph, 0));
            cudaGraphConditionalHandle handle;
            BFS_CUDA_TRY(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = handle;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cond = nullptr;
            cudaError_t ce = cudaGraphAddNode(&cond, graph, nullptr, nullptr, 0, &cp);
            if (ce != cudaSuccess) { cudaGraphDestroy(graph); return cuda_error(ce, "conditional node", __FILE__, __LINE__); }
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            cudaStream_t cs = nullptr;
            BFS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
            ce = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
            bfs_status bs = BFS_OK;
            if (ce == cudaSuccess) bs = level_body(cs, false, 0, handle);
            cudaError_t ce2 = cudaStreamEndCapture(cs, &body);
            cudaStreamDestroy(cs);
            if (ce != cudaSuccess || ce2 != cudaSuccess || bs != BFS_OK) {
                cudaGraphDestroy(graph);
                if (bs != BFS_OK) return bs;
                return cuda_error(ce != cudaSuccess ? ce : ce2, "capture of the level body", __FILE__, __LINE__);
            }
            cudaGraphExec_t exec = nullptr;
            ce = cudaGraphInstantiate(&exec, graph, 0);
            if (ce != cudaSuccess) { cudaGraphDestroy(graph); return cuda_error(ce, "cudaGraphInstantiate(search)", __FILE__, __LINE__); }
            c.graph = graph;
            c.exec = exec;
            c.mode = mode;
            c.wbits = wbits;
            c.rowx = rowx ? 1 : 0;
            c.bottom_up = bu_kernels ? 1 : 0;
            c.adaptive = adaptive ? 1 : 0;
            c.dynamic = dynamic ? 1 : 0;
            c.parent = parent;
            c.level = level;
            sg = &c;
        }
        BFS_CUDA_TRY(cudaGraphLaunch(sg->exec, st));
        BFS_CUDA_TRY(cudaMemcpyAsync(W.h_counters, ctr, sizeof(uint64_t) * C_NUM, cudaMemcpyDeviceToHost, st));
        BFS_CUDA_TRY(cudaStreamSynchronize(st));
        const uint64_t* h = W.h_counters;
        if (h[C_ERROR] & 2ull) return set_error(BFS_ERR_INVALID_ARG, "trace capacity exceeded");
        if (h[C_ERROR])
            return set_error(BFS_ERR_CORRUPT, "device invariant check failed (code %llu)",
                             (unsigned long long)h[C_ERROR]);
        if (g->debug_checks) return check_outputs(L.n, root, parent, level, ctl, st);
        return BFS_OK;
    }

    int64_t frontier = 1;
    int64_t raw_bytes = 0;
    for (int j = 0; j < p; ++j) raw_bytes += 4 * ((L.range_len(j) + 31) / 32);
    raw_bytes *= p;
    for (int32_t k = 0;; ++k) {
        BFS_TRY(level_body(st, true, k, cudaGraphConditionalHandle{}));
        BFS_CUDA_TRY(cudaMemcpyAsync(W.h_counters, ctr, sizeof(uint64_t) * C_NUM, cudaMemcpyDeviceToHost, st));
        BFS_CUDA_TRY(cudaStreamSynchronize(st));
        const uint64_t* h = W.h_counters;
        if (h[C_ERROR] & 2ull) return set_error(BFS_ERR_INVALID_ARG, "trace capacity exceeded");
        if (h[C_ERROR])
            return set_error(BFS_ERR_CORRUPT, "device invariant check failed (code %llu) at level %d",
                             (unsigned long long)h[C_ERROR], k);
        if (stats->levels && k < stats->capacity_levels) {
            bfs_level_stats& ls = stats->levels[k];
            memset(&ls, 0, sizeof(ls));
            ls.frontier_vertices = frontier;
            ls.exchanged_vertices = (mode == BFS_MODE_COMPRESS_SIEVE) ? (int64_t)h[C_EXCHANGED] : p * frontier;
            ls.column_hits = (int64_t)h[C_HITS];
            ls.raw_bytes = raw_bytes;
            ls.wah_bytes = (mode == BFS_MODE_PLAIN) ? 0 : (int64_t)h[C_WAH_WORDS] * (wbits / 8);
            ls.edges_scanned = (int64_t)h[C_EDGES];
            ls.row_wah_bytes = (int64_t)h[C_ROW_WORDS] * (wbits / 8);
            ls.bottom_up = h[C_BOTTOM_UP] ? 1 : 0;
            ls.compress_chunks = (int64_t)h[C_ENC_CHUNKS];
            ls.row_compress_chunks = (int64_t)h[C_ROW_CHUNKS];
            if (timing) {
                ls.ms_compress_sieve = elapsed(W.ev[0], W.ev[1]);
                ls.ms_communication = elapsed(W.ev[1], W.ev[2]);
                ls.ms_traversing = elapsed(W.ev[2], W.ev[3]);
                ls.ms_row_compress = elapsed(W.ev[3], W.ev[5]);
                ls.ms_row_fold = elapsed(W.ev[5], W.ev[6]);
                ls.ms_reducing = elapsed(W.ev[6], W.ev[4]);
                ls.ms_directory_update = dynamic ? elapsed(W.ev[7], W.ev[0]) : 0.0f;
            }
        }
        stats->n_levels = k + 1;
        if (tracing) stats->trace_used = (int64_t)h[C_TRACE_USED];
        if (row_tracing) stats->row_trace_used = (int64_t)h[C_ROW_TRACE_USED];
        frontier = (int64_t)h[C_NEXT_COUNT];
        if (frontier == 0 || k + 1 >= max_levels) break;
    }
    if (g->debug_checks) return check_outputs(L.n, root, parent, level, ctl, st);
    return BFS_OK;
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" bfs_status bfs_check_search(bfs_graph_t g, int32_t root, const int32_t* parent, const int32_t* level,
                                       void* stream) {
    if (!g) return set_error(BFS_ERR_INVALID_ARG, "graph is NULL");
    if (root < 0 || (int64_t)root >= g->L.n) return set_error(BFS_ERR_INVALID_ARG, "root %d outside [0, %lld)", root, (long long)g->L.n);
    if (!is_device_pointer(parent) || !is_device_pointer(level))
        return set_error(BFS_ERR_INVALID_ARG, "parent and level must be device pointers");
    return check_outputs(g->L.n, root, parent, level, nullptr, static_cast<cudaStream_t>(stream));
}

extern "C" bfs_status bfs_run(bfs_graph_t g, int32_t root, int32_t* parent, int32_t* level, bfs_run_stats* stats,
                              void* stream) {
    if (!g) return set_error(BFS_ERR_INVALID_ARG, "graph is NULL");
    if (!parent || !level) return set_error(BFS_ERR_INVALID_ARG, "parent and level are required");
    if (root < 0 || (int64_t)root >= g->L.n) return set_error(BFS_ERR_INVALID_ARG, "root %d outside [0, %lld)", root, (long long)g->L.n);
    if (stats && stats->capacity_levels < 0) return set_error(BFS_ERR_INVALID_ARG, "negative capacity_levels");
    BusyGuard guard(g);
    if (!guard.ok) return set_error(BFS_ERR_BUSY, "another search on this graph is running");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool dev_p = is_device_pointer(parent), dev_l = is_device_pointer(level);
    if (dev_p != dev_l) return set_error(BFS_ERR_INVALID_ARG, "parent and level must both be host or both be device pointers");
    if (dev_p) {
        const bfs_status rs = run_search(g, root, parent, level, stats, st);
        if (rs != BFS_OK) g->W.tblk_dirty = true;     // the row partials may hold a level's marks
        return rs;
    }
    Workspace& W = g->W;
    if (!W.tmp_parent.ptr || !W.tmp_level.ptr) {
        bfs_status rc = W.tmp_parent.alloc(sizeof(int32_t) * g->L.n);
        if (rc == BFS_OK) rc = W.tmp_level.alloc(sizeof(int32_t) * g->L.n);
        if (rc != BFS_OK) { W.tmp_parent.release(); W.tmp_level.release(); return rc; }
    }
    {
        const bfs_status rs = run_search(g, root, W.tmp_parent.as<int32_t>(), W.tmp_level.as<int32_t>(), stats, st);
        if (rs != BFS_OK) { W.tblk_dirty = true; return rs; }
    }
    BFS_CUDA_TRY(cudaMemcpyAsync(parent, W.tmp_parent.ptr, sizeof(int32_t) * g->L.n, cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaMemcpyAsync(level, W.tmp_level.ptr, sizeof(int32_t) * g->L.n, cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    return BFS_OK;
}
