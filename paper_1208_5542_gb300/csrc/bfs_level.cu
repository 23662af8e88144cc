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
//                          by V_{i,j} and WAH-encoded (lines 9-10); block (i,j)
//                          decodes its stream (line 13) -- every decoded vertex
//                          has a nonempty column, so only its rank is looked up.
//   expansion (line 5):    for every decoded (u, block) item, every entry
//                          u -> v of its column: if v is not in pi, set t[v]
//                          and lower parent[v] to u (the (select, min) semiring).
//   reduce (lines 6-7):    t = t & ~pi; pi |= t; level[v] = k + 1 for v in t;
//                          |t| counted on the device; f <- t.
// The exchange itself (line 11) is the identity on one GPU: the receive buffer
// g' is the send buffer in HBM; its sizes are scanned for the statistics and
// packed into the caller's trace when one is requested.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"
#include "wah.cuh"

namespace bfsgb {

bfs_status launch_wah_encode_counted(const EncodeArgs& a, int wah_bits, unsigned long long* setbits,
                                     cudaStream_t st);

namespace {

constexpr int kNT = 256;
constexpr int kChunkWords = 1024;     // stream words per expansion unit (4 per thread)
constexpr int kWordsPerThread = kChunkWords / kNT;
constexpr int kPlainUnitWords = kNT;  // raw 32-bit frontier words per PLAIN unit

struct Unit {
    int32_t block;
    int32_t stream;
    int64_t word0;
    int64_t gbase;
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
    Unit* units;
    Item* pieces;
    int64_t piece_cap;
    unsigned long long* ctr;
    int sieve;                // 1: DIR-WAH streams (no directory test at the receiver)
    int nstreams;
};

__device__ __forceinline__ int64_t range_begin(const LevelArgs& a, int64_t b) {
    const int64_t x = b * a.nb;
    return x < a.n ? x : a.n;
}

// Visit entry u -> v of the expansion: if v was not visited before this
// level, lower parent[v] to u and set t[v].  Both updates are reductions whose
// results are not used (fire-and-forget at L2); the only dependent load is the
// visited word, read through the read-only path (pi does not change during the
// expansion).
__device__ __forceinline__ void visit(const LevelArgs& a, int32_t v, int32_t u) {
    const uint32_t w = (uint32_t)v >> 5;
    const uint32_t m = 1u << ((uint32_t)v & 31u);
    if (__ldg(a.pi + w) & m) return;
    atomicMin(reinterpret_cast<unsigned int*>(a.parent) + v, (unsigned int)u);   // -1 is the largest unsigned
    atomicOr(a.t + w, m);
}

constexpr uint32_t kHub = 1024;     // columns longer than this are cut into pieces
constexpr uint32_t kPiece = 1024;   // entries per piece

// Expand one item per lane (u, offset of its column in ir, length; length 0 =
// none).  Columns longer than kHub go to the piece list; the rest are expanded
// by the warp with a load-balanced search over the lanes' entry counts, so
// every lane reads one entry per step and a step covers 32 consecutive entries
// of the concatenated columns.
__device__ __forceinline__ void warp_expand(const LevelArgs& a, int32_t u, int64_t beg, uint32_t len,
                                            unsigned long long& edges, unsigned long long& hits) {
    const uint32_t lane = lane_id();
    hits += (len > 0);
    if (__any_sync(0xffffffffu, len > kHub)) {
        if (len > kHub) {
            const uint32_t np = (len + kPiece - 1) / kPiece;
            const unsigned long long base = atomicAdd(a.ctr + C_PIECES, (unsigned long long)np);
            if (base + np <= (unsigned long long)a.piece_cap) {
                for (uint32_t k = 0; k < np; ++k) {
                    Item it;
                    it.u = u;
                    it.len = (len - k * kPiece < kPiece) ? len - k * kPiece : kPiece;
                    it.begin = beg + (int64_t)k * kPiece;
                    a.pieces[base + k] = it;
                }
            } else {
                atomicOr(a.ctr + C_ERROR, 8ull);        // piece list overflow (cannot happen by the bound)
            }
            len = 0;
        }
    }
    const uint32_t incl = warp_incl_sum(len);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - len;
    edges += len;
    for (uint32_t e0 = 0; e0 < total; e0 += 32) {
        const uint32_t e = e0 + lane;
        // owner: the first lane whose inclusive count exceeds e
        int lo = 0, hi = 31;
#pragma unroll
        for (int step = 0; step < 5; ++step) {
            const int mid = (lo + hi) >> 1;
            const uint32_t im = __shfl_sync(0xffffffffu, incl, mid);
            if (im > e) hi = mid; else lo = mid + 1;
        }
        const int o = lo;
        const int64_t ob = __shfl_sync(0xffffffffu, beg, o);
        const uint32_t oe = __shfl_sync(0xffffffffu, excl, o);
        const int32_t ou = __shfl_sync(0xffffffffu, u, o);
        if (e < total) {
            const int32_t v = __ldg(a.ir + ob + (int64_t)(e - oe));
            visit(a, v, ou);
        }
    }
}

// Column of source u_local in block b: (offset into ir, len); len 0 if empty.
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

__device__ __forceinline__ void flush_counts(const LevelArgs& a, unsigned long long edges, unsigned long long hits) {
    edges = warp_sum(edges);
    hits = warp_sum(hits);
    if (lane_id() == 0) {
        if (edges) atomicAdd(a.ctr + C_EDGES, edges);
        if (hits) atomicAdd(a.ctr + C_HITS, hits);
    }
}

// Pieces of long columns: one warp per piece, 32 consecutive entries per step.
__global__ void __launch_bounds__(kNT) expand_pieces(LevelArgs a) {
    const int64_t np = (int64_t)*reinterpret_cast<volatile unsigned long long*>(a.ctr + C_PIECES);
    const int64_t lim = np < a.piece_cap ? np : a.piece_cap;
    const int64_t gw0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t gws = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t pc = gw0; pc < lim; pc += gws) {
        const Item it = a.pieces[pc];
        uint32_t e = lane_id();
        for (; e + 96 < it.len; e += 128) {
            const int32_t v0 = __ldg(a.ir + it.begin + e);
            const int32_t v1 = __ldg(a.ir + it.begin + e + 32);
            const int32_t v2 = __ldg(a.ir + it.begin + e + 64);
            const int32_t v3 = __ldg(a.ir + it.begin + e + 96);
            visit(a, v0, it.u);
            visit(a, v1, it.u);
            visit(a, v2, it.u);
            visit(a, v3, it.u);
        }
        for (; e < it.len; e += 32) visit(a, __ldg(a.ir + it.begin + e), it.u);
    }
}

// ------------------------------------------------------------------ PLAIN --
// Unit = (block b, 256 raw frontier words of range j).  Thread t reads word t
// and keeps the bits whose column is nonempty (word-wise AND with V_{i,j}, the
// column index of the block); the warps then expand the unit's items.
__global__ void __launch_bounds__(kNT) expand_plain(LevelArgs a, int64_t units_per_block) {
    __shared__ uint32_t s_word[kNT];
    __shared__ uint32_t s_excl[kNT];
    __shared__ unsigned long long red[kNT / 32 + 1];
    const int64_t nunits = (int64_t)a.p * a.p * units_per_block;
    unsigned long long edges = 0, hits = 0;
    for (int64_t unit = blockIdx.x; unit < nunits; unit += gridDim.x) {
        const int64_t b = unit / units_per_block, c = unit % units_per_block;
        const int64_t j = b % a.p;
        const int64_t jb = range_begin(a, j), jl = range_begin(a, j + 1) - jb;
        const int64_t w = c * kPlainUnitWords + threadIdx.x;     // word of the slice
        uint32_t x = 0;
        if (w * 32 < jl) {
            x = bits32_at_cg(a.f, (uint64_t)(jb + w * 32));
            const int64_t left = jl - w * 32;
            if (left < 32) x &= (1u << left) - 1u;
            if (x) x &= __ldg(a.dir + b * a.dir_stride + w);
        }
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan<kNT>((unsigned long long)__popc(x), 0ull, OpSum(), red, &tot);
        if (tot == 0) continue;                                   // uniform
        s_word[threadIdx.x] = x;
        s_excl[threadIdx.x] = (uint32_t)ex;
        __syncthreads();
        if (threadIdx.x == 0) atomicAdd(a.ctr + C_ITEMS, tot);
        const BlockView bv = block_view(a, b);
        for (uint64_t q0 = (threadIdx.x & ~31u); q0 < tot; q0 += kNT) {
            const uint64_t q = q0 + lane_id();
            int32_t u = 0;
            int64_t begin = 0;
            uint32_t len = 0;
            if (q < tot) {
                int lo = 0, hi = kNT - 1;                          // last word with excl <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_excl[mid] <= q) lo = mid; else hi = mid - 1;
                }
                const int bitpos = select32(s_word[lo], (int)(q - s_excl[lo]));
                const int64_t ul = ((int64_t)c * kPlainUnitWords + lo) * 32 + bitpos;
                column_of(a, bv, ul, false, &begin, &len);
                u = (int32_t)(jb + ul);
            }
            warp_expand(a, u, begin, len, edges, hits);
        }
        __syncthreads();
    }
    flush_counts(a, edges, hits);
}

// -------------------------------------------------------------------- WAH --
// Per stream: group base of every chunk of kChunkWords words, and the units
// (block, stream, chunk) of the expansion.  One CTA per stream.
template <typename W>
__global__ void __launch_bounds__(kNT) stream_chunks(LevelArgs a) {
    __shared__ unsigned long long red[kNT / 32 + 1];
    __shared__ int64_t s_base;
    const int s = blockIdx.x;
    const W* in = static_cast<const W*>(a.xbuf) + (int64_t)s * a.slot_cap;
    const int64_t count = a.xcount[s];
    const int64_t nch = (count + kChunkWords - 1) / kChunkWords;
    unsigned long long gpos = 0;
    for (int64_t ch = 0; ch < nch; ++ch) {
        unsigned long long g = 0;
        for (int k = 0; k < kWordsPerThread; ++k) {
            const int64_t x = ch * kChunkWords + (int64_t)k * kNT + threadIdx.x;
            if (x < count) g += word_groups<W>(in[x]);
        }
        if (threadIdx.x == 0) a.chunk_base[(int64_t)s * a.chunks_per_slot + ch] = (int64_t)gpos;
        unsigned long long tot;
        block_excl_scan<kNT>(g, 0ull, OpSum(), red, &tot);
        gpos += tot;
    }
    const int copies = a.sieve ? 1 : a.p;       // COMPRESS: every block-row decodes stream j
    if (threadIdx.x == 0) {
        s_base = (int64_t)atomicAdd(a.ctr + C_UNITS, (unsigned long long)(nch * copies));
        atomicAdd(a.ctr + C_WAH_WORDS, (unsigned long long)count);
    }
    __syncthreads();
    for (int64_t q = threadIdx.x; q < nch * copies; q += kNT) {
        const int64_t ch = q % nch, i = q / nch;
        Unit un;
        un.block = a.sieve ? s : (int32_t)(i * a.p + s);
        un.stream = s;
        un.word0 = ch * kChunkWords;
        un.gbase = a.chunk_base[(int64_t)s * a.chunks_per_slot + ch];
        a.units[s_base + q] = un;
    }
}

// Fused decode + expansion of the units: words of one chunk -> (u, block)
// items -> entries.
template <typename W>
__global__ void __launch_bounds__(kNT) expand_wah(LevelArgs a) {
    using T = Wah<W>;
    constexpr int GB = T::GB;
    __shared__ W s_y[kChunkWords];
    __shared__ int64_t s_gs[kChunkWords];
    __shared__ uint32_t s_iex[kChunkWords];
    __shared__ unsigned long long red[kNT / 32 + 1];
    const int64_t nunits = (int64_t)*reinterpret_cast<volatile unsigned long long*>(a.ctr + C_UNITS);
    unsigned long long edges = 0, hits = 0;
    for (int64_t ui = blockIdx.x; ui < nunits; ui += gridDim.x) {
        const Unit un = a.units[ui];
        const int64_t b = un.block;
        const int64_t j = b % a.p;
        const int64_t jb = range_begin(a, j), jl = range_begin(a, j + 1) - jb;
        const int64_t G = jl / GB;
        const int r = (int)(jl % GB);
        const W* in = static_cast<const W*>(a.xbuf) + (int64_t)un.stream * a.slot_cap;
        const int64_t count = a.xcount[un.stream];
        // this thread's words: blocked, kWordsPerThread consecutive words
        W y[kWordsPerThread];
        unsigned long long glen[kWordsPerThread];
        unsigned long long gsum = 0;
#pragma unroll
        for (int k = 0; k < kWordsPerThread; ++k) {
            const int64_t x = un.word0 + (int64_t)threadIdx.x * kWordsPerThread + k;
            y[k] = (x < count) ? in[x] : W(0);
            glen[k] = (x < count) ? word_groups<W>(y[k]) : 0ull;
            gsum += glen[k];
        }
        unsigned long long tot;
        unsigned long long gs = (unsigned long long)un.gbase +
                                block_excl_scan<kNT>(gsum, 0ull, OpSum(), red, &tot);
        unsigned long long icount = 0;
        uint32_t ic[kWordsPerThread];
#pragma unroll
        for (int k = 0; k < kWordsPerThread; ++k) {
            const int64_t x = un.word0 + (int64_t)threadIdx.x * kWordsPerThread + k;
            uint32_t c = 0;
            if (x < count) {
                if (gs < (unsigned long long)G) {
                    if (is_fill<W>(y[k])) c = (y[k] & T::VAL) ? (uint32_t)(glen[k] * GB) : 0u;
                    else c = (uint32_t)T::popc(T::from_payload(y[k]));
                } else if (r > 0) {
                    c = (uint32_t)T::popc(T::from_active(y[k], r));      // the active word
                    glen[k] = 0;
                }
            }
            ic[k] = c;
            s_y[threadIdx.x * kWordsPerThread + k] = y[k];
            s_gs[threadIdx.x * kWordsPerThread + k] = (int64_t)gs;
            gs += glen[k];
            icount += c;
        }
        unsigned long long items;
        unsigned long long iex = block_excl_scan<kNT>(icount, 0ull, OpSum(), red, &items);
#pragma unroll
        for (int k = 0; k < kWordsPerThread; ++k) {
            s_iex[threadIdx.x * kWordsPerThread + k] = (uint32_t)iex;
            iex += ic[k];
        }
        __syncthreads();
        if (threadIdx.x == 0 && items) atomicAdd(a.ctr + C_ITEMS, items);
        const BlockView bv = block_view(a, b);
        for (uint64_t q0 = (threadIdx.x & ~31u); q0 < items; q0 += kNT) {
            const uint64_t q = q0 + lane_id();
            int32_t u = 0;
            int64_t begin = 0;
            uint32_t len = 0;
            if (q < items) {
                int lo = 0, hi = kChunkWords - 1;                  // last word with iex <= q
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (s_iex[mid] <= q) lo = mid; else hi = mid - 1;
                }
                // words with no items share the same iex: step back over none (lo is the last
                // word with iex <= q; it has items because q < next word's iex)
                const W yy = s_y[lo];
                const int64_t g0 = s_gs[lo];
                const int kk = (int)(q - s_iex[lo]);
                int64_t ul;
                if (g0 >= G) ul = G * GB + T::select(T::from_active(yy, r), kk);
                else if (is_fill<W>(yy)) ul = g0 * GB + kk;
                else ul = g0 * GB + T::select(T::from_payload(yy), kk);
                column_of(a, bv, ul, !a.sieve, &begin, &len);
                u = (int32_t)(jb + ul);
            }
            warp_expand(a, u, begin, len, edges, hits);
        }
        __syncthreads();
    }
    flush_counts(a, edges, hits);
}

// ---------------------------------------------------------------- reduce --
// t = t & ~pi; pi |= t; level of the new vertices; |t|; clear the old
// frontier (it becomes the next t); frontier summary of t.
__global__ void __launch_bounds__(kNT) reduce_level(uint32_t* __restrict__ t, uint32_t* __restrict__ pi,
                                                    uint32_t* __restrict__ f_old, uint8_t* __restrict__ fsum,
                                                    int64_t words, int64_t n, int32_t* __restrict__ level,
                                                    int32_t next_level, unsigned long long* ctr) {
    const int64_t nwarps = (words + 31) / 32;
    const int64_t gw0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t gstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gw = gw0; gw < nwarps; gw += gstride) {
        const int64_t w = gw * 32 + lane_id();
        uint32_t x = 0;
        if (w < words) {
            x = t[w] & ~pi[w];
            if (x) {
                pi[w] |= x;
                uint32_t y = x;
                while (y) {
                    const int bpos = __ffs(y) - 1;
                    y &= y - 1;
                    const int64_t v = w * 32 + bpos;
                    if (v < n) level[v] = next_level;
                }
            }
            t[w] = x;
            f_old[w] = 0u;
        }
        const uint32_t any = __ballot_sync(0xffffffffu, x != 0u);
        const int cnt = warp_sum(__popc(x));
        if (lane_id() == 0) {
            fsum[gw] = any ? 1 : 0;
            if (cnt) atomicAdd(ctr + C_NEXT_COUNT, (unsigned long long)cnt);
        }
    }
}

__global__ void init_search(int32_t* __restrict__ level, int32_t* __restrict__ parent, int64_t n,
                            uint32_t* __restrict__ pi, uint32_t* __restrict__ fa, uint32_t* __restrict__ fb,
                            int64_t words, uint8_t* __restrict__ fsum, int64_t fsum_len) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        level[v] = -1;
        parent[v] = -1;
    }
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words; w += stride) {
        pi[w] = 0u;
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

// Pack the streams of this exchange into the trace (receive buffer g').
__global__ void __launch_bounds__(kNT) trace_offsets(const int64_t* __restrict__ counts, int nslots, int u32_per_word,
                                                     int64_t* __restrict__ slot_off, int64_t* __restrict__ trace_counts,
                                                     unsigned long long* ctr, int64_t capacity) {
    __shared__ unsigned long long red[kNT / 32 + 1];
    const unsigned long long used = ctr[C_TRACE_USED];
    unsigned long long carry = 0;
    for (int s0 = 0; s0 < nslots; s0 += kNT) {
        const int s = s0 + threadIdx.x;
        const unsigned long long c = (s < nslots) ? (unsigned long long)counts[s] * u32_per_word : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan<kNT>(c, 0ull, OpSum(), red, &tot);
        if (s < nslots) {
            slot_off[s] = (int64_t)(used + carry + ex);
            trace_counts[s] = counts[s];
        }
        carry += tot;
    }
    if (threadIdx.x == 0) {
        if (used + carry > (unsigned long long)capacity) {
            ctr[C_ERROR] |= 2ull;                 // trace overflow
            ctr[C_TRACE_USED] = (unsigned long long)capacity + 1;
        } else {
            ctr[C_TRACE_USED] = used + carry;
        }
    }
}

__global__ void trace_copy(const uint32_t* __restrict__ xbuf, int64_t slot_cap_u32, const int64_t* __restrict__ counts,
                           int u32_per_word, const int64_t* __restrict__ slot_off, uint32_t* __restrict__ trace,
                           int64_t capacity) {
    const int s = blockIdx.y;
    const int64_t c = counts[s] * u32_per_word;
    const int64_t off = slot_off[s];
    if (off + c > capacity) return;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < c; x += (int64_t)gridDim.x * blockDim.x)
        trace[off + x] = xbuf[(int64_t)s * slot_cap_u32 + x];
}

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

}  // namespace

// ------------------------------------------------------------- workspace --
bfs_status ensure_workspace(bfs_graph* g, cudaStream_t st) {
    (void)st;
    Workspace& W = g->W;
    const Layout& L = g->L;
    if (W.bm_words) return BFS_OK;
    const int64_t p2 = (int64_t)L.p * L.p;
    W.bm_words = ((L.n + 31) / 32 + 4 + 3) / 4 * 4;
    W.fsum_len = (W.bm_words + 31) / 32 + 64;
    const int64_t cap32 = L.nb / 31 + 2, cap64 = L.nb / 63 + 2;
    W.slot_cap = cap32;                                   // in words of the current width (set per run)
    W.chunk_words = kChunkWords;
    W.chunks_per_slot = (cap32 + kChunkWords - 1) / kChunkWords;
    const int64_t xbytes = p2 * std::max<int64_t>(4 * cap32, 8 * cap64);
    BFS_TRY(W.pi.alloc(4 * W.bm_words));
    BFS_TRY(W.fa.alloc(4 * W.bm_words));
    BFS_TRY(W.fb.alloc(4 * W.bm_words));
    BFS_TRY(W.fsum.alloc(W.fsum_len));
    BFS_TRY(W.xbuf.alloc(xbytes));
    BFS_TRY(W.xcount.alloc(sizeof(int64_t) * p2));
    BFS_TRY(W.chunk_base.alloc(sizeof(int64_t) * p2 * W.chunks_per_slot));
    BFS_TRY(W.units.alloc(sizeof(Unit) * p2 * W.chunks_per_slot));
    BFS_TRY(W.counters.alloc(sizeof(unsigned long long) * C_NUM));
    // pieces: sum over long columns of ceil(len/kPiece) <= nnz/kPiece + nnz/kHub
    W.piece_cap = L.nnz / kPiece + L.nnz / kHub + 16;
    BFS_TRY(W.pieces.alloc(sizeof(Item) * W.piece_cap));
    if (!W.h_counters) {
        void* h = nullptr;
        BFS_CUDA_TRY(cudaMallocHost(&h, sizeof(uint64_t) * C_NUM));
        W.h_counters = static_cast<uint64_t*>(h);
    }
    if (!W.events) {
        for (auto& e : W.ev) BFS_CUDA_TRY(cudaEventCreate(&e));
        W.events = true;
    }
    return BFS_OK;
}

void free_workspace(bfs_graph* g) {
    Workspace& W = g->W;
    W.pi.release(); W.fa.release(); W.fb.release(); W.fsum.release(); W.xbuf.release();
    W.xcount.release(); W.chunk_base.release(); W.units.release(); W.counters.release(); W.pieces.release();
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
    const int grid = sm_count() * 8;
    DevBuf slot_off;
    if (tracing) BFS_TRY(slot_off.alloc(sizeof(int64_t) * nslots));
    if (stats) { stats->n_levels = 0; stats->trace_used = 0; }

    init_search<<<sm_count() * 4, kNT, 0, st>>>(level, parent, L.n, W.pi.as<uint32_t>(), W.fa.as<uint32_t>(),
                                                W.fb.as<uint32_t>(), W.bm_words, W.fsum.as<uint8_t>(), W.fsum_len);
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
    a.units = static_cast<Unit*>(W.units.ptr);
    a.pieces = W.pieces.as<Item>();
    a.piece_cap = W.piece_cap;
    a.ctr = ctr;
    a.sieve = (mode == BFS_MODE_COMPRESS_SIEVE);
    a.nstreams = nslots;

    EncodeArgs ea;
    memset(&ea, 0, sizeof(ea));
    ea.dir = (mode == BFS_MODE_COMPRESS_SIEVE) ? L.dir.as<uint32_t>() : nullptr;
    ea.dir_stride = L.dir_stride;
    ea.p = p;
    ea.nb = L.nb;
    ea.n = L.n;
    ea.sieve = a.sieve;
    ea.nslots = nslots;
    ea.fsum = W.fsum.as<uint8_t>();
    ea.out = W.xbuf.ptr;
    ea.slot_cap = slot_cap;
    ea.counts = W.xcount.as<int64_t>();

    uint32_t* f = W.fa.as<uint32_t>();
    uint32_t* t = W.fb.as<uint32_t>();
    int64_t frontier = 1;
    int64_t raw_bytes = 0;
    for (int j = 0; j < p; ++j) raw_bytes += 4 * ((L.range_len(j) + 31) / 32);
    raw_bytes *= p;
    const int64_t units_per_block = (L.nb + 32LL * kPlainUnitWords - 1) / (32LL * kPlainUnitWords);

    for (int32_t k = 0;; ++k) {
        if (k > 0) {   // per-level counters; the error flag and the trace cursor persist
            BFS_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(unsigned long long) * C_ERROR, st));
            BFS_CUDA_TRY(cudaMemsetAsync(ctr + C_WAH_WORDS, 0, sizeof(unsigned long long) * (C_NUM - C_WAH_WORDS), st));
        }
        a.f = f;
        a.t = t;
        ea.frontier = f;
        if (timing) cudaEventRecord(W.ev[0], st);
        if (mode == BFS_MODE_PLAIN) {
            if (timing) { cudaEventRecord(W.ev[1], st); cudaEventRecord(W.ev[2], st); }
            expand_plain<<<grid, kNT, 0, st>>>(a, units_per_block);
            BFS_CUDA_TRY(cudaGetLastError());
        } else {
            BFS_TRY(launch_wah_encode_counted(ea, wbits, ctr + C_EXCHANGED, st));
            if (wbits == 32) stream_chunks<uint32_t><<<nslots, kNT, 0, st>>>(a);
            else stream_chunks<unsigned long long><<<nslots, kNT, 0, st>>>(a);
            BFS_CUDA_TRY(cudaGetLastError());
            if (timing) cudaEventRecord(W.ev[1], st);
            if (tracing && k < stats->capacity_levels) {
                const int u32pw = wbits / 32;
                trace_offsets<<<1, kNT, 0, st>>>(W.xcount.as<int64_t>(), nslots, u32pw, slot_off.as<int64_t>(),
                                                 stats->trace_counts + (int64_t)k * nslots, ctr,
                                                 stats->trace_capacity);
                dim3 tg(8, nslots);
                trace_copy<<<tg, kNT, 0, st>>>(W.xbuf.as<uint32_t>(), slot_cap * u32pw, W.xcount.as<int64_t>(), u32pw,
                                               slot_off.as<int64_t>(), stats->trace_words, stats->trace_capacity);
                BFS_CUDA_TRY(cudaGetLastError());
            }
            if (timing) cudaEventRecord(W.ev[2], st);
            if (wbits == 32) expand_wah<uint32_t><<<grid, kNT, 0, st>>>(a);
            else expand_wah<unsigned long long><<<grid, kNT, 0, st>>>(a);
            BFS_CUDA_TRY(cudaGetLastError());
        }
        expand_pieces<<<grid, kNT, 0, st>>>(a);
        BFS_CUDA_TRY(cudaGetLastError());
        if (timing) cudaEventRecord(W.ev[3], st);
        reduce_level<<<std::min<int64_t>((W.bm_words + 255) / 256 + 1, sm_count() * 16), kNT, 0, st>>>(
            t, W.pi.as<uint32_t>(), f, W.fsum.as<uint8_t>(), W.bm_words, L.n, level, k + 1, ctr);
        BFS_CUDA_TRY(cudaGetLastError());
        if (timing) cudaEventRecord(W.ev[4], st);
        BFS_CUDA_TRY(cudaMemcpyAsync(W.h_counters, ctr, sizeof(uint64_t) * C_NUM, cudaMemcpyDeviceToHost, st));
        BFS_CUDA_TRY(cudaStreamSynchronize(st));
        const uint64_t* h = W.h_counters;
        if (h[C_ERROR] & 2ull) return set_error(BFS_ERR_INVALID_ARG, "trace capacity exceeded");
        if (h[C_ERROR]) return set_error(BFS_ERR_CORRUPT, "device invariant check failed (code %llu)",
                                         (unsigned long long)h[C_ERROR]);
        if (stats) {
            if (stats->levels && k < stats->capacity_levels) {
                bfs_level_stats& ls = stats->levels[k];
                memset(&ls, 0, sizeof(ls));
                ls.frontier_vertices = frontier;
                ls.exchanged_vertices = (mode == BFS_MODE_COMPRESS_SIEVE) ? (int64_t)h[C_EXCHANGED] : p * frontier;
                ls.column_hits = (int64_t)h[C_HITS];
                ls.raw_bytes = raw_bytes;
                ls.wah_bytes = (mode == BFS_MODE_PLAIN) ? 0 : (int64_t)h[C_WAH_WORDS] * (wbits / 8);
                ls.edges_scanned = (int64_t)h[C_EDGES];
                if (timing) {
                    ls.ms_compress_sieve = elapsed(W.ev[0], W.ev[1]);
                    ls.ms_communication = elapsed(W.ev[1], W.ev[2]);
                    ls.ms_traversing = elapsed(W.ev[2], W.ev[3]);
                    ls.ms_reducing = elapsed(W.ev[3], W.ev[4]);
                }
            }
            stats->n_levels = k + 1;
            if (tracing) stats->trace_used = (int64_t)h[C_TRACE_USED];
        }
        frontier = (int64_t)h[C_NEXT_COUNT];
        if (frontier == 0) break;
        std::swap(f, t);
    }
    return BFS_OK;
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

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
    if (dev_p) return run_search(g, root, parent, level, stats, st);
    Workspace& W = g->W;
    if (!W.tmp_parent.ptr) {
        BFS_TRY(W.tmp_parent.alloc(sizeof(int32_t) * g->L.n));
        BFS_TRY(W.tmp_level.alloc(sizeof(int32_t) * g->L.n));
    }
    BFS_TRY(run_search(g, root, W.tmp_parent.as<int32_t>(), W.tmp_level.as<int32_t>(), stats, st));
    BFS_CUDA_TRY(cudaMemcpyAsync(parent, W.tmp_parent.ptr, sizeof(int32_t) * g->L.n, cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaMemcpyAsync(level, W.tmp_level.ptr, sizeof(int32_t) * g->L.n, cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    return BFS_OK;
}
