// wah.cu -- WAH compress (Sec. IV, Table 3; the compress steps of Alg. 2 and 3),
// fused with the cross-directory sieve (Alg. 3, Sec. V-A), and the standalone
// codec entry points of the C ABI.
//
// Encoder: one CTA per exchange slot walks the slot's groups in tiles of
// kTile groups.  Inside a tile every thread classifies kK consecutive groups
// (all-zero / all-one / literal); a block scan of "head" flags (a literal, or
// a group whose type differs from its predecessor) gives every word its index,
// and a block max-scan of head positions gives every group the start of its
// run, so the group that ends a fill run writes the merged fill word.  The open
// run, the word count and the previous type carry from tile to tile.  Tiles
// whose frontier bits are all zero (frontier summary: one byte per 1024 bits)
// are skipped without loading a word.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "internal.h"
#include "wah.cuh"

namespace bfsgb {
namespace {

constexpr int kNT = 256;          // threads per encoder CTA
constexpr int kK = 4;             // groups per thread per tile
constexpr int kTile = kNT * kK;   // groups per tile
static_assert(kTile == kEncChunkGroups, "the encoder's chunk is the unit of its chunk index");

struct SlotGeom {
    int64_t src0;      // first bitmap bit of the slot's source range
    int64_t nbits;     // bits in the slot
    const uint32_t* dirb;   // directory of the slot's block, or nullptr
};

__device__ __forceinline__ SlotGeom slot_geom(const EncodeArgs& a, int s) {
    const int j = a.sieve ? (a.row_slots ? (int)((uint32_t)s / (uint32_t)a.p) : (int)((uint32_t)s % (uint32_t)a.p))
                          : s;
    int64_t b0 = (int64_t)j * a.nb, b1 = b0 + a.nb;
    if (b0 > a.n) b0 = a.n;
    if (b1 > a.n) b1 = a.n;
    SlotGeom g;
    g.src0 = b0;
    g.nbits = b1 - b0;
    g.dirb = a.sieve ? a.dir + (int64_t)s * a.dir_stride : nullptr;
    return g;
}

// True if the frontier-summary bytes q0..q1 (inclusive) are all zero; the
// summary is padded to whole 32-bit words.
__device__ __forceinline__ bool fsum_zero(const uint8_t* fsum, int64_t q0, int64_t q1) {
    const uint32_t* w = reinterpret_cast<const uint32_t*>(fsum);
    const int64_t a = q0 >> 2, b = q1 >> 2;
    for (int64_t i = a; i <= b; ++i) {
        uint32_t x = __ldcg(w + i);
        if (i == a) x &= 0xffffffffu << (8 * (q0 & 3));
        if (i == b) x &= 0xffffffffu >> (8 * (3 - (q1 & 3)));
        if (x) return false;
    }
    return true;
}

template <typename W>
__device__ __forceinline__ W load_group(const EncodeArgs& a, const SlotGeom& sg, int64_t g) {
    W x = Wah<W>::group(a.frontier, (uint64_t)(sg.src0 + g * Wah<W>::GB));
    if (sg.dirb && x) x &= Wah<W>::group(sg.dirb, (uint64_t)(g * Wah<W>::GB));
    return x;
}

template <typename W>
__global__ void __launch_bounds__(kNT) wah_encode_kernel(EncodeArgs a, unsigned long long* setbits) {
    using T = Wah<W>;
    constexpr int GB = T::GB;
    const int s = blockIdx.x;
    const SlotGeom sg = slot_geom(a, s);
    const int64_t G = sg.nbits / GB;
    const int r = (int)(sg.nbits % GB);
    W* out = static_cast<W*>(a.out) + (int64_t)s * a.slot_cap;

    __shared__ int64_t sm64[kNT / 32 + 1];
    __shared__ unsigned long long smu[kNT / 32 + 1];
    __shared__ uint8_t sm_first[kNT], sm_last[kNT];
    __shared__ int sm_flag;
    __shared__ int sm_next_type;
    __shared__ int sm_carry_type;
    __shared__ int64_t sm_carry_start;

    int64_t nw = 0;            // words assigned so far (the open run's word included)
    int prev_type = -1;        // type of the group before the tile (-1: none)
    int64_t run_start = 0;     // start group of the run holding the group before the tile
    unsigned long long ones = 0;

    for (int64_t tb = 0; tb < G;) {
        int64_t tend = (tb + kTile < G) ? tb + kTile : G;
        // ---- zero skip from the frontier summary: lane l of warp 0 tests tile
        // tb + l*kTile; a run of leading all-zero tiles extends the zero fill ----
        if (a.fsum) {
            if (threadIdx.x < 32) {
                const int64_t t0 = tb + (int64_t)lane_id() * kTile;
                bool zero = false;
                if (t0 < G) {
                    const int64_t t1 = (t0 + kTile < G) ? t0 + kTile : G;
                    zero = fsum_zero(a.fsum, (sg.src0 + t0 * GB) >> 10, (sg.src0 + t1 * GB - 1) >> 10);
                }
                const uint32_t zmask = __ballot_sync(0xffffffffu, zero);
                if (threadIdx.x == 0) sm_flag = __ffs(~zmask) - 1;      // leading zero tiles (0..31)
                if (threadIdx.x == 0 && zmask == 0xffffffffu) sm_flag = 32;
            }
            __syncthreads();
            const int nz = sm_flag;
            __syncthreads();
            if (nz > 0) {
                const int64_t skip_end = (tb + (int64_t)nz * kTile < G) ? tb + (int64_t)nz * kTile : G;
                if (prev_type != G_ZERO) { nw += 1; run_start = tb; prev_type = G_ZERO; }
                if (skip_end == G && threadIdx.x == 0) out[nw - 1] = fill_word<W>(G_ZERO, (uint64_t)(G - run_start));
                tb = skip_end;
                continue;
            }
        }
        // ---- classify this thread's groups ----
        const int64_t g0 = tb + (int64_t)threadIdx.x * kK;
        W x[kK];
        int ty[kK];
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            const int64_t g = g0 + k;
            if (g < tend) {
                x[k] = load_group<W>(a, sg, g);
                ty[k] = group_type<W>(x[k]);
                ones += (unsigned long long)T::popc(x[k]);
            } else {
                x[k] = W(0);
                ty[k] = G_NONE;
            }
        }
        // a zero run carried into this tile (possibly across skipped tiles) ends
        // here if the tile opens with another type: write its fill word (when the
        // run ended in a processed tile the same word was already written there)
        if (threadIdx.x == 0 && prev_type == G_ZERO && ty[0] != G_ZERO)
            out[nw - 1] = fill_word<W>(G_ZERO, (uint64_t)(tb - run_start));
        sm_first[threadIdx.x] = (uint8_t)ty[0];
        sm_last[threadIdx.x] = (uint8_t)ty[kK - 1];
        if (threadIdx.x == 0) sm_next_type = (tend < G) ? group_type<W>(load_group<W>(a, sg, tend)) : G_NONE;
        __syncthreads();
        const int prev0 = (threadIdx.x == 0) ? prev_type : (int)sm_last[threadIdx.x - 1];
        // heads and last head position of this thread
        bool h[kK];
        int hc = 0;
        int64_t lastpos = -1;
        int pt = prev0;
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            h[k] = (ty[k] != G_NONE) && (ty[k] == G_LIT || ty[k] != pt);
            if (h[k]) { ++hc; lastpos = g0 + k; }
            pt = ty[k];
        }
        int64_t tot_h;
        const int64_t excl_h = block_excl_scan<kNT>((int64_t)hc, (int64_t)0, OpSum(), sm64, &tot_h);
        int64_t dummy;
        const int64_t excl_pos = block_excl_scan<kNT>(lastpos, (int64_t)-1, OpMax(), sm64, &dummy);
        // ---- write literals and the fill words of runs that end here ----
        int64_t cur_start = excl_pos > run_start ? excl_pos : run_start;
        int64_t widx = nw + excl_h - 1;
#pragma unroll
        for (int k = 0; k < kK; ++k) {
            const int64_t g = g0 + k;
            if (ty[k] == G_NONE) break;
            if (h[k]) { cur_start = g; ++widx; }
            int nt;
            if (k + 1 < kK) nt = ty[k + 1];
            else nt = (threadIdx.x + 1 < kNT) ? (int)sm_first[threadIdx.x + 1] : G_NONE;
            if (g + 1 == tend) nt = sm_next_type;
            if (ty[k] == G_LIT) {
                out[widx] = T::to_payload(x[k]);
            } else if (nt != ty[k]) {
                out[widx] = fill_word<W>(ty[k], (uint64_t)(g - cur_start + 1));
            }
            if (g + 1 == tend) { sm_carry_type = ty[k]; sm_carry_start = cur_start; }
        }
        __syncthreads();
        nw += tot_h;
        prev_type = sm_carry_type;
        run_start = sm_carry_start;
        __syncthreads();
        tb = tend;
    }
    if (setbits) {
        unsigned long long tot;
        block_excl_scan<kNT>(ones, 0ull, OpSum(), smu, &tot);
        if (threadIdx.x == 0 && tot) atomicAdd(setbits, tot);
    }
    if (threadIdx.x == 0) {
        int64_t total = nw;
        if (r > 0) {
            const uint64_t pos = (uint64_t)(sg.src0 + G * GB);
            W y = T::tail(a.frontier, pos, r);
            if (a.invert_frontier) y = ~y & (W)((W(1) << r) - W(1));
            if (sg.dirb && y) y &= T::tail(sg.dirb, (uint64_t)(G * GB), r);
            if (a.dir_clear) {              // the tail words no chunk of the write pass owns
                uint32_t* d = a.dir_clear + (int64_t)s * a.dir_stride;
                for (int64_t w = (G * GB + 31) >> 5; w < (sg.nbits + 31) >> 5; ++w) d[w] = 0u;
            }
            if (setbits && y) atomicAdd(setbits, (unsigned long long)T::popc(y));
            out[total++] = T::to_active(y, r);
        }
        a.counts[s] = total;
    }
}

// ------------------------------------------------- parallel slot encoder --
// The same stream as wah_encode_kernel, built in three data-parallel passes
// over (slot, chunk of kTile groups):
//   1. enc_chunk_sums32 / enc_chunk_sums64: one warp per chunk tests the
//      frontier summary (a chunk without frontier bits is flagged all-zero and
//      not read) and, for the others, stages the chunk in shared memory and
//      takes its head count (its first group counted as a head), first and
//      last group type and last head position;
//   2. enc_chunk_scan: per slot, one warp scans the chunk sums (an all-zero
//      chunk is one zero run): a chunk whose first group continues the previous
//      chunk's fill run merges with it; this gives every chunk its first word
//      index and the start of the run it opens with, the slot's word count and
//      the active word, and writes the fill word of every zero run that ends
//      in an all-zero chunk.  The last slot to finish (a counter, no waiting)
//      lays out the decoder's units over all slots;
//   3. enc_chunk_write32 / enc_chunk_write64: one warp per flagged chunk
//      writes its words, each lane's word indices and run starts taken from
//      the scanned head masks and the chunk's carry from pass 2.
// With unit_base set, the group at which every 32nd word opens is recorded
// as the word is written (the decoder's unit bases).

// 31-bit groups of a whole chunk, staged in shared memory: the warp copies
// the chunk's frontier words and directory words with asynchronous 16-byte
// copies (all in flight together; one round trip per chunk), then every
// group is two shared-memory words funnel-shifted.
constexpr int kEW = 128;          // threads per staging encoder CTA (4 warps)
constexpr int kEWBlocks = 6;      // CTAs per SM the staging passes are compiled for: as many as their shared
                                  // memory allows (registers capped at 80; uncapped they held 5)
constexpr int kStageWords = 1060; // >= the words of one chunk (1024 x 31 bits) + alignment and funnel slack,
                                  // and >= the padded output words of a chunk (the frontier buffer is reused)

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}

struct Stage32 {
    const uint32_t* f;     // frontier words from a 16-byte boundary at or before group tb
    const uint32_t* d;     // directory words from group tb (or nullptr: no sieve)
    uint32_t off;          // bit of group tb in f
    uint32_t fx;           // xor mask of the frontier operand (all ones: complemented)
    int64_t tb;
};

__device__ __forceinline__ Stage32 stage_chunk(const EncodeArgs& a, const SlotGeom& sg, int64_t tb, int64_t tend,
                                               uint32_t* fbuf, uint32_t* dbuf) {
    const int lane = (int)lane_id();
    const int64_t fbit0 = sg.src0 + 31 * tb;
    const int64_t fw0 = (fbit0 >> 5) & ~(int64_t)3;
    const int64_t flast = ((sg.src0 + 31 * tend - 1) >> 5) + 1;    // the upper funnel word of the last group
    int64_t fend = (flast + 1 + 3) & ~(int64_t)3;
    if (fend > a.frontier_words) fend = a.frontier_words;
    for (int64_t i = lane; 4 * i < fend - fw0; i += 32) cp_async16(fbuf + 4 * i, a.frontier + fw0 + 4 * i);
    Stage32 st;
    st.f = fbuf;
    st.off = (uint32_t)(fbit0 - 32 * fw0);
    st.fx = a.invert_frontier ? 0xffffffffu : 0u;
    st.tb = tb;
    st.d = nullptr;
    if (sg.dirb) {
        const int64_t dw0 = (31 * tb) >> 5;                          // tb is a multiple of 1024: 16-byte aligned
        const int64_t dlast = ((31 * tend - 1) >> 5) + 1;
        int64_t dend = (dlast + 1 + 3) & ~(int64_t)3;
        if (dend > a.dir_stride) dend = a.dir_stride;
        for (int64_t i = lane; 4 * i < dend - dw0; i += 32) cp_async16(dbuf + 4 * i, sg.dirb + dw0 + 4 * i);
        st.d = dbuf;
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    return st;
}

struct ChunkSum {
    uint32_t heads;
    uint32_t types;        // first type | last type << 8
    int64_t last_head;     // group index of the chunk's last head
    uint32_t ones;         // set bits of the chunk (adaptive format only)
};
struct ChunkBase {
    int64_t words;         // index of the next word to open at the chunk's first group
    int64_t run_start;     // start group of the run open before the chunk
    int32_t prev_type;     // type of the group before the chunk (-1 at the slot start)
    int32_t next_type;     // type of the group after the chunk (G_NONE at the slot end)
    int64_t ones_before;   // set bits of the slot before the chunk (adaptive format only)
};


// The write pass is the last reader of a chunk's directory words: zero the
// nonzero ones among the words [w0, w1) that hold its groups (the staged copy
// d starts at word w0), so that the operand is clear for its next use.
__device__ __forceinline__ void clear_consumed(const EncodeArgs& a, int s, int64_t w0, int64_t w1, const uint32_t* d) {
    uint32_t* dst = a.dir_clear + (int64_t)s * a.dir_stride;
    for (int64_t k = lane_id(); k < w1 - w0; k += 32)
        if (d[k]) dst[w0 + k] = 0u;
}

// One warp per slot (blockDim.x = 32).
template <typename W>
__global__ void enc_chunk_scan(EncodeArgs a, const ChunkSum* sums, const uint8_t* flags, ChunkBase* bases,
                               int64_t cps, unsigned long long* setbits) {
    using T = Wah<W>;
    constexpr int GB = T::GB;
    const int s = blockIdx.x;
    if (a.skip && *a.skip) {                // a level without this exchange: empty streams
        if (lane_id() == 0) a.counts[s] = 0;
        return;
    }
    const SlotGeom sg = slot_geom(a, s);
    const int64_t G = sg.nbits / GB;
    const int r = (int)(sg.nbits % GB);
    const int64_t nch = (G + kTile - 1) / kTile;
    const int lane = (int)lane_id();
    W* out = static_cast<W*>(a.out) + (int64_t)s * a.slot_cap;
    int64_t* ub = a.unit_base ? a.unit_base + (int64_t)s * a.unit_stride : nullptr;
    auto sum_of = [&](int64_t c) -> ChunkSum {
        ChunkSum cs;
        if (flags[(int64_t)s * cps + c]) return sums[(int64_t)s * cps + c];
        cs.heads = 1;                                   // an all-zero chunk: one zero run
        cs.types = G_ZERO | (G_ZERO << 8);
        cs.last_head = c * kTile;
        cs.ones = 0;
        return cs;
    };
    // Lane l takes chunks [l*K, (l+1)*K) in order.  Pass 1: the lane's summary
    // (words, last head, first and last type) with the merges between its own
    // chunks applied; a scan over the lanes with the merge rule gives every lane
    // what comes before it; pass 2 walks the chunks again with that carry.
    struct Agg { int64_t w, h; int f, l; };       // f, l < 0: no chunk
    auto combine = [](const Agg& A, const Agg& B) -> Agg {   // A then B
        if (B.f < 0) return A;
        if (A.f < 0) return B;
        const bool m = A.l == B.f && B.f != G_LIT;           // B's first group continues A's last run
        Agg R;
        R.w = A.w + B.w - (m ? 1 : 0);
        R.h = (m && B.w == 1) ? A.h : (A.h > B.h ? A.h : B.h);
        R.f = A.f;
        R.l = B.l;
        return R;
    };
    const int64_t K = (nch + 31) / 32;
    const int64_t c_lo = (int64_t)lane * K, c_hi = (c_lo + K < nch) ? c_lo + K : nch;
    Agg mine{0, -1, -1, -1};
    bool bits = false;                                  // a chunk of the lane holds a set bit
    int64_t my_ones = 0;                                // set bits of the lane's chunks (adaptive)
    for (int64_t c = c_lo; c < c_hi; ++c) {
        const ChunkSum cs = sum_of(c);
        Agg one{(int64_t)cs.heads, cs.last_head, (int)(cs.types & 0xff), (int)((cs.types >> 8) & 0xff)};
        mine = combine(mine, one);
        bits |= !(cs.heads == 1 && (cs.types & 0xff) == G_ZERO);   // not one zero run
        if (a.adaptive) my_ones += cs.ones;
    }
    bits = __any_sync(0xffffffffu, bits);
    int64_t ones_before = 0, ones_total = 0;
    if (a.adaptive) {
        const int64_t oi = warp_incl_sum(my_ones);
        ones_before = oi - my_ones;
        ones_total = __shfl_sync(0xffffffffu, oi, 31);
    }
    Agg incl = mine;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        Agg y;
        y.w = __shfl_up_sync(0xffffffffu, incl.w, d);
        y.h = __shfl_up_sync(0xffffffffu, incl.h, d);
        y.f = __shfl_up_sync(0xffffffffu, incl.f, d);
        y.l = __shfl_up_sync(0xffffffffu, incl.l, d);
        if (lane >= d) incl = combine(y, incl);
    }
    Agg before_me;
    before_me.w = __shfl_up_sync(0xffffffffu, incl.w, 1);
    before_me.h = __shfl_up_sync(0xffffffffu, incl.h, 1);
    before_me.f = __shfl_up_sync(0xffffffffu, incl.f, 1);
    before_me.l = __shfl_up_sync(0xffffffffu, incl.l, 1);
    if (lane == 0) before_me = Agg{0, -1, -1, -1};
    // the trailing r bits of the slot (every lane), and the format of the slot
    W y = W(0);
    if (r > 0) {
        const uint64_t pos = (uint64_t)(sg.src0 + G * GB);
        y = T::tail(a.frontier, pos, r);
        if (a.invert_frontier) y = ~y & (W)((W(1) << r) - W(1));
        if (sg.dirb && y) y &= T::tail(sg.dirb, (uint64_t)(G * GB), r);
    }
    const int64_t wah_total = __shfl_sync(0xffffffffu, incl.w, 31) + (r > 0 ? 1 : 0);
    int fm = FMT_WAH;
    if (a.adaptive) {
        // the smallest in bytes, the lower format on a tie (every element is 4 bytes)
        const int64_t list_total = ones_total + T::popc(y), raw_total = (sg.nbits + 31) >> 5;
        fm = (wah_total <= list_total && wah_total <= raw_total) ? FMT_WAH
             : (list_total <= raw_total ? FMT_LIST : FMT_RAW);
    }
    if (fm != FMT_WAH) ub = nullptr;                    // no WAH units in this slot
    int64_t words = before_me.w, hmax = before_me.h;
    int prev_last = before_me.l;
    for (int64_t c = c_lo; c < c_hi; ++c) {
        const ChunkSum cs = sum_of(c);
        const int first = (int)(cs.types & 0xff), last = (int)((cs.types >> 8) & 0xff);
        const bool merge = prev_last >= 0 && prev_last == first && first != G_LIT;
        const int64_t eff = (int64_t)cs.heads - (merge ? 1 : 0);
        const int64_t h = (merge && cs.heads == 1) ? (int64_t)-1 : cs.last_head;
        ChunkBase cb;
        cb.words = words;
        cb.run_start = merge ? hmax : c * kTile;
        cb.prev_type = prev_last;
        const int nxt = (c + 1 < nch) ? (int)(sum_of(c + 1).types & 0xff) : G_NONE;
        cb.next_type = nxt;
        cb.ones_before = ones_before;
        if (a.adaptive) ones_before += sum_of(c).ones;
        bases[(int64_t)s * cps + c] = cb;
        if (a.chunk_first) {                // where a decoder of this chunk alone starts
            a.chunk_first[2 * ((int64_t)s * cps + c)] = merge ? cb.words - 1 : cb.words;
            a.chunk_first[2 * ((int64_t)s * cps + c) + 1] = merge ? cb.run_start : c * kTile;
        }
        if (!flags[(int64_t)s * cps + c] && fm == FMT_WAH) {
            // an all-zero chunk: its zero run opens a word here unless it merges
            if (!merge && ub && (cb.words & 31) == 0) ub[cb.words >> 5] = c * kTile;
            if (nxt != G_ZERO) {     // the run ends at the chunk's last group
                const int64_t tend = ((c + 1) * kTile < G) ? (c + 1) * kTile : G;
                const int64_t start = merge ? cb.run_start : c * kTile;
                out[merge ? cb.words - 1 : cb.words] = fill_word<W>(G_ZERO, (uint64_t)(tend - start));
            }
        }
        words += eff;
        hmax = h > hmax ? h : hmax;
        prev_last = last;
    }
    words = __shfl_sync(0xffffffffu, incl.w, 31);    // the slot's words before the active word
    if (lane == 0) {
        int64_t total = words;
        if (r > 0) {
            if (a.dir_clear) {              // the tail words no chunk of the write pass owns
                uint32_t* d = a.dir_clear + (int64_t)s * a.dir_stride;
                for (int64_t w = (G * GB + 31) >> 5; w < (sg.nbits + 31) >> 5; ++w) d[w] = 0u;
            }
            if (setbits && y) atomicAdd(setbits, (unsigned long long)T::popc(y));
            if (fm == FMT_WAH) {
                if (ub && (total & 31) == 0) ub[total >> 5] = G;
                out[total++] = T::to_active(y, r);
            }
            bits |= y != W(0);
        }
        if (fm == FMT_LIST) {               // the offsets of the trailing bits close the vector
            total = ones_total;
            for (W x = y; x; x &= x - W(1)) out[total++] = (W)(G * GB + T::select(x, 0));
        } else if (fm == FMT_RAW) {
            total = (sg.nbits + 31) >> 5;   // written by enc_raw32
        }
        a.counts[s] = total;
        if (a.fmt) a.fmt[s] = (uint8_t)fm;
        if (a.slot_bits) a.slot_bits[s] = bits ? 1 : 0;
        if (a.wah_words) atomicAdd(a.wah_words, (unsigned long long)total);
    }
    if (!a.plan_base) return;
    // The last slot to finish lays out the decoder's units: block (i,j) of the
    // p x p grid (row-major) decodes stream s = i*p+j (sieved) or j, in chunks
    // of 32 words; plan_base is the exclusive scan of the chunk counts.
    __shared__ bool s_last;
    if (lane == 0) {
        __threadfence();
        s_last = atomicAdd(a.plan_done, 1u) == (unsigned)(a.nslots - 1);
    }
    __syncwarp();
    if (!s_last) return;
    __threadfence();
    const int64_t nblocks = (int64_t)a.p * a.p;
    unsigned long long carry = 0;
    for (int64_t b0 = 0; b0 < nblocks; b0 += 32) {
        const int64_t b = b0 + lane;
        unsigned long long nch = 0;
        if (b < nblocks) {
            const int64_t stream = a.sieve ? b : b % a.p;
            nch = (unsigned long long)((__ldcg(a.counts + stream) + 31) / 32);
        }
        unsigned long long incl = nch;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        if (b < nblocks) a.plan_base[b] = (int64_t)(carry + incl - nch);
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) {
        a.plan_base[nblocks] = (int64_t)carry;
        *a.plan_units = carry;
        *a.plan_done = 0u;                       // ready for the next level
    }
}


// 31-bit groups, lane-sequential: the chunk is staged in shared memory; lane
// l takes groups 32l .. 32l+31, combining their words into c = f & V (in
// registers, aligned to its first group), a group being two words of c
// funnel-shifted; its groups are classified into zero / one masks, from which
// head, run-end and word-index masks follow by bit operations, and the lanes'
// partial results are combined by warp scans.
// The lane's 32 combined words c[k] = bits 32k.. of the sieved groups
// 32*lane .. 32*lane+31 of the chunk (c = f & V aligned to the chunk's first
// group; c[31] is past the lane's 992 bits).  Lanes read 31 words apart: no
// bank conflicts.
__device__ __forceinline__ void lane_cwords(const Stage32& st, uint32_t (&c)[32]) {
    const int lane = (int)lane_id();
    const uint32_t sh = st.off & 31u;
    const uint32_t* f = st.f + 31 * lane + (st.off >> 5);
    if (st.d) {
        const uint32_t* d = st.d + 31 * lane;
#pragma unroll
        for (int k = 0; k < 32; ++k) c[k] = (__funnelshift_r(f[k], f[k + 1], sh) ^ st.fx) & d[k];
    } else {
#pragma unroll
        for (int k = 0; k < 32; ++k) c[k] = __funnelshift_r(f[k], f[k + 1], sh);
    }
}

// Group i (0..31) of the lane (it starts at bit 31i: word (31i)/32, shift (31i)%32).
__device__ __forceinline__ uint32_t lane_group(const uint32_t (&c)[32], int i) {
    const int b = 31 * i;
    return __funnelshift_r(c[b >> 5], c[(b >> 5) + 1], (uint32_t)(b & 31)) & 0x7fffffffu;
}

// Zero / one / valid masks of the lane's groups (bit i = group 32*lane + i).
__device__ __forceinline__ void lane_masks(const uint32_t (&c)[32], int ng, uint32_t& zm, uint32_t& om,
                                           uint32_t& vm) {
    const int nv = ng - 32 * (int)lane_id();
    vm = nv >= 32 ? 0xffffffffu : (nv > 0 ? (1u << nv) - 1u : 0u);
    zm = 0u;
    om = 0u;
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const uint32_t x = lane_group(c, i);
        zm |= (x == 0u ? 1u : 0u) << i;
        om |= (x == 0x7fffffffu ? 1u : 0u) << i;
    }
    zm &= vm;
    om &= vm;
}

__device__ __forceinline__ int mask_type(uint32_t zm, uint32_t om, int i) {
    return ((zm >> i) & 1u) ? G_ZERO : (((om >> i) & 1u) ? G_ONE : G_LIT);
}

// Set bits of the lane's valid groups (ng groups in the chunk): its 31 words,
// the last lane's cut at the chunk end.
__device__ __forceinline__ uint32_t lane_popc(const uint32_t (&c)[32], int ng) {
    const int nv = ng - 32 * (int)lane_id();
    uint32_t cnt = 0;
    if (nv >= 32) {
#pragma unroll
        for (int k = 0; k < 31; ++k) cnt += __popc(c[k]);
    } else if (nv > 0) {
        const int nbits = nv * 31;
#pragma unroll
        for (int k = 0; k < 31; ++k) {
            const int left = nbits - 32 * k;
            const uint32_t m = left >= 32 ? 0xffffffffu : (left > 0 ? (1u << left) - 1u : 0u);
            cnt += __popc(c[k] & m);
        }
    }
    return cnt;
}

__global__ void __launch_bounds__(kEW, kEWBlocks) enc_chunk_sums32(EncodeArgs a, ChunkSum* sums, uint8_t* flags, int64_t cps,
                                                        unsigned long long* setbits) {
    if (a.skip && *a.skip) return;
    __shared__ __align__(16) uint32_t s_f[kEW / 32][kStageWords];
    __shared__ __align__(16) uint32_t s_d[kEW / 32][kStageWords];
    const int64_t n = (int64_t)a.nslots * cps;
    const int lane = (int)lane_id();
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long ones = 0;
    for (int64_t q = wid; q < n; q += nw) {
        const int s = (int)((uint32_t)q / (uint32_t)cps);          // slots x chunks fit in 32 bits
        const int64_t c = (int64_t)((uint32_t)q - (uint32_t)s * (uint32_t)cps);
        const SlotGeom sg = slot_geom(a, s);
        const int64_t G = sg.nbits / 31;
        const int64_t tb = c * kTile;
        bool live = false;
        int64_t tend = tb;
        if (tb < G && !(a.slot_live && !a.slot_live[s])) {
            tend = (tb + kTile < G) ? tb + kTile : G;
            bool nz = true;
            if (a.fsum) {
                const int64_t q0 = (sg.src0 + tb * 31) >> 10, q1 = (sg.src0 + tend * 31 - 1) >> 10;
                const int64_t w = (q0 >> 2) + lane;
                uint32_t x = 0;
                if (w <= (q1 >> 2)) {
                    x = __ldcg(reinterpret_cast<const uint32_t*>(a.fsum) + w);
                    if (w == (q0 >> 2)) x &= 0xffffffffu << (8 * (q0 & 3));
                    if (w == (q1 >> 2)) x &= 0xffffffffu >> (8 * (3 - (q1 & 3)));
                }
                nz = x != 0u;
            }
            live = __any_sync(0xffffffffu, nz);
        }
        if (lane == 0) flags[q] = live ? 1 : 0;
        if (!live) continue;
        if (lane == 0 && a.live_chunks) atomicAdd(a.live_chunks, 1ull);
        const Stage32 st = stage_chunk(a, sg, tb, tend, s_f[threadIdx.x >> 5], s_d[threadIdx.x >> 5]);
        const int ng = (int)(tend - tb);
        uint32_t cwd[32];
        lane_cwords(st, cwd);
        // set bits of the lane's groups (a statistic when asked for, and the
        // size of the sparse vector with the adaptive format): its 31 words,
        // the last lane's cut at the chunk end
        uint32_t lane_ones = 0;
        if (setbits || a.adaptive) {
            lane_ones = lane_popc(cwd, ng);
            ones += lane_ones;
        }
        uint32_t zm, om, vm;
        lane_masks(cwd, ng, zm, om, vm);
        uint32_t pz = __shfl_up_sync(0xffffffffu, zm, 1) >> 31, po = __shfl_up_sync(0xffffffffu, om, 1) >> 31;
        if (lane == 0) { pz = 0u; po = 0u; }              // the chunk's first group counts as a head
        const uint32_t hm = (vm & ~(zm | om)) | (zm & ~((zm << 1) | pz)) | (om & ~((om << 1) | po));
        const int heads = warp_sum(__popc(hm));
        int lh = hm ? 32 * lane + 31 - __clz(hm) : -1;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) { const int y = __shfl_xor_sync(0xffffffffu, lh, d); lh = y > lh ? y : lh; }
        const int lastl = (ng - 1) >> 5;                       // the lane holding the chunk's last group
        const int lastty = mask_type(__shfl_sync(0xffffffffu, zm, lastl), __shfl_sync(0xffffffffu, om, lastl),
                                     (ng - 1) & 31);
        const uint32_t chunk_ones = a.adaptive ? warp_sum(lane_ones) : 0u;
        if (lane == 0) {
            ChunkSum cs;
            cs.heads = (uint32_t)heads;
            cs.types = (uint32_t)mask_type(zm, om, 0) | ((uint32_t)lastty << 8);
            cs.last_head = lh >= 0 ? tb + lh : -1;
            cs.ones = chunk_ones;
            sums[q] = cs;
        }
        __syncwarp();           // the staging buffers are reused by the next chunk
    }
    if (setbits) {
        ones = warp_sum(ones);
        if (lane == 0 && ones) atomicAdd(setbits, ones);
    }
}

constexpr int kOutWords = kTile + 2;     // the chunk's words, from the one before its first head
// Local word k sits at k + k/32: consecutive lanes write 32 apart without
// bank conflicts.
__device__ __forceinline__ int opad(int k) { return k + (k >> 5); }

__global__ void __launch_bounds__(kEW, kEWBlocks) enc_chunk_write32(EncodeArgs a, const ChunkBase* bases, const uint8_t* flags,
                                                         int64_t cps) {
    __shared__ __align__(16) uint32_t s_f[kEW / 32][kStageWords];
    __shared__ __align__(16) uint32_t s_d[kEW / 32][kStageWords];
    static_assert(kOutWords + kOutWords / 32 + 1 <= kStageWords, "output words overflow the frontier buffer");
    if (a.skip && *a.skip) return;
    const int64_t n = (int64_t)a.nslots * cps;
    const int lane = (int)lane_id();
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t* ob = s_f[threadIdx.x >> 5];      // the words, once the frontier words are in registers
    for (int64_t q = wid; q < n; q += nw) {
        if (!flags[q]) continue;
        const int s = (int)((uint32_t)q / (uint32_t)cps);          // slots x chunks fit in 32 bits
        const int fm = a.adaptive ? (int)a.fmt[s] : FMT_WAH;
        if (fm == FMT_RAW) continue;                                // enc_raw32 writes the raw words
        const int64_t c = (int64_t)((uint32_t)q - (uint32_t)s * (uint32_t)cps);
        const SlotGeom sg = slot_geom(a, s);
        const int64_t G = sg.nbits / 31;
        const int64_t tb = c * kTile;
        const int64_t tend = (tb + kTile < G) ? tb + kTile : G;
        const ChunkBase cb = bases[q];
        uint32_t* out = static_cast<uint32_t*>(a.out) + (int64_t)s * a.slot_cap;
        int64_t* ub = a.unit_base ? a.unit_base + (int64_t)s * a.unit_stride : nullptr;
        const Stage32 st = stage_chunk(a, sg, tb, tend, s_f[threadIdx.x >> 5], s_d[threadIdx.x >> 5]);
        const int ng = (int)(tend - tb);
        uint32_t cwd[32];
        lane_cwords(st, cwd);
        if (a.dir_clear) clear_consumed(a, s, (31 * tb) >> 5, (31 * tend + 31) >> 5, st.d);
        if (fm == FMT_LIST) {
            // the sparse vector: every set bit's offset in the slice, in order; the
            // lane's bits start at bit 31 * (tb + 32 * lane) of the slice
            const uint32_t mine = lane_popc(cwd, ng);
            const uint32_t incl = warp_incl_sum(mine);
            int64_t at = cb.ones_before + (int64_t)(incl - mine);
            const int nv = ng - 32 * lane;
            const int nbits = nv >= 32 ? 992 : (nv > 0 ? nv * 31 : 0);
            const uint32_t base = (uint32_t)(31 * (tb + 32 * lane));
#pragma unroll
            for (int k = 0; k < 31; ++k) {
                const int left = nbits - 32 * k;
                uint32_t x = cwd[k] & (left >= 32 ? 0xffffffffu : (left > 0 ? (1u << left) - 1u : 0u));
                while (x) {
                    out[at++] = base + 32u * (uint32_t)k + (uint32_t)(__ffs(x) - 1);
                    x &= x - 1u;
                }
            }
            __syncwarp();
            continue;
        }
        __syncwarp();           // the frontier buffer now takes the output words
        uint32_t zm, om, vm;
        lane_masks(cwd, ng, zm, om, vm);
        const int r0 = 32 * lane;
        const int nv = ng - r0;
        // types around the lane's groups: the one before (the previous lane's
        // last group, or the chunk's carry) and the one after
        uint32_t pz = __shfl_up_sync(0xffffffffu, zm, 1) >> 31, po = __shfl_up_sync(0xffffffffu, om, 1) >> 31;
        if (lane == 0) { pz = cb.prev_type == G_ZERO; po = cb.prev_type == G_ONE; }
        uint32_t nz = __shfl_down_sync(0xffffffffu, zm, 1) & 1u, no = __shfl_down_sync(0xffffffffu, om, 1) & 1u;
        if (nv <= 32) { nz = cb.next_type == G_ZERO; no = cb.next_type == G_ONE; }
        const uint32_t lit = vm & ~(zm | om);
        const uint32_t hm = lit | (zm & ~((zm << 1) | pz)) | (om & ~((om << 1) | po));
        const int last = nv >= 32 ? 31 : nv - 1;                 // the lane's last group (if any)
        const uint32_t zend = nv > 0 ? zm & ~((zm >> 1) | (nz << last)) : 0u;
        const uint32_t oend = nv > 0 ? om & ~((om >> 1) | (no << last)) : 0u;
        const int hc = __popc(hm);
        int incl = hc, hmax = hm ? r0 + 31 - __clz(hm) : -1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            const int z = __shfl_up_sync(0xffffffffu, hmax, d);
            if (lane >= d) { incl += y; hmax = z > hmax ? z : hmax; }
        }
        const int H = __shfl_sync(0xffffffffu, incl, 31);
        int hprev = __shfl_up_sync(0xffffffffu, hmax, 1);
        if (lane == 0) hprev = -1;
        const int li0 = incl - hc;                    // local index of the word open before this lane's groups
        const int64_t st0 = hprev >= 0 ? tb + hprev : cb.run_start;   // start of the run open before them
        if (nv > 0) {
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const uint32_t bit = 1u << i;
                const uint32_t hb = hm & (i == 31 ? 0xffffffffu : (bit << 1) - 1u);   // heads up to group i
                const int li = li0 + __popc(hb);
                if (lit & bit) {
                    ob[opad(li)] = __brev(lane_group(cwd, i)) >> 1;
                } else if ((zend | oend) & bit) {
                    const int64_t start = hb ? tb + r0 + 31 - __clz(hb) : st0;
                    ob[opad(li)] = 0x80000000u | ((oend & bit) ? 0x40000000u : 0u) | (uint32_t)(tb + r0 + i - start + 1);
                }
            }
            // the decoder's unit base: the lane's heads open words cb.words + li0 .. + hc - 1;
            // at most one of them is a multiple of 32
            if (ub && hc > 0) {
                int j = (int)((1 - cb.words - li0) & 31);          // head ordinal (1-based) whose word is 32k
                if (j == 0) j = 32;
                if (j <= hc) ub[(cb.words - 1 + li0 + j) >> 5] = tb + r0 + select32(hm, j - 1);
            }
        }
        // word 0 (a run carried in) is written here when the chunk's first group
        // continues it and the run ends in the chunk; word H (the last opened)
        // when the chunk's last group is a literal or ends its run
        const uint32_t hm0 = __shfl_sync(0xffffffffu, hm, 0);
        const int lastl = (ng - 1) >> 5, lastb = (ng - 1) & 31;
        const uint32_t lit_l = __shfl_sync(0xffffffffu, lit, lastl);
        const uint32_t end_l = __shfl_sync(0xffffffffu, zend | oend, lastl);
        const bool last_lit = (lit_l >> lastb) & 1u, last_end = (end_l >> lastb) & 1u;
        const bool w0 = !(hm0 & 1u) && (H > 0 || last_end);
        const bool wH = H > 0 ? (last_lit || last_end) : w0;         // with no head, word H is word 0
        __syncwarp();
        // words cb.words .. cb.words + H - 2 are always complete here; the one
        // before (a run carried in) and the last one (a run carried out) only
        // when their run ends in this chunk
        const int lo = w0 ? 0 : 1, hi = wH ? H : H - 1;
        for (int k = lo + lane; k <= hi; k += 32) out[cb.words - 1 + k] = ob[opad(k)];
        __syncwarp();           // the staging buffers are reused by the next chunk
    }
}

// 63-bit groups (64-bit words), lane-sequential like the 31-bit passes: a
// chunk of 1024 groups is 64,512 bits, lane l owns groups 32l .. 32l+31, which
// start at word 63l of the chunk (a stride of 63 words: no bank conflicts), and
// takes them in two halves of 16 groups (1,008 bits; the second half starts
// 16 bits into word 31), each from 33 combined words c = f & V in registers;
// a group spans at most three of them.
constexpr int kEW64 = 64;                 // threads per CTA (2 warps: shared memory per warp is ~17 KB)
constexpr int kStage64 = 2176;            // words: a chunk (2,016) + alignment and funnel slack, and the
                                          // padded 64-bit output words (2 x 1,059) of the write pass

__device__ __forceinline__ Stage32 stage_chunk63(const EncodeArgs& a, const SlotGeom& sg, int64_t tb, int64_t tend,
                                                 uint32_t* fbuf, uint32_t* dbuf) {
    const int lane = (int)lane_id();
    const int64_t fbit0 = sg.src0 + 63 * tb;
    const int64_t fw0 = (fbit0 >> 5) & ~(int64_t)3;
    const int64_t flast = ((sg.src0 + 63 * tend - 1) >> 5) + 1;
    int64_t fend = (flast + 1 + 3) & ~(int64_t)3;
    if (fend > a.frontier_words) fend = a.frontier_words;
    for (int64_t i = lane; 4 * i < fend - fw0; i += 32) cp_async16(fbuf + 4 * i, a.frontier + fw0 + 4 * i);
    Stage32 st;
    st.f = fbuf;
    st.off = (uint32_t)(fbit0 - 32 * fw0);
    st.fx = a.invert_frontier ? 0xffffffffu : 0u;
    st.tb = tb;
    st.d = nullptr;
    if (sg.dirb) {
        const int64_t dw0 = (63 * tb) >> 5;                          // 2,016 words per chunk: 16-byte aligned
        const int64_t dlast = ((63 * tend - 1) >> 5) + 1;
        int64_t dend = (dlast + 1 + 3) & ~(int64_t)3;
        if (dend > a.dir_stride) dend = a.dir_stride;
        for (int64_t i = lane; 4 * i < dend - dw0; i += 32) cp_async16(dbuf + 4 * i, sg.dirb + dw0 + 4 * i);
        st.d = dbuf;
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    return st;
}

// The 33 combined words of half h of the lane's groups.
__device__ __forceinline__ void half_cwords63(const Stage32& st, int h, uint32_t (&c)[33]) {
    const int lane = (int)lane_id();
    const uint32_t sh = st.off & 31u;
    const int w0 = 63 * lane + 31 * h;
    const uint32_t* f = st.f + w0 + (st.off >> 5);
    if (st.d) {
        const uint32_t* d = st.d + w0;
#pragma unroll
        for (int k = 0; k < 33; ++k) c[k] = (__funnelshift_r(f[k], f[k + 1], sh) ^ st.fx) & d[k];
    } else {
#pragma unroll
        for (int k = 0; k < 33; ++k) c[k] = __funnelshift_r(f[k], f[k + 1], sh);
    }
}

// Group i (0..15) of half h from its combined words.
__device__ __forceinline__ unsigned long long half_group63(const uint32_t (&c)[33], int h, int i) {
    const int b = 16 * h + 63 * i;
    const int k = b >> 5;
    const uint32_t s = (uint32_t)(b & 31);
    const uint32_t lo = __funnelshift_r(c[k], c[k + 1], s), hi = __funnelshift_r(c[k + 1], c[k + 2], s);
    return (((unsigned long long)hi << 32) | lo) & 0x7fffffffffffffffull;
}

// Zero / one / valid masks of the lane's groups (bit i = group 32*lane + i) from
// the combined words of its two halves and, when asked for, their set bits.
__device__ __forceinline__ void lane_masks63(const uint32_t (&c0)[33], const uint32_t (&c1)[33], int ng, uint32_t& zm,
                                             uint32_t& om, uint32_t& vm, unsigned long long* ones) {
    const int nv = ng - 32 * (int)lane_id();
    vm = nv >= 32 ? 0xffffffffu : (nv > 0 ? (1u << nv) - 1u : 0u);
    zm = 0u;
    om = 0u;
#pragma unroll
    for (int bi = 0; bi < 32; ++bi) {
        const unsigned long long x = bi < 16 ? half_group63(c0, 0, bi) : half_group63(c1, 1, bi - 16);
        zm |= (x == 0ull ? 1u : 0u) << bi;
        om |= (x == 0x7fffffffffffffffull ? 1u : 0u) << bi;
        if (ones && bi < nv) *ones += (unsigned long long)__popcll(x);
    }
    zm &= vm;
    om &= vm;
}

__global__ void __launch_bounds__(kEW64) enc_chunk_sums64(EncodeArgs a, ChunkSum* sums, uint8_t* flags, int64_t cps,
                                                          unsigned long long* setbits) {
    if (a.skip && *a.skip) return;
    __shared__ __align__(16) uint32_t s_f[kEW64 / 32][kStage64];
    __shared__ __align__(16) uint32_t s_d[kEW64 / 32][kStage64];
    const int64_t n = (int64_t)a.nslots * cps;
    const int lane = (int)lane_id();
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long ones = 0;
    for (int64_t q = wid; q < n; q += nw) {
        const int s = (int)((uint32_t)q / (uint32_t)cps);
        const int64_t c = (int64_t)((uint32_t)q - (uint32_t)s * (uint32_t)cps);
        const SlotGeom sg = slot_geom(a, s);
        const int64_t G = sg.nbits / 63;
        const int64_t tb = c * kTile;
        bool live = false;
        int64_t tend = tb;
        if (tb < G && !(a.slot_live && !a.slot_live[s])) {
            tend = (tb + kTile < G) ? tb + kTile : G;
            bool nz = true;
            if (a.fsum) {
                const int64_t q0 = (sg.src0 + tb * 63) >> 10, q1 = (sg.src0 + tend * 63 - 1) >> 10;
                const int64_t w = (q0 >> 2) + lane;
                uint32_t x = 0;
                if (w <= (q1 >> 2)) {
                    x = __ldcg(reinterpret_cast<const uint32_t*>(a.fsum) + w);
                    if (w == (q0 >> 2)) x &= 0xffffffffu << (8 * (q0 & 3));
                    if (w == (q1 >> 2)) x &= 0xffffffffu >> (8 * (3 - (q1 & 3)));
                }
                nz = x != 0u;
            }
            live = __any_sync(0xffffffffu, nz);
        }
        if (lane == 0) flags[q] = live ? 1 : 0;
        if (!live) continue;
        if (lane == 0 && a.live_chunks) atomicAdd(a.live_chunks, 1ull);
        const Stage32 st = stage_chunk63(a, sg, tb, tend, s_f[threadIdx.x >> 5], s_d[threadIdx.x >> 5]);
        const int ng = (int)(tend - tb);
        uint32_t c0[33], c1[33];
        half_cwords63(st, 0, c0);
        half_cwords63(st, 1, c1);
        uint32_t zm, om, vm;
        lane_masks63(c0, c1, ng, zm, om, vm, setbits ? &ones : nullptr);
        uint32_t pz = __shfl_up_sync(0xffffffffu, zm, 1) >> 31, po = __shfl_up_sync(0xffffffffu, om, 1) >> 31;
        if (lane == 0) { pz = 0u; po = 0u; }              // the chunk's first group counts as a head
        const uint32_t hm = (vm & ~(zm | om)) | (zm & ~((zm << 1) | pz)) | (om & ~((om << 1) | po));
        const int heads = warp_sum(__popc(hm));
        int lh = hm ? 32 * lane + 31 - __clz(hm) : -1;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) { const int y = __shfl_xor_sync(0xffffffffu, lh, d); lh = y > lh ? y : lh; }
        const int lastl = (ng - 1) >> 5;
        const int lastty = mask_type(__shfl_sync(0xffffffffu, zm, lastl), __shfl_sync(0xffffffffu, om, lastl),
                                     (ng - 1) & 31);
        if (lane == 0) {
            ChunkSum cs;
            cs.heads = (uint32_t)heads;
            cs.types = (uint32_t)mask_type(zm, om, 0) | ((uint32_t)lastty << 8);
            cs.last_head = lh >= 0 ? tb + lh : -1;
            sums[q] = cs;
        }
        __syncwarp();
    }
    if (setbits) {
        ones = warp_sum(ones);
        if (lane == 0 && ones) atomicAdd(setbits, ones);
    }
}

__global__ void __launch_bounds__(kEW64) enc_chunk_write64(EncodeArgs a, const ChunkBase* bases, const uint8_t* flags,
                                                           int64_t cps) {
    using T = Wah<unsigned long long>;
    __shared__ __align__(16) uint32_t s_f[kEW64 / 32][kStage64];
    __shared__ __align__(16) uint32_t s_d[kEW64 / 32][kStage64];
    static_assert(2 * (kOutWords + kOutWords / 32 + 1) <= kStage64, "output words overflow the frontier buffer");
    if (a.skip && *a.skip) return;
    const int64_t n = (int64_t)a.nslots * cps;
    const int lane = (int)lane_id();
    const int64_t wid = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long* ob = reinterpret_cast<unsigned long long*>(s_f[threadIdx.x >> 5]);
    for (int64_t q = wid; q < n; q += nw) {
        if (!flags[q]) continue;
        const int s = (int)((uint32_t)q / (uint32_t)cps);
        const int64_t c = (int64_t)((uint32_t)q - (uint32_t)s * (uint32_t)cps);
        const SlotGeom sg = slot_geom(a, s);
        const int64_t G = sg.nbits / 63;
        const int64_t tb = c * kTile;
        const int64_t tend = (tb + kTile < G) ? tb + kTile : G;
        const ChunkBase cb = bases[q];
        unsigned long long* out = static_cast<unsigned long long*>(a.out) + (int64_t)s * a.slot_cap;
        int64_t* ub = a.unit_base ? a.unit_base + (int64_t)s * a.unit_stride : nullptr;
        const Stage32 st = stage_chunk63(a, sg, tb, tend, s_f[threadIdx.x >> 5], s_d[threadIdx.x >> 5]);
        const int ng = (int)(tend - tb);
        uint32_t c0[33], c1[33];
        half_cwords63(st, 0, c0);
        half_cwords63(st, 1, c1);
        if (a.dir_clear) clear_consumed(a, s, (63 * tb) >> 5, (63 * tend + 31) >> 5, st.d);
        uint32_t zm, om, vm;
        lane_masks63(c0, c1, ng, zm, om, vm, nullptr);
        const int r0 = 32 * lane;
        const int nv = ng - r0;
        uint32_t pz = __shfl_up_sync(0xffffffffu, zm, 1) >> 31, po = __shfl_up_sync(0xffffffffu, om, 1) >> 31;
        if (lane == 0) { pz = cb.prev_type == G_ZERO; po = cb.prev_type == G_ONE; }
        uint32_t nz = __shfl_down_sync(0xffffffffu, zm, 1) & 1u, no = __shfl_down_sync(0xffffffffu, om, 1) & 1u;
        if (nv <= 32) { nz = cb.next_type == G_ZERO; no = cb.next_type == G_ONE; }
        const uint32_t lit = vm & ~(zm | om);
        const uint32_t hm = lit | (zm & ~((zm << 1) | pz)) | (om & ~((om << 1) | po));
        const int last = nv >= 32 ? 31 : nv - 1;
        const uint32_t zend = nv > 0 ? zm & ~((zm >> 1) | (nz << last)) : 0u;
        const uint32_t oend = nv > 0 ? om & ~((om >> 1) | (no << last)) : 0u;
        const int hc = __popc(hm);
        int incl = hc, hmax = hm ? r0 + 31 - __clz(hm) : -1;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, d);
            const int z = __shfl_up_sync(0xffffffffu, hmax, d);
            if (lane >= d) { incl += y; hmax = z > hmax ? z : hmax; }
        }
        const int H = __shfl_sync(0xffffffffu, incl, 31);
        int hprev = __shfl_up_sync(0xffffffffu, hmax, 1);
        if (lane == 0) hprev = -1;
        const int li0 = incl - hc;
        const int64_t st0 = hprev >= 0 ? tb + hprev : cb.run_start;
        // every lane has read its frontier words: the buffer now takes the output words
        __syncwarp();
        if (nv > 0) {
#pragma unroll
            for (int bi = 0; bi < 32; ++bi) {
                const uint32_t bit = 1u << bi;
                const uint32_t hb = hm & (bi == 31 ? 0xffffffffu : (bit << 1) - 1u);
                const int li = li0 + __popc(hb);
                if (lit & bit) {
                    ob[opad(li)] = T::to_payload(bi < 16 ? half_group63(c0, 0, bi) : half_group63(c1, 1, bi - 16));
                } else if ((zend | oend) & bit) {
                    const int64_t start = hb ? tb + r0 + 31 - __clz(hb) : st0;
                    ob[opad(li)] = fill_word<unsigned long long>((oend & bit) ? G_ONE : G_ZERO,
                                                                 (uint64_t)(tb + r0 + bi - start + 1));
                }
            }
            if (ub && hc > 0) {
                int j = (int)((1 - cb.words - li0) & 31);
                if (j == 0) j = 32;
                if (j <= hc) ub[(cb.words - 1 + li0 + j) >> 5] = tb + r0 + select32(hm, j - 1);
            }
        }
        const uint32_t hm0 = __shfl_sync(0xffffffffu, hm, 0);
        const int lastl = (ng - 1) >> 5, lastb = (ng - 1) & 31;
        const uint32_t lit_l = __shfl_sync(0xffffffffu, lit, lastl);
        const uint32_t end_l = __shfl_sync(0xffffffffu, zend | oend, lastl);
        const bool last_lit = (lit_l >> lastb) & 1u, last_end = (end_l >> lastb) & 1u;
        const bool w0 = !(hm0 & 1u) && (H > 0 || last_end);
        const bool wH = H > 0 ? (last_lit || last_end) : w0;
        __syncwarp();
        const int lo = w0 ? 0 : 1, hi = wH ? H : H - 1;
        for (int k = lo + lane; k <= hi; k += 32) out[cb.words - 1 + k] = ob[opad(k)];
        __syncwarp();
    }
}

// The raw bitmap of every slot whose adaptive format is FMT_RAW: word w =
// bits 32w .. 32w+31 of the slice (the frontier at the slot's range, sieved by
// the slot's directory), bits past the slice cleared.
__global__ void __launch_bounds__(kNT) enc_raw32(EncodeArgs a) {
    if (a.skip && *a.skip) return;
    for (int s = blockIdx.y; s < a.nslots; s += gridDim.y) {
        if (a.fmt[s] != FMT_RAW) continue;
        const SlotGeom sg = slot_geom(a, s);
        const int64_t words = (sg.nbits + 31) >> 5;
        uint32_t* out = static_cast<uint32_t*>(a.out) + (int64_t)s * a.slot_cap;
        for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words;
             w += (int64_t)gridDim.x * blockDim.x) {
            uint32_t x = bits32_at(a.frontier, (uint64_t)(sg.src0 + 32 * w));
            if (sg.dirb) x &= __ldg(sg.dirb + w);
            const int64_t left = sg.nbits - 32 * w;
            if (left < 32) x &= (1u << left) - 1u;
            out[w] = x;
        }
    }
}

// ------------------------------------------------------- standalone decode --
// One CTA decodes the stream into the zeroed output (cta_wah_decode_or);
// malformed streams set *err.
template <typename W>
__global__ void __launch_bounds__(kNT) wah_decode_bitmap_kernel(DecodeArgs a) {
    __shared__ unsigned long long smu[kNT / 32 + 1];
    cta_wah_decode_or<W, kNT>(static_cast<const W*>(a.words), a.nwords, a.nbits, a.bits, 0ull, a.err, smu);
}

}  // namespace

bfs_status launch_wah_encode(const EncodeArgs& a, int wah_bits, cudaStream_t st) {
    if (a.nslots <= 0) return BFS_OK;
    if (wah_bits == 32)
        wah_encode_kernel<uint32_t><<<a.nslots, kNT, 0, st>>>(a, nullptr);
    else
        wah_encode_kernel<unsigned long long><<<a.nslots, kNT, 0, st>>>(a, nullptr);
    BFS_CUDA_TRY(cudaGetLastError());
    return BFS_OK;
}

int64_t parallel_encode_chunks(int64_t max_nbits, int wah_bits) {
    const int64_t G = max_nbits / (wah_bits - 1);
    return (G + kTile - 1) / kTile + 1;
}

bfs_status launch_wah_encode_parallel(const EncodeArgs& a, int wah_bits, void* sums, void* bases, int64_t cps,
                                      void* flags, unsigned long long* setbits, int grid, cudaStream_t st) {
    if (a.nslots <= 0) return BFS_OK;
    ChunkSum* cs = static_cast<ChunkSum*>(sums);
    ChunkBase* cb = static_cast<ChunkBase*>(bases);
    uint8_t* fl = static_cast<uint8_t*>(flags);
    if (a.adaptive && (wah_bits != 32 || !a.fmt)) return set_error(BFS_ERR_INVALID_ARG, "adaptive format needs 32-bit words");
    if (wah_bits == 32) {
        enc_chunk_sums32<<<grid, kEW, 0, st>>>(a, cs, fl, cps, setbits);
        enc_chunk_scan<uint32_t><<<a.nslots, 32, 0, st>>>(a, cs, fl, cb, cps, setbits);
        enc_chunk_write32<<<grid, kEW, 0, st>>>(a, cb, fl, cps);
        if (a.adaptive) {
            dim3 rg(8, (unsigned)std::min(a.nslots, 65535));
            enc_raw32<<<rg, kNT, 0, st>>>(a);
        }
    } else {
        enc_chunk_sums64<<<grid * 2, kEW64, 0, st>>>(a, cs, fl, cps, setbits);
        enc_chunk_scan<unsigned long long><<<a.nslots, 32, 0, st>>>(a, cs, fl, cb, cps, setbits);
        enc_chunk_write64<<<grid * 2, kEW64, 0, st>>>(a, cb, fl, cps);
    }
    BFS_CUDA_TRY(cudaGetLastError());
    return BFS_OK;
}

size_t parallel_encode_sum_bytes() { return sizeof(ChunkSum); }
size_t parallel_encode_base_bytes() { return sizeof(ChunkBase); }

bfs_status launch_wah_decode_bitmap(const DecodeArgs& a, int wah_bits, cudaStream_t st) {
    if (wah_bits == 32)
        wah_decode_bitmap_kernel<uint32_t><<<1, kNT, 0, st>>>(a);
    else
        wah_decode_bitmap_kernel<unsigned long long><<<1, kNT, 0, st>>>(a);
    BFS_CUDA_TRY(cudaGetLastError());
    return BFS_OK;
}

// ---------------------------------------------- allocation-free decoder --
// Scratch of bfs_wah_decode_static: element 0 is the error word, the rest a
// zeroed staging copy of the output bitmap (room for kStaticDecodeMaxBits
// bits plus two words of padding).  Every device that loads the library holds
// this array until the process exits; all calls on a device share it.
constexpr int64_t kStaticDecodeMaxBits = (int64_t)1 << 23;                 // 8,388,608 bits
constexpr int64_t kStaticDecodeWords = kStaticDecodeMaxBits / 32 + 2;      // uint32 staging words
static __device__ __align__(256) unsigned long long g_decode_scratch[1 + (kStaticDecodeWords + 1) / 2];

namespace {
std::mutex g_scratch_mu;
void* g_scratch_addr[256] = {};
}

// Device address of g_decode_scratch on the current device, resolved once per
// device (the name is only a host-side stand-in in host code).
bfs_status static_decode_scratch(void** out) {
    int dev = 0;
    BFS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 256) return set_error(BFS_ERR_INVALID_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        BFS_CUDA_TRY(cudaGetSymbolAddress(&p, g_decode_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return BFS_OK;
}

}  // namespace bfsgb

using namespace bfsgb;

extern "C" {

bfs_status bfs_wah_encode(const uint32_t* bits, int64_t nbits, int32_t word_bits, void* words,
                          int64_t capacity_words, int64_t* nwords, void* stream) {
    if (word_bits != 32 && word_bits != 64) return set_error(BFS_ERR_INVALID_ARG, "word_bits must be 32 or 64");
    if (nbits < 0 || !nwords || (nbits > 0 && (!bits || !words)))
        return set_error(BFS_ERR_INVALID_ARG, "bad encode arguments");
    const int64_t bound = nbits / (word_bits - 1) + 1;
    if (capacity_words < bound)
        return set_error(BFS_ERR_INVALID_ARG, "capacity %lld below the bound %lld", (long long)capacity_words, (long long)bound);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    EncodeArgs a;
    memset(&a, 0, sizeof(a));
    a.frontier = bits;
    a.p = 1;
    a.nb = nbits;
    a.n = nbits;
    a.sieve = 0;
    a.nslots = 1;
    a.out = words;
    a.slot_cap = capacity_words;
    a.counts = nwords;
    if (nbits == 0) {
        BFS_CUDA_TRY(cudaMemsetAsync(nwords, 0, sizeof(int64_t), st));
        return BFS_OK;
    }
    return launch_wah_encode(a, word_bits, st);
}

bfs_status bfs_wah_decode(const void* words, int64_t nwords, int64_t nbits, int32_t word_bits, uint32_t* bits,
                          void* stream) {
    if (word_bits != 32 && word_bits != 64) return set_error(BFS_ERR_INVALID_ARG, "word_bits must be 32 or 64");
    if (nbits < 0 || nwords < 0 || (nwords > 0 && !words) || (nbits > 0 && !bits))
        return set_error(BFS_ERR_INVALID_ARG, "bad decode arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t out_words = (nbits + 31) / 32;
    DevBuf err, pad;
    BFS_TRY(err.alloc(sizeof(unsigned long long)));
    BFS_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(unsigned long long), st));
    // the kernel may OR into the word after the last one: decode into a padded copy
    BFS_TRY(pad.alloc(sizeof(uint32_t) * (out_words + 2)));
    BFS_CUDA_TRY(cudaMemsetAsync(pad.ptr, 0, pad.bytes, st));
    DecodeArgs a;
    a.words = words;
    a.nwords = nwords;
    a.nbits = nbits;
    a.bits = pad.as<uint32_t>();
    a.err = err.as<unsigned long long>();
    BFS_TRY(launch_wah_decode_bitmap(a, word_bits, st));
    unsigned long long h_err = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_err, err.ptr, sizeof(h_err), cudaMemcpyDeviceToHost, st));
    if (out_words > 0)
        BFS_CUDA_TRY(cudaMemcpyAsync(bits, pad.ptr, sizeof(uint32_t) * out_words, cudaMemcpyDeviceToDevice, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) return set_error(BFS_ERR_CORRUPT, "malformed WAH stream");
    return BFS_OK;
}

bfs_status bfs_wah_decode_static(const void* words, int64_t nwords, int64_t nbits, int32_t word_bits, uint32_t* bits,
                                 void* stream) {
    if (word_bits != 32 && word_bits != 64) return set_error(BFS_ERR_INVALID_ARG, "word_bits must be 32 or 64");
    if (nbits < 0 || nwords < 0 || (nwords > 0 && !words) || (nbits > 0 && !bits))
        return set_error(BFS_ERR_INVALID_ARG, "bad decode arguments");
    if (nbits > kStaticDecodeMaxBits)
        return set_error(BFS_ERR_INVALID_ARG, "nbits %lld above the %lld-bit limit of the static scratch",
                         (long long)nbits, (long long)kStaticDecodeMaxBits);
    void* scratch = nullptr;
    BFS_TRY(static_decode_scratch(&scratch));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned long long* err = static_cast<unsigned long long*>(scratch);
    uint32_t* staging = reinterpret_cast<uint32_t*>(err + 1);
    const int64_t out_words = (nbits + 31) / 32;
    // the array keeps the previous call's contents: clear the error word and the staging words used
    BFS_CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(unsigned long long), st));
    BFS_CUDA_TRY(cudaMemsetAsync(staging, 0, sizeof(uint32_t) * (out_words + 2), st));
    DecodeArgs a;
    a.words = words;
    a.nwords = nwords;
    a.nbits = nbits;
    a.bits = staging;
    a.err = err;
    BFS_TRY(launch_wah_decode_bitmap(a, word_bits, st));
    unsigned long long h_err = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_err, err, sizeof(h_err), cudaMemcpyDeviceToHost, st));
    if (out_words > 0)
        BFS_CUDA_TRY(cudaMemcpyAsync(bits, staging, sizeof(uint32_t) * out_words, cudaMemcpyDeviceToDevice, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) return set_error(BFS_ERR_CORRUPT, "malformed WAH stream");
    return BFS_OK;
}

}  // extern "C"
