// wah.cu -- WAH compress (Sec. IV, Table 3; Alg. 2 line 7, Alg. 3 line 10),
// fused with the cross-directory sieve (Alg. 3 line 9), and the standalone
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

struct SlotGeom {
    int64_t src0;      // first bitmap bit of the slot's source range
    int64_t nbits;     // bits in the slot
    const uint32_t* dirb;   // directory of the slot's block, or nullptr
};

__device__ __forceinline__ SlotGeom slot_geom(const EncodeArgs& a, int s) {
    const int j = a.sieve ? (s % a.p) : s;
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
            if (sg.dirb && y) y &= T::tail(sg.dirb, (uint64_t)(G * GB), r);
            if (setbits && y) atomicAdd(setbits, (unsigned long long)T::popc(y));
            out[total++] = T::to_active(y, r);
        }
        a.counts[s] = total;
    }
}

// ------------------------------------------------- parallel slot encoder --
// The same stream as wah_encode_kernel, built in data-parallel passes over
// (slot, chunk of kTile groups):
//   0. enc_chunk_flags: one thread per chunk tests the frontier summary and
//      appends the chunks with any frontier bit to a work list;
//   1. enc_chunk_sums: one warp per listed chunk, 32 groups per step: its
//      head count (its first group counted as a head), first and last group
//      type and last head position, from ballots of the head flags;
//   2. enc_chunk_scan: per slot, one warp scans the chunk sums (an all-zero
//      chunk is one zero run): a chunk whose first group continues the previous
//      chunk's fill run merges with it; this gives every chunk its first word
//      index and the start of the run it opens with, the slot's word count and
//      the active word, and writes the fill word of every zero run that ends
//      in an all-zero chunk;
//   3. enc_chunk_write: one warp per listed chunk writes its words, each
//      lane's word index and run start taken from the ballot of the head flags
//      and the chunk's carry from pass 2.
// With unit_base set, the group at which every 32nd word opens is recorded
// as the word is written (the decoder's unit bases).
constexpr int kU = 8;             // 32-group steps whose loads a warp issues together

// Groups gb + 32k + lane (k < kU) of a slot, 0 at and beyond group G.  For
// 31-bit groups a step of 32 groups is exactly 31 words of the directory and
// at most 32 words of the frontier: every lane loads one word of each
// (coalesced), and its group is funnel-shifted from the two words it spans,
// fetched by shuffles.  The directory is not read when the frontier words of
// all kU steps are zero.  63-bit groups are read per lane.
template <typename W>
__device__ __forceinline__ void warp_groups(const EncodeArgs& a, const SlotGeom& sg, int64_t gb, int64_t G,
                                            W (&x)[kU]) {
    const int lane = (int)lane_id();
    if constexpr (sizeof(W) == 4) {
        uint32_t fw[kU], dw[kU];
        const int64_t last = G * 31;                                // bits of the full groups
        const int64_t fmax = last > 0 ? (sg.src0 + last - 1) >> 5 : -1;
        const int64_t dmax = last > 0 ? (last - 1) >> 5 : -1;
        const int64_t p0 = sg.src0 + gb * 31;
        const uint32_t sh0 = (uint32_t)(p0 & 31);
        bool any = false;
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int64_t w = (p0 >> 5) + 31 * k + lane;
            fw[k] = (w <= fmax) ? __ldg(a.frontier + w) : 0u;
            any |= fw[k] != 0u;
        }
        const bool sieve = sg.dirb != nullptr;
        const bool need_dir = sieve && __any_sync(0xffffffffu, any);
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int64_t w = ((gb * 31) >> 5) + 31 * k + lane;
            dw[k] = (need_dir && lane < 31 && w <= dmax) ? __ldg(sg.dirb + w) : 0u;
        }
        const uint32_t rel = 31u * (uint32_t)lane + sh0;
        const int fa = (int)(rel >> 5), fb = fa + 1 < 32 ? fa + 1 : 31;
        const int da = (31 * lane) >> 5;
        const uint32_t dsh = (31u * (uint32_t)lane) & 31u;
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const uint32_t lo = __shfl_sync(0xffffffffu, fw[k], fa);
            const uint32_t hi = __shfl_sync(0xffffffffu, fw[k], fb);
            uint32_t v = __funnelshift_r(lo, hi, rel & 31u) & 0x7fffffffu;
            if (sieve) {
                const uint32_t dlo = __shfl_sync(0xffffffffu, dw[k], da);
                const uint32_t dhi = __shfl_sync(0xffffffffu, dw[k], da + 1);
                v &= __funnelshift_r(dlo, dhi, dsh) & 0x7fffffffu;
            }
            x[k] = (gb + 32 * k + lane < G) ? (W)v : W(0);
        }
    } else {
        const SlotGeom g = sg;
#pragma unroll
        for (int k = 0; k < kU; ++k) {
            const int64_t gi = gb + 32 * k + lane;
            x[k] = (gi < G) ? load_group<W>(a, g, gi) : W(0);
        }
    }
}

struct ChunkSum {
    uint32_t heads;
    uint32_t types;        // first type | last type << 8
    int64_t last_head;     // group index of the chunk's last head
};
struct ChunkBase {
    int64_t words;         // index of the next word to open at the chunk's first group
    int64_t run_start;     // start group of the run open before the chunk
    int32_t prev_type;     // type of the group before the chunk (-1 at the slot start)
    int32_t next_type;     // type of the group after the chunk (G_NONE at the slot end)
};

template <typename W>
__global__ void enc_chunk_flags(EncodeArgs a, int64_t cps, uint8_t* flags, int64_t* list,
                                unsigned long long* nlist) {
    constexpr int GB = Wah<W>::GB;
    const int64_t total = (int64_t)a.nslots * cps;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q - (int64_t)lane_id() < total;
         q += (int64_t)gridDim.x * blockDim.x) {
        bool live = false;
        if (q < total) {
            const int s = (int)(q / cps);
            const int64_t c = q % cps;
            const SlotGeom sg = slot_geom(a, s);
            const int64_t G = sg.nbits / GB;
            const int64_t tb = c * kTile;
            if (tb < G) {
                const int64_t tend = (tb + kTile < G) ? tb + kTile : G;
                live = !a.fsum || !fsum_zero(a.fsum, (sg.src0 + tb * GB) >> 10, (sg.src0 + tend * GB - 1) >> 10);
            }
            flags[q] = live ? 1 : 0;
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, live);
        if (ball) {
            unsigned long long base = 0;
            if (lane_id() == 0) base = atomicAdd(nlist, (unsigned long long)__popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (live) list[base + __popc(ball & ((1u << lane_id()) - 1u))] = q;
        }
    }
}

template <typename W>
__global__ void __launch_bounds__(kNT) enc_chunk_sums(EncodeArgs a, ChunkSum* sums, int64_t cps,
                                                      const int64_t* list, const unsigned long long* nlist,
                                                      unsigned long long* setbits) {
    using T = Wah<W>;
    constexpr int GB = T::GB;
    const unsigned long long n = *nlist;
    const int lane = (int)lane_id();
    const unsigned long long wid = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    unsigned long long ones = 0;
    for (unsigned long long li = wid; li < n; li += nw) {
        const int64_t q = list[li];
        const int s = (int)(q / cps);
        const int64_t c = q % cps;
        const SlotGeom sg = slot_geom(a, s);
        const int64_t G = sg.nbits / GB;
        const int64_t tb = c * kTile;
        const int64_t tend = (tb + kTile < G) ? tb + kTile : G;
        int prev = -1, first = G_NONE;
        uint32_t heads = 0;
        int64_t last_head = -1;
        for (int64_t gb = tb; gb < tend; gb += 32 * kU) {
            W x[kU];                  // the loads of kU steps are issued together
            warp_groups<W>(a, sg, gb, tend, x);
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                const int64_t g0 = gb + 32 * k;
                if (g0 >= tend) break;
                const bool valid = g0 + lane < tend;
                const int ty = valid ? group_type<W>(x[k]) : G_NONE;
                ones += (unsigned long long)T::popc(x[k]);
                int pt = __shfl_up_sync(0xffffffffu, ty, 1);
                if (lane == 0) pt = prev;
                const uint32_t b = __ballot_sync(0xffffffffu, valid && (ty == G_LIT || ty != pt));
                heads += __popc(b);
                if (b) last_head = g0 + 31 - __clz(b);
                if (g0 == tb) first = __shfl_sync(0xffffffffu, ty, 0);
                const int lv = (tend - g0 < 32) ? (int)(tend - g0 - 1) : 31;
                prev = __shfl_sync(0xffffffffu, ty, lv);
            }
        }
        if (lane == 0) {
            ChunkSum cs;
            cs.heads = heads;
            cs.types = (uint32_t)first | ((uint32_t)prev << 8);
            cs.last_head = last_head;
            sums[q] = cs;
        }
    }
    if (setbits) {
        ones = warp_sum(ones);
        if (lane == 0 && ones) atomicAdd(setbits, ones);
    }
}

// One warp per slot (blockDim.x = 32).
template <typename W>
__global__ void enc_chunk_scan(EncodeArgs a, const ChunkSum* sums, const uint8_t* flags, ChunkBase* bases,
                               int64_t cps, unsigned long long* setbits) {
    using T = Wah<W>;
    constexpr int GB = T::GB;
    const int s = blockIdx.x;
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
        return cs;
    };
    int64_t words = 0, hmax = -1;
    int prev_last = -1;
    for (int64_t c0 = 0; c0 < nch; c0 += 32) {
        const int64_t c = c0 + lane;
        ChunkSum cs;
        cs.heads = 0;
        cs.types = G_NONE | (G_NONE << 8);
        cs.last_head = -1;
        if (c < nch) cs = sum_of(c);
        const int first = (int)(cs.types & 0xff), last = (int)((cs.types >> 8) & 0xff);
        int before = __shfl_up_sync(0xffffffffu, last, 1);
        if (lane == 0) before = prev_last;
        const bool merge = (c < nch) && before == first && first != G_LIT && before >= 0;
        const int64_t eff = (c < nch) ? (int64_t)cs.heads - (merge ? 1 : 0) : 0;
        const int64_t h = (c < nch) ? ((merge && cs.heads == 1) ? (int64_t)-1 : cs.last_head) : (int64_t)-1;
        int64_t incl = eff, hin = h;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, incl, d);
            const int64_t z = __shfl_up_sync(0xffffffffu, hin, d);
            if (lane >= d) { incl += y; hin = z > hin ? z : hin; }
        }
        int64_t hex = __shfl_up_sync(0xffffffffu, hin, 1);
        if (lane == 0) hex = -1;
        hex = hex > hmax ? hex : hmax;
        int nxt = __shfl_down_sync(0xffffffffu, first, 1);
        if (c < nch) {
            ChunkBase cb;
            cb.words = words + incl - eff;
            cb.run_start = merge ? hex : c * kTile;
            cb.prev_type = before;
            if (c + 1 >= nch) nxt = G_NONE;
            else if (lane == 31) nxt = (int)(sum_of(c + 1).types & 0xff);
            cb.next_type = nxt;
            bases[(int64_t)s * cps + c] = cb;
            if (!flags[(int64_t)s * cps + c]) {
                // an all-zero chunk: its zero run opens a word here unless it merges
                if (!merge && ub && (cb.words & 31) == 0) ub[cb.words >> 5] = c * kTile;
                if (nxt != G_ZERO) {     // the run ends at the chunk's last group
                    const int64_t tend = ((c + 1) * kTile < G) ? (c + 1) * kTile : G;
                    const int64_t start = merge ? cb.run_start : c * kTile;
                    out[merge ? cb.words - 1 : cb.words] = fill_word<W>(G_ZERO, (uint64_t)(tend - start));
                }
            }
        }
        words += __shfl_sync(0xffffffffu, incl, 31);
        const int64_t hb = __shfl_sync(0xffffffffu, hin, 31);
        hmax = hb > hmax ? hb : hmax;
        const int last_lane = (c0 + 32 > nch) ? (int)((nch - 1) % 32) : 31;
        prev_last = __shfl_sync(0xffffffffu, last, last_lane);
    }
    if (lane == 0) {
        int64_t total = words;
        if (r > 0) {
            const uint64_t pos = (uint64_t)(sg.src0 + G * GB);
            W y = T::tail(a.frontier, pos, r);
            if (sg.dirb && y) y &= T::tail(sg.dirb, (uint64_t)(G * GB), r);
            if (setbits && y) atomicAdd(setbits, (unsigned long long)T::popc(y));
            if (ub && (total & 31) == 0) ub[total >> 5] = G;
            out[total++] = T::to_active(y, r);
        }
        a.counts[s] = total;
        if (a.wah_words) atomicAdd(a.wah_words, (unsigned long long)total);
    }
}

template <typename W>
__global__ void __launch_bounds__(kNT) enc_chunk_write(EncodeArgs a, const ChunkBase* bases, int64_t cps,
                                                       const int64_t* list, const unsigned long long* nlist) {
    using T = Wah<W>;
    constexpr int GB = T::GB;
    const unsigned long long n = *nlist;
    const int lane = (int)lane_id();
    const uint32_t le_mask = 0xffffffffu >> (31 - lane);        // lanes 0..lane
    const unsigned long long wid = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long li = wid; li < n; li += nw) {
        const int64_t q = list[li];
        const int s = (int)(q / cps);
        const int64_t c = q % cps;
        const SlotGeom sg = slot_geom(a, s);
        const int64_t G = sg.nbits / GB;
        const int64_t tb = c * kTile;
        const int64_t tend = (tb + kTile < G) ? tb + kTile : G;
        const ChunkBase cb = bases[q];
        W* out = static_cast<W*>(a.out) + (int64_t)s * a.slot_cap;
        int64_t* ub = a.unit_base ? a.unit_base + (int64_t)s * a.unit_stride : nullptr;
        int64_t base = cb.words;          // next word to open
        int64_t run_start = cb.run_start;
        int prev = cb.prev_type;
        for (int64_t gb = tb; gb < tend; gb += 32 * kU) {
            W x[kU];
            int tys[kU];
            warp_groups<W>(a, sg, gb, tend, x);
#pragma unroll
            for (int k = 0; k < kU; ++k) tys[k] = (gb + 32 * k + lane < tend) ? group_type<W>(x[k]) : G_NONE;
#pragma unroll
            for (int k = 0; k < kU; ++k) {
                const int64_t g0 = gb + 32 * k;
                if (g0 >= tend) break;
                const int64_t g = g0 + lane;
                const bool valid = g < tend;
                const int ty = tys[k];
                int pt = __shfl_up_sync(0xffffffffu, ty, 1);
                if (lane == 0) pt = prev;
                const bool h = valid && (ty == G_LIT || ty != pt);
                const uint32_t b = __ballot_sync(0xffffffffu, h);
                int nt = __shfl_down_sync(0xffffffffu, ty, 1);
                const int nt31 = (k + 1 < kU) ? __shfl_sync(0xffffffffu, tys[k + 1 < kU ? k + 1 : k], 0) : G_NONE;
                if (valid) {
                    const uint32_t bl = b & le_mask;
                    const int64_t widx = base + __popc(bl) - 1;
                    const int64_t start = bl ? g0 + 31 - __clz(bl) : run_start;
                    if (g + 1 == tend) nt = cb.next_type;
                    else if (lane == 31) nt = (k + 1 < kU) ? nt31 : group_type<W>(load_group<W>(a, sg, g + 1));
                    if (ty == G_LIT) out[widx] = T::to_payload(x[k]);
                    else if (nt != ty) out[widx] = fill_word<W>(ty, (uint64_t)(g - start + 1));
                    if (h && ub && (widx & 31) == 0) ub[widx >> 5] = g;
                }
                base += __popc(b);
                if (b) run_start = g0 + 31 - __clz(b);
                const int lv = (tend - g0 < 32) ? (int)(tend - g0 - 1) : 31;
                prev = __shfl_sync(0xffffffffu, ty, lv);
            }
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

bfs_status launch_wah_encode_counted(const EncodeArgs& a, int wah_bits, unsigned long long* setbits,
                                     cudaStream_t st) {
    if (a.nslots <= 0) return BFS_OK;
    if (wah_bits == 32)
        wah_encode_kernel<uint32_t><<<a.nslots, kNT, 0, st>>>(a, setbits);
    else
        wah_encode_kernel<unsigned long long><<<a.nslots, kNT, 0, st>>>(a, setbits);
    BFS_CUDA_TRY(cudaGetLastError());
    return BFS_OK;
}

int64_t parallel_encode_chunks(int64_t max_nbits, int wah_bits) {
    const int64_t G = max_nbits / (wah_bits - 1);
    return (G + kTile - 1) / kTile + 1;
}

bfs_status launch_wah_encode_parallel(const EncodeArgs& a, int wah_bits, void* sums, void* bases, int64_t cps,
                                      void* flags, void* list, unsigned long long* nlist, unsigned long long* setbits,
                                      int grid, cudaStream_t st) {
    if (a.nslots <= 0) return BFS_OK;
    ChunkSum* cs = static_cast<ChunkSum*>(sums);
    ChunkBase* cb = static_cast<ChunkBase*>(bases);
    uint8_t* fl = static_cast<uint8_t*>(flags);
    int64_t* li = static_cast<int64_t*>(list);
    BFS_CUDA_TRY(cudaMemsetAsync(nlist, 0, sizeof(unsigned long long), st));
    const int64_t total = (int64_t)a.nslots * cps;
    const int fgrid = (int)std::min<int64_t>((total + kNT - 1) / kNT, grid);
    if (wah_bits == 32) {
        enc_chunk_flags<uint32_t><<<fgrid, kNT, 0, st>>>(a, cps, fl, li, nlist);
        enc_chunk_sums<uint32_t><<<grid, kNT, 0, st>>>(a, cs, cps, li, nlist, setbits);
        enc_chunk_scan<uint32_t><<<a.nslots, 32, 0, st>>>(a, cs, fl, cb, cps, setbits);
        enc_chunk_write<uint32_t><<<grid, kNT, 0, st>>>(a, cb, cps, li, nlist);
    } else {
        enc_chunk_flags<unsigned long long><<<fgrid, kNT, 0, st>>>(a, cps, fl, li, nlist);
        enc_chunk_sums<unsigned long long><<<grid, kNT, 0, st>>>(a, cs, cps, li, nlist, setbits);
        enc_chunk_scan<unsigned long long><<<a.nslots, 32, 0, st>>>(a, cs, fl, cb, cps, setbits);
        enc_chunk_write<unsigned long long><<<grid, kNT, 0, st>>>(a, cb, cps, li, nlist);
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
