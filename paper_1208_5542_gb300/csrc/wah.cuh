// wah.cuh -- the word-aligned hybrid word format (Sec. IV, Table 3) on the device.
//
// A w-bit word covers groups of GB = w-1 bitmap bits.  Bit q of a group is
// bitmap bit (group start + q); in the word the first bit of the group is the
// most significant payload bit.  Literal: top bit 0 + payload.  Fill: top bit
// 1, next bit the fill value, low w-2 bits the run length in groups.  Active
// word (when nbits mod GB != 0): the r trailing bits right-aligned, first bit
// highest.
#pragma once

#include <cstdint>

#include "common.cuh"

namespace bfsgb {

enum GroupType : int { G_ZERO = 0, G_ONE = 1, G_LIT = 2, G_NONE = 3 };

// Groups per chunk of the data-parallel encoder (its unit of work, and the
// unit of the chunk index it records for decoders of one chunk).
constexpr int kEncChunkGroups = 1024;

// Formats of an exchanged slice under the level-adaptive exchange (the
// smallest of the three; ties to the lower number): its WAH stream (Sec. IV),
// its sparse vector of set-bit offsets (Sec. II, Table 2), its raw bitmap.
enum SliceFormat : int { FMT_WAH = 0, FMT_LIST = 1, FMT_RAW = 2 };

// Position of the set bit of rank k in x (k = 0 is the lowest set bit),
// by halving on popcounts; k must be < popc(x).
__device__ __forceinline__ int select32(uint32_t v, int k) {
    int pos = 0, c;
    c = __popc(v & 0xffffu); if (k >= c) { k -= c; v >>= 16; pos += 16; }
    c = __popc(v & 0xffu);   if (k >= c) { k -= c; v >>= 8;  pos += 8; }
    c = __popc(v & 0xfu);    if (k >= c) { k -= c; v >>= 4;  pos += 4; }
    c = __popc(v & 0x3u);    if (k >= c) { k -= c; v >>= 2;  pos += 2; }
    c = (int)(v & 1u);       if (k >= c) { pos += 1; }
    return pos;
}

template <typename W> struct Wah;

template <> struct Wah<uint32_t> {
    static constexpr int GB = 31;
    static constexpr uint32_t TOP = 0x80000000u;
    static constexpr uint32_t VAL = 0x40000000u;
    static constexpr uint32_t CNT = 0x3fffffffu;
    static constexpr uint32_t ONES = 0x7fffffffu;
    // group bits (bit q = bitmap bit pos+q) of a bitmap
    __device__ static __forceinline__ uint32_t group(const uint32_t* bm, uint64_t pos) {
        return bits32_at(bm, pos) & ONES;
    }
    __device__ static __forceinline__ uint32_t group_cg(const uint32_t* bm, uint64_t pos) {
        return bits32_at_cg(bm, pos) & ONES;
    }
    // r < 31 bits starting at pos
    __device__ static __forceinline__ uint32_t tail(const uint32_t* bm, uint64_t pos, int r) {
        return bits32_at(bm, pos) & ((1u << r) - 1u);
    }
    // group bits -> literal payload (first bit most significant) and back
    __device__ static __forceinline__ uint32_t to_payload(uint32_t x) { return __brev(x) >> 1; }
    __device__ static __forceinline__ uint32_t from_payload(uint32_t y) { return __brev(y << 1); }
    // r trailing bits -> active word and back
    __device__ static __forceinline__ uint32_t to_active(uint32_t x, int r) { return __brev(x) >> (32 - r); }
    __device__ static __forceinline__ uint32_t from_active(uint32_t y, int r) { return __brev(y << (32 - r)); }
    __device__ static __forceinline__ int popc(uint32_t x) { return __popc(x); }
    // position of the set bit of rank k (k = 0 for the lowest; k < popc(x))
    __device__ static __forceinline__ int select(uint32_t x, int k) { return select32(x, k); }
};

template <> struct Wah<unsigned long long> {
    static constexpr int GB = 63;
    static constexpr unsigned long long TOP = 0x8000000000000000ull;
    static constexpr unsigned long long VAL = 0x4000000000000000ull;
    static constexpr unsigned long long CNT = 0x3fffffffffffffffull;
    static constexpr unsigned long long ONES = 0x7fffffffffffffffull;
    __device__ static __forceinline__ unsigned long long group(const uint32_t* bm, uint64_t pos) {
        return bits64_at(bm, pos) & ONES;
    }
    __device__ static __forceinline__ unsigned long long group_cg(const uint32_t* bm, uint64_t pos) {
        return bits64_at(bm, pos) & ONES;
    }
    __device__ static __forceinline__ unsigned long long tail(const uint32_t* bm, uint64_t pos, int r) {
        return bits64_at(bm, pos) & ((1ull << r) - 1ull);
    }
    __device__ static __forceinline__ unsigned long long to_payload(unsigned long long x) { return __brevll(x) >> 1; }
    __device__ static __forceinline__ unsigned long long from_payload(unsigned long long y) { return __brevll(y << 1); }
    __device__ static __forceinline__ unsigned long long to_active(unsigned long long x, int r) {
        return __brevll(x) >> (64 - r);
    }
    __device__ static __forceinline__ unsigned long long from_active(unsigned long long y, int r) {
        return __brevll(y << (64 - r));
    }
    __device__ static __forceinline__ int popc(unsigned long long x) { return __popcll(x); }
    __device__ static __forceinline__ int select(unsigned long long x, int k) {
        const uint32_t lo = (uint32_t)x;
        const int pl = __popc(lo);
        if (k < pl) return select32(lo, k);
        return 32 + select32((uint32_t)(x >> 32), k - pl);
    }
};

template <typename W>
__device__ __forceinline__ int group_type(W x) {
    return x == W(0) ? G_ZERO : (x == Wah<W>::ONES ? G_ONE : G_LIT);
}

template <typename W>
__device__ __forceinline__ W fill_word(int type, uint64_t count) {
    return Wah<W>::TOP | (type == G_ONE ? Wah<W>::VAL : W(0)) | (W)count;
}

template <typename W>
__device__ __forceinline__ bool is_fill(W y) { return (y & Wah<W>::TOP) != W(0); }

// Groups covered by a word of the body (a fill's run length, else 1).
template <typename W>
__device__ __forceinline__ uint64_t word_groups(W y) {
    return is_fill(y) ? (uint64_t)(y & Wah<W>::CNT) : 1ull;
}

// OR bit q of a bitmap of nbits bits into bits[(bit0 + q) / 32], for every
// bit set in the WAH stream in[0, nwords).  One CTA of NT threads walks the
// stream in tiles of NT words (one per thread), scanning run lengths to place
// each word.  Malformed streams (a fill of length 0, groups past nbits, a
// missing or oversized active word, trailing words) set *err; smu needs NT/32+1
// elements.  Words of the output entirely inside a 1-fill are stored whole.
template <typename W, int NT>
__device__ void cta_wah_decode_or(const W* in, int64_t nwords, int64_t nbits, uint32_t* bits, uint64_t bit0,
                                  unsigned long long* err, unsigned long long* smu) {
    using T = Wah<W>;
    constexpr int GB = T::GB;
    const int64_t G = nbits / GB;
    const int r = (int)(nbits % GB);
    unsigned long long gpos = 0;     // groups consumed before the tile
    auto or_bits = [&](uint64_t bq, uint32_t part) {
        const uint64_t w = bq >> 5;
        const uint32_t sh = (uint32_t)(bq & 31);
        atomicOr(bits + w, part << sh);
        if (sh && (part >> (32 - sh))) atomicOr(bits + w + 1, part >> (32 - sh));
    };
    for (int64_t wb = 0; wb < nwords; wb += NT) {
        const int64_t x = wb + threadIdx.x;
        const bool valid = x < nwords;
        const W y = valid ? in[x] : W(0);
        const unsigned long long len = valid ? (unsigned long long)word_groups<W>(y) : 0ull;
        unsigned long long tot;
        const unsigned long long gs = gpos + block_excl_scan<NT>(len, 0ull, OpSum(), smu, &tot);
        if (valid) {
            bool bad = false;
            if (gs < (unsigned long long)G) {
                if (is_fill<W>(y)) {
                    if (len == 0 || gs + len > (unsigned long long)G) bad = true;
                    else if (y & T::VAL) {
                        const uint64_t b1 = bit0 + (gs + len) * GB;
                        uint64_t b = bit0 + gs * GB;
                        while (b < b1) {
                            const uint64_t w = b >> 5;
                            const uint32_t lo = (uint32_t)(b & 31);
                            const uint64_t take = (b1 - b < 32 - lo) ? b1 - b : 32 - lo;
                            const uint32_t mask = (take == 32) ? 0xffffffffu : (((1u << take) - 1u) << lo);
                            if (mask == 0xffffffffu) bits[w] = mask;
                            else atomicOr(bits + w, mask);
                            b += take;
                        }
                    }
                } else {
                    const W v = T::from_payload(y);
                    for (int q = 0; q < GB; q += 32) {
                        const int nbit = (GB - q < 32) ? GB - q : 32;
                        uint32_t part = (uint32_t)(v >> q);
                        if (nbit < 32) part &= (1u << nbit) - 1u;
                        if (part) or_bits(bit0 + gs * GB + q, part);
                    }
                }
            } else if (gs == (unsigned long long)G && r > 0 && x == nwords - 1) {
                if ((y >> r) != W(0)) bad = true;
                else {
                    const W v = T::from_active(y, r);
                    for (int q = 0; q < r; q += 32) {
                        const int nbit = (r - q < 32) ? r - q : 32;
                        uint32_t part = (uint32_t)(v >> q);
                        if (nbit < 32) part &= (1u << nbit) - 1u;
                        if (part) or_bits(bit0 + gs * GB + q, part);
                    }
                }
            } else {
                bad = true;           // word past the groups, or misplaced active word
            }
            if (bad) atomicOr(err, 1ull);
        }
        gpos += tot;
    }
    if (threadIdx.x == 0 && gpos != (unsigned long long)G + (r > 0 ? 1ull : 0ull)) atomicOr(err, 1ull);
}

}  // namespace bfsgb
