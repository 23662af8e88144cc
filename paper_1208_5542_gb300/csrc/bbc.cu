// bbc.cu -- byte-aligned bitmap code (BBC, Antoshenkov) of one bitmap: the
// other bitmap code Sec. IV names beside WAH and PLWAH.  The paper does not
// define it; the reading (include/bfs_gb300.h, bfs_bbc_encode) is:
//   byte k of the bitmap holds bits 8k .. 8k+7, bit 8k most significant;
//   gap byte of value b: 0x00 / 0xFF; map byte: any other; a map byte is odd
//   for b when it differs from the gap byte of value b in one bit;
//   a run is a fill of F gap bytes of value b, then a tail of T <= 15 map
//   bytes or one odd byte (its position in the header):
//     1bFFTTTT  F <= 3, tail          01bFFPPP  F <= 3, odd byte
//     001bTTTT  F >= 4, tail          0001bPPP  F >= 4, odd byte
//   (F >= 4 follows the header as a base-128 counter, low group first);
//   a unit (a maximal fill and the maximal map bytes after it) is one run
//   with the fill and up to 15 map bytes, then runs of F = 0 with 15 each; a
//   final one-byte tail that is odd becomes an odd-byte run.
//
// Encoding is data parallel over bytes and units: flags mark the bytes that
// open a unit and the first map byte of each unit; scans number the units;
// every unit's size follows from its fill and map lengths (and, for the odd
// rule, its last byte); a scan of the sizes places the units; one pass writes
// the first header of each unit, one the map bytes and the later headers.
// Decoding splits the stream into chunks: a record is at most 25 bytes, so a
// chunk's first header lies within its first 25 bytes.  Every chunk is parsed
// from each of the 25 possible entries (where it leaves the chunk, the records
// and bytes it produced); one thread chains the entries from the stream's
// start; then every chunk is parsed again from its real entry, one warp per
// chunk writing the one-fills and the tails into the zeroed output.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace bfsgb {
namespace {

constexpr int kBT = 256;                    // threads per CTA
constexpr int kBPerThread = 16;             // bytes per thread in the flag passes
constexpr int64_t kBTile = kBT * kBPerThread;
constexpr int kMaxRecord = 25;              // header + 9 counter bytes + 15 tail bytes
constexpr int64_t kChunk = 1024;            // stream bytes per decoding chunk
constexpr int64_t kBbcMaxBits = (int64_t)1 << 31;

// Multiprocessors of the current device (grid sizes).
int bbc_sms() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

__device__ __forceinline__ uint32_t brev8(uint32_t x) { return __brev(x) >> 24; }

// Byte k of the bitmap, bit 8k most significant; bits past nbits read as 0.
__device__ __forceinline__ uint32_t bmp_byte(const uint32_t* bits, int64_t nbits, int64_t k) {
    uint32_t x = brev8((bits[k >> 2] >> (8 * (k & 3))) & 0xFFu);
    const int64_t left = nbits - 8 * k;
    if (left < 8) x &= (0xFF00u >> left) & 0xFFu;
    return x;
}

// 0 / 1: a gap byte of that value; 2: a map byte.
__device__ __forceinline__ int bclass(uint32_t x) { return x == 0u ? 0 : (x == 0xFFu ? 1 : 2); }

// Position of the odd bit of x for fill value b (0 = most significant), or -1.
__device__ __forceinline__ int odd_pos(uint32_t x, int b) {
    const uint32_t d = x ^ (b ? 0xFFu : 0u);
    return (d && !(d & (d - 1u))) ? 7 - (31 - __clz(d)) : -1;
}

__device__ __forceinline__ int counter_len(int64_t f) {
    int n = 1;
    while (f >= 128) { f >>= 7; ++n; }
    return n;
}

// The odd position and fill value of a unit's final one-byte tail x: for the
// unit's first run with a fill the fill's value only, otherwise b = 0 first
// and b = 1 second.  Returns -1 (and *rb = the run's b) when it is not odd.
__device__ __forceinline__ int final_odd(uint32_t x, bool first_run, int64_t F, int bf, int* rb) {
    if (first_run && F > 0) { *rb = bf; return odd_pos(x, bf); }
    int p = odd_pos(x, 0);
    if (p >= 0) { *rb = 0; return p; }
    p = odd_pos(x, 1);
    if (p >= 0) { *rb = 1; return p; }
    *rb = first_run ? bf : 0;
    return -1;
}

struct Unit {
    int64_t start, mp, end;     // first byte, first map byte (-1: none), one past the last byte
};

__device__ __forceinline__ Unit unit_of(const int32_t* unit_pos, const int32_t* map_pos, uint32_t U, int64_t nbytes,
                                        uint32_t u) {
    Unit x;
    x.start = unit_pos[u];
    x.end = (u + 1 < U) ? unit_pos[u + 1] : nbytes;
    x.mp = map_pos[u];
    return x;
}

// ---------------------------------------------------------------- encode --
// Flags of every byte (1: opens a unit, 2: the first map byte of a unit) and
// the units opened per tile.
__global__ void __launch_bounds__(kBT) bbc_flags(const uint32_t* __restrict__ bits, int64_t nbits, int64_t nbytes,
                                                 uint8_t* __restrict__ flags, uint32_t* __restrict__ tile_units) {
    __shared__ uint32_t s_sum[kBT / 32];
    const int64_t ntiles = (nbytes + kBTile - 1) / kBTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t k0 = t * kBTile + (int64_t)threadIdx.x * kBPerThread;
        uint32_t units = 0;
        int prev = (k0 > 0 && k0 <= nbytes) ? bclass(bmp_byte(bits, nbits, k0 - 1)) : -1;
        for (int i = 0; i < kBPerThread; ++i) {
            const int64_t k = k0 + i;
            if (k >= nbytes) break;
            const int c = bclass(bmp_byte(bits, nbits, k));
            const bool us = (c < 2 && c != prev) || (k == 0 && c == 2);
            const bool ms = c == 2 && (k == 0 || prev < 2);
            flags[k] = (uint8_t)((us ? 1 : 0) | (ms ? 2 : 0));
            units += us ? 1u : 0u;
            prev = c;
        }
        const uint32_t w = warp_sum(units);
        if (lane_id() == 0) s_sum[threadIdx.x >> 5] = w;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t s = 0;
            for (int i = 0; i < kBT / 32; ++i) s += s_sum[i];
            tile_units[t] = s;
        }
        __syncthreads();
    }
}

// Exclusive scan of n values in one CTA (in place); *total gets their sum.
__global__ void __launch_bounds__(1024) scan_one_cta(uint32_t* __restrict__ v, int64_t n, uint32_t* __restrict__ total) {
    __shared__ uint32_t s_w[33];
    uint32_t carry = 0;
    for (int64_t b = 0; b < n; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const uint32_t x = i < n ? v[i] : 0u;
        const uint32_t incl = warp_incl_sum(x);
        if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x < 32) {
            const uint32_t t = threadIdx.x < (blockDim.x >> 5) ? s_w[threadIdx.x] : 0u;
            const uint32_t ti = warp_incl_sum(t);
            s_w[threadIdx.x] = ti - t;
            if (threadIdx.x == 31) s_w[32] = ti;
        }
        __syncthreads();
        if (i < n) v[i] = carry + s_w[threadIdx.x >> 5] + incl - x;
        carry += s_w[32];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// Unit numbers: every unit's first byte and first map byte.
__global__ void __launch_bounds__(kBT) bbc_number(const uint8_t* __restrict__ flags, int64_t nbytes,
                                                  const uint32_t* __restrict__ tile_base, int32_t* __restrict__ unit_pos,
                                                  int32_t* __restrict__ map_pos) {
    __shared__ uint32_t s_w[kBT / 32 + 1];
    const int64_t ntiles = (nbytes + kBTile - 1) / kBTile;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t k0 = t * kBTile + (int64_t)threadIdx.x * kBPerThread;
        uint32_t mine = 0;
        for (int i = 0; i < kBPerThread && k0 + i < nbytes; ++i) mine += flags[k0 + i] & 1u;
        const uint32_t incl = warp_incl_sum(mine);
        if (lane_id() == 31) s_w[threadIdx.x >> 5] = incl;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t s = 0;
            for (int i = 0; i < kBT / 32; ++i) { const uint32_t y = s_w[i]; s_w[i] = s; s += y; }
        }
        __syncthreads();
        uint32_t before = tile_base[t] + s_w[threadIdx.x >> 5] + incl - mine;   // units opened before k0
        for (int i = 0; i < kBPerThread && k0 + i < nbytes; ++i) {
            const uint32_t f = flags[k0 + i];
            if (f & 1u) unit_pos[before++] = (int32_t)(k0 + i);
            if (f & 2u) map_pos[before - 1] = (int32_t)(k0 + i);     // the unit opened last holds it
        }
        __syncthreads();
    }
}

// Bytes of every unit.
__global__ void __launch_bounds__(kBT) bbc_sizes(const uint32_t* __restrict__ bits, int64_t nbits, int64_t nbytes,
                                                 const int32_t* __restrict__ unit_pos,
                                                 const int32_t* __restrict__ map_pos, const uint32_t* __restrict__ nunits,
                                                 uint32_t* __restrict__ sizes) {
    const uint32_t U = *nunits;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x) {
        const Unit x = unit_of(unit_pos, map_pos, U, nbytes, u);
        const int64_t F = (x.mp >= 0 ? x.mp : x.end) - x.start;
        const int64_t L = x.mp >= 0 ? x.end - x.mp : 0;
        const int bf = F > 0 ? bclass(bmp_byte(bits, nbits, x.start)) : 0;
        int64_t size = (L == 0 ? 1 : (L + 14) / 15) + (F >= 4 ? counter_len(F) : 0) + L;
        if (L % 15 == 1) {
            int rb;
            if (final_odd(bmp_byte(bits, nbits, x.end - 1), L == 1, F, bf, &rb) >= 0) size -= 1;
        }
        sizes[u] = (uint32_t)size;
    }
}

__device__ __forceinline__ int64_t put_counter(uint8_t* out, int64_t at, int64_t f) {
    do {
        uint32_t g = (uint32_t)(f & 0x7F);
        f >>= 7;
        if (f) g |= 0x80u;
        out[at++] = (uint8_t)g;
    } while (f);
    return at;
}

// The first run's header (and counter) of every unit; its odd byte when the
// unit's only map byte is odd.
__global__ void __launch_bounds__(kBT) bbc_heads(const uint32_t* __restrict__ bits, int64_t nbits, int64_t nbytes,
                                                 const int32_t* __restrict__ unit_pos,
                                                 const int32_t* __restrict__ map_pos, const uint32_t* __restrict__ nunits,
                                                 const uint32_t* __restrict__ offs, uint8_t* __restrict__ out) {
    const uint32_t U = *nunits;
    for (uint32_t u = blockIdx.x * blockDim.x + threadIdx.x; u < U; u += gridDim.x * blockDim.x) {
        const Unit x = unit_of(unit_pos, map_pos, U, nbytes, u);
        const int64_t F = (x.mp >= 0 ? x.mp : x.end) - x.start;
        const int64_t L = x.mp >= 0 ? x.end - x.mp : 0;
        const int bf = F > 0 ? bclass(bmp_byte(bits, nbits, x.start)) : 0;
        int64_t at = offs[u];
        int rb = bf, pos = -1;
        if (L == 1) pos = final_odd(bmp_byte(bits, nbits, x.end - 1), true, F, bf, &rb);
        if (pos >= 0) {
            if (F <= 3) out[at++] = (uint8_t)(0x40 | (rb << 5) | ((int)F << 3) | pos);
            else { out[at++] = (uint8_t)(0x10 | (rb << 3) | pos); put_counter(out, at, F); }
        } else {
            const int T = (int)(L < 15 ? L : 15);
            if (F <= 3) out[at++] = (uint8_t)(0x80 | (bf << 6) | ((int)F << 4) | T);
            else { out[at++] = (uint8_t)(0x20 | (bf << 4) | T); put_counter(out, at, F); }
        }
    }
}

// Every map byte (one thread per byte): its unit by binary search, its run
// and place; the first byte of every later run also writes that run's header.
__global__ void __launch_bounds__(kBT) bbc_tails(const uint32_t* __restrict__ bits, int64_t nbits, int64_t nbytes,
                                                 const int32_t* __restrict__ unit_pos,
                                                 const int32_t* __restrict__ map_pos, const uint32_t* __restrict__ nunits,
                                                 const uint32_t* __restrict__ offs, uint8_t* __restrict__ out) {
    const uint32_t U = *nunits;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nbytes; k += stride) {
        const uint32_t xb = bmp_byte(bits, nbits, k);
        if (bclass(xb) < 2) continue;
        uint32_t lo = 0, hi = U - 1;                     // the last unit opened at or before k
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if ((int64_t)unit_pos[mid] <= k) lo = mid; else hi = mid - 1;
        }
        const Unit x = unit_of(unit_pos, map_pos, U, nbytes, lo);
        const int64_t F = x.mp - x.start;
        const int64_t L = x.end - x.mp;
        const int64_t q = k - x.mp;                      // the byte's place among the unit's map bytes
        const int64_t r = q / 15, i = q - 15 * r;
        const int64_t hdr0 = 1 + (F >= 4 ? counter_len(F) : 0);
        const int64_t base = offs[lo];
        if (q == L - 1 && L % 15 == 1) {                 // a final one-byte tail: odd or not
            int rb;
            const int pos = final_odd(xb, r == 0, F, F > 0 ? bclass(bmp_byte(bits, nbits, x.start)) : 0, &rb);
            if (pos >= 0) {
                if (r > 0) out[base + hdr0 + 15 + (r - 1) * 16] = (uint8_t)(0x40 | (rb << 5) | pos);
                continue;                                // run 0's odd byte: bbc_heads wrote it
            }
        }
        if (r == 0) {
            out[base + hdr0 + i] = (uint8_t)xb;
        } else {
            const int64_t rs = base + hdr0 + 15 + (r - 1) * 16;
            if (i == 0) {
                const int64_t T = (L - 15 * r < 15) ? L - 15 * r : 15;
                out[rs] = (uint8_t)(0x80 | T);
            }
            out[rs + 1 + i] = (uint8_t)xb;
        }
    }
}

__global__ void bbc_total(const uint32_t* offs, const uint32_t* sizes, const uint32_t* nunits, int64_t* nout) {
    const uint32_t U = *nunits;
    *nout = U ? (int64_t)offs[U - 1] + sizes[U - 1] : 0;
}

// ---------------------------------------------------------------- decode --
// One record from position at: fills F bytes of value b, then T tail bytes
// from tail_at, or one odd byte.  Returns the position after it, or -1 if
// the header is unused, the counter is cut or too long, or the record runs
// past the stream.
struct Rec {
    int64_t f, tail_at;
    int b, t, odd;
};

__device__ __forceinline__ int64_t parse_rec(const uint8_t* in, int64_t nin, int64_t at, Rec* r) {
    const uint32_t h = in[at++];
    r->odd = -1;
    r->t = 0;
    bool counter = false;
    if (h & 0x80u) { r->b = (h >> 6) & 1; r->f = (h >> 4) & 3; r->t = h & 15; }
    else if (h & 0x40u) { r->b = (h >> 5) & 1; r->f = (h >> 3) & 3; r->odd = h & 7; }
    else if (h & 0x20u) { r->b = (h >> 4) & 1; r->t = h & 15; counter = true; }
    else if (h & 0x10u) { r->b = (h >> 3) & 1; r->odd = h & 7; counter = true; }
    else return -1;
    if (counter) {
        int64_t f = 0;
        int shift = 0;
        for (;;) {
            if (at >= nin || shift > 49) return -1;
            const uint32_t g = in[at++];
            f |= (int64_t)(g & 0x7Fu) << shift;
            shift += 7;
            if (!(g & 0x80u)) break;
        }
        r->f = f;
    }
    r->tail_at = at;
    if (r->odd < 0) {
        if (r->t > nin - at) return -1;
        at += r->t;
    }
    return at;
}

__device__ __forceinline__ int64_t rec_bytes(const Rec& r) { return r.f + (r.odd >= 0 ? 1 : r.t); }

// Per chunk and entry e in [0, kMaxRecord): parse from chunk start + e until
// the position reaches the chunk's end; exit = position - end (0 .. 24), or
// 255 when a record is malformed; bytes = output bytes of the records.
__global__ void __launch_bounds__(kBT) bbc_entries(const uint8_t* __restrict__ in, int64_t nin,
                                                   uint8_t* __restrict__ exits, int64_t* __restrict__ outb) {
    const int64_t nch = (nin + kChunk - 1) / kChunk;
    const int64_t total = nch * kMaxRecord;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total; x += stride) {
        const int64_t c = x / kMaxRecord;
        const int e = (int)(x - c * kMaxRecord);
        const int64_t c0 = c * kChunk, c1 = (c0 + kChunk < nin) ? c0 + kChunk : nin;
        int64_t at = c0 + e, bytes = 0;
        uint8_t ex = 255;
        if (at <= c1) {
            while (at < c1) {
                Rec r;
                at = parse_rec(in, nin, at, &r);
                if (at < 0) break;
                bytes += rec_bytes(r);
            }
            if (at >= c1) ex = (uint8_t)(at - c1);
        }
        exits[x] = ex;
        outb[x] = bytes;
    }
}

// The real entry of every chunk, chained from the stream's start by one
// thread through shared-memory copies of the exit tables (kChainChunks chunks
// at a time); then the output bytes of every chunk from its real entry.  The
// last chunk must end exactly at the stream's end.
constexpr int kChainChunks = 1536;

__global__ void __launch_bounds__(1024) bbc_chain(const uint8_t* __restrict__ exits, const int64_t* __restrict__ outb,
                                                  int64_t nin, uint8_t* __restrict__ entry, uint32_t* __restrict__ sel,
                                                  unsigned long long* err) {
    __shared__ uint8_t s_ex[kChainChunks * kMaxRecord];
    __shared__ int s_e;
    const int64_t nch = (nin + kChunk - 1) / kChunk;
    if (threadIdx.x == 0) s_e = 0;
    for (int64_t c0 = 0; c0 < nch; c0 += kChainChunks) {
        const int64_t cn = (nch - c0 < kChainChunks) ? nch - c0 : kChainChunks;
        __syncthreads();
        for (int64_t x = threadIdx.x; x < cn * kMaxRecord; x += blockDim.x) s_ex[x] = exits[c0 * kMaxRecord + x];
        __syncthreads();
        if (threadIdx.x == 0) {
            int e = s_e;
            for (int64_t c = 0; c < cn; ++c) {
                entry[c0 + c] = (uint8_t)e;
                const uint8_t ex = s_ex[c * kMaxRecord + e];
                if (ex == 255) { *err = 1; e = 0; break; }
                e = ex;
            }
            s_e = e;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && s_e != 0) *err = 1;
    __syncthreads();
    for (int64_t c = threadIdx.x; c < nch; c += blockDim.x)
        sel[c] = (uint32_t)outb[c * kMaxRecord + entry[c]];
}

// One warp per chunk: parse from its real entry; write the one-fill bytes and
// the tails (bytes past nbytes are an error; the output was zeroed).
__global__ void __launch_bounds__(kBT) bbc_expand(const uint8_t* __restrict__ in, int64_t nin, int64_t nbytes,
                                                  const uint8_t* __restrict__ entry, const uint32_t* __restrict__ out_base,
                                                  uint8_t* __restrict__ out8, unsigned long long* err) {
    const int64_t nch = (nin + kChunk - 1) / kChunk;
    const int lane = (int)lane_id();
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t ws = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = w0; c < nch; c += ws) {
        const int64_t c0 = c * kChunk, c1 = (c0 + kChunk < nin) ? c0 + kChunk : nin;
        int64_t at = c0 + entry[c], k = out_base[c];
        while (at < c1) {
            Rec r;
            at = parse_rec(in, nin, at, &r);           // every lane parses the same record
            if (at < 0 || rec_bytes(r) > nbytes - k) {
                if (lane == 0) atomicOr(err, 1ull);
                break;
            }
            if (r.b)
                for (int64_t q = lane; q < r.f; q += 32) out8[k + q] = 0xFF;
            k += r.f;
            if (r.odd >= 0) {
                if (lane == 0) out8[k] = (uint8_t)brev8((r.b ? 0xFFu : 0u) ^ (0x80u >> r.odd));
                k += 1;
            } else {
                if (lane < r.t) out8[k + lane] = (uint8_t)brev8(in[r.tail_at + lane]);
                k += r.t;
            }
        }
    }
}

// Bits past nbits in the last decoded byte must be 0.
__global__ void bbc_padding(const uint8_t* out8, int64_t nbits, unsigned long long* err) {
    const int64_t nbytes = (nbits + 7) / 8;
    const int r = (int)(nbits & 7);
    if (r && (out8[nbytes - 1] >> r)) *err = 1;        // stored LSB-first: bit j of the byte = bit 8k+j
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" {

bfs_status bfs_bbc_encode(const uint32_t* bits, int64_t nbits, uint8_t* bytes, int64_t capacity_bytes,
                          int64_t* nbytes_out, void* stream) {
    if (nbits < 0 || nbits >= kBbcMaxBits)
        return set_error(BFS_ERR_INVALID_ARG, "nbits %lld outside [0, 2^31)", (long long)nbits);
    if (!nbytes_out || (nbits > 0 && (!bits || !bytes))) return set_error(BFS_ERR_INVALID_ARG, "bad encode arguments");
    const int64_t nbytes = (nbits + 7) / 8;
    const int64_t bound = nbytes + nbytes / 15 + 11;
    if (capacity_bytes < bound)
        return set_error(BFS_ERR_INVALID_ARG, "capacity %lld below the bound %lld", (long long)capacity_bytes,
                         (long long)bound);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (nbits == 0) {
        BFS_CUDA_TRY(cudaMemsetAsync(nbytes_out, 0, sizeof(int64_t), st));
        return BFS_OK;
    }
    const int64_t ntiles = (nbytes + kBTile - 1) / kBTile;
    const int sms = bbc_sms();
    DevBuf flags, tiles, cnt, upos, mpos, sizes, offs;
    BFS_TRY(flags.alloc((size_t)nbytes));
    BFS_TRY(tiles.alloc(sizeof(uint32_t) * (size_t)ntiles));
    BFS_TRY(cnt.alloc(sizeof(uint32_t) * 2));
    BFS_TRY(upos.alloc(sizeof(int32_t) * (size_t)nbytes));
    BFS_TRY(mpos.alloc(sizeof(int32_t) * (size_t)nbytes));
    BFS_TRY(sizes.alloc(sizeof(uint32_t) * (size_t)nbytes));
    BFS_TRY(offs.alloc(sizeof(uint32_t) * (size_t)nbytes));
    const int grid = (int)std::min<int64_t>(std::max<int64_t>(ntiles, 1), (int64_t)sms * 8);
    const int egrid = (int)std::min<int64_t>((nbytes + kBT - 1) / kBT, (int64_t)sms * 16);
    BFS_CUDA_TRY(cudaMemsetAsync(mpos.ptr, 0xFF, mpos.bytes, st));
    uint32_t* nunits = cnt.as<uint32_t>();
    bbc_flags<<<grid, kBT, 0, st>>>(bits, nbits, nbytes, flags.as<uint8_t>(), tiles.as<uint32_t>());
    scan_one_cta<<<1, 1024, 0, st>>>(tiles.as<uint32_t>(), ntiles, nunits);
    bbc_number<<<grid, kBT, 0, st>>>(flags.as<uint8_t>(), nbytes, tiles.as<uint32_t>(), upos.as<int32_t>(),
                                     mpos.as<int32_t>());
    bbc_sizes<<<egrid, kBT, 0, st>>>(bits, nbits, nbytes, upos.as<int32_t>(), mpos.as<int32_t>(), nunits,
                                     sizes.as<uint32_t>());
    BFS_CUDA_TRY(cudaMemcpyAsync(offs.ptr, sizes.ptr, sizes.bytes, cudaMemcpyDeviceToDevice, st));
    uint32_t h_units = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_units, nunits, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    scan_one_cta<<<1, 1024, 0, st>>>(offs.as<uint32_t>(), (int64_t)h_units, nunits + 1);
    bbc_heads<<<egrid, kBT, 0, st>>>(bits, nbits, nbytes, upos.as<int32_t>(), mpos.as<int32_t>(), nunits,
                                     offs.as<uint32_t>(), bytes);
    bbc_tails<<<egrid, kBT, 0, st>>>(bits, nbits, nbytes, upos.as<int32_t>(), mpos.as<int32_t>(), nunits,
                                     offs.as<uint32_t>(), bytes);
    bbc_total<<<1, 1, 0, st>>>(offs.as<uint32_t>(), sizes.as<uint32_t>(), nunits, nbytes_out);
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaStreamSynchronize(st));          // the scratch is released on return
    return BFS_OK;
}

bfs_status bfs_bbc_decode(const uint8_t* bytes, int64_t nbytes_in, int64_t nbits, uint32_t* bits, void* stream) {
    if (nbits < 0 || nbits >= kBbcMaxBits)
        return set_error(BFS_ERR_INVALID_ARG, "nbits %lld outside [0, 2^31)", (long long)nbits);
    if (nbytes_in < 0 || (nbytes_in > 0 && !bytes) || (nbits > 0 && !bits))
        return set_error(BFS_ERR_INVALID_ARG, "bad decode arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t nbytes = (nbits + 7) / 8;
    if (nbits > 0) BFS_CUDA_TRY(cudaMemsetAsync(bits, 0, sizeof(uint32_t) * (size_t)((nbits + 31) / 32), st));
    if (nbytes_in == 0) {
        if (nbytes != 0) return set_error(BFS_ERR_CORRUPT, "malformed BBC stream (empty for %lld bits)", (long long)nbits);
        return BFS_OK;
    }
    const int64_t nch = (nbytes_in + kChunk - 1) / kChunk;
    const int sms = bbc_sms();
    DevBuf exits, outb, entry, obase, err, tot;
    BFS_TRY(exits.alloc((size_t)(nch * kMaxRecord)));
    BFS_TRY(outb.alloc(sizeof(int64_t) * (size_t)(nch * kMaxRecord)));
    BFS_TRY(entry.alloc((size_t)nch));
    BFS_TRY(obase.alloc(sizeof(uint32_t) * (size_t)nch));
    BFS_TRY(err.alloc(sizeof(unsigned long long)));
    BFS_TRY(tot.alloc(sizeof(uint32_t)));
    BFS_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(unsigned long long), st));
    const int grid = (int)std::min<int64_t>((nch * kMaxRecord + kBT - 1) / kBT, (int64_t)sms * 16);
    bbc_entries<<<grid, kBT, 0, st>>>(bytes, nbytes_in, exits.as<uint8_t>(), outb.as<int64_t>());
    bbc_chain<<<1, 1024, 0, st>>>(exits.as<uint8_t>(), outb.as<int64_t>(), nbytes_in, entry.as<uint8_t>(),
                                  obase.as<uint32_t>(), err.as<unsigned long long>());
    scan_one_cta<<<1, 1024, 0, st>>>(obase.as<uint32_t>(), nch, tot.as<uint32_t>());
    unsigned long long h_err = 0;
    uint32_t h_tot = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_err, err.ptr, sizeof(h_err), cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_tot, tot.ptr, sizeof(h_tot), cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err || (int64_t)h_tot != nbytes) return set_error(BFS_ERR_CORRUPT, "malformed BBC stream");
    const int xgrid = (int)std::min<int64_t>((nch * 32 + kBT - 1) / kBT, (int64_t)sms * 16);
    bbc_expand<<<xgrid, kBT, 0, st>>>(bytes, nbytes_in, nbytes, entry.as<uint8_t>(), obase.as<uint32_t>(),
                                      reinterpret_cast<uint8_t*>(bits), err.as<unsigned long long>());
    bbc_padding<<<1, 1, 0, st>>>(reinterpret_cast<const uint8_t*>(bits), nbits, err.as<unsigned long long>());
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_err, err.ptr, sizeof(h_err), cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) return set_error(BFS_ERR_CORRUPT, "malformed BBC stream");
    return BFS_OK;
}

}  // extern "C"
