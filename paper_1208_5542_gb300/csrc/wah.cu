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
