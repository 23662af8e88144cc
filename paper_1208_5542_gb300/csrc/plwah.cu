// plwah.cu -- position-list word-aligned hybrid (PLWAH) code of one bitmap:
// the alternative bitmap code Sec. IV names beside WAH (Deliege and
// Pedersen).  32-bit words over 31-bit groups, as the 32-bit WAH code; a fill
// word keeps 25 bits of run length and uses bits 29..25 for the position
// (1 = first bit of the group, 0 = none) of the one odd bit of the group right
// after its run, which is then not written.
//
// PLWAH of a bitmap is its WAH stream with every literal that follows a fill
// word and differs from the fill value in one bit folded into that fill word
// (runs stay below 2^25 groups under the size limit of the entry points), so
// both directions are word-parallel transcodings around the WAH kernels: one
// CTA walks the stream in tiles, a block scan places the output words.
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace bfsgb {
namespace {

constexpr int kPT = 1024;                             // threads of the transcoding CTA
constexpr uint32_t kTop = 0x80000000u, kVal = 0x40000000u, kOnes = 0x7fffffffu;
constexpr uint32_t kCount25 = (1u << 25) - 1u;
constexpr int64_t kPlwahMaxBits = 31LL * ((1LL << 25) - 1);   // every run below 2^25 groups

// Exclusive scan of one value per thread over the CTA; returns the thread's
// offset and the total in *total.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* s_warp, uint32_t* total) {
    const uint32_t incl = warp_incl_sum(x);
    const int w = threadIdx.x >> 5;
    if (lane_id() == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        const uint32_t t = (lane_id() < (uint32_t)(blockDim.x >> 5)) ? s_warp[lane_id()] : 0u;
        const uint32_t ti = warp_incl_sum(t);
        s_warp[lane_id()] = ti - t;
        if (lane_id() == 31) s_warp[32] = ti;
    }
    __syncthreads();
    const uint32_t out = incl - x + s_warp[w];
    *total = s_warp[32];
    __syncthreads();                                  // s_warp is reused by the next tile
    return out;
}

// The odd bit of a literal against fill value v: its place (1..31), or 0 if
// the literal differs from the fill pattern in more or fewer than one bit.
__device__ __forceinline__ uint32_t odd_place(uint32_t lit, uint32_t v) {
    const uint32_t diff = lit ^ (v ? kOnes : 0u);
    return (diff && !(diff & (diff - 1u))) ? (uint32_t)__clz(diff) : 0u;   // bit 30 (first) -> 1
}

// WAH (32-bit words, runs < 2^25 groups) -> PLWAH.  A literal word k is
// folded when word k-1 is a fill and the literal is one bit off its value;
// the active word (the last word when nbits mod 31 != 0) is copied.
__global__ void __launch_bounds__(kPT) plwah_from_wah(const uint32_t* __restrict__ wah, const int64_t* __restrict__ nw_p,
                                                      int64_t nbits, uint32_t* __restrict__ out,
                                                      int64_t* __restrict__ out_count) {
    __shared__ uint32_t s_warp[33];
    const int64_t nw = *nw_p;
    const bool has_active = (nbits % 31) != 0;
    auto is_fill = [&](int64_t k) { return !(has_active && k == nw - 1) && (wah[k] & kTop); };
    int64_t carry = 0;
    for (int64_t base = 0; base < nw; base += kPT) {
        const int64_t k = base + threadIdx.x;
        uint32_t emit = 0, word = 0;
        if (k < nw) {
            const uint32_t w = wah[k];
            const bool active = has_active && k == nw - 1;
            bool folded = false;
            if (!active && !(w & kTop) && k > 0 && is_fill(k - 1))
                folded = odd_place(w, wah[k - 1] & kVal) != 0u;
            if (!folded) {
                emit = 1;
                word = w;
                if (is_fill(k)) {
                    uint32_t q = 0;
                    if (k + 1 < nw && !(has_active && k + 1 == nw - 1) && !(wah[k + 1] & kTop))
                        q = odd_place(wah[k + 1], w & kVal);
                    word = kTop | (w & kVal) | (q << 25) | (w & kCount25);
                }
            }
        }
        uint32_t total;
        const uint32_t pos = block_excl_scan(emit, s_warp, &total);
        if (emit) out[carry + pos] = word;
        carry += total;
    }
    if (threadIdx.x == 0) *out_count = carry;
}

// PLWAH -> WAH: a fill word with a position becomes the fill and the literal
// it stands for.  A fill of length 0 is flagged (the WAH decoder checks the
// rest of the structure).
__global__ void __launch_bounds__(kPT) wah_from_plwah(const uint32_t* __restrict__ pl, int64_t nw, int64_t nbits,
                                                      uint32_t* __restrict__ out, int64_t* __restrict__ out_count,
                                                      unsigned long long* __restrict__ err) {
    __shared__ uint32_t s_warp[33];
    const bool has_active = (nbits % 31) != 0;
    int64_t carry = 0;
    for (int64_t base = 0; base < nw; base += kPT) {
        const int64_t k = base + threadIdx.x;
        uint32_t c = 0, w = 0, q = 0;
        bool fill = false;
        if (k < nw) {
            w = pl[k];
            fill = !(has_active && k == nw - 1) && (w & kTop);
            c = 1;
            if (fill) {
                q = (w >> 25) & 31u;
                if ((w & kCount25) == 0u) atomicOr(err, 1ull);
                if (q) c = 2;
            }
        }
        uint32_t total;
        const uint32_t pos = block_excl_scan(c, s_warp, &total);
        if (k < nw) {
            if (fill) {
                out[carry + pos] = kTop | (w & kVal) | (w & kCount25);
                if (q) out[carry + pos + 1] = ((w & kVal) ? kOnes : 0u) ^ (1u << (31 - q));
            } else {
                out[carry + pos] = w;
            }
        }
        carry += total;
    }
    if (threadIdx.x == 0) *out_count = carry;
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" {

bfs_status bfs_plwah_encode(const uint32_t* bits, int64_t nbits, uint32_t* words, int64_t capacity_words,
                            int64_t* nwords, void* stream) {
    if (nbits < 0 || nbits > kPlwahMaxBits)
        return set_error(BFS_ERR_INVALID_ARG, "nbits %lld outside [0, %lld]", (long long)nbits, (long long)kPlwahMaxBits);
    if (!nwords || (nbits > 0 && (!bits || !words))) return set_error(BFS_ERR_INVALID_ARG, "bad encode arguments");
    const int64_t bound = nbits / 31 + 1;
    if (capacity_words < bound)
        return set_error(BFS_ERR_INVALID_ARG, "capacity %lld below the bound %lld", (long long)capacity_words,
                         (long long)bound);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (nbits == 0) {
        BFS_CUDA_TRY(cudaMemsetAsync(nwords, 0, sizeof(int64_t), st));
        return BFS_OK;
    }
    DevBuf wah, cnt;
    BFS_TRY(wah.alloc(sizeof(uint32_t) * (size_t)(bound + 1)));
    BFS_TRY(cnt.alloc(sizeof(int64_t)));
    EncodeArgs a;
    memset(&a, 0, sizeof(a));
    a.frontier = bits;
    a.p = 1;
    a.nb = nbits;
    a.n = nbits;
    a.sieve = 0;
    a.nslots = 1;
    a.out = wah.ptr;
    a.slot_cap = bound + 1;
    a.counts = cnt.as<int64_t>();
    BFS_TRY(launch_wah_encode(a, 32, st));
    plwah_from_wah<<<1, kPT, 0, st>>>(wah.as<uint32_t>(), cnt.as<int64_t>(), nbits, words, nwords);
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaStreamSynchronize(st));          // the scratch is released on return
    return BFS_OK;
}

bfs_status bfs_plwah_decode(const uint32_t* words, int64_t nwords, int64_t nbits, uint32_t* bits, void* stream) {
    if (nbits < 0 || nbits > kPlwahMaxBits)
        return set_error(BFS_ERR_INVALID_ARG, "nbits %lld outside [0, %lld]", (long long)nbits, (long long)kPlwahMaxBits);
    if (nwords < 0 || (nwords > 0 && !words) || (nbits > 0 && !bits))
        return set_error(BFS_ERR_INVALID_ARG, "bad decode arguments");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    DevBuf wah, cnt, err;
    BFS_TRY(wah.alloc(sizeof(uint32_t) * (size_t)(2 * nwords + 1)));
    BFS_TRY(cnt.alloc(sizeof(int64_t)));
    BFS_TRY(err.alloc(sizeof(unsigned long long)));
    BFS_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, sizeof(int64_t), st));
    BFS_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, sizeof(unsigned long long), st));
    if (nwords > 0) {
        wah_from_plwah<<<1, kPT, 0, st>>>(words, nwords, nbits, wah.as<uint32_t>(), cnt.as<int64_t>(),
                                          err.as<unsigned long long>());
        BFS_CUDA_TRY(cudaGetLastError());
    }
    int64_t h_cnt = 0;
    unsigned long long h_err = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_cnt, cnt.ptr, sizeof(h_cnt), cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_err, err.ptr, sizeof(h_err), cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) return set_error(BFS_ERR_CORRUPT, "malformed PLWAH stream (a fill of length 0)");
    const bfs_status rc = bfs_wah_decode(wah.ptr, h_cnt, nbits, 32, bits, stream);
    if (rc == BFS_ERR_CORRUPT) return set_error(BFS_ERR_CORRUPT, "malformed PLWAH stream");
    return rc;
}

}  // extern "C"
