// common.cuh -- device helpers shared by the kernels of libbfs_gb300.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace bfsgb {

constexpr int kWarp = 32;

// 32 bits of a little-endian bitmap starting at bit `pos` (bit q of the result
// = bitmap bit pos+q).  Reads words pos/32 and pos/32 + 1.
__device__ __forceinline__ uint32_t bits32_at(const uint32_t* __restrict__ bm, uint64_t pos) {
    const uint64_t w = pos >> 5;
    const uint32_t sh = static_cast<uint32_t>(pos & 31u);
    const uint32_t lo = __ldg(bm + w);
    const uint32_t hi = __ldg(bm + w + 1);
    return __funnelshift_r(lo, hi, sh);
}

// Same, but through L2 only (for bitmaps written earlier in the same kernel
// sequence without an intervening launch boundary guarantee on L1).
__device__ __forceinline__ uint32_t bits32_at_cg(const uint32_t* bm, uint64_t pos) {
    const uint64_t w = pos >> 5;
    const uint32_t sh = static_cast<uint32_t>(pos & 31u);
    const uint32_t lo = __ldcg(bm + w);
    const uint32_t hi = __ldcg(bm + w + 1);
    return __funnelshift_r(lo, hi, sh);
}

// 64 bits starting at bit `pos` (reads three words).
__device__ __forceinline__ uint64_t bits64_at(const uint32_t* __restrict__ bm, uint64_t pos) {
    const uint64_t w = pos >> 5;
    const uint32_t sh = static_cast<uint32_t>(pos & 31u);
    const uint32_t a = __ldg(bm + w), b = __ldg(bm + w + 1), c = __ldg(bm + w + 2);
    const uint32_t lo = __funnelshift_r(a, b, sh);
    const uint32_t hi = __funnelshift_r(b, c, sh);
    return (static_cast<uint64_t>(hi) << 32) | lo;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_incl_sum(T x) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, d);
        if (static_cast<int>(lane_id()) >= d) x += y;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_incl_max(T x) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, d);
        if (static_cast<int>(lane_id()) >= d) x = y > x ? y : x;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
}

// Block-wide inclusive sum over NT threads (NT a multiple of 32, <= 1024).
// `smem` needs NT/32 + 1 elements.  Returns the inclusive prefix; *total gets
// the block total.  Contains __syncthreads (call from all threads).
template <int NT, typename T>
__device__ __forceinline__ T block_incl_sum(T x, T* smem, T* total) {
    constexpr int NW = NT / 32;
    const int w = threadIdx.x >> 5;
    T incl = warp_incl_sum(x);
    if (lane_id() == 31) smem[w] = incl;
    __syncthreads();
    if (w == 0) {
        T s = (lane_id() < NW) ? smem[lane_id()] : T(0);
        s = warp_incl_sum(s);
        if (lane_id() < NW) smem[lane_id()] = s;
    }
    __syncthreads();
    T pre = (w > 0) ? smem[w - 1] : T(0);
    *total = smem[NW - 1];
    __syncthreads();
    return pre + incl;
}

// Block-wide inclusive max (same contract as block_incl_sum).
template <int NT, typename T>
__device__ __forceinline__ T block_incl_max(T x, T* smem, T* total) {
    constexpr int NW = NT / 32;
    const int w = threadIdx.x >> 5;
    T incl = warp_incl_max(x);
    if (lane_id() == 31) smem[w] = incl;
    __syncthreads();
    if (w == 0) {
        T s = (lane_id() < NW) ? smem[lane_id()] : smem[0];
        s = warp_incl_max(s);
        if (lane_id() < NW) smem[lane_id()] = s;
    }
    __syncthreads();
    T r = incl;
    if (w > 0) { T p = smem[w - 1]; r = p > r ? p : r; }
    *total = smem[NW - 1];
    __syncthreads();
    return r;
}

struct OpSum {
    template <typename T> __device__ __forceinline__ T operator()(T a, T b) const { return a + b; }
};
struct OpMax {
    template <typename T> __device__ __forceinline__ T operator()(T a, T b) const { return a > b ? a : b; }
};

// Block-wide exclusive scan over NT threads with an associative op and its
// identity.  `smem` needs NT/32 + 1 elements.  Returns the exclusive prefix
// (identity for thread 0); *total gets the reduction of all threads.
// Contains __syncthreads (call from all threads).
template <int NT, typename T, typename Op>
__device__ __forceinline__ T block_excl_scan(T x, T identity, Op op, T* smem, T* total) {
    constexpr int NW = NT / 32;
    const int w = threadIdx.x >> 5;
    const int l = (int)lane_id();
    T incl = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, incl, d);
        if (l >= d) incl = op(y, incl);
    }
    T excl = __shfl_up_sync(0xffffffffu, incl, 1);
    if (l == 0) excl = identity;
    if (l == 31) smem[w] = incl;
    __syncthreads();
    if (w == 0) {
        T v = (l < NW) ? smem[l] : identity;
        T vi = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, vi, d);
            if (l >= d) vi = op(y, vi);
        }
        T ve = __shfl_up_sync(0xffffffffu, vi, 1);
        if (l == 0) ve = identity;
        if (l < NW) smem[l] = ve;                 // exclusive prefix of warp totals
        if (l == NW - 1) smem[NW] = vi;           // block total
    }
    __syncthreads();
    const T res = op(smem[w], excl);
    *total = smem[NW];
    __syncthreads();
    return res;
}

}  // namespace bfsgb
