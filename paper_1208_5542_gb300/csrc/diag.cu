// diag.cu -- bfs_measure_scatter_reads: the rate of scattered 4-byte reads
// (the bound of the expansion's visited test on its L1/L2 path).  Every
// thread of one 1024-thread CTA per SM reads `iterations` words at
// pseudo-random addresses of the region through the read-only path, as the
// visited test does, four independent reads in flight.
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace bfsgb {
namespace {

constexpr int kDT = 1024;
constexpr int kStreams = 4;        // independent reads in flight per thread

// Every thread walks kStreams xorshift32 sequences (Marsaglia, 2003: x ^= x << 13;
// x ^= x >> 17; x ^= x << 5) and reads one word per step of each at the masked
// (power-of-two region) or reduced position: a few integer operations per read,
// the reads independent of each other and of the values read.
__device__ __forceinline__ uint32_t xorshift32(uint32_t x) {
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    return x;
}

template <bool POW2>
__global__ void __launch_bounds__(kDT, 1) scatter_reads(const uint32_t* __restrict__ region, uint32_t nwords,
                                                          int32_t iterations, uint32_t* __restrict__ sink) {
    uint32_t x[kStreams], acc = 0;
    const uint32_t id = blockIdx.x * kDT + threadIdx.x;
#pragma unroll
    for (int k = 0; k < kStreams; ++k) x[k] = (id * kStreams + k) * 2654435761u | 1u;     // nonzero seeds
    const uint32_t mask = nwords - 1u;
    for (int32_t i = 0; i < iterations; i += kStreams) {
#pragma unroll
        for (int k = 0; k < kStreams; ++k) {
            x[k] = xorshift32(x[k]);
            acc += __ldg(region + (POW2 ? (x[k] & mask) : (x[k] % nwords)));
        }
    }
    if (acc == 0x9e3779b9u) sink[0] = acc;     // keeps the reads; practically never taken
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" bfs_status bfs_measure_scatter_reads(int64_t region_bytes, int32_t iterations, double* reads_per_s,
                                                void* stream) {
    if (!reads_per_s) return set_error(BFS_ERR_INVALID_ARG, "reads_per_s is NULL");
    if (region_bytes < 4096 || region_bytes > (1LL << 30))
        return set_error(BFS_ERR_INVALID_ARG, "region_bytes %lld outside [4096, 1 GiB]", (long long)region_bytes);
    if (iterations < 1) return set_error(BFS_ERR_INVALID_ARG, "iterations must be >= 1");
    iterations = (iterations + kStreams - 1) / kStreams * kStreams;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0, sms = 0;
    BFS_CUDA_TRY(cudaGetDevice(&dev));
    BFS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const uint32_t nwords = (uint32_t)(region_bytes / 4);
    DevBuf region, sink;
    BFS_TRY(region.alloc(4 * (size_t)nwords));
    BFS_TRY(sink.alloc(4));
    BFS_CUDA_TRY(cudaMemsetAsync(region.ptr, 1, 4 * (size_t)nwords, st));
    cudaEvent_t e0, e1;
    BFS_CUDA_TRY(cudaEventCreate(&e0));
    BFS_CUDA_TRY(cudaEventCreate(&e1));
    const bool pow2 = (nwords & (nwords - 1)) == 0;
    auto launch = [&]() {
        if (pow2) scatter_reads<true><<<sms, kDT, 0, st>>>(region.as<uint32_t>(), nwords, iterations, sink.as<uint32_t>());
        else scatter_reads<false><<<sms, kDT, 0, st>>>(region.as<uint32_t>(), nwords, iterations, sink.as<uint32_t>());
    };
    launch();                                   // warm-up
    cudaEventRecord(e0, st);
    launch();
    cudaEventRecord(e1, st);
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return cuda_error(err, "scatter_reads", __FILE__, __LINE__);
    *reads_per_s = (double)sms * kDT * (double)iterations / (ms * 1e-3);
    return BFS_OK;
}
