// diag.cu -- bfs_measure_scatter_reads: the rate of scattered 4-byte reads
// (the bound of the expansion's visited test on its L1/L2 path).  Every
// thread of one 1024-thread CTA per SM reads `iterations` words at hashed
// addresses of the region through the read-only path, as the visited test does.
#include <cstring>

#include "common.cuh"
#include "internal.h"

namespace bfsgb {
namespace {

constexpr int kDT = 1024;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {     // an integer hash (xorshift-multiply rounds)
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

__global__ void __launch_bounds__(kDT, 1) scatter_reads(const uint32_t* __restrict__ region, uint32_t nwords,
                                                          int32_t iterations, uint32_t* __restrict__ sink) {
    uint32_t acc = 0, h = blockIdx.x * kDT + threadIdx.x;
    for (int32_t i = 0; i < iterations; ++i) {
        h = mix32(h + (uint32_t)i);
        acc += __ldg(region + (h % nwords));
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
    scatter_reads<<<sms, kDT, 0, st>>>(region.as<uint32_t>(), nwords, iterations, sink.as<uint32_t>());   // warm-up
    cudaEventRecord(e0, st);
    scatter_reads<<<sms, kDT, 0, st>>>(region.as<uint32_t>(), nwords, iterations, sink.as<uint32_t>());
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
