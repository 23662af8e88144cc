// graph_build.cu -- the blocked layout of the adjacency (Eq. 1-4) built on the
// device, and the graph-management entry points of the C ABI.
//
// Layout (one-time per graph, amortised over every search as the paper
// assumes for its cross directory, Sec. V-B): the directed entries u -> v are
// counted per (block-row i = range of v, source u); a per-block segmented scan
// of those counts gives the block-local column offsets; set counts give the
// directory V_{i,j} (Eq. 4); a scan of directory popcounts gives the rank of
// every nonempty column; the entries are then scattered column by column.
#include <atomic>
#include <cstdarg>
#include <cstring>
#include <new>
#include <utility>

#include "common.cuh"
#include "internal.h"

namespace bfsgb {

// ------------------------------------------------------------------ errors --
namespace {
thread_local bfs_status t_last_status = BFS_OK;
thread_local char t_last_msg[512] = "no error";
}

bfs_status set_error(bfs_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_last_msg, sizeof(t_last_msg), fmt, ap);
    va_end(ap);
    t_last_status = s;
    return s;
}

bfs_status cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    bfs_status s = (e == cudaErrorMemoryAllocation) ? BFS_ERR_OUT_OF_MEMORY : BFS_ERR_CUDA;
    return set_error(s, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
}

bool is_device_pointer(const void* p) {
    if (!p) return false;
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Allocation-failure injection (bfs_debug_fail_allocation): the armed
// allocation fails as if the device were out of memory.  0 = disarmed.
std::atomic<int64_t> g_fail_countdown{0};

bfs_status DevBuf::alloc(size_t nbytes) {
    release();
    if (nbytes == 0) nbytes = 16;
    int64_t k = g_fail_countdown.load();
    while (k > 0 && !g_fail_countdown.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) return set_error(BFS_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu bytes): injected failure", nbytes);
    cudaError_t e = cudaMalloc(&ptr, nbytes);
    if (e != cudaSuccess) {
        ptr = nullptr;
        cudaGetLastError();
        return set_error(BFS_ERR_OUT_OF_MEMORY, "cudaMalloc(%zu bytes): %s", nbytes, cudaGetErrorString(e));
    }
    bytes = nbytes;
    return BFS_OK;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

// ------------------------------------------------------------ build kernels --
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int64_t kScanTile = (int64_t)kScanThreads * kScanItems;

// Count entries per (block-row of the destination, source) and flag bad ids.
__global__ void count_entries(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                              int symmetrize, int64_t n, int64_t nb, int64_t row_stride,
                              uint32_t* __restrict__ cnt, unsigned long long* err) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        if (a < 0 || a >= n || b < 0 || b >= n) {
            atomicOr(err, 1ull);
            continue;
        }
        atomicAdd(cnt + (int64_t)(b / nb) * row_stride + a, 1u);
        if (symmetrize) atomicAdd(cnt + (int64_t)(a / nb) * row_stride + b, 1u);
    }
}

// Directory words: bit q of word w of block b = (count of column 32w+q > 0).
// One warp per word; also writes the word's popcount into rank (scanned later).
__global__ void directory_words(const uint32_t* __restrict__ cnt, int64_t nblocks, int64_t nb,
                                int64_t words_per_block, int64_t dir_stride,
                                uint32_t* __restrict__ dir, uint32_t* __restrict__ rank) {
    const int64_t warps = nblocks * words_per_block;
    const int64_t gw0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t gstride = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gw = gw0; gw < warps; gw += gstride) {
        const int64_t b = gw / words_per_block, w = gw % words_per_block;
        const int64_t x = w * 32 + lane_id();
        const uint32_t c = (x < nb) ? cnt[b * nb + x] : 0u;
        const uint32_t bits = __ballot_sync(0xffffffffu, c != 0u);
        if (lane_id() == 0) {
            dir[b * dir_stride + w] = bits;
            rank[b * dir_stride + w] = __popc(bits);
        }
    }
}

// Segmented scan, phase A: sums of tiles of kScanTile elements; segments of
// length seg_len (uniform), tiles never cross a segment boundary.
__global__ void __launch_bounds__(kScanThreads)
scan_tile_sums(const uint32_t* __restrict__ a, int64_t nseg, int64_t seg_len, int64_t seg_stride,
               int64_t tiles_per_seg, unsigned long long* __restrict__ tile_sum) {
    __shared__ unsigned long long sm[kScanThreads / 32 + 1];
    const int64_t tile = blockIdx.x;
    const int64_t s = tile / tiles_per_seg, t = tile % tiles_per_seg;
    if (s >= nseg) return;
    const int64_t base = s * seg_stride + t * kScanTile;
    const int64_t lim = seg_len - t * kScanTile;
    unsigned long long acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t x = (int64_t)k * kScanThreads + threadIdx.x;
        if (x < lim) acc += a[base + x];
    }
    unsigned long long tot;
    block_incl_sum<kScanThreads>(acc, sm, &tot);
    if (threadIdx.x == 0) tile_sum[tile] = tot;
}

// Phase B: per segment, exclusive scan of its tile sums; segment totals.
__global__ void __launch_bounds__(kScanThreads)
scan_tile_offsets(unsigned long long* __restrict__ tile_sum, int64_t nseg, int64_t tiles_per_seg,
                  unsigned long long* __restrict__ seg_total) {
    __shared__ unsigned long long sm[kScanThreads / 32 + 1];
    const int64_t s = blockIdx.x;
    if (s >= nseg) return;
    unsigned long long carry = 0;
    for (int64_t t0 = 0; t0 < tiles_per_seg; t0 += kScanThreads) {
        const int64_t t = t0 + threadIdx.x;
        const unsigned long long v = (t < tiles_per_seg) ? tile_sum[s * tiles_per_seg + t] : 0ull;
        unsigned long long tot;
        const unsigned long long incl = block_incl_sum<kScanThreads>(v, sm, &tot);
        if (t < tiles_per_seg) tile_sum[s * tiles_per_seg + t] = carry + incl - v;
        carry += tot;
    }
    if (threadIdx.x == 0) seg_total[s] = carry;
}

// Phase C: exclusive scan inside each tile plus the tile offset, in place.
// Elements are loaded blocked (thread t owns elements t*kScanItems ...).
__global__ void __launch_bounds__(kScanThreads)
scan_tiles_apply(uint32_t* __restrict__ a, int64_t nseg, int64_t seg_len, int64_t seg_stride,
                 int64_t tiles_per_seg, const unsigned long long* __restrict__ tile_off) {
    __shared__ unsigned long long sm[kScanThreads / 32 + 1];
    const int64_t tile = blockIdx.x;
    const int64_t s = tile / tiles_per_seg, t = tile % tiles_per_seg;
    if (s >= nseg) return;
    const int64_t base = s * seg_stride + t * kScanTile;
    const int64_t lim = seg_len - t * kScanTile;
    uint32_t v[kScanItems];
    unsigned long long acc = 0;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t x = (int64_t)threadIdx.x * kScanItems + k;
        v[k] = (x < lim) ? a[base + x] : 0u;
        acc += v[k];
    }
    unsigned long long tot;
    const unsigned long long incl = block_incl_sum<kScanThreads>(acc, sm, &tot);
    unsigned long long run = tile_off[tile] + incl - acc;
    for (int k = 0; k < kScanItems; ++k) {
        const int64_t x = (int64_t)threadIdx.x * kScanItems + k;
        if (x < lim) a[base + x] = (uint32_t)run;
        run += v[k];
    }
}

// Column pointers: for every nonempty column (u_local) of block b, cp of its
// rank = the block-local offset of the column; plus the closing entry.
__global__ void column_pointers(const uint32_t* __restrict__ off, const uint32_t* __restrict__ dir,
                                const uint32_t* __restrict__ rank, int64_t nblocks, int64_t nb,
                                int64_t dir_stride, const int64_t* __restrict__ cp_base,
                                const unsigned long long* __restrict__ nnz_b,
                                const unsigned long long* __restrict__ nnzc_b, uint32_t* __restrict__ cp) {
    const int64_t total = nblocks * nb;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < total;
         x += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = x / nb, ul = x % nb;
        const uint32_t dw = dir[b * dir_stride + (ul >> 5)];
        const uint32_t bit = 1u << (ul & 31);
        if (dw & bit) {
            const uint32_t c = rank[b * dir_stride + (ul >> 5)] + __popc(dw & (bit - 1u));
            cp[cp_base[b] + c] = off[b * nb + ul];
        }
        if (ul == 0) cp[cp_base[b] + (int64_t)nnzc_b[b]] = (uint32_t)nnz_b[b];
    }
}

// Scatter every entry into its column (order inside a column is arbitrary).
__global__ void scatter_entries(const int32_t* __restrict__ src, const int32_t* __restrict__ dst, int64_t m,
                                int symmetrize, int64_t nb, int p, int64_t row_stride,
                                uint32_t* __restrict__ off, const int64_t* __restrict__ ir_base,
                                int32_t* __restrict__ ir) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        {
            const int64_t i = b / nb, j = a / nb;
            const uint32_t pos = atomicAdd(off + i * row_stride + a, 1u);
            ir[ir_base[i * p + j] + pos] = b;
        }
        if (symmetrize) {
            const int64_t i = a / nb, j = b / nb;
            const uint32_t pos = atomicAdd(off + i * row_stride + b, 1u);
            ir[ir_base[i * p + j] + pos] = a;
        }
    }
}

// Degree of every vertex u (range j): the lengths of its columns in blocks
// (i, j), i = 0 .. p-1, saturated at 2^32 - 1.
__global__ void vertex_degrees(const uint32_t* __restrict__ dir, const uint32_t* __restrict__ rank,
                               int64_t dir_stride, const uint32_t* __restrict__ cp,
                               const int64_t* __restrict__ cp_base, int p, int64_t nb, int64_t n,
                               uint32_t* __restrict__ deg) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = u / nb, ul = u - j * nb;
        const uint32_t bit = 1u << (ul & 31);
        uint64_t d = 0;
        for (int i = 0; i < p; ++i) {
            const int64_t b = (int64_t)i * p + j;
            const uint32_t dw = dir[b * dir_stride + (ul >> 5)];
            if (!(dw & bit)) continue;
            const int64_t c = cp_base[b] + rank[b * dir_stride + (ul >> 5)] + __popc(dw & (bit - 1u));
            d += cp[c + 1] - cp[c];
        }
        deg[u] = d > 0xffffffffull ? 0xffffffffu : (uint32_t)d;
    }
}

// Bitmap of the vertices without entries: no search reaches them from
// another vertex, and a bottom-up level need not scan them.
__global__ void isolated_bits(const uint32_t* __restrict__ deg, int64_t n, int64_t words, uint32_t* __restrict__ iso) {
    for (int64_t w = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
        uint32_t x = 0;
        for (int b = 0; b < 32; ++b) {
            const int64_t v = w * 32 + b;
            if (v < n && deg[v] == 0) x |= 1u << b;
        }
        iso[w] = x;
    }
}

// Bottom-up layout, step 1: exclusive scan of the degrees in tiles of 1024,
// in 64 bits, with every tile's total.
__global__ void __launch_bounds__(1024) degree_tile_scan(const uint32_t* __restrict__ deg, int64_t n,
                                                         int64_t* __restrict__ ptr, int64_t* __restrict__ tile_sum) {
    __shared__ int64_t warp_tot[32];
    const int64_t x = blockIdx.x * 1024LL + threadIdx.x;
    const int64_t d = x < n ? (int64_t)deg[x] : 0;
    int64_t incl = d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane_id() >= o) incl += y;
    }
    if (lane_id() == 31) warp_tot[threadIdx.x >> 5] = incl;
    __syncthreads();
    if (threadIdx.x < 32) {
        int64_t t = warp_tot[threadIdx.x], ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, ti, o);
            if ((int)threadIdx.x >= o) ti += y;
        }
        warp_tot[threadIdx.x] = ti - t;
        if (threadIdx.x == 31) tile_sum[blockIdx.x] = ti;
    }
    __syncthreads();
    if (x <= n) ptr[x] = incl - d + warp_tot[threadIdx.x >> 5];      // ptr[n]: the entries before n in its tile
}

// Step 2: add the tiles' scanned totals; ptr[n] = the total.
__global__ void degree_tile_add(int64_t* __restrict__ ptr, int64_t n, const int64_t* __restrict__ tile_base) {
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x <= n; x += (int64_t)gridDim.x * blockDim.x)
        ptr[x] += tile_base[x >> 10];
}

// Step 3: the columns of every vertex v (range i) in blocks (0,i), (1,i), ...
// copied back to back from bu_ptr[v]: its neighbours grouped by range j in
// ascending order (in any order inside a range).
__global__ void bottom_up_rows(const uint32_t* __restrict__ dir, const uint32_t* __restrict__ rank,
                               int64_t dir_stride, const uint32_t* __restrict__ cp,
                               const int64_t* __restrict__ cp_base, const int64_t* __restrict__ ir_base,
                               const int32_t* __restrict__ ir, int p, int64_t nb, int64_t n,
                               const int64_t* __restrict__ ptr, int32_t* __restrict__ adj) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = v / nb, vl = v - i * nb;
        const uint32_t bit = 1u << (vl & 31);
        int64_t pos = ptr[v];
        for (int j = 0; j < p; ++j) {
            const int64_t b = (int64_t)j * p + i;
            const uint32_t dw = dir[b * dir_stride + (vl >> 5)];
            if (!(dw & bit)) continue;
            const int64_t c = cp_base[b] + rank[b * dir_stride + (vl >> 5)] + __popc(dw & (bit - 1u));
            const int32_t* col = ir + ir_base[b];
            const uint32_t c0 = cp[c], c1 = cp[c + 1];
            for (uint32_t e = c0; e < c1; ++e) adj[pos++] = col[e];
        }
    }
}

// CSR -> per-entry source ids.
__global__ void expand_rows(const int64_t* __restrict__ row_ptr, int64_t n, int32_t* __restrict__ src) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x)
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) src[e] = (int32_t)u;
}

__global__ void check_csr(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col, int64_t n,
                          int64_t nnz, unsigned long long* err) {
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
         u += (int64_t)gridDim.x * blockDim.x) {
        if (row_ptr[u] > row_ptr[u + 1] || row_ptr[u] < 0 || row_ptr[u + 1] > nnz) atomicOr(err, 1ull);
    }
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz;
         e += (int64_t)gridDim.x * blockDim.x)
        if (col[e] < 0 || col[e] >= n) atomicOr(err, 1ull);
}

int grid_for(int64_t work, int threads) {
    int64_t g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 64) g = 152 * 64;
    return (int)g;
}

// In-place segmented exclusive scan of `a` (nseg segments of seg_len
// elements, segment s at s*seg_stride); seg_total[s] receives the totals.
bfs_status segmented_scan(uint32_t* a, int64_t nseg, int64_t seg_len, int64_t seg_stride,
                          std::vector<uint64_t>& totals, cudaStream_t st) {
    const int64_t tiles_per_seg = seg_len > 0 ? (seg_len + kScanTile - 1) / kScanTile : 1;
    DevBuf tile_sum, seg_total;
    BFS_TRY(tile_sum.alloc(sizeof(unsigned long long) * nseg * tiles_per_seg));
    BFS_TRY(seg_total.alloc(sizeof(unsigned long long) * nseg));
    const int64_t ntiles = nseg * tiles_per_seg;
    if (ntiles > 0x7fffffffLL) return set_error(BFS_ERR_INVALID_ARG, "graph too large for the layout scan");
    scan_tile_sums<<<(unsigned)ntiles, kScanThreads, 0, st>>>(a, nseg, seg_len, seg_stride, tiles_per_seg,
                                                              tile_sum.as<unsigned long long>());
    BFS_CUDA_TRY(cudaGetLastError());
    scan_tile_offsets<<<(unsigned)nseg, kScanThreads, 0, st>>>(tile_sum.as<unsigned long long>(), nseg,
                                                               tiles_per_seg, seg_total.as<unsigned long long>());
    BFS_CUDA_TRY(cudaGetLastError());
    totals.assign(nseg, 0);
    BFS_CUDA_TRY(cudaMemcpyAsync(totals.data(), seg_total.ptr, sizeof(uint64_t) * nseg, cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int64_t s = 0; s < nseg; ++s)
        if (totals[s] > 0xffffffffull)
            return set_error(BFS_ERR_INVALID_ARG, "a block holds 2^32 or more entries; use a larger grid");
    scan_tiles_apply<<<(unsigned)ntiles, kScanThreads, 0, st>>>(a, nseg, seg_len, seg_stride, tiles_per_seg,
                                                                tile_sum.as<unsigned long long>());
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    return BFS_OK;
}

}  // namespace

bfs_status build_layout(bfs_graph* g, int64_t n, int64_t m, const int32_t* d_src, const int32_t* d_dst,
                        int symmetrize, cudaStream_t st) {
    Layout& L = g->L;
    const int p = L.p;
    L.n = n;
    L.nb = (n + p - 1) / p;
    L.nnz = symmetrize ? 2 * m : m;
    const int64_t nb = L.nb;
    const int64_t nblocks = (int64_t)p * p;
    const int64_t row_stride = (int64_t)p * nb;
    const int64_t words_per_block = (nb + 31) / 32;
    L.dir_stride = ((words_per_block + 3 + 3) / 4) * 4;   // >= 3 words of padding, 16-byte rows

    DevBuf cnt, err;
    BFS_TRY(cnt.alloc(sizeof(uint32_t) * nblocks * nb));
    BFS_TRY(err.alloc(sizeof(unsigned long long)));
    BFS_CUDA_TRY(cudaMemsetAsync(cnt.ptr, 0, cnt.bytes, st));
    BFS_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, err.bytes, st));
    count_entries<<<grid_for(m, 256), 256, 0, st>>>(d_src, d_dst, m, symmetrize, n, nb, row_stride,
                                                    cnt.as<uint32_t>(), err.as<unsigned long long>());
    BFS_CUDA_TRY(cudaGetLastError());
    unsigned long long h_err = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_err, err.ptr, sizeof(h_err), cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) return set_error(BFS_ERR_INVALID_ARG, "an edge names a vertex outside [0, %lld)", (long long)n);

    // directory + popcounts
    BFS_TRY(L.dir.alloc(sizeof(uint32_t) * nblocks * L.dir_stride));
    BFS_TRY(L.rank.alloc(sizeof(uint32_t) * nblocks * L.dir_stride));
    BFS_CUDA_TRY(cudaMemsetAsync(L.dir.ptr, 0, L.dir.bytes, st));
    BFS_CUDA_TRY(cudaMemsetAsync(L.rank.ptr, 0, L.rank.bytes, st));
    directory_words<<<grid_for(nblocks * words_per_block * 32, 256), 256, 0, st>>>(
        cnt.as<uint32_t>(), nblocks, nb, words_per_block, L.dir_stride, L.dir.as<uint32_t>(), L.rank.as<uint32_t>());
    BFS_CUDA_TRY(cudaGetLastError());

    // rank = exclusive scan of popcounts per block; nnzc_b = totals
    std::vector<uint64_t> nnzc_b, nnz_b;
    BFS_TRY(segmented_scan(L.rank.as<uint32_t>(), nblocks, L.dir_stride, L.dir_stride, nnzc_b, st));
    // block-local column offsets = exclusive scan of counts per block; nnz_b = totals
    BFS_TRY(segmented_scan(cnt.as<uint32_t>(), nblocks, nb, nb, nnz_b, st));

    L.cp_base.assign(nblocks, 0);
    L.ir_base.assign(nblocks, 0);
    L.nnzc.assign(nblocks, 0);
    L.nnz_b.assign(nblocks, 0);
    int64_t cpt = 0, irt = 0;
    for (int64_t b = 0; b < nblocks; ++b) {
        L.cp_base[b] = cpt;
        L.ir_base[b] = irt;
        L.nnzc[b] = (int64_t)nnzc_b[b];
        L.nnz_b[b] = (int64_t)nnz_b[b];
        cpt += (int64_t)nnzc_b[b] + 1;
        irt += (int64_t)nnz_b[b];
    }
    L.nnzc_total = cpt - nblocks;
    if (irt != L.nnz) return set_error(BFS_ERR_CUDA, "layout build lost entries (%lld of %lld)", (long long)irt, (long long)L.nnz);

    BFS_TRY(L.cp.alloc(sizeof(uint32_t) * (cpt > 0 ? cpt : 1)));
    BFS_TRY(L.ir.alloc(sizeof(int32_t) * (L.nnz > 0 ? L.nnz : 1)));
    BFS_TRY(L.cp_base_d.alloc(sizeof(int64_t) * nblocks));
    BFS_TRY(L.ir_base_d.alloc(sizeof(int64_t) * nblocks));
    DevBuf d_nnz_b, d_nnzc_b;
    BFS_TRY(d_nnz_b.alloc(sizeof(uint64_t) * nblocks));
    BFS_TRY(d_nnzc_b.alloc(sizeof(uint64_t) * nblocks));
    BFS_CUDA_TRY(cudaMemcpyAsync(L.cp_base_d.ptr, L.cp_base.data(), sizeof(int64_t) * nblocks, cudaMemcpyHostToDevice, st));
    BFS_CUDA_TRY(cudaMemcpyAsync(L.ir_base_d.ptr, L.ir_base.data(), sizeof(int64_t) * nblocks, cudaMemcpyHostToDevice, st));
    BFS_CUDA_TRY(cudaMemcpyAsync(d_nnz_b.ptr, nnz_b.data(), sizeof(uint64_t) * nblocks, cudaMemcpyHostToDevice, st));
    BFS_CUDA_TRY(cudaMemcpyAsync(d_nnzc_b.ptr, nnzc_b.data(), sizeof(uint64_t) * nblocks, cudaMemcpyHostToDevice, st));

    column_pointers<<<grid_for(nblocks * nb, 256), 256, 0, st>>>(
        cnt.as<uint32_t>(), L.dir.as<uint32_t>(), L.rank.as<uint32_t>(), nblocks, nb, L.dir_stride,
        L.cp_base_d.as<int64_t>(), d_nnz_b.as<unsigned long long>(), d_nnzc_b.as<unsigned long long>(),
        L.cp.as<uint32_t>());
    BFS_CUDA_TRY(cudaGetLastError());
    scatter_entries<<<grid_for(m, 256), 256, 0, st>>>(d_src, d_dst, m, symmetrize, nb, p, row_stride,
                                                      cnt.as<uint32_t>(), L.ir_base_d.as<int64_t>(), L.ir.as<int32_t>());
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    return BFS_OK;
}

bfs_status ensure_degrees(bfs_graph* g, cudaStream_t st) {
    Layout& L = g->L;
    if (L.deg.ptr) return BFS_OK;
    DevBuf deg, iso;
    BFS_TRY(deg.alloc(sizeof(uint32_t) * L.n));
    vertex_degrees<<<grid_for(L.n, 256), 256, 0, st>>>(L.dir.as<uint32_t>(), L.rank.as<uint32_t>(), L.dir_stride,
                                                       L.cp.as<uint32_t>(), L.cp_base_d.as<int64_t>(), L.p, L.nb,
                                                       L.n, deg.as<uint32_t>());
    BFS_CUDA_TRY(cudaGetLastError());
    const int64_t iso_words = ((L.n + 31) / 32 + 4 + 3) / 4 * 4;        // the search bitmaps' padded size
    BFS_TRY(iso.alloc(sizeof(uint32_t) * iso_words));
    isolated_bits<<<grid_for(iso_words, 256), 256, 0, st>>>(deg.as<uint32_t>(), L.n, iso_words, iso.as<uint32_t>());
    BFS_CUDA_TRY(cudaGetLastError());
    // the bottom-up rows: offsets = scan of the degrees, then the columns
    const int64_t tiles = (L.n + 1 + 1023) / 1024;
    DevBuf ptr, adj, tsum;
    BFS_TRY(ptr.alloc(sizeof(int64_t) * (L.n + 1)));
    BFS_TRY(adj.alloc(sizeof(int32_t) * (L.nnz > 0 ? L.nnz : 1)));
    BFS_TRY(tsum.alloc(sizeof(int64_t) * tiles));
    degree_tile_scan<<<tiles, 1024, 0, st>>>(deg.as<uint32_t>(), L.n, ptr.as<int64_t>(), tsum.as<int64_t>());
    BFS_CUDA_TRY(cudaGetLastError());
    std::vector<int64_t> h(tiles);
    BFS_CUDA_TRY(cudaMemcpyAsync(h.data(), tsum.ptr, sizeof(int64_t) * tiles, cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    int64_t run = 0;
    for (int64_t t = 0; t < tiles; ++t) {
        const int64_t x = h[t];
        h[t] = run;
        run += x;
    }
    if (run != L.nnz)
        return set_error(BFS_ERR_CUDA, "bottom-up rows: degrees sum to %lld, not %lld entries", (long long)run,
                         (long long)L.nnz);
    BFS_CUDA_TRY(cudaMemcpyAsync(tsum.ptr, h.data(), sizeof(int64_t) * tiles, cudaMemcpyHostToDevice, st));
    degree_tile_add<<<grid_for(L.n + 1, 256), 256, 0, st>>>(ptr.as<int64_t>(), L.n, tsum.as<int64_t>());
    BFS_CUDA_TRY(cudaGetLastError());
    bottom_up_rows<<<grid_for(L.n, 256), 256, 0, st>>>(L.dir.as<uint32_t>(), L.rank.as<uint32_t>(), L.dir_stride,
                                                       L.cp.as<uint32_t>(), L.cp_base_d.as<int64_t>(),
                                                       L.ir_base_d.as<int64_t>(), L.ir.as<int32_t>(), L.p, L.nb,
                                                       L.n, ptr.as<int64_t>(), adj.as<int32_t>());
    BFS_CUDA_TRY(cudaGetLastError());
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    std::swap(L.deg.ptr, deg.ptr);
    std::swap(L.deg.bytes, deg.bytes);
    std::swap(L.iso.ptr, iso.ptr);
    std::swap(L.iso.bytes, iso.bytes);
    std::swap(L.bu_ptr.ptr, ptr.ptr);
    std::swap(L.bu_ptr.bytes, ptr.bytes);
    std::swap(L.bu_adj.ptr, adj.ptr);
    std::swap(L.bu_adj.bytes, adj.bytes);
    return BFS_OK;
}

// --------------------------------------------------------- entry helpers --
namespace {

bfs_status check_options(const bfs_options* o, int64_t n) {
    if (!o) return BFS_OK;
    if (o->grid_r != o->grid_c) return set_error(BFS_ERR_INVALID_ARG, "grid must be square (grid_r == grid_c)");
    if (o->grid_r < 1 || o->grid_r > 1024 || o->grid_r > n)
        return set_error(BFS_ERR_INVALID_ARG, "grid size %d outside [1, min(n, 1024)]", o->grid_r);
    if (o->mode < 0 || o->mode > 2) return set_error(BFS_ERR_INVALID_ARG, "unknown mode %d", o->mode);
    if (o->wah_word_bits != 32 && o->wah_word_bits != 64)
        return set_error(BFS_ERR_INVALID_ARG, "wah_word_bits must be 32 or 64");
    return BFS_OK;
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

bfs_status create_common(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int symmetrize,
                         const bfs_options* opt, void* stream, bfs_graph_t* out, bool src_is_device_scratch) {
    bfs_options o;
    bfs_options_default(&o);
    if (opt) o = *opt;
    BFS_TRY(check_options(&o, n));
    cudaStream_t st = as_stream(stream);
    bfs_graph* g = new (std::nothrow) bfs_graph();
    if (!g) return set_error(BFS_ERR_OUT_OF_MEMORY, "host allocation of the graph handle");
    g->L.p = o.grid_r;
    g->mode = o.mode;
    g->wah_bits = o.wah_word_bits;
    g->debug_checks = o.debug_checks ? 1 : 0;
    g->autotune = o.autotune ? 1 : 0;
    g->row_exchange = o.row_exchange ? 1 : 0;
    g->symmetric = symmetrize ? 1 : 0;
    cudaGetDevice(&g->device);

    DevBuf dsrc, ddst;
    const int32_t* s_ptr = src;
    const int32_t* d_ptr = dst;
    bfs_status rc = BFS_OK;
    if (!src_is_device_scratch) {
        if (m > 0 && !is_device_pointer(src)) {
            rc = dsrc.alloc(sizeof(int32_t) * m);
            if (rc == BFS_OK && cudaMemcpyAsync(dsrc.ptr, src, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = set_error(BFS_ERR_CUDA, "copy of src to the device failed");
            s_ptr = dsrc.as<int32_t>();
        }
        if (rc == BFS_OK && m > 0 && !is_device_pointer(dst)) {
            rc = ddst.alloc(sizeof(int32_t) * m);
            if (rc == BFS_OK && cudaMemcpyAsync(ddst.ptr, dst, sizeof(int32_t) * m, cudaMemcpyHostToDevice, st) != cudaSuccess)
                rc = set_error(BFS_ERR_CUDA, "copy of dst to the device failed");
            d_ptr = ddst.as<int32_t>();
        }
    }
    if (rc == BFS_OK) rc = build_layout(g, n, m, s_ptr, d_ptr, symmetrize, st);
    if (rc == BFS_OK) rc = ensure_workspace(g, st);
    if (rc != BFS_OK) {
        cudaStreamSynchronize(st);
        free_workspace(g);
        delete g;
        return rc;
    }
    *out = g;
    return BFS_OK;
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" {

void bfs_options_default(bfs_options* opt) {
    if (!opt) return;
    opt->grid_r = 1;
    opt->grid_c = 1;
    opt->mode = BFS_MODE_COMPRESS_SIEVE;
    opt->wah_word_bits = 32;
    opt->autotune = 0;
    opt->debug_checks = 0;
    opt->row_exchange = 1;
}

const char* bfs_status_string(bfs_status s) {
    switch (s) {
        case BFS_OK: return "BFS_OK";
        case BFS_ERR_INVALID_ARG: return "BFS_ERR_INVALID_ARG";
        case BFS_ERR_OUT_OF_MEMORY: return "BFS_ERR_OUT_OF_MEMORY";
        case BFS_ERR_CUDA: return "BFS_ERR_CUDA";
        case BFS_ERR_TIMEOUT: return "BFS_ERR_TIMEOUT";
        case BFS_ERR_CORRUPT: return "BFS_ERR_CORRUPT";
        case BFS_ERR_BUSY: return "BFS_ERR_BUSY";
        case BFS_ERR_NOT_FOUND: return "BFS_ERR_NOT_FOUND";
    }
    return "BFS_ERR_UNKNOWN";
}

bfs_status bfs_debug_fail_allocation(int64_t k) {
    if (k < 0) return set_error(BFS_ERR_INVALID_ARG, "k must be >= 0");
    g_fail_countdown.store(k);
    return BFS_OK;
}

bfs_status bfs_last_error(char* buf, int64_t len) {
    if (buf && len > 0) {
        strncpy(buf, t_last_msg, (size_t)len - 1);
        buf[len - 1] = '\0';
    }
    return t_last_status;
}

bfs_status bfs_graph_create_edges(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t symmetrize,
                                  const bfs_options* opt, void* stream, bfs_graph_t* out) {
    if (!out) return set_error(BFS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 0x7fffffffLL) return set_error(BFS_ERR_INVALID_ARG, "n_vertices %lld outside [1, 2^31-1]", (long long)n);
    if (m < 0 || (m > 0 && (!src || !dst))) return set_error(BFS_ERR_INVALID_ARG, "bad edge arrays");
    if ((symmetrize ? 2 * m : m) > (int64_t)0x7fffffff * 16)
        return set_error(BFS_ERR_INVALID_ARG, "too many entries");
    return create_common(n, m, src, dst, symmetrize ? 1 : 0, opt, stream, out, false);
}

bfs_status bfs_graph_create_csr(int64_t n, const int64_t* row_ptr, const int32_t* col, const bfs_options* opt,
                                void* stream, bfs_graph_t* out) {
    if (!out) return set_error(BFS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n < 1 || n > 0x7fffffffLL) return set_error(BFS_ERR_INVALID_ARG, "n_vertices %lld outside [1, 2^31-1]", (long long)n);
    if (!row_ptr) return set_error(BFS_ERR_INVALID_ARG, "row_ptr is NULL");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool rp_dev = is_device_pointer(row_ptr);
    int64_t first = 0, nnz = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&first, row_ptr, sizeof(int64_t), rp_dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st));
    BFS_CUDA_TRY(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof(int64_t), rp_dev ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (first != 0 || nnz < 0) return set_error(BFS_ERR_INVALID_ARG, "row_ptr[0] must be 0 and row_ptr[n] >= 0");
    if (nnz > 0 && !col) return set_error(BFS_ERR_INVALID_ARG, "col is NULL");
    DevBuf drp, dcol, dsrc, err;
    const int64_t* rp = row_ptr;
    const int32_t* cl = col;
    if (!rp_dev) {
        BFS_TRY(drp.alloc(sizeof(int64_t) * (n + 1)));
        BFS_CUDA_TRY(cudaMemcpyAsync(drp.ptr, row_ptr, sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
        rp = drp.as<int64_t>();
    }
    if (nnz > 0 && !is_device_pointer(col)) {
        BFS_TRY(dcol.alloc(sizeof(int32_t) * nnz));
        BFS_CUDA_TRY(cudaMemcpyAsync(dcol.ptr, col, sizeof(int32_t) * nnz, cudaMemcpyHostToDevice, st));
        cl = dcol.as<int32_t>();
    }
    BFS_TRY(err.alloc(sizeof(unsigned long long)));
    BFS_CUDA_TRY(cudaMemsetAsync(err.ptr, 0, err.bytes, st));
    check_csr<<<grid_for(n > nnz ? n : nnz, 256), 256, 0, st>>>(rp, cl, n, nnz, err.as<unsigned long long>());
    BFS_CUDA_TRY(cudaGetLastError());
    unsigned long long h_err = 0;
    BFS_CUDA_TRY(cudaMemcpyAsync(&h_err, err.ptr, sizeof(h_err), cudaMemcpyDeviceToHost, st));
    BFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (h_err) return set_error(BFS_ERR_INVALID_ARG, "row_ptr is not nondecreasing or col names a vertex outside [0, n)");
    BFS_TRY(dsrc.alloc(sizeof(int32_t) * (nnz > 0 ? nnz : 1)));
    expand_rows<<<grid_for(n, 256), 256, 0, st>>>(rp, n, dsrc.as<int32_t>());
    BFS_CUDA_TRY(cudaGetLastError());
    return create_common(n, nnz, dsrc.as<int32_t>(), cl, 0, opt, stream, out, true);
}

bfs_status bfs_graph_destroy(bfs_graph_t g) {
    if (!g) return BFS_OK;
    if (g->busy.load()) return set_error(BFS_ERR_BUSY, "graph is in use");
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    free_msbfs(g);
    free_workspace(g);
    delete g;
    cudaSetDevice(cur);
    return BFS_OK;
}

bfs_status bfs_graph_footprint(bfs_graph_t g, int64_t* bytes) {
    if (!g || !bytes) return set_error(BFS_ERR_INVALID_ARG, "NULL argument");
    const Layout& L = g->L;
    const Workspace& W = g->W;
    int64_t b = (int64_t)(L.dir.bytes + L.rank.bytes + L.cp.bytes + L.ir.bytes + L.cp_base_d.bytes + L.ir_base_d.bytes +
                          L.deg.bytes + L.iso.bytes + L.bu_ptr.bytes + L.bu_adj.bytes);
    b += (int64_t)(W.pi.bytes + W.fa.bytes + W.fb.bytes + W.fsum.bytes + W.xbuf.bytes + W.xcount.bytes +
                   W.chunk_base.bytes + W.units.bytes + W.counters.bytes + W.tmp_parent.bytes + W.tmp_level.bytes +
                   W.pieces.bytes + W.level_scratch.bytes + W.row_meta.bytes + W.tblk.bytes + W.rowbuf.bytes +
                   W.rowcount.bytes + W.rowfirst.bytes + W.rowlive.bytes + W.xfmt.bytes + W.enc_sums.bytes + W.enc_bases.bytes + W.enc_flags.bytes +
                   W.enc_done.bytes + W.gbits.bytes + W.colfirst.bytes + W.ddir.bytes);
    *bytes = b;
    return BFS_OK;
}

bfs_status bfs_graph_info(bfs_graph_t g, bfs_graph_info_t* info) {
    if (!g || !info) return set_error(BFS_ERR_INVALID_ARG, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->n_vertices = g->L.n;
    info->n_entries = g->L.nnz;
    info->p = g->L.p;
    info->mode = g->mode;
    info->wah_word_bits = g->wah_bits;
    info->range_size = g->L.nb;
    info->row_exchange = g->row_exchange;
    info->exchange_format = g->adaptive ? BFS_FORMAT_ADAPTIVE : BFS_FORMAT_WAH;
    info->direction = g->direction;
    info->dynamic_directory = g->dynamic_dir;
    info->nonempty_columns = g->L.nnzc_total;
    return BFS_OK;
}

bfs_status bfs_graph_set_mode(bfs_graph_t g, int32_t mode, int32_t wah_word_bits) {
    if (!g) return set_error(BFS_ERR_INVALID_ARG, "graph is NULL");
    if (mode < 0 || mode > 2) return set_error(BFS_ERR_INVALID_ARG, "unknown mode %d", mode);
    if (wah_word_bits != 32 && wah_word_bits != 64) return set_error(BFS_ERR_INVALID_ARG, "wah_word_bits must be 32 or 64");
    if (g->busy.load()) return set_error(BFS_ERR_BUSY, "graph is in use");
    std::lock_guard<std::mutex> lk(g->mu);
    g->mode = mode;
    g->wah_bits = wah_word_bits;
    return BFS_OK;
}

bfs_status bfs_graph_set_row_exchange(bfs_graph_t g, int32_t enabled) {
    if (!g) return set_error(BFS_ERR_INVALID_ARG, "graph is NULL");
    if (g->busy.load()) return set_error(BFS_ERR_BUSY, "graph is in use");
    std::lock_guard<std::mutex> lk(g->mu);
    g->row_exchange = enabled ? 1 : 0;
    return BFS_OK;
}

bfs_status bfs_graph_set_exchange_format(bfs_graph_t g, int32_t format) {
    if (!g) return set_error(BFS_ERR_INVALID_ARG, "graph is NULL");
    if (format != BFS_FORMAT_WAH && format != BFS_FORMAT_ADAPTIVE)
        return set_error(BFS_ERR_INVALID_ARG, "unknown exchange format %d", format);
    if (g->busy.load()) return set_error(BFS_ERR_BUSY, "graph is in use");
    std::lock_guard<std::mutex> lk(g->mu);
    g->adaptive = format == BFS_FORMAT_ADAPTIVE ? 1 : 0;
    return BFS_OK;
}

bfs_status bfs_graph_set_dynamic_directory(bfs_graph_t g, int32_t enabled) {
    if (!g) return set_error(BFS_ERR_INVALID_ARG, "graph is NULL");
    if (enabled != 0 && enabled != 1) return set_error(BFS_ERR_INVALID_ARG, "enabled must be 0 or 1");
    if (g->busy.load()) return set_error(BFS_ERR_BUSY, "graph is in use");
    std::lock_guard<std::mutex> lk(g->mu);
    g->dynamic_dir = enabled;
    return BFS_OK;
}

bfs_status bfs_graph_set_direction(bfs_graph_t g, int32_t policy, int32_t alpha, int32_t beta) {
    if (!g) return set_error(BFS_ERR_INVALID_ARG, "graph is NULL");
    if (policy < BFS_DIRECTION_TOP_DOWN || policy > BFS_DIRECTION_BOTTOM_UP)
        return set_error(BFS_ERR_INVALID_ARG, "unknown direction policy %d", policy);
    if (alpha < 1 || alpha > 1000000 || beta < 1 || beta > 1000000)
        return set_error(BFS_ERR_INVALID_ARG, "alpha and beta must lie in [1, 1000000]");
    if (policy != BFS_DIRECTION_TOP_DOWN && !g->symmetric)
        return set_error(BFS_ERR_INVALID_ARG, "bottom-up levels need an undirected graph (created with symmetrize = 1)");
    if (g->busy.load()) return set_error(BFS_ERR_BUSY, "graph is in use");
    std::lock_guard<std::mutex> lk(g->mu);
    if (policy != BFS_DIRECTION_TOP_DOWN) {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(g->device);
        const bfs_status rc = ensure_degrees(g, nullptr);
        cudaSetDevice(cur);
        BFS_TRY(rc);
    }
    g->direction = policy;
    g->alpha = alpha;
    g->beta = beta;
    return BFS_OK;
}

bfs_status bfs_graph_directory(bfs_graph_t g, int32_t i, int32_t j, uint32_t* out_words, void* stream) {
    if (!g || !out_words) return set_error(BFS_ERR_INVALID_ARG, "NULL argument");
    const int p = g->L.p;
    if (i < 0 || i >= p || j < 0 || j >= p) return set_error(BFS_ERR_INVALID_ARG, "block (%d,%d) outside the %dx%d grid", i, j, p, p);
    const int64_t words = (g->L.range_len(j) + 31) / 32;
    if (words == 0) return BFS_OK;
    const uint32_t* src = g->L.dir.as<uint32_t>() + ((int64_t)i * p + j) * g->L.dir_stride;
    BFS_CUDA_TRY(cudaMemcpyAsync(out_words, src, sizeof(uint32_t) * words, cudaMemcpyDeviceToDevice,
                                 static_cast<cudaStream_t>(stream)));
    return BFS_OK;
}

}  // extern "C"
