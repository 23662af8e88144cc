// msbfs.cu -- batched multi-source BFS: up to 64 searches at once, bit-parallel.
//
// Every vertex holds three 64-bit lane words (bit r = search r): vis (visited),
// f (frontier) and nxt (next).  One level is the boolean SpMV of Sec. III-A
// applied to all 64 lane vectors at once:
//   nxt[v] |= f[u] & ~vis[v]     for every entry u -> v of a nonempty column
// of a block whose source u is active (f[u] != 0); the directory V_{i,j}
// (Eq. 4) sieves the (vertex, block) pairs, exactly as in the single search.
// Then new = nxt & ~vis; vis |= new; f = new; level[r][v] = k + 1 for every new
// bit r; and the next level's active list is the set of v with new != 0.
// Optional parents: parent[r][v] = the smallest u of lane r's previous level
// with an entry u -> v, by a (select, min) reduction per new lane bit.
//
// The whole batch is one CUDA-graph launch: the initialisation, then a
// conditional WHILE node whose body is one level (expand, long-column pieces,
// reduce, and a one-thread kernel that decides whether to iterate again from
// the active count).  No host round trip per level.  Kernels read their
// arguments from a device-resident state block, so the graph is built once per
// graph handle and reused by every call.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace bfsgb {
namespace {

constexpr int kMT = 256;            // threads of the small kernels
constexpr uint32_t kMsCoop = 32;    // columns of at least this many entries take the whole warp
constexpr uint32_t kMsHub = 1024;   // longer columns are cut into pieces
constexpr uint32_t kMsPiece = 1024;

// Device-resident arguments and counters of a batch (one per graph).
struct MsState {
    // graph layout (constant)
    const uint32_t* dir;
    const uint32_t* rank;
    int64_t dir_stride;
    const uint32_t* cp;
    const int64_t* cp_base;
    const int64_t* ir_base;
    const int32_t* ir;
    int p;
    int64_t nb, n;
    // lane words and active lists (constant buffers)
    unsigned long long* vis;
    unsigned long long* f[2];
    unsigned long long* nxt;
    int32_t* act[2];
    Item* pieces;
    int64_t piece_cap;
    // per call
    const int32_t* roots;       // device copy of the roots
    int32_t n_roots;
    int32_t max_levels;         // iteration limit (n + 1 at most)
    int32_t* levels;            // [n_roots][n]
    int32_t* parents;           // [n_roots][n] or nullptr
    // per level
    int32_t cur;                // index of the current f / act buffers
    int32_t level;              // k
    unsigned long long act_count[2];
    unsigned long long act_next;     // hand-out cursor over the current active list
    unsigned long long piece_count;
    unsigned long long piece_next;
    unsigned long long edges;        // entries scanned (all levels)
    unsigned long long levels_done;  // levels performed
};

__device__ __forceinline__ int64_t ms_range_begin(const MsState& s, int64_t b) {
    const int64_t x = b * s.nb;
    return x < s.n ? x : s.n;
}

// ------------------------------------------------------------------ init --
__global__ void ms_reset(MsState* S) {
    S->cur = 0;
    S->level = 0;
    S->act_count[0] = 0;
    S->act_count[1] = 0;
    S->act_next = 0;
    S->piece_count = 0;
    S->piece_next = 0;
    S->edges = 0;
    S->levels_done = 0;
}

__global__ void ms_clear(MsState* S) {
    const MsState& s = *S;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t v = tid; v < s.n; v += stride) {
        s.vis[v] = 0ull;
        s.f[0][v] = 0ull;
        s.f[1][v] = 0ull;
        s.nxt[v] = 0ull;
    }
    const int64_t total = (int64_t)s.n_roots * s.n;
    for (int64_t x = tid; x < total; x += stride) {
        s.levels[x] = -1;
        if (s.parents) s.parents[x] = -1;
    }
}

__global__ void ms_roots(MsState* S) {
    MsState& s = *S;
    const int r = threadIdx.x;
    if (r >= s.n_roots) return;
    const int32_t v = s.roots[r];
    const unsigned long long bit = 1ull << r;
    const unsigned long long old = atomicOr(s.vis + v, bit);
    atomicOr(s.f[0] + v, bit);
    s.levels[(int64_t)r * s.n + v] = 0;
    if (s.parents) s.parents[(int64_t)r * s.n + v] = v;
    if (old == 0ull) {                       // first lane at this vertex: make it active
        const unsigned long long pos = atomicAdd(&s.act_count[0], 1ull);
        s.act[0][pos] = v;
    }
}

// ----------------------------------------------------------------- level --
struct MsVisit {
    const MsState* s;
    __device__ __forceinline__ void operator()(int32_t v, int32_t u, unsigned long long fu) const {
        const unsigned long long nb = fu & ~__ldg(s->vis + v);     // vis does not change during the expansion
        if (!nb) return;
        atomicOr(s->nxt + v, nb);
        if (s->parents) {
            unsigned long long m = nb;
            while (m) {
                const int r = __ffsll((long long)m) - 1;
                m &= m - 1;
                atomicMin(reinterpret_cast<unsigned int*>(s->parents + (int64_t)r * s->n + v), (unsigned int)u);
            }
        }
    }
};

__device__ __forceinline__ void ms_column(const MsVisit& vis, const int32_t* ir, int32_t u, unsigned long long fu,
                                          int64_t beg, uint32_t len) {
    const int32_t* col = ir + beg;
    for (uint32_t e = lane_id(); e < len; e += 32) vis(__ldg(col + e), u, fu);
}

// One item per lane (u, f[u], column); long columns go to the piece list,
// columns of at least kMsCoop entries take the whole warp, the rest share the
// warp through a load-balanced search over their entry counts.
__device__ __forceinline__ void ms_warp_expand(MsState& s, const MsVisit& vis, int32_t u, unsigned long long fu,
                                               int64_t beg, uint32_t len, unsigned long long& edges) {
    edges += len;
    if (__any_sync(0xffffffffu, len > kMsHub)) {
        if (len > kMsHub) {
            const uint32_t np = (len + kMsPiece - 1) / kMsPiece;
            const unsigned long long base = atomicAdd(&s.piece_count, (unsigned long long)np);
            for (uint32_t k = 0; k < np && base + k < (unsigned long long)s.piece_cap; ++k) {
                Item it;
                it.u = u;
                it.len = (len - k * kMsPiece < kMsPiece) ? len - k * kMsPiece : kMsPiece;
                it.begin = beg + (int64_t)k * kMsPiece;
                s.pieces[base + k] = it;
            }
            len = 0;
        }
    }
    uint32_t coop = __ballot_sync(0xffffffffu, len >= kMsCoop);
    while (coop) {
        const int src = __ffs(coop) - 1;
        coop &= coop - 1;
        ms_column(vis, s.ir, __shfl_sync(0xffffffffu, u, src), __shfl_sync(0xffffffffu, fu, src),
                  __shfl_sync(0xffffffffu, beg, src), __shfl_sync(0xffffffffu, len, src));
    }
    if (len >= kMsCoop) len = 0;
    const uint32_t incl = warp_incl_sum(len);
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const uint32_t excl = incl - len;
    for (uint32_t e0 = 0; e0 < total; e0 += 32) {
        const uint32_t e = e0 + lane_id();
        int lo = 0, hi = 31;
#pragma unroll
        for (int step = 0; step < 5; ++step) {
            const int mid = (lo + hi) >> 1;
            const uint32_t im = __shfl_sync(0xffffffffu, incl, mid);
            if (im > e) hi = mid; else lo = mid + 1;
        }
        const int64_t ob = __shfl_sync(0xffffffffu, beg, lo);
        const uint32_t oe = __shfl_sync(0xffffffffu, excl, lo);
        const int32_t ou = __shfl_sync(0xffffffffu, u, lo);
        const unsigned long long of = __shfl_sync(0xffffffffu, fu, lo);
        if (e < total) vis(__ldg(s.ir + ob + (int64_t)(e - oe)), ou, of);
    }
}

// Expansion: warps take 32 active vertices at a time; for every block-row i,
// the vertices whose column of block (i, j(u)) is nonempty (directory test)
// are expanded.
__global__ void ms_expand(MsState* S) {
    MsState& s = *S;
    const MsVisit vis{S};
    const int cur = s.cur;
    const int32_t* act = s.act[cur];
    const unsigned long long nact = s.act_count[cur];
    const unsigned long long* f = s.f[cur];
    unsigned long long edges = 0;
    for (;;) {
        unsigned long long base = 0;
        if (lane_id() == 0) base = atomicAdd(&s.act_next, 32ull);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= nact) break;
        const unsigned long long q = base + lane_id();
        int32_t u = 0;
        unsigned long long fu = 0;
        int64_t j = 0, ul = 0;
        if (q < nact) {
            u = act[q];
            fu = f[u];
            j = u / s.nb;
            ul = u - j * s.nb;
        }
        for (int i = 0; i < s.p; ++i) {
            int64_t beg = 0;
            uint32_t len = 0;
            if (fu) {
                const int64_t b = (int64_t)i * s.p + j;
                const uint32_t* dirb = s.dir + b * s.dir_stride;
                const uint32_t dw = __ldg(dirb + (ul >> 5));
                const uint32_t bit = 1u << (ul & 31);
                if (dw & bit) {
                    const uint32_t c = __ldg(s.rank + b * s.dir_stride + (ul >> 5)) + __popc(dw & (bit - 1u));
                    const uint32_t* cpb = s.cp + __ldg(s.cp_base + b);
                    const uint32_t c0 = __ldg(cpb + c), c1 = __ldg(cpb + c + 1);
                    beg = __ldg(s.ir_base + b) + c0;
                    len = c1 - c0;
                }
            }
            if (__any_sync(0xffffffffu, len > 0)) ms_warp_expand(s, vis, u, fu, beg, len, edges);
        }
    }
    edges = warp_sum(edges);
    if (lane_id() == 0 && edges) atomicAdd(&s.edges, edges);
}

__global__ void ms_pieces(MsState* S) {
    MsState& s = *S;
    const MsVisit vis{S};
    const unsigned long long* f = s.f[s.cur];
    const unsigned long long np = min(s.piece_count, (unsigned long long)s.piece_cap);
    for (;;) {
        unsigned long long pc = 0;
        if (lane_id() == 0) pc = atomicAdd(&s.piece_next, 1ull);
        pc = __shfl_sync(0xffffffffu, pc, 0);
        if (pc >= np) break;
        const Item it = s.pieces[pc];
        ms_column(vis, s.ir, it.u, f[it.u], it.begin, it.len);
    }
}

// new = nxt & ~vis; vis |= new; f' = new; level of every new lane; next active list.
__global__ void __launch_bounds__(kMT) ms_reduce(MsState* S) {
    MsState& s = *S;
    const int cur = s.cur, nxt_i = cur ^ 1;
    unsigned long long* fn = s.f[nxt_i];
    int32_t* actn = s.act[nxt_i];
    const int32_t lv = s.level + 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nwarp_iters = (s.n + stride - 1) / stride;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    for (int64_t it = 0; it < nwarp_iters; ++it) {
        const int64_t v = it * stride + tid;
        unsigned long long nv = 0;
        if (v < s.n) {
            const unsigned long long x = s.nxt[v];
            if (x) {
                s.nxt[v] = 0ull;
                nv = x & ~s.vis[v];
                if (nv) {
                    s.vis[v] |= nv;
                    unsigned long long m = nv;
                    while (m) {
                        const int r = __ffsll((long long)m) - 1;
                        m &= m - 1;
                        s.levels[(int64_t)r * s.n + v] = lv;
                    }
                }
            }
            fn[v] = nv;
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, nv != 0ull);
        if (ball) {
            unsigned long long base = 0;
            if (lane_id() == 0) base = atomicAdd(&s.act_count[nxt_i], (unsigned long long)__popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (nv) actn[base + __popc(ball & ((1u << lane_id()) - 1u))] = (int32_t)v;
        }
    }
}

// One thread: switch to the next level and decide whether to iterate again.
__global__ void ms_finalize(MsState* S, cudaGraphConditionalHandle handle) {
    MsState& s = *S;
    const int nxt_i = s.cur ^ 1;
    const unsigned long long cnt = s.act_count[nxt_i];
    s.act_count[s.cur] = 0;
    s.cur = nxt_i;
    s.level += 1;
    s.levels_done += 1;
    s.act_next = 0;
    s.piece_count = 0;
    s.piece_next = 0;
    cudaGraphSetConditional(handle, (cnt > 0 && s.level < s.max_levels) ? 1u : 0u);
}

int ms_sm_count() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    return v > 0 ? v : 1;
}

}  // namespace

// ---------------------------------------------------------- host side --
struct MsContext {
    DevBuf vis, f0, f1, nxt, act0, act1, pieces, state, roots;
    int64_t piece_cap = 0;
    cudaGraph_t graph[2] = {nullptr, nullptr};       // [without parents, with parents]
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    int expand_ctas_per_sm = 4;                       // launch shape, set by the autotuner
    int expand_threads = 256;
    ~MsContext() {
        for (int k = 0; k < 2; ++k) {
            if (exec[k]) cudaGraphExecDestroy(exec[k]);
            if (graph[k]) cudaGraphDestroy(graph[k]);
        }
    }
    void drop_graphs() {
        for (int k = 0; k < 2; ++k) {
            if (exec[k]) cudaGraphExecDestroy(exec[k]);
            if (graph[k]) cudaGraphDestroy(graph[k]);
            exec[k] = nullptr;
            graph[k] = nullptr;
        }
    }
};

void free_msbfs(bfs_graph* g) {
    delete g->ms;
    g->ms = nullptr;
}

namespace {

bfs_status ms_ensure(bfs_graph* g) {
    if (g->ms) return BFS_OK;
    MsContext* c = new (std::nothrow) MsContext();
    if (!c) return set_error(BFS_ERR_OUT_OF_MEMORY, "host allocation");
    const Layout& L = g->L;
    const int64_t n = L.n;
    bfs_status rc = BFS_OK;
    c->piece_cap = L.nnz / kMsPiece + L.nnz / kMsHub + 16;
    if (rc == BFS_OK) rc = c->vis.alloc(8 * n);
    if (rc == BFS_OK) rc = c->f0.alloc(8 * n);
    if (rc == BFS_OK) rc = c->f1.alloc(8 * n);
    if (rc == BFS_OK) rc = c->nxt.alloc(8 * n);
    if (rc == BFS_OK) rc = c->act0.alloc(4 * n);
    if (rc == BFS_OK) rc = c->act1.alloc(4 * n);
    if (rc == BFS_OK) rc = c->pieces.alloc(sizeof(Item) * c->piece_cap);
    if (rc == BFS_OK) rc = c->state.alloc(sizeof(MsState));
    if (rc == BFS_OK) rc = c->roots.alloc(sizeof(int32_t) * 64);
    if (rc != BFS_OK) { delete c; return rc; }
    MsState h;
    memset(&h, 0, sizeof(h));
    h.dir = L.dir.as<uint32_t>();
    h.rank = L.rank.as<uint32_t>();
    h.dir_stride = L.dir_stride;
    h.cp = L.cp.as<uint32_t>();
    h.cp_base = L.cp_base_d.as<int64_t>();
    h.ir_base = L.ir_base_d.as<int64_t>();
    h.ir = L.ir.as<int32_t>();
    h.p = L.p;
    h.nb = L.nb;
    h.n = n;
    h.vis = c->vis.as<unsigned long long>();
    h.f[0] = c->f0.as<unsigned long long>();
    h.f[1] = c->f1.as<unsigned long long>();
    h.nxt = c->nxt.as<unsigned long long>();
    h.act[0] = c->act0.as<int32_t>();
    h.act[1] = c->act1.as<int32_t>();
    h.pieces = c->pieces.as<Item>();
    h.piece_cap = c->piece_cap;
    h.roots = c->roots.as<int32_t>();
    cudaError_t e = cudaMemcpy(c->state.ptr, &h, sizeof(h), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { delete c; return cuda_error(e, "cudaMemcpy(state)", __FILE__, __LINE__); }
    g->ms = c;
    return BFS_OK;
}

// Build the batch graph: reset, clear, roots, then WHILE(level) { expand,
// pieces, reduce, finalize }.
bfs_status ms_build_graph(bfs_graph* g, int with_parents, cudaStream_t st) {
    MsContext* c = g->ms;
    if (c->exec[with_parents]) return BFS_OK;
    MsState* S = c->state.as<MsState>();
    const int sms = ms_sm_count();
    cudaGraph_t graph = nullptr;
    BFS_CUDA_TRY(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle handle;
    BFS_CUDA_TRY(cudaGraphConditionalHandleCreate(&handle, graph, 1, cudaGraphCondAssignDefault));
    // prologue nodes, captured
    cudaStream_t cs = nullptr;
    BFS_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    BFS_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    ms_reset<<<1, 1, 0, cs>>>(S);
    ms_clear<<<sms * 8, kMT, 0, cs>>>(S);
    ms_roots<<<1, 64, 0, cs>>>(S);
    cudaGraph_t captured = nullptr;
    cudaError_t ce = cudaStreamEndCapture(cs, &captured);
    if (ce != cudaSuccess) {
        cudaStreamDestroy(cs);
        cudaGraphDestroy(graph);
        return cuda_error(ce, "capture of the batch prologue", __FILE__, __LINE__);
    }
    // the conditional loop after the prologue
    size_t nleaf = 0;
    BFS_CUDA_TRY(cudaGraphGetNodes(graph, nullptr, &nleaf));
    std::vector<cudaGraphNode_t> nodes(nleaf);
    BFS_CUDA_TRY(cudaGraphGetNodes(graph, nodes.data(), &nleaf));
    cudaGraphNode_t last = nullptr;
    for (auto nd : nodes) {                      // the prologue is a chain: its sink is the only node without successors
        size_t nout = 0;
        BFS_CUDA_TRY(cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nout));
        if (nout == 0) last = nd;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = handle;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond = nullptr;
    BFS_CUDA_TRY(cudaGraphAddNode(&cond, graph, &last, nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    BFS_CUDA_TRY(cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    ms_expand<<<sms * c->expand_ctas_per_sm, c->expand_threads, 0, cs>>>(S);
    ms_pieces<<<sms * 4, kMT, 0, cs>>>(S);
    ms_reduce<<<sms * 8, kMT, 0, cs>>>(S);
    ms_finalize<<<1, 1, 0, cs>>>(S, handle);
    ce = cudaStreamEndCapture(cs, &body);
    cudaStreamDestroy(cs);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_error(ce, "capture of the batch level body", __FILE__, __LINE__);
    }
    (void)with_parents;
    cudaGraphExec_t exec = nullptr;
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_error(ce, "cudaGraphInstantiate(batch)", __FILE__, __LINE__);
    }
    c->graph[with_parents] = graph;
    c->exec[with_parents] = exec;
    (void)st;
    return BFS_OK;
}

struct MsCall {
    const int32_t* roots;
    int32_t n_roots;
    int32_t max_levels;
    int32_t* levels;
    int32_t* parents;
};

bfs_status ms_run(bfs_graph* g, const int32_t* roots_host, int32_t n_roots, int32_t* levels, int32_t* parents,
                  bfs_batch_stats* stats, cudaStream_t st) {
    BFS_TRY(ms_ensure(g));
    MsContext* c = g->ms;
    const int wp = parents ? 1 : 0;
    BFS_TRY(ms_build_graph(g, wp, st));
    // per-call fields of the state block
    BFS_CUDA_TRY(cudaMemcpyAsync(c->roots.ptr, roots_host, sizeof(int32_t) * n_roots, cudaMemcpyHostToDevice, st));
    MsCall call{c->roots.as<int32_t>(), n_roots, (int32_t)std::min<int64_t>(g->L.n + 1, 0x7fffffff), levels, parents};
    BFS_CUDA_TRY(cudaMemcpyAsync(reinterpret_cast<char*>(c->state.ptr) + offsetof(MsState, roots), &call,
                                 sizeof(MsCall), cudaMemcpyHostToDevice, st));
    BFS_CUDA_TRY(cudaGraphLaunch(c->exec[wp], st));
    if (stats) {
        MsState h;
        BFS_CUDA_TRY(cudaMemcpyAsync(&h, c->state.ptr, sizeof(h), cudaMemcpyDeviceToHost, st));
        BFS_CUDA_TRY(cudaStreamSynchronize(st));
        stats->n_levels = (int32_t)h.levels_done;
        stats->edges_scanned = (int64_t)h.edges;
    }
    return BFS_OK;
}

}  // namespace
}  // namespace bfsgb

using namespace bfsgb;

extern "C" bfs_status bfs_run_batch(bfs_graph_t g, const int32_t* roots, int32_t n_roots, int32_t* levels,
                                    int32_t* parents, bfs_batch_stats* stats, void* stream) {
    if (!g) return set_error(BFS_ERR_INVALID_ARG, "graph is NULL");
    if (!roots || !levels) return set_error(BFS_ERR_INVALID_ARG, "roots and levels are required");
    if (n_roots < 1 || n_roots > 64) return set_error(BFS_ERR_INVALID_ARG, "n_roots %d outside [1, 64]", n_roots);
    if (!is_device_pointer(levels) || (parents && !is_device_pointer(parents)))
        return set_error(BFS_ERR_INVALID_ARG, "levels and parents must be device pointers");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t hroots[64];
    if (is_device_pointer(roots)) {
        BFS_CUDA_TRY(cudaMemcpyAsync(hroots, roots, sizeof(int32_t) * n_roots, cudaMemcpyDeviceToHost, st));
        BFS_CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        memcpy(hroots, roots, sizeof(int32_t) * n_roots);
    }
    for (int r = 0; r < n_roots; ++r)
        if (hroots[r] < 0 || (int64_t)hroots[r] >= g->L.n)
            return set_error(BFS_ERR_INVALID_ARG, "root %d outside [0, %lld)", hroots[r], (long long)g->L.n);
    int expect = 0;
    if (!g->busy.compare_exchange_strong(expect, 1)) return set_error(BFS_ERR_BUSY, "another search on this graph is running");
    bfs_status rc = ms_run(g, hroots, n_roots, levels, parents, stats, st);
    if (rc == BFS_OK && !stats) {
        cudaError_t e = cudaStreamSynchronize(st);     // hroots is read by an async copy
        if (e != cudaSuccess) rc = cuda_error(e, "cudaStreamSynchronize", __FILE__, __LINE__);
    }
    g->busy.store(0);
    return rc;
}

extern "C" bfs_status bfs_batch_autotune(bfs_graph_t g, const int32_t* roots, int32_t n_roots, int32_t* levels,
                                         int32_t* best_threads, int32_t* best_ctas_per_sm, void* stream) {
    if (!g || !roots || !levels) return set_error(BFS_ERR_INVALID_ARG, "NULL argument");
    if (n_roots < 1 || n_roots > 64) return set_error(BFS_ERR_INVALID_ARG, "n_roots %d outside [1, 64]", n_roots);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BFS_TRY(ms_ensure(g));
    MsContext* c = g->ms;
    static const int threads[] = {128, 256, 512, 1024};
    static const int ctas[] = {1, 2, 4, 8, 16};
    cudaEvent_t e0, e1;
    BFS_CUDA_TRY(cudaEventCreate(&e0));
    BFS_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int bt = c->expand_threads, bc = c->expand_ctas_per_sm;
    bfs_status rc = BFS_OK;
    for (int t : threads) {
        for (int k : ctas) {
            if (t * k > 2048) continue;                 // threads resident per SM
            c->drop_graphs();
            c->expand_threads = t;
            c->expand_ctas_per_sm = k;
            float ms = 0.f;
            for (int rep = 0; rep < 2 && rc == BFS_OK; ++rep) {
                cudaEventRecord(e0, st);
                rc = bfs_run_batch(g, roots, n_roots, levels, nullptr, nullptr, stream);
                cudaEventRecord(e1, st);
                cudaEventSynchronize(e1);
                cudaEventElapsedTime(&ms, e0, e1);
            }
            if (rc != BFS_OK) break;
            if (ms < best) { best = ms; bt = t; bc = k; }
        }
        if (rc != BFS_OK) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->drop_graphs();
    c->expand_threads = bt;
    c->expand_ctas_per_sm = bc;
    if (rc != BFS_OK) return rc;
    if (best_threads) *best_threads = bt;
    if (best_ctas_per_sm) *best_ctas_per_sm = bc;
    return BFS_OK;
}

