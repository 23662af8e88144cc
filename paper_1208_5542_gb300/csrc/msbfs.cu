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
    unsigned long long parent_mask;  // lanes whose parents are computed (with parents != nullptr)
    // per level
    int32_t cur;                // index of the current f / act buffers
    int32_t level;              // k
    unsigned long long act_count[2];
    unsigned long long act_next;     // hand-out cursor over the current active list
    unsigned long long piece_count;
    unsigned long long piece_next;
    unsigned long long edges;        // entries scanned (all levels)
    unsigned long long levels_done;  // levels performed
    // continuous batching (server): lane r's level of v is (iteration + 1) - lane_start[r]
    int32_t lane_start[64];
    unsigned long long alive;        // lanes that reached a new vertex in this iteration
    int64_t nnz;                     // entries of the layout
    unsigned long long err;          // first failed bounds check: code, then two values
    unsigned long long err_a, err_b;
};

// A bounds check failed: keep the first one's code and values (the access is skipped).
__device__ __forceinline__ void ms_fault(MsState* S, unsigned long long code, unsigned long long x,
                                         unsigned long long y) {
    if (atomicCAS(&S->err, 0ull, code) == 0ull) {
        S->err_a = x;
        S->err_b = y;
    }
}

// ------------------------------------------------------------------ init --
__global__ void ms_reset(MsState* S) {
    for (int r = 0; r < 64; ++r) S->lane_start[r] = 0;
    S->alive = 0;
    S->cur = 0;
    S->level = 0;
    S->act_count[0] = 0;
    S->act_count[1] = 0;
    S->act_next = 0;
    S->piece_count = 0;
    S->piece_next = 0;
    S->edges = 0;
    S->levels_done = 0;
    S->err = 0;
    S->err_a = 0;
    S->err_b = 0;
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
        if ((uint64_t)(uint32_t)v >= (uint64_t)s->n) { ms_fault(const_cast<MsState*>(s), 2, (uint32_t)v, (uint32_t)u); return; }
        const unsigned long long nb = fu & ~__ldg(s->vis + v);     // vis does not change during the expansion
        if (!nb) return;
        atomicOr(s->nxt + v, nb);
        if (s->parents) {
            unsigned long long m = nb & s->parent_mask;
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
            if ((uint64_t)(uint32_t)u >= (uint64_t)s.n) { ms_fault(S, 1, q, (uint32_t)u); u = 0; }
            else fu = f[u];
            j = (uint32_t)u / (uint32_t)s.nb;                 // ids and ranges are below 2^31
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
        if ((uint64_t)(uint32_t)it.u >= (uint64_t)s.n || it.begin < 0 || it.begin + (int64_t)it.len > s.nnz) {
            if (lane_id() == 0) ms_fault(S, 6, pc, (uint64_t)it.begin);
            continue;
        }
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
                        s.levels[(int64_t)r * s.n + v] = lv - s.lane_start[r];
                    }
                }
            }
            fn[v] = nv;
        }
        const uint32_t ball = __ballot_sync(0xffffffffu, nv != 0ull);
        unsigned long long any = nv;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) any |= __shfl_xor_sync(0xffffffffu, any, d);
        if (any && lane_id() == 0) atomicOr(&s.alive, any);
        if (ball) {
            unsigned long long base = 0;
            if (lane_id() == 0) base = atomicAdd(&s.act_count[nxt_i], (unsigned long long)__popc(ball));
            base = __shfl_sync(0xffffffffu, base, 0);
            const unsigned long long at = base + __popc(ball & ((1u << lane_id()) - 1u));
            if (nv) {
                if (at < (unsigned long long)s.n) actn[at] = (int32_t)v;
                else ms_fault(S, 3, at, (uint64_t)v);
            }
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

// One server iteration ends: switch buffers, advance the iteration.
__global__ void ms_step_end(MsState* S) {
    MsState& s = *S;
    const int nxt_i = s.cur ^ 1;
    s.act_count[s.cur] = 0;
    s.cur = nxt_i;
    s.level += 1;
    s.levels_done += 1;
    s.act_next = 0;
    s.piece_count = 0;
    s.piece_next = 0;
}

// Admission, phase A: lanes in `mask` start over -- clear their bits in every
// lane word and their level rows.
__global__ void ms_admit_clear(MsState* S, unsigned long long mask, const int32_t* lanes, int nlanes) {
    MsState& s = *S;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const unsigned long long keep = ~mask;
    for (int64_t v = tid; v < s.n; v += stride) {
        if (s.vis[v] & mask) s.vis[v] &= keep;
        if (s.f[s.cur][v] & mask) s.f[s.cur][v] &= keep;
        if (s.nxt[v] & mask) s.nxt[v] &= keep;
    }
    const int64_t total = (int64_t)nlanes * s.n;
    for (int64_t x = tid; x < total; x += stride) {
        const int64_t q = x / s.n;
        const int r = lanes[q];
        if (r < 0 || r >= 64) { ms_fault(S, 7, (uint64_t)x, (uint64_t)r); continue; }
        s.levels[(int64_t)r * s.n + (x - q * s.n)] = -1;
        if (s.parents) s.parents[(int64_t)r * s.n + (x - q * s.n)] = -1;
    }
    if (tid == 0) s.alive = 0;
}

// Admission, phase B: lane lanes[q] starts from roots[q] at this iteration,
// computing parents when want_parents[q] != 0.
__global__ void ms_admit_roots(MsState* S, const int32_t* lanes, const int32_t* roots, const int32_t* want_parents,
                               int nlanes) {
    MsState& s = *S;
    const int q = threadIdx.x;
    if (q >= nlanes) return;
    const int r = lanes[q];
    const int32_t v = roots[q];
    if (r < 0 || r >= 64 || (uint64_t)(uint32_t)v >= (uint64_t)s.n) { ms_fault(S, 4, (uint64_t)r, (uint32_t)v); return; }
    const unsigned long long bit = 1ull << r;
    if (want_parents[q]) atomicOr(&s.parent_mask, bit);
    else atomicAnd(&s.parent_mask, ~bit);
    atomicOr(s.vis + v, bit);
    const unsigned long long old = atomicOr(s.f[s.cur] + v, bit);
    s.levels[(int64_t)r * s.n + v] = 0;
    if (s.parents) s.parents[(int64_t)r * s.n + v] = v;
    s.lane_start[r] = s.level;
    if (old == 0ull) {
        const unsigned long long pos = atomicAdd(&s.act_count[s.cur], 1ull);
        if (pos < (unsigned long long)s.n) s.act[s.cur][pos] = v;
        else ms_fault(S, 5, pos, (uint32_t)v);
    }
}

__global__ void ms_clear_alive(MsState* S) { S->alive = 0; }

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
    h.nnz = L.nnz;
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
    unsigned long long parent_mask;
};

bfs_status ms_run(bfs_graph* g, const int32_t* roots_host, int32_t n_roots, int32_t* levels, int32_t* parents,
                  bfs_batch_stats* stats, cudaStream_t st) {
    BFS_TRY(ms_ensure(g));
    MsContext* c = g->ms;
    const int wp = parents ? 1 : 0;
    BFS_TRY(ms_build_graph(g, wp, st));
    // per-call fields of the state block
    BFS_CUDA_TRY(cudaMemcpyAsync(c->roots.ptr, roots_host, sizeof(int32_t) * n_roots, cudaMemcpyHostToDevice, st));
    MsCall call{c->roots.as<int32_t>(), n_roots, (int32_t)std::min<int64_t>(g->L.n + 1, 0x7fffffff), levels, parents,
                parents ? ~0ull : 0ull};
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
    if (g->autotune && !g->batch_tuned) {       // bfs_options.autotune: tune on the first batch's roots
        g->batch_tuned = true;
        BFS_TRY(bfs_batch_autotune(g, hroots, n_roots, levels, nullptr, nullptr, stream));
    }
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


// ===================================================================== server
// Continuous batching over resident graphs.  Every graph keeps up to 64 lanes
// of the bit-parallel search resident on the device; a server thread runs
// iterations (one BFS level of every running lane) on each graph's own stream,
// so the graphs' work overlaps on the GPU.  At every iteration boundary queued
// requests are admitted into free lanes (a lane admitted at iteration s reports
// level = iteration + 1 - s), and lanes whose frontier emptied are retired:
// their level row is copied to a result buffer and the request completes.
// Graphs are admitted against an HBM budget by their footprint (layout, lane
// state and level rows); results awaiting collection count against it too, and
// admission of new requests pauses while they would not fit.
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

namespace bfsgb {
namespace {

struct ServeGraph {
    bfs_graph* g = nullptr;
    int lanes = 0;
    cudaStream_t stream = nullptr;
    DevBuf levels;                   // [lanes][n]
    DevBuf parents;                  // [lanes][n]: the smallest previous-level neighbour
    DevBuf admit;                    // lanes[64], roots[64], want_parents[64]
    bool lane_parents[64] = {};      // the query running in lane r asked for parents
    int32_t* h_admit = nullptr;      // pinned staging of `admit`
    unsigned long long* h_alive = nullptr;   // pinned copy of the alive mask
    cudaGraphExec_t step = nullptr;  // expand, pieces, reduce, step end
    cudaGraph_t step_graph = nullptr;
    int64_t lane_ticket[64];
    unsigned long long running = 0;
    std::deque<int64_t> pending;
    int64_t footprint = 0;
    int64_t iterations = 0;
    bool inflight = false;           // an iteration is on the stream
    unsigned long long before = 0;   // lanes running in it
};

struct Request {
    int32_t graph = 0;
    int32_t root = 0;
    int state = 0;                   // 0 queued, 1 running, 2 done
    bool parents = false;            // submitted with BFS_QUERY_PARENTS
    std::chrono::steady_clock::time_point t_submit, t_done;
    int32_t* result = nullptr;       // device, once done: the level row (n), then the parent row (n) if asked
};

}  // namespace
}  // namespace bfsgb

struct bfs_server {
    int64_t budget = 0;
    int64_t used = 0;                // resident graphs
    int64_t results_bytes = 0;       // results awaiting collection
    int max_lanes = 64;
    std::vector<bfsgb::ServeGraph*> graphs;
    std::unordered_map<int64_t, bfsgb::Request> req;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    bool failed = false;
    char fail_msg[256] = {0};
    int64_t next_ticket = 1;
    int64_t queue_limit = 1 << 20;   // queued requests accepted before BFS_ERR_BUSY
    int64_t submitted = 0, completed = 0, rejected = 0, queued = 0;
    int64_t iterations = 0;
    int peak_lanes = 0;
    std::vector<double> lat_us;
    std::chrono::steady_clock::time_point t0;
    int device = 0;
};

namespace bfsgb {
namespace {

constexpr int64_t kMaxQueued = 1 << 20;      // default queue limit (bfs_server_set_queue_limit)

bfs_status build_step_graph(ServeGraph* sg) {
    MsContext* c = sg->g->ms;
    MsState* S = c->state.as<MsState>();
    const int sms = ms_sm_count();
    BFS_CUDA_TRY(cudaStreamBeginCapture(sg->stream, cudaStreamCaptureModeThreadLocal));
    ms_expand<<<sms * c->expand_ctas_per_sm, c->expand_threads, 0, sg->stream>>>(S);
    ms_pieces<<<sms * 4, kMT, 0, sg->stream>>>(S);
    ms_reduce<<<sms * 8, kMT, 0, sg->stream>>>(S);
    ms_step_end<<<1, 1, 0, sg->stream>>>(S);
    cudaGraph_t graph = nullptr;
    BFS_CUDA_TRY(cudaStreamEndCapture(sg->stream, &graph));
    cudaGraphExec_t exec = nullptr;
    cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) { cudaGraphDestroy(graph); return cuda_error(e, "cudaGraphInstantiate(step)", __FILE__, __LINE__); }
    sg->step_graph = graph;
    sg->step = exec;
    return BFS_OK;
}

void release_graph(ServeGraph* sg) {
    if (sg->stream) cudaStreamSynchronize(sg->stream);
    if (sg->step) cudaGraphExecDestroy(sg->step);
    if (sg->step_graph) cudaGraphDestroy(sg->step_graph);
    if (sg->h_admit) cudaFreeHost(sg->h_admit);
    if (sg->h_alive) cudaFreeHost(sg->h_alive);
    if (sg->stream) cudaStreamDestroy(sg->stream);
    sg->levels.release();
    sg->parents.release();
    sg->admit.release();
    if (sg->g) sg->g->busy.store(0);
}

void fail(bfs_server* s, const char* what) {
    std::lock_guard<std::mutex> lk(s->mu);
    s->failed = true;
    snprintf(s->fail_msg, sizeof(s->fail_msg), "%s", what);
    s->cv_done.notify_all();
}

// Every graph advances on its own: when its iteration has finished (a stream
// query, no waiting on the other graphs) its lanes whose frontier emptied are
// retired, queued requests are admitted into free lanes, and the next
// iteration is launched.  Returns whether any graph made progress.
bool finish_iteration(bfs_server* s, ServeGraph* sg) {
    if (sg->h_alive[2]) {
        char msg[160];
        snprintf(msg, sizeof(msg), "bounds check %llu failed on the device (%llu, %llu)",
                 (unsigned long long)sg->h_alive[2], (unsigned long long)sg->h_alive[3],
                 (unsigned long long)sg->h_alive[4]);
        fail(s, msg);
        return false;
    }
    const unsigned long long done = sg->before & ~sg->h_alive[0];
    const int64_t n = sg->g->L.n;
    std::vector<std::pair<int64_t, int32_t*>> fin;
    for (int r = 0; r < sg->lanes; ++r) {
        if (!(done & (1ull << r))) continue;
        void* buf = nullptr;
        const int rows = sg->lane_parents[r] ? 2 : 1;
        if (cudaMallocAsync(&buf, rows * sizeof(int32_t) * n, sg->stream) != cudaSuccess) { fail(s, "result allocation failed"); return false; }
        cudaMemcpyAsync(buf, sg->levels.as<int32_t>() + (int64_t)r * n, sizeof(int32_t) * n,
                        cudaMemcpyDeviceToDevice, sg->stream);
        if (rows == 2)
            cudaMemcpyAsync(static_cast<int32_t*>(buf) + n, sg->parents.as<int32_t>() + (int64_t)r * n,
                            sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, sg->stream);
        fin.push_back({sg->lane_ticket[r], static_cast<int32_t*>(buf)});
        sg->lane_ticket[r] = -1;
    }
    if (!fin.empty() && cudaStreamSynchronize(sg->stream) != cudaSuccess) { fail(s, "result copy failed"); return false; }
    std::lock_guard<std::mutex> lk(s->mu);
    sg->running &= ~done;
    ++sg->iterations;
    ++s->iterations;
    const auto now = std::chrono::steady_clock::now();
    for (auto& f : fin) {
        Request& q = s->req[f.first];
        q.state = 2;
        q.result = f.second;
        q.t_done = now;
        s->results_bytes += (q.parents ? 2 : 1) * sizeof(int32_t) * n;
        ++s->completed;
        s->lat_us.push_back(std::chrono::duration<double, std::micro>(now - q.t_submit).count());
    }
    if (!fin.empty()) s->cv_done.notify_all();
    return true;
}

bool launch_iteration(bfs_server* s, ServeGraph* sg) {
    std::unique_lock<std::mutex> lk(s->mu);
    // admission into free lanes, while the results would fit in the budget
    int nadm = 0;
    unsigned long long mask = 0;
    for (int r = 0; r < sg->lanes && !sg->pending.empty(); ++r) {
        if (sg->running & (1ull << r)) continue;
        // the result of a lane: its level row (and parent row)
        const int64_t row = (s->req[sg->pending.front()].parents ? 8 : 4) * sg->g->L.n;
        if (s->used + s->results_bytes + row > s->budget) break;     // wait for results to be collected
        const int64_t t = sg->pending.front();
        sg->pending.pop_front();
        --s->queued;
        Request& q = s->req[t];
        q.state = 1;
        sg->lane_ticket[r] = t;
        sg->running |= 1ull << r;
        sg->h_admit[nadm] = r;
        sg->h_admit[64 + nadm] = q.root;
        sg->h_admit[128 + nadm] = q.parents ? 1 : 0;
        sg->lane_parents[r] = q.parents;
        mask |= 1ull << r;
        ++nadm;
    }
    if (!sg->running) return false;
    MsState* S = sg->g->ms->state.as<MsState>();
    if (nadm) {
        int32_t* d = sg->admit.as<int32_t>();
        if (cudaMemcpyAsync(d, sg->h_admit, sizeof(int32_t) * 192, cudaMemcpyHostToDevice, sg->stream) != cudaSuccess) {
            lk.unlock(); fail(s, "admission copy failed"); return false;
        }
        ms_admit_clear<<<ms_sm_count() * 4, kMT, 0, sg->stream>>>(S, mask, d, nadm);
        ms_admit_roots<<<1, 64, 0, sg->stream>>>(S, d, d + 64, d + 128, nadm);
    } else {
        ms_clear_alive<<<1, 1, 0, sg->stream>>>(S);
    }
    if (cudaGraphLaunch(sg->step, sg->stream) != cudaSuccess) {
        lk.unlock(); fail(s, "iteration launch failed"); return false;
    }
    cudaMemcpyAsync(sg->h_alive, reinterpret_cast<char*>(S) + offsetof(MsState, alive),
                    sizeof(unsigned long long) * 5, cudaMemcpyDeviceToHost, sg->stream);   // alive, nnz, err, a, b
    sg->before = sg->running;
    sg->inflight = true;
    int lanes_now = 0;
    for (ServeGraph* x : s->graphs) lanes_now += __builtin_popcountll(x->running);
    if (lanes_now > s->peak_lanes) s->peak_lanes = lanes_now;
    return true;
}

bool serve_pass(bfs_server* s) {
    std::vector<ServeGraph*> gs;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        gs = s->graphs;
    }
    bool progressed = false;
    for (ServeGraph* sg : gs) {
        if (sg->inflight) {
            const cudaError_t q = cudaStreamQuery(sg->stream);
            if (q == cudaErrorNotReady) continue;
            sg->inflight = false;
            if (q != cudaSuccess) { fail(s, "iteration failed on the device"); return false; }
            if (!finish_iteration(s, sg)) return false;
            progressed = true;
        }
        if (launch_iteration(s, sg)) progressed = true;
        {
            std::lock_guard<std::mutex> lk(s->mu);
            if (s->failed) return false;
        }
    }
    return progressed;
}

void serve_loop(bfs_server* s) {
    cudaSetDevice(s->device);
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop || s->failed) break;
            bool work = false;
            for (ServeGraph* sg : s->graphs) work |= sg->inflight || (sg->running != 0) || !sg->pending.empty();
            if (!work) s->cv_work.wait_for(lk, std::chrono::milliseconds(1));
            if (s->stop) break;
        }
        if (!serve_pass(s)) {            // iterations in flight and nothing finished yet
            std::unique_lock<std::mutex> lk(s->mu);
            if (s->stop || s->failed) break;
            s->cv_work.wait_for(lk, std::chrono::microseconds(20));
        }
    }
    // leave no iteration in flight
    std::vector<ServeGraph*> gs;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        gs = s->graphs;
    }
    for (ServeGraph* sg : gs)
        if (sg->inflight) { cudaStreamSynchronize(sg->stream); sg->inflight = false; }
}

}  // namespace
}  // namespace bfsgb

extern "C" {

bfs_status bfs_server_create(int64_t hbm_budget_bytes, int32_t max_lanes, bfs_server_t* out) {
    if (!out || hbm_budget_bytes <= 0 || max_lanes < 1 || max_lanes > 64)
        return set_error(BFS_ERR_INVALID_ARG, "bad server arguments (budget > 0, 1 <= max_lanes <= 64)");
    bfs_server* s = new (std::nothrow) bfs_server();
    if (!s) return set_error(BFS_ERR_OUT_OF_MEMORY, "host allocation");
    s->budget = hbm_budget_bytes;
    s->max_lanes = max_lanes;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    s->worker = std::thread(serve_loop, s);
    *out = s;
    return BFS_OK;
}

bfs_status bfs_server_add_graph(bfs_server_t s, bfs_graph_t g, int32_t* graph_id) {
    if (!s || !g || !graph_id) return set_error(BFS_ERR_INVALID_ARG, "NULL argument");
    int expect = 0;
    if (!g->busy.compare_exchange_strong(expect, 1)) return set_error(BFS_ERR_BUSY, "graph is in use");
    ServeGraph* sg = new (std::nothrow) ServeGraph();
    if (!sg) { g->busy.store(0); return set_error(BFS_ERR_OUT_OF_MEMORY, "host allocation"); }
    sg->g = g;
    for (auto& t : sg->lane_ticket) t = -1;
    const int64_t n = g->L.n;
    int64_t layout = 0;
    bfs_graph_footprint(g, &layout);
    const int64_t lane_state = 32 * n + 8 * n + (int64_t)sizeof(Item) * (g->L.nnz / kMsPiece + g->L.nnz / kMsHub + 16);
    int lanes = s->max_lanes;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        while (lanes > 0 && s->used + layout + lane_state + 8 * n * (int64_t)lanes > s->budget) lanes /= 2;
    }
    if (lanes == 0) {
        delete sg;
        g->busy.store(0);
        return set_error(BFS_ERR_OUT_OF_MEMORY, "graph does not fit the server's HBM budget");
    }
    sg->lanes = lanes;
    sg->footprint = layout + lane_state + 8 * n * (int64_t)lanes;
    bfs_status rc = ms_ensure(g);
    if (rc == BFS_OK) rc = sg->levels.alloc(sizeof(int32_t) * n * lanes);
    if (rc == BFS_OK) rc = sg->parents.alloc(sizeof(int32_t) * n * lanes);
    if (rc == BFS_OK) rc = sg->admit.alloc(sizeof(int32_t) * 192);
    if (rc == BFS_OK && cudaMallocHost(reinterpret_cast<void**>(&sg->h_admit), sizeof(int32_t) * 192) != cudaSuccess)
        rc = set_error(BFS_ERR_OUT_OF_MEMORY, "pinned host allocation");
    if (rc == BFS_OK && cudaMallocHost(reinterpret_cast<void**>(&sg->h_alive), sizeof(unsigned long long) * 5) != cudaSuccess)
        rc = set_error(BFS_ERR_OUT_OF_MEMORY, "pinned host allocation");
    if (rc == BFS_OK && cudaStreamCreateWithFlags(&sg->stream, cudaStreamNonBlocking) != cudaSuccess)
        rc = set_error(BFS_ERR_CUDA, "stream creation failed");
    if (rc == BFS_OK) {
        MsState* S = g->ms->state.as<MsState>();
        MsCall call{g->ms->roots.as<int32_t>(), lanes, 0x7fffffff, sg->levels.as<int32_t>(), sg->parents.as<int32_t>(),
                    0ull};
        if (cudaMemcpyAsync(reinterpret_cast<char*>(S) + offsetof(MsState, roots), &call, sizeof(call),
                            cudaMemcpyHostToDevice, sg->stream) != cudaSuccess)
            rc = set_error(BFS_ERR_CUDA, "state copy failed");
        if (rc == BFS_OK) {
            ms_reset<<<1, 1, 0, sg->stream>>>(S);
            ms_clear<<<ms_sm_count() * 8, kMT, 0, sg->stream>>>(S);
            if (cudaStreamSynchronize(sg->stream) != cudaSuccess) rc = set_error(BFS_ERR_CUDA, "lane state initialisation failed");
        }
    }
    if (rc == BFS_OK) rc = build_step_graph(sg);
    if (rc != BFS_OK) {
        release_graph(sg);
        delete sg;
        return rc;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    s->used += sg->footprint;
    s->graphs.push_back(sg);
    *graph_id = (int32_t)s->graphs.size() - 1;
    return BFS_OK;
}

bfs_status bfs_server_submit(bfs_server_t s, int32_t graph_id, int32_t root, int64_t* ticket) {
    return bfs_server_submit_ex(s, graph_id, root, 0, ticket);
}

bfs_status bfs_server_submit_ex(bfs_server_t s, int32_t graph_id, int32_t root, int32_t flags, int64_t* ticket) {
    if (!s || !ticket) return set_error(BFS_ERR_INVALID_ARG, "NULL argument");
    if (flags & ~BFS_QUERY_PARENTS) return set_error(BFS_ERR_INVALID_ARG, "unknown query flags 0x%x", flags);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed) return set_error(BFS_ERR_CUDA, "server failed: %s", s->fail_msg);
    if (graph_id < 0 || graph_id >= (int32_t)s->graphs.size()) return set_error(BFS_ERR_NOT_FOUND, "unknown graph id %d", graph_id);
    ServeGraph* sg = s->graphs[graph_id];
    if (root < 0 || (int64_t)root >= sg->g->L.n) return set_error(BFS_ERR_INVALID_ARG, "root %d outside [0, %lld)", root, (long long)sg->g->L.n);
    if (s->queued >= s->queue_limit) { ++s->rejected; return set_error(BFS_ERR_BUSY, "server queue is full"); }
    const int64_t t = s->next_ticket++;
    Request q;
    q.graph = graph_id;
    q.root = root;
    q.parents = (flags & BFS_QUERY_PARENTS) != 0;
    q.t_submit = std::chrono::steady_clock::now();
    s->req.emplace(t, q);
    sg->pending.push_back(t);
    ++s->queued;
    ++s->submitted;
    *ticket = t;
    s->cv_work.notify_one();
    return BFS_OK;
}

bfs_status bfs_server_set_queue_limit(bfs_server_t s, int64_t limit) {
    if (!s || limit < 1 || limit > kMaxQueued)
        return set_error(BFS_ERR_INVALID_ARG, "queue limit outside [1, %lld]", (long long)kMaxQueued);
    std::lock_guard<std::mutex> lk(s->mu);
    s->queue_limit = limit;
    return BFS_OK;
}

bfs_status bfs_server_poll(bfs_server_t s, int64_t ticket, int32_t* done) {
    if (!s || !done) return set_error(BFS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->req.find(ticket);
    if (it == s->req.end()) return set_error(BFS_ERR_NOT_FOUND, "unknown ticket %lld", (long long)ticket);
    *done = it->second.state == 2;
    return BFS_OK;
}

bfs_status bfs_server_wait(bfs_server_t s, int64_t ticket, int64_t timeout_us, int32_t* level, int32_t* parent) {
    if (!s) return set_error(BFS_ERR_INVALID_ARG, "NULL server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->req.find(ticket);
    if (it == s->req.end()) return set_error(BFS_ERR_NOT_FOUND, "unknown ticket %lld", (long long)ticket);
    if (parent && !it->second.parents)
        return set_error(BFS_ERR_INVALID_ARG, "request %lld was submitted without BFS_QUERY_PARENTS", (long long)ticket);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us < 0 ? 0 : timeout_us);
    while (s->req[ticket].state != 2 && !s->failed) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && s->req[ticket].state != 2)
            return set_error(BFS_ERR_TIMEOUT, "request %lld not finished", (long long)ticket);
    }
    if (s->failed) return set_error(BFS_ERR_CUDA, "server failed: %s", s->fail_msg);
    Request q = s->req[ticket];
    s->req.erase(ticket);
    ServeGraph* sg = s->graphs[q.graph];
    const int64_t n = sg->g->L.n;
    s->results_bytes -= (q.parents ? 2 : 1) * sizeof(int32_t) * n;
    lk.unlock();
    bfs_status rc = BFS_OK;
    // the result was allocated stream-ordered and completed before the request
    // was marked done: copy it out and free it stream-ordered on the legacy stream
    if (level) {
        cudaError_t e = cudaMemcpyAsync(level, q.result, sizeof(int32_t) * n, cudaMemcpyDefault, 0);
        if (e != cudaSuccess) rc = cuda_error(e, "result copy", __FILE__, __LINE__);
    }
    if (parent && rc == BFS_OK) {
        cudaError_t e = cudaMemcpyAsync(parent, q.result + n, sizeof(int32_t) * n, cudaMemcpyDefault, 0);
        if (e != cudaSuccess) rc = cuda_error(e, "result copy", __FILE__, __LINE__);
    }
    cudaFreeAsync(q.result, 0);
    cudaError_t e = cudaStreamSynchronize(0);
    if (rc == BFS_OK && e != cudaSuccess) rc = cuda_error(e, "result copy", __FILE__, __LINE__);
    s->cv_work.notify_one();
    return rc;
}

bfs_status bfs_server_stats(bfs_server_t s, bfs_server_stats_t* st) {
    if (!s || !st) return set_error(BFS_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    memset(st, 0, sizeof(*st));
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->queued = s->queued;
    st->iterations = s->iterations;
    st->peak_lanes = s->peak_lanes;
    st->graphs = (int32_t)s->graphs.size();
    st->hbm_used_bytes = s->used + s->results_bytes;
    std::vector<double> v = s->lat_us;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
        st->p50_us = pct(0.50);
        st->p99_us = pct(0.99);
        st->max_us = v.back();
    }
    return BFS_OK;
}

bfs_status bfs_server_destroy(bfs_server_t s) {
    if (!s) return BFS_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& kv : s->req)
        if (kv.second.result) cudaFreeAsync(kv.second.result, 0);
    cudaStreamSynchronize(0);
    for (ServeGraph* sg : s->graphs) {
        release_graph(sg);
        delete sg;
    }
    delete s;
    return BFS_OK;
}

}  // extern "C"
