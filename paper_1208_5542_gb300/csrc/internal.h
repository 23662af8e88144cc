// internal.h -- host-side structures shared by the translation units of
// libbfs_gb300 (graph layout, search workspace, error reporting, launchers).
#pragma once

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "bfs_gb300.h"

struct bfs_graph;

namespace bfsgb {

// ---------------------------------------------------------------- errors --
bfs_status set_error(bfs_status s, const char* fmt, ...);
bfs_status cuda_error(cudaError_t e, const char* what, const char* file, int line);

#define BFS_CUDA_TRY(expr)                                                        \
    do {                                                                          \
        cudaError_t e__ = (expr);                                                 \
        if (e__ != cudaSuccess) return ::bfsgb::cuda_error(e__, #expr, __FILE__, __LINE__); \
    } while (0)

#define BFS_TRY(expr)                                                             \
    do {                                                                          \
        bfs_status s__ = (expr);                                                  \
        if (s__ != BFS_OK) return s__;                                            \
    } while (0)

// Kind of pointer the caller handed over.
bool is_device_pointer(const void* p);

// ---------------------------------------------------------- device arrays --
// Owning device buffer (cudaMalloc / cudaFree).
struct DevBuf {
    void* ptr = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { release(); }
    bfs_status alloc(size_t nbytes);
    void release();
    template <typename T> T* as() const { return static_cast<T*>(ptr); }
};

// ------------------------------------------------------------ the layout --
// Blocks b = i*p + j: block-row i = destinations in range i, block column j =
// sources in range j.  Per block: directory V_{i,j} (range_len(j) bits, padded
// to dir_stride uint32 words), rank[w] = set directory bits before word w,
// cp = nnzc_b + 1 block-local offsets into the block's part of ir, ir = global
// destination ids, block after block, column after column.
struct Layout {
    int64_t n = 0;          // vertices
    int p = 1;              // grid p x p
    int64_t nb = 0;         // range size ceil(n/p)
    int64_t nnz = 0;        // directed entries
    int64_t dir_stride = 0; // uint32 words per block directory (padded)
    int64_t nnzc_total = 0; // nonempty columns over all blocks
    DevBuf dir, rank, cp, ir, cp_base_d, ir_base_d;
    DevBuf deg;             // entries per source vertex (uint32, saturated), computed for bottom-up levels
    DevBuf iso;             // bitmap of the vertices without entries (bottom-up levels mark them visited)
    DevBuf bu_ptr, bu_adj;  // bottom-up levels: the columns of v in blocks (0,i) .. (p-1,i) back to back
                            // (int64 offsets n+1, int32 ids), grouped by range in ascending order
    std::vector<int64_t> cp_base, ir_base, nnzc, nnz_b;   // host copies, p*p
    int64_t range_begin(int b) const { int64_t x = (int64_t)b * nb; return x < n ? x : n; }
    int64_t range_len(int b) const { return range_begin(b + 1) - range_begin(b); }
};

// Work item of the expansion: source u with its column of one block.
struct __align__(16) Item {
    int32_t u;
    uint32_t len;
    int64_t begin;
};

// Device counters of one search (uint64 slots).
enum Counter : int {
    C_NEXT_COUNT = 0,    // vertices in the next frontier
    C_UNITS,             // work units of the expansion (WAH chunks)
    C_ITEMS,             // decoded (vertex, block) items
    C_HITS,              // items with a nonempty column
    C_EDGES,             // adjacency entries scanned
    C_ERROR,             // nonzero: an invariant failed (code)
    C_TRACE_USED,        // uint32 elements of the trace written so far
    C_ROW_TRACE_USED,    // uint32 elements of the row-buffer trace written so far
    C_WAH_WORDS,         // words of all streams of this level
    C_EXCHANGED,         // set bits carried by the exchange
    C_PIECES,            // pieces of long columns queued for the piece kernel
    C_ROW_WORDS,         // WAH words of the compressed row exchange
    C_NEXT_DEGREE,       // degree sum of the next frontier (direction choice)
    C_BOTTOM_UP,         // 1: this level ran bottom-up
    C_ENC_CHUNKS,        // chunks read by the column encoder (statistics only)
    C_ROW_CHUNKS,        // chunks read by the row encoder (statistics only)
    C_NUM
};

// The level loop of one search configuration as an instantiated CUDA graph
// (a conditional WHILE node around one level).
struct SearchGraph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int mode = -1, wbits = 0, rowx = 0, bottom_up = 0, adaptive = 0, dynamic = 0;
    int32_t* parent = nullptr;
    int32_t* level = nullptr;
};

// Per-search workspace (owned by the graph, reused by every search).
struct Workspace {
    int64_t bm_words = 0;       // uint32 words of an n-bit bitmap (padded)
    int64_t fsum_len = 0;       // bytes of the frontier summary (1 per 1024 bits)
    int64_t slot_cap = 0;       // words (of the WAH width) per exchange slot
    int64_t chunk_words = 0;    // words per expansion chunk of a stream
    int64_t chunks_per_slot = 0;
    int slots = 0;              // exchange slots of the current mode
    int wah_bits = 0;
    int mode = -1;
    DevBuf pi, fa, fb, fsum, xbuf, xcount, chunk_base, units, counters, pieces;
    DevBuf level_scratch;       // per-level work counters (3 per row)
    DevBuf row_meta;            // per-row piece bases and capacities
    int64_t piece_cap = 0;      // capacity of `pieces` (Item entries)
    int64_t win_words = 0;      // shared-memory row window of the expansion (0: none)
    DevBuf tblk;                // row exchange: per-block partial next bitmaps t_{i,j} (dir layout)
    DevBuf rowbuf, rowcount, rowfirst;   // row exchange: row buffers, their word counts, chunk index
    DevBuf rowlive;             // row exchange: 1 for a block whose column stream carried a vertex
    bool tblk_dirty = false;    // a search stopped mid-level: clear the partials before the next one
    DevBuf enc_sums, enc_bases;  // chunk summaries of the parallel encoder
    DevBuf enc_flags;            // chunks with frontier bits
    DevBuf enc_done;             // slots finished by the encoder's scan
    DevBuf ctl;                  // the level values kept on the device
    DevBuf gbits;                // exchanged streams decoded into one bitmap (bottom-up levels)
    DevBuf colfirst;             // the column encoder's per-chunk first words (bottom-up decode)
    DevBuf xfmt;                 // per-slot format of the level-adaptive exchange
    DevBuf ddir;                 // dynamic cross directory: the search's copy D_{i,j} of the directories
    SearchGraph sgraph[2];       // level loops as CUDA graphs, most recent configurations
    int sgraph_next = 0;
    int64_t enc_cps = 0;         // encoder chunks per slot
    int64_t row_cap = 0;        // words (of the WAH width) per row buffer
    DevBuf tmp_parent, tmp_level;      // for searches with host outputs
    uint64_t* h_counters = nullptr;    // pinned mirror of the counters
    cudaEvent_t ev[8] = {};
    bool events = false;
};

struct MsContext;    // batched search state (msbfs.cu)
void free_msbfs(bfs_graph* g);

}  // namespace bfsgb

struct bfs_graph {
    bfsgb::Layout L;
    bfsgb::Workspace W;
    int mode = BFS_MODE_COMPRESS_SIEVE;
    int wah_bits = 32;
    int debug_checks = 0;        // 1: bfs_run checks its outputs (bfs_check_search) before returning
    int autotune = 0;            // 1: the first bfs_run_batch picks the batch launch shape
    bool batch_tuned = false;
    int row_exchange = 0;
    int adaptive = 0;            // level-adaptive exchange format (bfs_graph_set_exchange_format)
    int dynamic_dir = 0;         // dynamic cross directory (bfs_graph_set_dynamic_directory)
    int symmetric = 0;           // built with symmetrize = 1: in-neighbours = out-neighbours
    int direction = BFS_DIRECTION_TOP_DOWN;
    int alpha = 14, beta = 24;   // switch thresholds of the hybrid
    int device = 0;
    std::atomic<int> busy{0};
    std::mutex mu;
    bfsgb::MsContext* ms = nullptr;
};

namespace bfsgb {

// graph_build.cu
bfs_status build_layout(bfs_graph* g, int64_t n, int64_t m, const int32_t* d_src,
                        const int32_t* d_dst, int symmetrize, cudaStream_t st);
bfs_status ensure_workspace(bfs_graph* g, cudaStream_t st);
bfs_status ensure_degrees(bfs_graph* g, cudaStream_t st);
void free_workspace(bfs_graph* g);

// wah.cu
struct EncodeArgs {
    const uint32_t* frontier;   // bitmap read by the encoder
    int64_t frontier_words;     // its readable words (a multiple of 4)
    const uint32_t* dir;        // directories (sieve) or nullptr
    int64_t dir_stride;
    int p;
    int64_t nb, n;
    int sieve;                  // 1: slot s = i*p + j sieved by V_{i,j}; 0: slot = j
    int nslots;
    const uint8_t* fsum;        // frontier summary or nullptr
    void* out;
    int64_t slot_cap;
    int64_t* counts;
    int64_t* unit_base;         // or nullptr: group start of every word 32k of slot s at [s * unit_stride + k]
    int64_t unit_stride;
    unsigned long long* wah_words;   // or nullptr: words of all slots are added here
    int64_t* plan_base;         // or nullptr: the decoder's units per block, p*p + 1 entries
    unsigned long long* plan_units;  // their total
    unsigned int* plan_done;    // slots finished (zero between uses)
    // the row exchange of the fold (slot s = i*p + j carries range i, not j):
    int row_slots;              // 1: slot s covers range s / p; the bitmap read at its range is
                                //    `frontier`, combined as ~frontier & dir (with invert_frontier)
    int invert_frontier;        // 1: the frontier operand enters complemented (the sieve by not(pi))
    uint32_t* dir_clear;        // or nullptr: the directory operand, zeroed as the passes consume it
    int64_t* chunk_first;       // or nullptr: per (slot, chunk) the word holding the chunk's first
                                //   group and that word's first group, 2 entries
    const int32_t* skip;        // or nullptr: the passes do nothing while *skip != 0 (the counts
                                //   are set to 0)
    unsigned long long* live_chunks;   // or nullptr: chunks the passes read are counted here
    int adaptive;               // 1: each slot goes as the smallest of WAH stream, sparse vector of
                                //    set-bit offsets and raw bitmap (32-bit words only); the scan
                                //    writes the choice to fmt[s] and counts[s] = its elements
    uint8_t* fmt;               // per-slot format (SliceFormat), with adaptive
    uint8_t* slot_bits;         // or nullptr: the scan writes 1 for a slot whose stream carries a set bit
    const uint8_t* slot_live;   // or nullptr: a slot with slot_live[s] == 0 is all zero (not read)
};
bfs_status launch_wah_encode(const EncodeArgs& a, int wah_bits, cudaStream_t st);

struct DecodeArgs {             // standalone decode into a bitmap
    const void* words;
    int64_t nwords;
    int64_t nbits;
    uint32_t* bits;
    unsigned long long* err;
};
bfs_status launch_wah_decode_bitmap(const DecodeArgs& a, int wah_bits, cudaStream_t st);

}  // namespace bfsgb
