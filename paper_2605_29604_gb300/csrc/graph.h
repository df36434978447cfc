// graph.h -- the library's graph handle and host-side helpers (host code only).
#pragma once

#include <atomic>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "internal.h"
#include "tcmis.h"

namespace tcmis {

// Records code + message for the calling thread and returns the code.
int set_error(int code, const std::string& msg);
int set_cuda_error(cudaError_t e, const char* what);
void clear_error();

// Device buffers of one solve in flight: vertex words, worklists, the in-set
// bits and row-block lists of the tile kernels, the control block, phase
// timestamps, seeds (one per graph of a batch) and the result bytes.
struct Workspace {
    int64_t cap = 0;       // vertices held (a multiple of 16)
    int32_t seed_cap = 0;  // seeds held
    uint32_t* word = nullptr;
    int4* wl0 = nullptr;  // worklists of row records
    int4* wl1 = nullptr;
    int4* wlp = nullptr;
    uint32_t* inbits = nullptr;
    int32_t* rbl0 = nullptr;
    int32_t* rbl1 = nullptr;
    Ctl* ctl = nullptr;
    PhaseTimes* times = nullptr;
    uint64_t* seeds = nullptr;
    uint8_t* out = nullptr;
    int64_t bytes = 0;
};

// Allocate a workspace for graphs of up to n vertices and `count` seeds
// (frees and reallocates when it is too small); returns the CUDA error.
cudaError_t ws_reserve(Workspace& w, int64_t n, int32_t count);
void ws_free(Workspace& w);
int64_t ws_bytes_for(int64_t n, int32_t count);

// Device buffers of one graph (or one block-diagonal union of graphs) plus
// the workspace of the handle's own solves.
struct GraphData {
    int device = 0;
    int32_t n = 0;          // vertices (union size, padding included)
    int64_t arcs = 0;       // stored arcs
    int32_t* rp = nullptr;  // n + 1
    int32_t* col = nullptr; // arcs, padded to a multiple of 4 plus 4
    // batch segments (count == 0 for a single graph)
    int32_t count = 0;
    int32_t* blk_seg = nullptr;
    int32_t* voff = nullptr;
    int32_t* nv = nullptr;
    int32_t* garcs = nullptr;
    int64_t* roff = nullptr;
    uint64_t* seeds_host = nullptr;  // pinned staging, count entries
    std::vector<int32_t> h_nv;       // per graph vertices (host copy)
    int64_t result_bytes = 0;        // sum of the graphs' n
    // tile-CSR (built on demand)
    TileCsr tiles;
    int64_t tile_footprint = 0;
    // stored payload of the 16 x 16 tiles for a tensor-core form that reads
    // one (int8 or fp16, built on first use; kind -1 = none)
    void* tpay = nullptr;
    int32_t tpay_kind = -1;
    // multi-seed solves on the tiles: one in-set bit vector per solve
    uint32_t* inb8 = nullptr;
    // degree-ordered rows and degree bins of the CSR kernel
    int32_t* col_sel = nullptr;
    int32_t* split = nullptr;
    int4* order0 = nullptr;       // round-0 row records grouped by bin
    uint8_t* r0class = nullptr;   // round-0 classes (with a degree-ordered adjacency)
    int32_t* sure_out = nullptr;  // sure round-0 exclusions
    uint32_t* word8 = nullptr;    // multi-seed solves: 8 words per vertex (lazily)
    int32_t* s0_rp = nullptr;     // the tested subgraph (when it is small)
    int32_t* s0_col = nullptr;
    int32_t* s0_pre = nullptr;
    int4* order0_s0 = nullptr;
    int64_t s0_bytes = 0;
    int64_t s0_arcs = 0;
    int2* keyed = nullptr;        // vertices whose words a solve reads (with s0_col)
    uint8_t* out0 = nullptr;      // result bytes decided at create time
    int32_t n_keyed = 0;
    int32_t n_tested = 0;             // vertices of the tested subgraph
    int32_t* dyn_mark = nullptr;      // mis_repair: pass stamp of each vertex (lazily)
    int* dyn_cnt = nullptr;           // mis_repair: list counters
    int32_t dyn_stamp = 0;            // mis_repair: last pass stamp issued
    int64_t tested_prefix_arcs = 0;   // arcs of their selection prefixes
    int32_t n_sure_in = 0;
    int32_t n_sure_out = 0;
    int32_t bin_off[6] = {0, 0, 0, 0, 0, 0};
    int32_t n_isolated = 0;
    int32_t thr[4] = {0, 0, 0, 0};
    unsigned* flags = nullptr;
    // workspace of the handle's own solves (mis_solve / mis_solve_ex)
    Workspace ws;
    Ctl* ctl_host = nullptr;           // pinned
    PhaseTimes* times_host = nullptr;  // pinned
    int64_t footprint = 0;
};

}  // namespace tcmis

struct mis_graph {
    tcmis::GraphData d;
    mis_options opt{};
    int32_t path = MIS_PATH_CSR;  // resolved path
    int32_t tpr = 0;              // forced lanes per row (0 = degree bins)
    int32_t grid = 0;             // persistent grid size (CSR kernel)
    int32_t tile_grid = 0;        // persistent grid size (tile kernels)
    int32_t tile_slots = 8;       // tile kernels: lanes (tiles in flight) per row block
    int32_t csr_pending = 0;      // CSR kernel: Phase 1 lists non-candidates for Phase 2
    int32_t tile_payload = 0;     // tensor-core tile path: payload form (MIS_TILE_*)
    tcmis::ClusterPlan cluster;   // cluster path: its launch shape
    int32_t csr_range0 = 1;       // CSR kernel: round 0 tests bin 0 by vertex ranges
    int32_t multi_form = 0;       // multi-seed solves off the tile path (MIS_MULTI_*)
    int32_t multi_tc_fill = 32;   // MIS_MULTI_ROWS_TC: Phase 2 on tensor cores while at
                                  // least multi_tc_fill / 256 of the listed entries are undecided
                                  // (graphs without round-0 classes only)
    cudaStream_t own_stream = nullptr;
    cudaStream_t last_stream = nullptr;
    int32_t last_path = 0;
    std::mutex mu;
    std::atomic<int> inflight{0};       // served requests not yet finished
    std::atomic<bool> destroy_pending{false};
    std::atomic<int> replays{0};        // live captured solves (they hold device pointers)
};

// A captured solve (mis_capture): an executable CUDA graph of one solve.
struct mis_replay {
    mis_graph* g = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    uint64_t* seeds_pinned = nullptr;  // the captured seeds, read by every replay
    int32_t path = 0;                  // round kernel captured
    bool counted = false;              // counted in g->replays
};

namespace tcmis {

// api.cu
int solve_async(mis_graph* g, const uint64_t* seeds, uint8_t* out_dev, cudaStream_t s);
// One solve of g on stream s in workspace w; seeds (host, one per graph of
// the handle) are staged through `seeds_pinned`.  blocks: 0 = the graph's own
// persistent grid; 1 = the round kernel as one block through an ordinary
// launch (a lone block needs no co-scheduling); > 1 = a cooperative grid of
// at most that many blocks.
int solve_in(mis_graph* g, Workspace& w, const uint64_t* seeds, uint64_t* seeds_pinned,
             uint8_t* out_dev, cudaStream_t s, int blocks);
// k multi-seed solves of single graph g on stream s in workspace w (word8:
// kMaxMulti words per vertex; out_dev: k * n bytes); blocks as for solve_in.
int solve_multi_in(mis_graph* g, Workspace& w, uint32_t* word8, int k, const uint64_t* seeds,
                   uint8_t* out_dev, cudaStream_t s, int blocks);
void free_graph(mis_graph* g);

int autotune(mis_graph* g, int reps, mis_tuning* out);

// serve.cu
void serve_release_graph(mis_graph* g);

}  // namespace tcmis
