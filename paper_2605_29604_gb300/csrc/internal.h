// internal.h -- host-side declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tcmis {

struct Ctl;
struct PhaseTimes;

// Per-graph parameters of Eq. 1 for a block-diagonal union (count == 0: one
// graph, seed in `seed0`, average degree from row_ptr[n] / n).
struct SegTable {
    int32_t count = 0;
    const int32_t* blk_seg = nullptr;  // per 16-vertex block of the union: graph index
    const int32_t* voff = nullptr;     // per graph: first vertex in the union
    const int32_t* nv = nullptr;       // per graph: vertices
    const int32_t* arcs = nullptr;     // per graph: arcs (its own row_ptr[n])
    const int64_t* roff = nullptr;     // per graph: first byte of its result
    const uint64_t* seed = nullptr;    // per graph: seed
};

// Solves of one graph in one multi-seed launch (kernels_multi.cu): at most
// kMaxMulti, one seed each.
constexpr int kMaxMulti = 8;
struct MultiSeeds {
    uint64_t seed[kMaxMulti];
};

// Everything one persistent solve launch needs.
struct SolveArgs {
    const int32_t* rp = nullptr;   // row_ptr, n+1
    const int32_t* col = nullptr;  // col_idx, padded by >= 4 entries
    int32_t n = 0;                 // vertices (of the union for a batch)
    uint32_t* word = nullptr;      // packed per-vertex state, n
    // Worklists hold row records {v, row begin, end of the selection prefix,
    // row end} (int4), so that a scan needs no row_ptr lookup.
    int4* wl0 = nullptr;           // worklists, n each
    int4* wl1 = nullptr;
    int4* wlp = nullptr;           // pending list of Phase 2 (non-candidates), n
    Ctl* ctl = nullptr;            // control block (zeroed before launch)
    PhaseTimes* times = nullptr;   // phase timestamps (nullable)
    uint8_t* out = nullptr;        // result bytes (device), nullable
    SegTable seg;                  // batch segments
    uint64_t seed0 = 0;            // single-graph seed
    long long spin_cap = 0;        // barrier poll limit
    int32_t max_rounds = 0;        // round cap (error beyond)
    // degree bins of the CSR kernel
    const int32_t* col_sel = nullptr; // rows sorted by neighbour degree (padded like col)
    const int32_t* split = nullptr;   // neighbours of degree <= deg(v) + 1 (nullable)
    const int4* order0 = nullptr;     // round-0 records: real non-isolated vertices by bin
    int32_t bin_off[6] = {0, 0, 0, 0, 0, 0};  // bin j occupies [bin_off[j], bin_off[j+1])
    int32_t n_isolated = 0;           // real vertices of degree 0 (not in order0)
    // Round-0 decisions known at create time (see build_round0_classes):
    // r0class[v] = 1 marks a sure round-0 candidate (written in the MIS at
    // init), sure_out lists the sure round-0 exclusions (written out in
    // round 0's Phase 2); neither is in order0.  Null / 0 when unused.
    const uint8_t* r0class = nullptr;
    const int32_t* sure_out = nullptr;
    // The adjacency of every scan but round 0's selection test: the tested
    // subgraph's rows where the graph has one (order0_s0[i] is then
    // order0[i]'s row in it), else col_sel itself (order0_s0 null).
    const int32_t* col_s0 = nullptr;
    const int4* order0_s0 = nullptr;
    // With these (single graphs with a tested subgraph): the solve computes
    // the keys of keyed[0 .. n_keyed) only, starts the result from out0 and
    // marks its candidates in it as it selects them (no output pass).
    const int2* keyed = nullptr;
    const uint8_t* out0 = nullptr;
    int32_t n_keyed = 0;
    // 1 (single graphs): the CSR kernel writes the result as it decides --
    // the create-time part at init, candidates as they are selected -- and
    // counts the MIS size on the way, so it needs no output pass and a small
    // last worklist can be finished by one block
    int32_t direct = 0;
    int32_t n_sure_in = 0;
    int32_t n_sure_out = 0;
    int32_t priority = 0;             // priority heuristic (kPrioEq1, kPrioHash, kPrioEq1Q8)
    // > 0: round 0 tests bin 0 (degree 1 .. range0_max) by vertex ranges over
    // row_ptr instead of its order0 list (graphs without round-0 classes)
    int32_t range0_max = 0;
    int32_t thr[4] = {0, 0, 0, 0};    // the degree bins' upper bounds (bins 0..3)
    int32_t pending = 0;              // 1: Phase 1 lists its non-candidates for Phase 2
                                      // (in wlp); 0: Phase 2 triages W_r itself
    // tile-CSR (used by the tile kernels only)
    const int32_t* trp = nullptr;    // row block rb owns tiles [trp[rb], trp[rb+1])
    const int32_t* tcol = nullptr;   // column block of each tile
    const uint64_t* tbits = nullptr; // T*T/64 words of row-major 0/1 bits per tile
    const void* tpay = nullptr;      // stored int8 / fp16 tile payload (tensor-core forms)
    int32_t nrb = 0;                 // row blocks = ceil(n / T)
    uint32_t* inbits = nullptr;      // bit v set once v is in the MIS (nrb*T bits)
    int32_t* rbl0 = nullptr;         // row-block worklists, nrb each
    int32_t* rbl1 = nullptr;
};

// mem.cu: device memory from the stream-ordered pool (reused across
// creates); callers synchronise their streams before dev_free.
// dev_alloc_deferred leaves the allocation ordered on the legacy stream
// only: dev_alloc_fence makes every deferred allocation before it usable on
// any stream.
cudaError_t dev_alloc(void** p, size_t bytes);
cudaError_t dev_alloc_deferred(void** p, size_t bytes);
cudaError_t dev_alloc_fence();
void dev_free(void* p);
// mem.cu: small pinned host blocks from never-returned slabs (larger
// requests: cudaMallocHost); null on failure.
void* host_small_alloc(size_t bytes);
void host_small_free(void* p);

// Launch configuration chosen by the host.
struct LaunchCfg {
    int grid = 0;
    int block = 0;
};

// kernels_csr.cu
cudaError_t launch_csr_solve(const SolveArgs& a, int grid, cudaStream_t s);
// The same kernel as a single block through an ordinary launch (a lone block
// needs no co-scheduling guarantee for its barriers).
cudaError_t launch_csr_solve_single(const SolveArgs& a, cudaStream_t s);
int csr_max_coresident_blocks(int device);
int csr_block_size();
// Where round 0's vertices go: order0 bins, or decided without a test.
struct Round0Plan {
    int32_t bin_off[6];   // order0 bin j occupies [bin_off[j], bin_off[j+1])
    int32_t n_isolated;   // degree 0: in the MIS at init
    int32_t n_sure_in;    // r0class 1: in the MIS at init
    int32_t n_sure_out;   // r0class 2: listed in sure_out
};

// Round-0 row records grouped by degree bin (thr: inclusive upper degree of
// bins 0..3; split: selection-prefix lengths, nullable = whole rows).
// Isolated vertices and the classes of r0class (nullable) are left out of
// order0; the sure exclusions are listed in sure_out.
cudaError_t build_bins(const int32_t* rp, const int32_t* split, const uint8_t* r0class,
                       int32_t n, const SegTable& seg, const int32_t thr[4], int4* order0,
                       int32_t* sure_out, const int32_t* s0_rp, const int32_t* s0_pre,
                       int4* order0_s0, Round0Plan* plan, cudaStream_t s);
// (with s0_rp, s0_pre and order0_s0 non-null, order0_s0[i] is order0[i]'s row
// in the tested subgraph below)

// The tested subgraph: the class-0 vertices' adjacency restricted to class-0
// neighbours, each row in col_sel's order (s0_pre = its selection-prefix
// length).  Built only when it has at most max_arcs arcs (else all outputs
// null); the caller owns what it returns.
cudaError_t build_s0_graph(const int32_t* rp, const int32_t* col_sel, const int32_t* split,
                           const uint8_t* r0class, int32_t n, int64_t max_arcs, int32_t** s0_rp,
                           int32_t** s0_col, int32_t** s0_pre, int64_t* s0_arcs,
                           cudaStream_t s);
// The keyed vertices of a graph with a tested subgraph (S0 and the vertices
// of S0 rows' selection prefixes; {vertex, degree}, sorted by vertex) and the
// result bytes known at create time (out0[v] = 1 for isolated vertices and
// sure candidates; padded to a multiple of 16).  Device arrays, owned by the
// caller.  Also counts the tested vertices and the arcs of their selection
// prefixes.
cudaError_t build_keyed(const int32_t* rp, const int32_t* col_sel, const int32_t* split,
                        const uint8_t* r0class, int32_t n, int2** keyed, int32_t* n_keyed,
                        uint8_t** out0, int32_t* n_tested, int64_t* prefix_arcs,
                        cudaStream_t s);

// Create-time round-0 classes from the degree-ordered rows (col_sel, split):
// 1 = sure candidate (empty selection prefix: every neighbour has degree >=
// deg + 2, so none can outrank it, whatever the seed); 2 = sure exclusion (not
// class 1, with a class-1 neighbour); 0 = the rest (tested in round 0).
cudaError_t build_round0_classes(const int32_t* rp, const int32_t* col_sel, const int32_t* split,
                                 int32_t n, const SegTable& seg, uint8_t* r0class,
                                 cudaStream_t s);

// kernels_multi.cu: k <= kMaxMulti solves of the graph of `a` (a.seg unused);
// word8 holds kMaxMulti words per vertex (n padded to 16); a.out receives
// k * n result bytes, solve s at a.out + s * n.
cudaError_t launch_multi_solve(const SolveArgs& a, uint32_t* word8, int k,
                               const MultiSeeds& seeds, int grid, cudaStream_t s);
int multi_max_coresident_blocks(int device);
// The same with Phase 2 on tensor cores (kernels_multi.cu, multi_rows_tc_kernel):
// the selection test on the CSR rows of `a` (a graph without create-time
// round-0 structures), the exclusion test as the single-bit MMA over its
// 16 x 16 bitmask tiles (a.trp, a.tcol, a.tbits; a.rbl0/1 row-block lists,
// a.nrb).  inb4: 4 * a.nrb words of in-set bits, 16-byte aligned.  Phase 2
// stays on tensor cores while at least tc_fill / 256 of the listed row blocks'
// entries are undecided (then the CSR scan, for the rest of the solve).
// split: sparse tiles on CUDA cores where that saves an MMA (worth it only
// where row blocks have more than eight tiles).
cudaError_t launch_multi_rows_tc_solve(const SolveArgs& a, uint32_t* word8, uint32_t* inb4, int k,
                                      const MultiSeeds& seeds, int tc_fill, bool split, int grid,
                                      cudaStream_t s);
int multi_rows_tc_max_coresident_blocks(int device);

// kernels_push.cu: the push/decrement form of the rounds (uses the worklist
// buffers of `a` for its ready and excluded lists and per-vertex counts).
cudaError_t launch_push_solve(const SolveArgs& a, int grid, cudaStream_t s);
int push_max_coresident_blocks(int device);

// kernels_util.cu
// Input contract checks.  Flags are ORed into *d_flags; with check_symmetry,
// d_sym[0..1] (zeroed by the caller) receive the two arc-set hash sums, both
// zero exactly when the arc set equals its reverse (see kernels_util.cu).
cudaError_t launch_validate(const int32_t* rp, const int32_t* col, int32_t n, int64_t arcs,
                            int check_symmetry, unsigned* d_flags, unsigned long long* d_sym,
                            cudaStream_t s);
// The two halves of launch_validate: row pointers, then the arcs [a0, a1)
// (which trust the row pointers).
cudaError_t launch_validate_rowptr(const int32_t* rp, int32_t n, int64_t arcs, unsigned* d_flags,
                                   cudaStream_t s);
cudaError_t launch_validate_arcs(const int32_t* rp, const int32_t* col, int32_t n, int64_t a0,
                                 int64_t a1, int check_symmetry, unsigned* d_flags,
                                 unsigned long long* d_sym, cudaStream_t s);
cudaError_t launch_keys(const SolveArgs& a, uint32_t* out_key, cudaStream_t s);
cudaError_t launch_fill_seg(int32_t* blk_seg, const int32_t* voff, int32_t count,
                            int32_t nblk, cudaStream_t s);
cudaError_t launch_relocate(int32_t* rp, int32_t* col, int32_t n, int32_t arcs, int32_t voff,
                            int32_t aoff, cudaStream_t s);
cudaError_t launch_pad_rows(int32_t* dst_rp, int32_t from, int32_t to, int32_t value,
                            cudaStream_t s);

// kernels_order.cu
// Rows of col sorted by neighbour degree into col_sel (same offsets) and
// split[v] = neighbours of degree <= deg(v) + 1 (the whole row for very high
// degrees): the only neighbours that can outrank v under Eq. 1.
cudaError_t build_degree_order(const int32_t* rp, const int32_t* col, int32_t n, int64_t arcs,
                               const SegTable& seg, int32_t* col_sel, int32_t* split,
                               cudaStream_t s);
// The same prefix by a stable partition of each row (cheaper than the sort).
cudaError_t build_row_partition(const int32_t* rp, const int32_t* col, int32_t n, int64_t arcs,
                                const SegTable& seg, int32_t* col_sel, int32_t* split,
                                cudaStream_t s);

// kernels_tile.cu
struct TileCsr {
    int T = 0;
    int32_t nrb = 0;
    int64_t ntiles = 0;
    int32_t* trp = nullptr;
    int32_t* tcol = nullptr;
    uint64_t* tbits = nullptr;
};
// Non-empty T x T tiles of the adjacency (T = 8 or 16), bitmask payloads;
// allocates out's arrays (the caller frees them with cudaFree).
cudaError_t build_tiles(const int32_t* rp, const int32_t* col, int32_t n, int64_t arcs, int T,
                        TileCsr* out, cudaStream_t s);
// Persistent tile round kernel: T = 8 or 16 (tile size), S = 8 or 32 (lanes,
// i.e. tiles in flight, per row block); tc_payload = the payload form of the
// exclusion test on tensor cores (tile_tc.cuh; T = 16 only), -1 = popc on
// CUDA cores.
cudaError_t launch_tile_solve(const SolveArgs& a, int T, int S, int tc_payload, int grid,
                              cudaStream_t s);
int tile_max_coresident_blocks(int T, int S, int tc_payload, int device);
// kernels_cluster.cu: a single graph solved by one thread-block cluster (its
// vertex words in the CTAs' shared memory, cluster barriers between phases);
// graphs of up to cluster_max_vertices() vertices (0: no cluster fits).
int32_t cluster_max_vertices();
// The cluster for a graph (d_rp: its row_ptr on the device, n vertices): ncta
// CTAs of 2^shift words each, rows in shared memory or not, the dynamic
// shared memory of a CTA; false when none fits.  Sets the kernel's
// attributes; call it before a launch is captured.
struct ClusterPlan {
    int32_t ncta = 0;
    int32_t shift = 0;
    int32_t smem_rows = 0;
    int32_t replicated = 0;  // every CTA holds a replica of all vertex words
    int64_t smem_bytes = 0;
};
bool cluster_plan(const int32_t* d_rp, int32_t n, ClusterPlan* plan);
cudaError_t launch_cluster_solve(const SolveArgs& a, const ClusterPlan& p, cudaStream_t s);
// kernels_tile_multi.cu: k <= kMaxMulti solves of the graph of `a` on its
// 16 x 16 tiles (a.trp, a.tcol, a.tbits, a.tpay; a.rbl0/1 row-block lists),
// the exclusion test on tensor cores in payload form `payload` with the k
// solves as right-hand sides.  word8: kMaxMulti words per vertex (nrb * 16
// vertices); inb8: kMaxMulti bit vectors of tile_multi_bitvector_words(nrb)
// words each.  a.out receives solve s at a.out + s * n.
int32_t tile_multi_bitvector_words(int32_t nrb);
cudaError_t launch_tile_multi_solve(const SolveArgs& a, uint32_t* word8, uint32_t* inb8, int k,
                                    const MultiSeeds& seeds, int payload, int grid,
                                    cudaStream_t s);
int tile_multi_max_coresident_blocks(int payload, int device);
// The int8 (256 bytes per tile) or fp16 (512 bytes per tile) payload of a
// 16 x 16 tile-CSR for the tensor-core exclusion, expanded from its bitmask
// (tile_tc.cuh: kPayI8, kPayF16); allocates *out (freed with dev_free).
int64_t tile_payload_bytes(int64_t ntiles, int P);
cudaError_t build_tile_payload(const TileCsr& tiles, int P, void** out, cudaStream_t s);

// validation flag bits
constexpr unsigned kBadRowPtr = 1u;
constexpr unsigned kBadColRange = 2u;
constexpr unsigned kBadSelfLoop = 4u;
constexpr unsigned kBadOrder = 8u;
constexpr unsigned kBadSymmetry = 16u;

}  // namespace tcmis
