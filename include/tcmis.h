/*
 * tcmis.h -- C ABI of the GB300 (sm_103a) TC-MIS library, libtcmis.so.
 *
 * The library computes a maximal independent set (MIS) of an undirected,
 * unweighted graph with the round-synchronous, priority-based iteration of
 * TC-MIS (Nijhara & Banerjee), Algorithm 2:
 *
 *   priorities   P(v) = d / (d + deg(v) - eps(v))                  (Eq. 1, Sec. 2)
 *                d = average degree, eps(v) in [0, 1) a hashed perturbation;
 *                assigned once per solve and reused every round (Sec. 2).
 *   while A != {}:                                                 (Algorithm 2)
 *     Phase 1  C(v) = [P(v) > max over alive neighbours u of P(u)]  (selection test)
 *     Phase 2  N_c = A x C                                         (exclusion test)
 *     Phase 3  v joins the set if C(v) = 1; v leaves A if C(v) = 1 or N_c(v) > 0.
 *
 * Every phase of one round reads the state at the start of that round (the
 * H3 ordering of Sec. 3.3).  The result is therefore unique for a given
 * (graph, seed): it is the set that sequential greedy in decreasing priority
 * order produces.  Every path of the library (CSR kernel, tile kernels,
 * tensor-core kernel, batched and served solves) returns exactly that set.
 *
 * Exact priority rule (binary32, round-to-nearest, no FMA contraction):
 *   d      = float(row_ptr[n]) / float(n)        (arcs counted in both directions)
 *   h      = high 32 bits of mix(mix(seed) XOR v), mix = splitmix64 finaliser
 *   eps    = float(h >> 8) * 2^-24
 *   P      = d / ((d + float(deg(v))) - eps)
 *   ties in P are broken by the larger vertex id.
 *
 * Graph input contract (checked by mis_create*, violations give MIS_EINVAL):
 *   0 <= n < 2^31; row_ptr has n+1 entries, row_ptr[0] = 0, non-decreasing,
 *   row_ptr[n] < 2^31; every col_idx entry in [0, n); no self-loop; each row
 *   strictly increasing (sorted, no duplicates); symmetric (u in row v iff
 *   v in row u), because the paper's graphs are undirected (Sec. 4.1.2).
 *   n = 0 is valid and gives an empty result.
 *
 * Threading: every entry point may be called from any host thread.  Calls on
 * the same mis_graph are serialised by the library.  The serving entry points
 * (mis_submit / mis_poll / mis_wait) are driven by scheduler threads that the
 * library starts on first use.
 *
 * Errors: functions returning int give MIS_OK (0) or a negative MIS_E* code;
 * functions returning a pointer give NULL on error.  In both cases
 * mis_last_error() returns the code and a message for the calling thread.
 */
#ifndef TCMIS_H
#define TCMIS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    MIS_OK = 0,
    MIS_EINVAL = -1,     /* bad argument or graph violating the input contract */
    MIS_ENOMEM = -2,     /* device or host allocation failed, or HBM budget exceeded */
    MIS_EBUSY = -3,      /* no serving slot free / object in use */
    MIS_ETIMEDOUT = -4,  /* a bounded device-side wait gave up, or mis_wait timed out */
    MIS_EDEVICE = -5,    /* CUDA runtime error */
    MIS_EINTERNAL = -6,  /* internal invariant broken (e.g. round cap exceeded) */
    MIS_ENOTREADY = -7   /* request still in flight */
};

/* Which round kernel runs a solve. */
enum {
    MIS_PATH_AUTO = 0,     /* autotuner's choice, cached per density class */
    MIS_PATH_CSR = 1,      /* warp-per-row CSR kernel on CUDA cores */
    MIS_PATH_TILE = 2,     /* tile-CSR kernel, bitmask payload, popc on CUDA cores */
    MIS_PATH_TILE_TC = 3,  /* tile-CSR kernel, exclusion test as tensor-core MMA
                              (payload form: mis_set_tile_payload) */
    MIS_PATH_PUSH = 4,     /* CSR, work-efficient push/decrement rounds: a count of
                              undecided higher neighbours per vertex, decremented
                              as they are excluded; every arc read O(1) times */
    MIS_PATH_CLUSTER = 5,  /* single graphs of up to about half a million vertices:
                              one thread-block cluster (up to 16 SMs) keeps every
                              vertex word in its distributed shared memory and
                              separates the phases by the hardware cluster
                              barrier instead of a grid barrier */
    MIS_PATH_ROWS_TC = 6   /* reported by mis_get_stats only (not a value for
                              mis_set_path): multi-seed solves with the
                              selection test on the CSR rows and the exclusion
                              test on tensor cores (mis_set_multi_form) */
};

typedef struct mis_graph mis_graph;
typedef struct mis_replay mis_replay;
typedef int64_t mis_ticket;

typedef struct mis_options {
    int32_t path;            /* MIS_PATH_*; default MIS_PATH_AUTO */
    int32_t threads_per_row; /* CSR path: 0 = degree bins (rows of degree <= 8 get
                                one lane, <= 4096 four, <= 65536 a warp, beyond a
                                whole block), else 1, 4, 16, 32 or 512 lanes for
                                every row */
    int32_t check_symmetry;  /* 1 (default) = verify symmetry at create, 0 = trust */
    int32_t build_tiles;     /* 1 = build the 16 x 16 tile-CSR at create; -1 (default)
                                = when a tile path is first selected */
    int64_t spin_cap;        /* device barrier spin limit in polls; 0 = default
                                (about one second); the test suite uses small values */
    int32_t device;          /* CUDA device ordinal; default 0 */
    int32_t max_slots;       /* serving: concurrent solves per step; 0 = default (64) */
    int64_t hbm_budget;      /* serving: bytes of per-solve workspace admitted at
                                once; 0 = default (half of free device memory) */
    int32_t serve_blocks;    /* serving: most blocks one served solve may use (graphs
                                of up to 16384 vertices always use one); 0 = default
                                (half the SMs), so that several large requests share
                                the device */
    int32_t order_rows;      /* CSR kernel's copy of col_idx, made at create (seed-
                                independent): 1 (default) = each row stably partitioned
                                so that the neighbours able to outrank a vertex (degree
                                <= its degree + 1) come first and the selection test
                                scans only them; 2 = each row fully sorted by neighbour
                                degree (slower create, shorter exclusion scans);
                                0 = none (full rows) */
    int32_t priority;        /* priority heuristic (Sec. 3.3), fixed at create:
                                MIS_PRIORITY_EQ1 (default; H2/H3, Eq. 1),
                                MIS_PRIORITY_HASH (H1: random priority hash(v)),
                                MIS_PRIORITY_EQ1_Q8 (Eq. 1 discretised to 8 bits, ties
                                by vertex id).  The degree-ordered rows and the
                                create-time round-0 decisions rely on Eq. 1's degree
                                order; the other heuristics scan whole rows. */
} mis_options;

enum {
    MIS_PRIORITY_EQ1 = 0,
    MIS_PRIORITY_HASH = 1,
    MIS_PRIORITY_EQ1_Q8 = 2
};

/* Per-solve statistics of the last completed solve on a graph. */
typedef struct mis_stats {
    int32_t rounds;          /* while-loop iterations of Algorithm 2 */
    int32_t path;            /* MIS_PATH_* that ran */
    int32_t threads_per_row; /* CSR path: lanes per row forced for every row, or 0
                                when rows are binned by degree */
    int32_t status;          /* MIS_OK or the error of that solve */
    int32_t tile;            /* tile size of the graph's tile-CSR (0 = not built) */
    int32_t csr_pending;     /* CSR path: 1 when Phase 1 listed its non-candidates
                                for Phase 2, 0 when Phase 2 triaged the worklist */
    int64_t ntiles;          /* non-empty tiles of that tile-CSR */
    int64_t alive_sum;       /* sum over rounds of |A| at round start */
    int64_t mis_size;        /* |M| */
    int64_t alive_per_round[64]; /* |A| at the start of rounds 0..63 (0 beyond) */
    int64_t init_ns;         /* device time of the priority initialisation (Eq. 1) */
    int64_t select_ns[64];   /* device time of Phase 1 (selection test), rounds 0..63 */
    int64_t exclude_ns[64];  /* device time of Phases 2+3 (exclusion test, state
                                update, compaction), rounds 0..63 */
    int64_t sure_in;         /* CSR path: vertices known at create time to be round-0
                                candidates (every neighbour has degree >= deg + 2),
                                put in the MIS at init without a test */
    int64_t sure_out;        /* CSR path: neighbours of those, excluded in round 0
                                without a test */
    int64_t tested_arcs;     /* CSR path: arcs among the vertices neither of the
                                above nor isolated (the tested subgraph), whose
                                rows all scans but round 0's selection test read;
                                -1 when the graph keeps no copy of them (more
                                than half of the arcs) */
    int64_t keyed;           /* CSR path: vertices whose Eq. 1 key a solve computes
                                when the graph has a tested subgraph (its
                                vertices and those of their selection prefixes;
                                no other word is read); -1 = every vertex */
    int64_t tested_rows;     /* CSR path, with a tested subgraph: its vertices (the
                                rows round 0 tests); -1 without one */
    int64_t tested_prefix_arcs; /* ... and the arcs of their selection prefixes
                                (neighbours of degree <= deg + 1), which round
                                0's selection test reads; -1 without one */
    int32_t tile_payload;    /* MIS_PATH_TILE_TC: the MIS_TILE_* form that ran; -1
                                on other paths */
} mis_stats;

/* Fill *opt with the defaults listed above. */
void mis_options_init(mis_options *opt);

/*
 * Create a graph handle from a CSR graph in HOST memory (copied to the device;
 * the caller may free its arrays when the call returns).  Validates the input
 * contract on the device.  Returns NULL on error (see mis_last_error).
 *   n        number of vertices
 *   row_ptr  int32[n+1] row offsets
 *   col_idx  int32[row_ptr[n]] neighbour ids
 */
mis_graph *mis_create(int32_t n, const int32_t *row_ptr, const int32_t *col_idx);

/*
 * As mis_create, with options, and with row_ptr / col_idx either host
 * pointers (on_device = 0) or device pointers (on_device = 1; copied device
 * to device).  `stream` is a cudaStream_t (NULL = legacy default stream); the
 * call returns after the graph is resident.  `opt` may be NULL (defaults).
 */
mis_graph *mis_create_ex(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                         int32_t on_device, const mis_options *opt, void *stream);

/*
 * Block-diagonal disjoint union of `count` graphs, solved together in one
 * persistent launch.  Graph g (host CSR arrays ns[g], row_ptrs[g],
 * col_idxs[g]) keeps its own vertex ids, its own average degree d and its own
 * seed for Eq. 1, so its part of the result equals a standalone solve of g.
 * Vertex offsets inside the union are padded to multiples of 16.
 */
mis_graph *mis_create_batch(int32_t count, const int32_t *ns, const int32_t *const *row_ptrs,
                            const int32_t *const *col_idxs, const mis_options *opt);

/* Number of graphs in a handle (1 unless made by mis_create_batch) and the
 * total number of result bytes (sum of the graphs' n). */
int32_t mis_graph_count(const mis_graph *g);
int64_t mis_result_size(const mis_graph *g);

/*
 * Solve with seed `seed` and write the result to HOST memory:
 * out_status[v] = 1 if v is in the MIS, else 0 (n bytes; for a batch, the
 * graphs' results one after another, each graph's seed = seed + its index).
 * Blocks until done.
 */
int mis_solve(mis_graph *g, uint64_t seed, uint8_t *out_status);

/*
 * Asynchronous solve on `stream` (a cudaStream_t; NULL = legacy default).
 * `seeds` holds one seed per graph of the handle (mis_graph_count entries).
 * `out_status` is a DEVICE pointer to mis_result_size bytes.  Returns after
 * enqueueing; errors found on the device are reported by mis_get_stats (which
 * synchronises the stream).  The graph's device workspace is reused by the
 * next solve on the same handle, so solves on one handle must be ordered on
 * one stream.
 */
int mis_solve_ex(mis_graph *g, const uint64_t *seeds, uint8_t *out_status, void *stream);

/*
 * Several solves of one graph in one launch: k solves (1 <= k <= 8) with
 * seeds[0..k-1] (HOST array).  Each solve's result is the set mis_solve_ex
 * with that seed gives; solve s is written to out_status + s * n (DEVICE
 * buffer of k * n bytes).  The k solves share the graph and one worklist and
 * run their rounds of Algorithm 2 in lock step: with k right-hand sides the
 * exclusion product of Sec. 3.1 (Phase 2, N_c = A x C) becomes A x [C_1 ..
 * C_k], and every neighbour gather serves all k solves.  mis_get_stats then
 * reports rounds = the largest round count of the k solves, alive sets and
 * MIS sizes summed over the solves.  Single-graph handles only (MIS_EINVAL for
 * a batch, or k outside [1, 8]); MIS_EBUSY while served requests on `g` are in
 * flight; the extra device memory (32 bytes per vertex) is kept by the handle.
 * On a graph whose path is MIS_PATH_TILE_TC the solves run on its 16 x 16
 * tiles and the product A x [C_1 .. C_k] is a tensor-core MMA with the k
 * solves as k of its eight columns, in the graph's tile payload form
 * (mis_set_tile_payload); on any other path, on the CSR kernel's rows with
 * CUDA cores.  mis_get_stats reports the path that ran.
 */
int mis_solve_multi_ex(mis_graph *g, int32_t k, const uint64_t *seeds, uint8_t *out_status,
                       void *stream);

/*
 * The form of mis_solve_multi_ex on a graph whose path is not
 * MIS_PATH_TILE_TC (Sec. 3.1 Phase 2 as the product A x [C_1 .. C_k]):
 *   MIS_MULTI_ROWS     both tests on the CSR rows on CUDA cores (default)
 *   MIS_MULTI_ROWS_TC  the selection test on the CSR rows (per-vertex
 *                      worklists), the exclusion test over the graph's 16 x 16
 *                      bitmask tiles (Sec. 3.2) on the single-bit tensor-core
 *                      MMA (AND, then population count, int32 accumulation:
 *                      exact), the k solves as k of its eight columns.  The
 *                      16 x 16 tile-CSR is built on the first such solve and
 *                      kept by the handle (mis_footprint counts it); a graph
 *                      whose single solves run on 8 x 8 tiles (MIS_PATH_TILE,
 *                      tile size 8) is refused at solve time (MIS_EINVAL).
 *                      Phase 2 runs on the tensor cores while at least
 *                      one in eight of the entries of the row blocks still
 *                      listed is undecided, and as the CSR scan for the rest
 *                      of the solve (mis_autotune_multi may move that point).
 *                      mis_get_stats reports MIS_PATH_ROWS_TC.
 * Both forms give every solve the set and rounds of its single solve.
 * MIS_MULTI_ROWS_TC takes a single graph created without round-0 structures
 * (mis_options.order_rows = 0): MIS_EINVAL otherwise, and for unknown forms;
 * MIS_EBUSY while served requests on `g` are in flight.
 */
enum {
    MIS_MULTI_ROWS = 0,
    MIS_MULTI_ROWS_TC = 1
};
int mis_set_multi_form(mis_graph *g, int32_t form);

/* Autotuner for the form above: times mis_solve_multi_ex with k seeds (1 ..
 * k; median of `reps` launches, reps <= 0 means 3) in each form the graph can
 * take -- MIS_MULTI_ROWS_TC with its switch to the CSR scan at three points
 * (while 1/8, 3/8 or 25/32 of the listed entries are undecided) -- keeps the
 * fastest for later multi-seed solves on `g` and returns its form in *form
 * (may be NULL).  mis_set_multi_form restores the default switch point.  A graph that cannot take MIS_MULTI_ROWS_TC (see above)
 * gets MIS_MULTI_ROWS without timing.  Allocates k * n bytes of device output
 * for the timing and frees it.  Blocks the calling thread.  MIS_EINVAL for a
 * batch or k outside [1, 8], MIS_EBUSY while served requests on `g` are in
 * flight. */
int mis_autotune_multi(mis_graph *g, int32_t k, int32_t reps, int32_t *form);

/*
 * Captured solves (no counterpart in the paper: launch-overhead removal for
 * repeated solves, e.g. a batched union solved again and again).
 * mis_capture records what mis_solve_ex(g, seeds, out_status, stream) enqueues
 * -- control-block reset, seed upload, the one persistent round-kernel launch
 * -- into an executable CUDA graph; mis_replay_launch launches that graph on
 * `stream` (a cudaStream_t).  Each replay is a complete solve with the captured seeds
 * (copied at capture time) into the captured DEVICE buffer `out_status`, and
 * the captured path, bins and grid.  Replays use the handle's workspace like
 * mis_solve_ex: order them with the handle's other solves on one stream;
 * mis_get_stats reports the last one.  Destroy every replay of a handle
 * before the handle.  Errors: MIS_EINVAL (null or bad arguments), MIS_EBUSY
 * (served requests in flight on `g`), MIS_EDEVICE (capture or instantiation
 * refused by the driver), MIS_ENOMEM.
 */
int mis_capture(mis_graph *g, const uint64_t *seeds, uint8_t *out_status, mis_replay **replay);
int mis_replay_launch(mis_replay *replay, void *stream);
void mis_replay_destroy(mis_replay *replay);

/* Statistics of the last solve on `g`; synchronises that solve's stream and
 * returns its device-side status (MIS_OK, MIS_ETIMEDOUT, MIS_EINTERNAL). */
int mis_get_stats(mis_graph *g, mis_stats *stats);

/*
 * Priority keys of Eq. 1 as computed by the device (for testing): writes
 * uint32 key[v] = bit pattern of binary32 P(v) for deg(v) >= 1 and
 * 0xFFFFFFFF for isolated vertices, into the DEVICE buffer out_key
 * (mis_result_size entries).  Runs on `stream`.
 */
int mis_keys_ex(mis_graph *g, const uint64_t *seeds, uint32_t *out_key, void *stream);

/* Select the round kernel for later solves.  MIS_PATH_CSR (or AUTO): `param`
 * is the lanes per row as in mis_options.threads_per_row.  MIS_PATH_TILE:
 * `param` is the tile size, 8 or 16 (0 = 16); MIS_PATH_TILE_TC: 16 (or 0).
 * MIS_PATH_CLUSTER: single graphs that fit one cluster (MIS_EINVAL for a
 * batch or a larger graph; mis_cluster_max_vertices gives the limit).
 * The tile-CSR (non-empty tiles only, 0/1 bitmask payloads) is built on the
 * device the first time a tile size is selected. */
int mis_set_path(mis_graph *g, int32_t path, int32_t param);

/* The most vertices a graph may have for MIS_PATH_CLUSTER on the current
 * device (0 when no cluster fits). */
int32_t mis_cluster_max_vertices(void);

/* CSR path with degree bins: bounds[0..3] are the inclusive upper degrees of
 * bins 0..3 (1, 4, 16 and 32 lanes per row; bin 4, a block of 512 threads per
 * row, takes the rest).  Non-decreasing; -1 empties a bin.  Used by the
 * autotuner. */
int mis_set_csr_bins(mis_graph *g, const int32_t *bounds);

/* CSR path: how Phase 2 finds the vertices to test (Sec. 3.1: the exclusion
 * test concerns the undecided non-candidates of the round).  pending = 1:
 * Phase 1 appends each non-candidate's row to a pending list that Phase 2
 * scans; pending = 0 (default): Phase 2 reads the whole worklist and skips
 * the candidates by their state.  Same result either way; the faster one
 * depends on the graph (chosen by mis_autotune).  MIS_EINVAL for other
 * values, MIS_EBUSY while served requests on `g` are in flight. */
int mis_set_csr_pending(mis_graph *g, int32_t pending);

/* Tile payload forms of the tensor-core exclusion (MIS_PATH_TILE_TC), i.e.
 * of the product N_c = A x C of Sec. 3.1 Phase 2 over the non-empty 16 x 16
 * tiles.  The selection test always reads the tiles' bitmasks; the forms
 * differ in what the tensor cores read:
 *   MIS_TILE_BITS     the bitmask, expanded to fp16 0/1 fragments in registers
 *                     (mma m16n8k16, fp32 accumulation, one tile per MMA)
 *   MIS_TILE_BITS_B1  the bitmask itself on the single-bit MMA: AND, then
 *                     population count, int32 accumulation (m16n8k128, eight
 *                     tiles per MMA)
 *   MIS_TILE_INT8     stored 16 x 16 int8 0/1 tiles, 256 bytes each (m16n8k32,
 *                     int32 accumulation, two tiles per MMA)
 *   MIS_TILE_FP16     stored 16 x 16 fp16 0/1 tiles, 512 bytes each, the
 *                     paper's format (Sec. 3.2, Listing 1; m16n8k16, fp32)
 * All are exact (0/1 entries, sums below 2^24).  A stored payload is built on
 * the device from the bitmask the first time its form runs and is kept by the
 * handle (mis_footprint counts it). */
enum {
    MIS_TILE_BITS = 0,
    MIS_TILE_BITS_B1 = 1,
    MIS_TILE_INT8 = 2,
    MIS_TILE_FP16 = 3
};

/* The payload form of the tensor-core tile path for later solves (and for
 * the exclusion of multi-seed solves on that path); switches a graph already
 * on MIS_PATH_TILE_TC at once, building its stored payload if needed.
 * MIS_EINVAL for other values, MIS_ENOMEM when the payload does not fit,
 * MIS_EBUSY while served requests on `g` are in flight. */
int mis_set_tile_payload(mis_graph *g, int32_t payload);

/* The 16 x 16 tiles' payload in form `payload` copied into the DEVICE buffer
 * `out` on `stream` (for testing): MIS_TILE_BITS / MIS_TILE_BITS_B1 give the
 * bitmask (32 bytes per tile, as mis_tiles_ex), MIS_TILE_INT8 256 bytes per
 * tile (entry (i, j) at byte 16 i + j), MIS_TILE_FP16 512 bytes per tile (at
 * half 16 i + j); tiles in tile-CSR order (mis_get_stats: ntiles).  Builds
 * the 16 x 16 tile-CSR and the stored payload if needed; out may be NULL
 * (build only). */
int mis_tile_payload_ex(mis_graph *g, int32_t payload, void *out, void *stream);

/* CSR path, graphs created without the round-0 classes (order_rows = 0 or a
 * priority other than Eq. 1): how round 0 (Algorithm 2's first iteration,
 * every vertex alive) reaches the rows of degree bin 0.  on = 1 (default):
 * the warps split the vertex range and read row_ptr in sequence, one lane per
 * light row; on = 0: from the bin's create-time list of 16-byte row records.
 * Same result either way (chosen by mis_autotune).  MIS_EINVAL for other
 * values, MIS_EBUSY while served requests on `g` are in flight. */
int mis_set_csr_range0(mis_graph *g, int32_t on);

/* The autotuner's choice for a graph. */
typedef struct mis_tuning {
    int32_t path;        /* MIS_PATH_CSR, MIS_PATH_TILE or MIS_PATH_TILE_TC */
    int32_t param;       /* CSR: forced lanes per row (0 = degree bins); tile: size */
    int32_t bounds[4];   /* CSR degree-bin bounds (see mis_set_csr_bins) */
    int32_t grid;        /* persistent blocks in use */
    int32_t candidates;  /* configurations timed */
    float ms;            /* median solve time of the choice, ms */
    int32_t csr_pending; /* CSR: the mis_set_csr_pending mode of the choice */
    double arcs_per_tile;/* sampled arcs per non-empty 8 x 8 tile */
    int32_t csr_range0;  /* CSR: the mis_set_csr_range0 mode of the choice (0 when
                            the graph has round-0 classes) */
    int32_t tile_payload;/* MIS_PATH_TILE_TC: the MIS_TILE_* form of the choice,
                            else -1 */
} mis_tuning;

/*
 * Autotuner: times candidate configurations on `g` (median of `reps` solves
 * each, reps <= 0 means 3) -- CSR degree-bin bounds, grid sizes and both
 * mis_set_csr_pending modes, and the
 * tile paths (8 x 8 and 16 x 16 popc, 16 x 16 tensor core) when sampled tiles
 * hold enough arcs -- applies the fastest to `g` and caches it for the
 * graph's density class (average degree, size, tile locality, device).  Graphs
 * created later with path MIS_PATH_AUTO take the cached choice of their class.
 * The cache lives in the process and, if the environment variable
 * TCMIS_TUNE_CACHE names a file, in that file.  Blocks the calling thread;
 * MIS_EBUSY while served requests on `g` are in flight.  `chosen` may be NULL.
 */
int mis_autotune(mis_graph *g, int32_t reps, mis_tuning *chosen);

/* Blocks of the persistent round kernel for later solves on `g` (0 = default:
 * one per 256 vertices), clamped to what can be co-resident on the device;
 * mis_get_grid returns the value in use.  Used by the autotuner. */
int mis_set_grid(mis_graph *g, int32_t blocks);
int32_t mis_get_grid(const mis_graph *g);

/* Copy the graph's tile-CSR into DEVICE buffers on `stream` (for testing):
 * trp int32[nrb+1] (nrb = ceil(n / T)), tcol int32[ntiles], tbits uint64[ntiles
 * * T * T / 64] (row-major bits: bit i*T + j of a tile is entry (i, j)).  Sizes
 * come from mis_get_stats (tile, ntiles).  Any pointer may be NULL. */
int mis_tiles_ex(mis_graph *g, int32_t *trp, int32_t *tcol, uint64_t *tbits, void *stream);

/* Bytes of device memory held by the handle (graph + workspace). */
int64_t mis_footprint(const mis_graph *g);

/* ---------------------------------------------------------------- dynamic graphs
 *
 * The dynamic setting (edge insertions and deletions) that the paper's
 * conclusion names as future work.  Single graphs only (not a batch).
 *
 * mis_update_edges applies n_ins insertions and n_del deletions of undirected
 * edges to the resident graph.  ins and del are HOST arrays of vertex pairs
 * (u0, v0, u1, v1, ...), each with 0 <= u, v < n and u != v, else MIS_EINVAL.
 * Inserting an edge that exists, or deleting one that does not, changes
 * nothing.  The graph is rebuilt on the device (sorted, duplicate-free,
 * symmetric) with every create-time structure, as mis_create_ex builds them
 * from the new CSR; the handle keeps its options and its resolved path.
 * Synchronises `stream`.  MIS_EBUSY while served requests of the handle are
 * in flight or captured solves of it (mis_capture) exist, since both hold its
 * device memory; on any error the handle keeps its old graph.
 */
int mis_update_edges(mis_graph *g, int64_t n_ins, const int32_t *ins, int64_t n_del,
                     const int32_t *del, void *stream);

/*
 * mis_add_vertices appends k isolated vertices, ids n .. n+k-1 (n grows to
 * n+k; result buffers then need n+k bytes).  An isolated vertex is in every
 * maximal independent set, so the result of the grown graph is the old
 * result followed by k ones, and edges to the new vertices then go through
 * mis_update_edges and mis_repair.  A vertex is removed from the set problem
 * by deleting its edges (it is then isolated, hence in).  Same conditions as
 * mis_update_edges (single graph, no served request in flight, no captured
 * solve); synchronises `stream`.
 */
int mis_add_vertices(mis_graph *g, int32_t k, void *stream);

/*
 * mis_repair turns out_status (DEVICE, n bytes), the result of a solve with
 * `seed` of the graph as it was before some edge changes, into the result of
 * the same solve of the graph as it is now -- bit-identical to mis_solve_ex
 * with that seed -- by re-deciding only the vertices whose state can change.
 * changed: HOST pairs (u, v) of every edge inserted or deleted since
 * out_status was computed (a superset is fine).  Algorithm 2 with fixed keys
 * yields the greedy MIS in priority order, where a vertex is in exactly when
 * no neighbour that outranks it is in; so the repair re-decides the lower
 * endpoints of the changed edges, then, pass by pass, the lower-priority
 * neighbours of every vertex that flipped, until nothing flips; the other
 * vertices keep their state.  Requires MIS_PRIORITY_HASH
 * (H1, Sec. 3.3), whose keys do not depend on the graph: Eq. 1's keys divide
 * by the average degree, so an edge change moves every key (MIS_EINVAL: solve
 * again instead).  mis_size and rounds (nullable) receive |M| and the rounds
 * run over all passes.  Uses the handle's workspace (not concurrently with its
 * other solves); synchronises `stream`.
 */
int mis_repair(mis_graph *g, uint64_t seed, int64_t n_changed, const int32_t *changed,
               uint8_t *out_status, int64_t *mis_size, int32_t *rounds, void *stream);

/*
 * Release the handle.  If served requests on it are still in flight the
 * release is deferred until they finish.
 */
void mis_destroy(mis_graph *g);

/* ---------------------------------------------------------------- serving
 *
 * Continuous batching over resident graphs.  mis_submit queues a request
 * (graph, seed, HOST output buffer of n bytes that must stay valid until the
 * request completes).  A few scheduler threads per process share up to
 * max_slots solve slots, each slot with its own CUDA stream and workspace;
 * each thread loops over its own slots:
 *   retire  slots whose solve finished: the result is copied to the caller's
 *           buffer, then the request is reported done;
 *   admit   queued requests, oldest first, while a slot is free and the
 *           workspace bytes of the admitted requests fit the HBM budget;
 *   group   queued requests on the same single graph ride one slot together,
 *           up to 8, solved by one multi-seed launch (see mis_solve_multi_ex);
 *   launch  each admitted request or group as a whole solve on its slot's
 *           stream: one block for graphs of up to 16384 vertices, else a
 *           cooperative grid of at most serve_blocks blocks.
 * Requests that arrive while others run are admitted as slots and memory
 * free up, and their solves run on the device at the same time as the others'.
 */
int mis_submit(mis_graph *g, uint64_t seed, uint8_t *out_status, mis_ticket *ticket);

/* MIS_OK if the request finished (and its ticket is released), MIS_ENOTREADY
 * if still pending, or the negative error it finished with. */
int mis_poll(mis_ticket ticket);

/* Wait up to timeout_us microseconds (negative = forever); same returns as
 * mis_poll, MIS_ETIMEDOUT when the wait expires first. */
int mis_wait(mis_ticket ticket, int64_t timeout_us);

/* As mis_poll; when the request is done, *latency_ns (if not NULL) receives
 * the time from its mis_submit to the moment its result was in the caller's
 * buffer, measured by the library (steady clock). */
int mis_poll_ex(mis_ticket ticket, int64_t *latency_ns);

/* Configure the serving scheduler (before the first submit; opt as in
 * mis_create_ex: max_slots, hbm_budget, spin_cap, device). */
int mis_serve_configure(const mis_options *opt);

/* Stop the scheduler thread after draining in-flight requests. */
void mis_serve_shutdown(void);

/* ---------------------------------------------------------------- no allocation
 *
 * The paper has no counterpart to this entry point; it exists for callers
 * that must not allocate device memory (code running inside a custom
 * allocator, frameworks that reserve all device memory up front, loops that
 * cannot afford an allocation's latency or implicit synchronisation).
 *
 * Solves one graph on the calling thread's current CUDA device without any
 * allocation: no cudaMalloc, no cudaFree, no allocating library routine.
 *   n           number of vertices, 0 <= n <= 262144 (larger n: MIS_EINVAL)
 *   row_ptr     DEVICE int32[n+1]
 *   col_idx     DEVICE int32[row_ptr[n]] (no padding or alignment needed);
 *               may be NULL only when row_ptr[n] = 0 (else MIS_EINVAL)
 *   seed        seed of the hashed priority perturbation; the same meaning
 *               as mis_solve's seed
 *   out_status  DEVICE uint8[n]: 1 if the vertex is in the MIS, else 0
 *   stream      cudaStream_t (NULL = legacy default stream)
 * The result equals mis_solve's for the same graph and seed.  The call
 * enqueues on `stream` and waits for it before it returns; it returns MIS_OK,
 * MIS_EINVAL, MIS_ETIMEDOUT, MIS_EINTERNAL or MIS_EDEVICE.  The graph is NOT
 * validated: a graph that breaks the input contract gives an unspecified
 * set, but the kernel never reads or writes outside the buffers above.
 *
 * Scratch: the library holds one fixed array of 3 MiB + 1 KiB in device
 * memory on every GPU that loads it, until the process exits.  Each call
 * looks up that array's device address on the current device; the first
 * call on a device also loads the library's device code there.  All calls
 * share the array, and each call clears the part that must start at zero;
 * calls whose work overlaps on a GPU (different streams or threads) race and
 * must be serialised by the caller.
 */
int mis_solve_noalloc(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, uint64_t seed,
                      uint8_t *out_status, void *stream);

/* Thread-local code and message of the last failing call on this thread. */
int mis_last_error(const char **msg);

/* Library version string. */
const char *mis_version(void);

#ifdef __cplusplus
}
#endif

#endif /* TCMIS_H */
