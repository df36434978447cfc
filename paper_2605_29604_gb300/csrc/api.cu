// api.cu -- the C ABI (include/tcmis.h): graph handles, solves, statistics.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "common.cuh"
#include "graph.h"
#include "internal.h"
#include "tcmis.h"

namespace tcmis {

// autotuner section below: the process's cached choice for the graph's
// class (false if none); is_csr tells whether it is the CSR kernel's
namespace {
struct TuneChoice;
}
bool cached_choice(mis_graph* g, TuneChoice** c, bool* is_csr);
int apply_cached(mis_graph* g, TuneChoice* c);
void drop_choice(TuneChoice* c);

namespace {
thread_local int t_err_code = 0;
thread_local std::string t_err_msg;
constexpr long long kDefaultSpinCap = 20000000;  // polls of ~64 ns: about a second or more
}  // namespace

int set_error(int code, const std::string& msg) {
    t_err_code = code;
    t_err_msg = msg;
    return code;
}

int set_cuda_error(cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a sticky launch error on this thread
    return set_error(e == cudaErrorMemoryAllocation ? MIS_ENOMEM : MIS_EDEVICE, m);
}

void clear_error() {
    t_err_code = 0;
    t_err_msg.clear();
}

namespace {

template <class T>
cudaError_t dalloc(T** p, int64_t count, int64_t* footprint) {
    const size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    cudaError_t e = dev_alloc((void**)p, bytes);
    if (e == cudaSuccess && footprint) *footprint += (int64_t)bytes;
    return e;
}

// The same without the fence: a group of these is followed by one
// dev_alloc_fence before any of the buffers is used on another stream.
template <class T>
cudaError_t dalloc_deferred(T** p, int64_t count, int64_t* footprint) {
    const size_t bytes = sizeof(T) * (size_t)std::max<int64_t>(count, 1);
    cudaError_t e = dev_alloc_deferred((void**)p, bytes);
    if (e == cudaSuccess && footprint) *footprint += (int64_t)bytes;
    return e;
}

void dfree(void* p) { dev_free(p); }

}  // namespace

// TCMIS_CREATE_LOG set: the wall time of each create stage on stderr (the
// stages synchronise their streams, so the times are the device's)
struct StageLog {
    bool on = std::getenv("TCMIS_CREATE_LOG") != nullptr;
    std::chrono::steady_clock::time_point t = std::chrono::steady_clock::now();
    void mark(const char* what, cudaStream_t s) {
        if (!on) return;
        cudaStreamSynchronize(s);
        const auto now = std::chrono::steady_clock::now();
        std::fprintf(stderr, "tcmis create: %-24s %8.3f ms\n", what,
                     std::chrono::duration<double, std::milli>(now - t).count());
        t = now;
    }
};

// The control block and the phase times share one allocation, so that one
// memset before each solve resets both.
constexpr size_t kCtlTimesOffset = (sizeof(Ctl) + 255) / 256 * 256;
constexpr size_t kCtlBlockBytes = kCtlTimesOffset + sizeof(PhaseTimes);

cudaError_t reset_control(const Workspace& w, cudaStream_t s) {
    return cudaMemsetAsync(w.ctl, 0, kCtlBlockBytes, s);
}

int64_t ws_bytes_for(int64_t n, int32_t count) {
    const int64_t cap = (n + 15) / 16 * 16;
    return 4 * cap + 16 * cap * 3 + (cap / 32 + 1) * 4 + 2 * 4 * (cap / 8) +
           (int64_t)kCtlBlockBytes + 8 * std::max<int64_t>(count, 1) + cap;
}

void ws_free(Workspace& w) {
    dfree(w.word);
    dfree(w.wl0);
    dfree(w.wl1);
    dfree(w.wlp);
    dfree(w.inbits);
    dfree(w.rbl0);
    dfree(w.rbl1);
    dfree(w.ctl);  // w.times lies inside this block
    dfree(w.seeds);
    dfree(w.out);
    w = Workspace();
}

cudaError_t ws_reserve(Workspace& w, int64_t n, int32_t count) {
    const int64_t cap = (n + 15) / 16 * 16;
    if (w.word && w.cap >= cap && w.seed_cap >= std::max(count, 1)) return cudaSuccess;
    ws_free(w);
    cudaError_t e;
    int64_t b = 0;
    if ((e = dalloc_deferred(&w.word, cap, &b)) != cudaSuccess ||
        (e = dalloc_deferred(&w.wl0, cap, &b)) != cudaSuccess ||
        (e = dalloc_deferred(&w.wl1, cap, &b)) != cudaSuccess ||
        (e = dalloc_deferred(&w.wlp, cap, &b)) != cudaSuccess ||
        (e = dalloc_deferred(&w.inbits, cap / 32 + 1, &b)) != cudaSuccess ||
        (e = dalloc_deferred(&w.rbl0, cap / 8, &b)) != cudaSuccess ||
        (e = dalloc_deferred(&w.rbl1, cap / 8, &b)) != cudaSuccess ||
        (e = dalloc_deferred(reinterpret_cast<unsigned char**>(&w.ctl),
                             (int64_t)kCtlBlockBytes, &b)) != cudaSuccess ||
        (e = dalloc_deferred(&w.seeds, std::max(count, 1), &b)) != cudaSuccess ||
        (e = dalloc_deferred(&w.out, cap, &b)) != cudaSuccess ||
        (e = dev_alloc_fence()) != cudaSuccess) {
        dev_alloc_fence();
        ws_free(w);
        return e;
    }
    w.times = reinterpret_cast<PhaseTimes*>(reinterpret_cast<unsigned char*>(w.ctl) + kCtlTimesOffset);
    // pool memory is recycled: the control block must read as "no solve yet"
    if ((e = cudaMemset(w.ctl, 0, kCtlBlockBytes)) != cudaSuccess) {
        ws_free(w);
        return e;
    }
    w.cap = cap;
    w.seed_cap = std::max(count, 1);
    w.bytes = b;
    return cudaSuccess;
}

namespace {

// Default degree-bin bounds: bin 0 (one lane per row) up to degree 8, bin 1
// (4 lanes) up to 4096, bin 2 (16 lanes) unused, bin 3 (a warp) up to 65536,
// bin 4 (a block per row) beyond.  Narrow groups win because most scans stop
// at their first few arcs; the autotuner refines the bounds per graph.
constexpr int32_t kDefaultThr[4] = {8, 4096, 4096, 65536};

// Bin bounds that force every vertex into the bin of `tpr` lanes
// (0 = default bins; 512 = a whole block per row).
bool thresholds_for(int tpr, int32_t thr[4]) {
    const int32_t none = -1, all = INT32_MAX;
    int force;
    switch (tpr) {
        case 0:
            for (int k = 0; k < 4; ++k) thr[k] = kDefaultThr[k];
            return true;
        case 1: force = 0; break;
        case 4: force = 1; break;
        case 16: force = 2; break;
        case 32: force = 3; break;
        case 512: force = 4; break;
        default: return false;
    }
    for (int k = 0; k < 4; ++k) thr[k] = k < force ? none : all;
    return true;
}

// Persistent grid: one block per 256 vertices, at most the co-resident limit
// (3 blocks of 512 threads per SM); `request` > 0 overrides (clamped).
int pick_grid(mis_graph* g, int request = 0) {
    const int maxb = csr_max_coresident_blocks(g->d.device);
    if (maxb <= 0) return 0;
    long long want = request > 0 ? request : ((long long)g->d.n + 255) / 256;
    if (want < 1) want = 1;
    return (int)std::min<long long>(want, maxb);
}

SegTable seg_of(const GraphData& d) {
    SegTable t;
    t.count = d.count;
    t.blk_seg = d.blk_seg;
    t.voff = d.voff;
    t.nv = d.nv;
    t.arcs = d.garcs;
    t.roff = d.roff;
    t.seed = nullptr;  // per-solve seeds live in the workspace
    return t;
}

// (Re)build the round-0 list grouped by degree bin for thresholds thr.
int rebin(mis_graph* g, const int32_t thr[4], cudaStream_t s) {
    GraphData& d = g->d;
    for (int j = 0; j < 4; ++j) d.thr[j] = thr[j];
    Round0Plan plan;
    cudaError_t e = build_bins(d.rp, d.split, d.r0class, d.n, seg_of(d), d.thr, d.order0,
                               d.sure_out, d.s0_rp, d.s0_pre, d.order0_s0, &plan, s);
    if (e != cudaSuccess) return set_cuda_error(e, "degree binning");
    for (int j = 0; j < 6; ++j) d.bin_off[j] = plan.bin_off[j];
    d.n_isolated = plan.n_isolated;
    d.n_sure_in = plan.n_sure_in;
    d.n_sure_out = plan.n_sure_out;
    return MIS_OK;
}

void free_payload(GraphData& d) {
    if (d.tpay) d.footprint -= tile_payload_bytes(d.tiles.ntiles, d.tpay_kind);
    dfree(d.tpay);
    d.tpay = nullptr;
    d.tpay_kind = -1;
}

void free_tiles(GraphData& d) {
    free_payload(d);
    dfree(d.tiles.trp);
    dfree(d.tiles.tcol);
    dfree(d.tiles.tbits);
    d.tiles = TileCsr();
    d.footprint -= d.tile_footprint;
    d.tile_footprint = 0;
}

// Switch to a tile path with T x T tiles, building the tile-CSR when needed.
int use_tiles(mis_graph* g, int path, int T) {
    GraphData& d = g->d;
    if (T != 8 && T != 16) return set_error(MIS_EINVAL, "tile size must be 8 or 16");
    if (path == MIS_PATH_TILE_TC && T != 16)
        return set_error(MIS_EINVAL, "the tensor-core tile path uses 16 x 16 tiles");
    cudaError_t e = cudaSuccess;
    if (d.tiles.T != T) {
        if (g->last_stream) cudaStreamSynchronize(g->last_stream);
        free_tiles(d);
        e = build_tiles(d.rp, d.col, d.n, d.arcs, T, &d.tiles, g->own_stream);
        if (e != cudaSuccess) {
            free_tiles(d);
            return set_cuda_error(e, "tile-CSR conversion");
        }
        const int words = T * T / 64;
        d.tile_footprint = 4 * ((int64_t)d.tiles.nrb + 1) + 4 * d.tiles.ntiles +
                           8 * (int64_t)words * d.tiles.ntiles;
        d.footprint += d.tile_footprint;
    }
    const bool tc = path == MIS_PATH_TILE_TC;
    // the stored int8 / fp16 payload of a tensor-core form that reads one
    const int pay = g->tile_payload;
    if (tc && (pay == MIS_TILE_INT8 || pay == MIS_TILE_FP16) && d.tpay_kind != pay) {
        if (g->last_stream) cudaStreamSynchronize(g->last_stream);
        free_payload(d);
        void* p = nullptr;
        e = build_tile_payload(d.tiles, pay, &p, g->own_stream);
        if (e != cudaSuccess) return set_cuda_error(e, "tile payload");
        d.tpay = p;
        d.tpay_kind = pay;
        d.footprint += tile_payload_bytes(d.tiles.ntiles, pay);
    }
    // a row block with many tiles gets a whole warp of tile slots; 8 x 8 row
    // blocks with few tiles are taken one per lane (32 row blocks per warp
    // pass: the selection test is latency-bound), 16 x 16 ones by 8 lanes
    const double per_rb = d.tiles.nrb ? (double)d.tiles.ntiles / d.tiles.nrb : 0.0;
    g->tile_slots = tc ? 8 : (per_rb > 12.0 ? 32 : (T == 8 ? 1 : 8));
    const int maxb = tile_max_coresident_blocks(T, g->tile_slots, tc ? pay : -1, d.device);
    if (maxb <= 0) return set_error(MIS_EDEVICE, "no co-resident blocks for the tile kernel");
    long long want = ((long long)d.tiles.nrb + 63) / 64;
    if (want < 1) want = 1;
    g->tile_grid = (int)std::min<long long>(want, maxb);
    g->path = path;
    return MIS_OK;
}

// Allocate the per-solve workspace and choose the launch shape.
int finish_create(mis_graph* g) {
    GraphData& d = g->d;
    cudaError_t e;
    const int64_t col_alloc = ((d.arcs + 3) / 4) * 4 + 4;
    // the selection prefixes and round-0 classes hold for Eq. 1's degree order only
    const bool order = g->opt.order_rows != 0 && g->opt.priority == MIS_PRIORITY_EQ1;
    if ((e = dalloc_deferred(&d.order0, d.n, &d.footprint)) != cudaSuccess ||
        (order && (e = dalloc_deferred(&d.r0class, d.n, &d.footprint)) != cudaSuccess) ||
        (order && (e = dalloc_deferred(&d.sure_out, d.n, &d.footprint)) != cudaSuccess) ||
        (order && (e = dalloc_deferred(&d.col_sel, col_alloc, &d.footprint)) != cudaSuccess) ||
        (order && (e = dalloc_deferred(&d.split, d.n, &d.footprint)) != cudaSuccess) ||
        (e = ws_reserve(d.ws, d.n, d.count)) != cudaSuccess) {  // its fence covers these
        dev_alloc_fence();
        return set_cuda_error(e, "workspace allocation");
    }
    d.footprint += d.ws.bytes;
    d.ctl_host = static_cast<Ctl*>(host_small_alloc(sizeof(Ctl)));
    d.times_host = static_cast<PhaseTimes*>(host_small_alloc(sizeof(PhaseTimes)));
    if (!d.ctl_host || !d.times_host) return set_cuda_error(cudaErrorMemoryAllocation, "pinned allocation");
    std::memset(d.ctl_host, 0, sizeof(Ctl));
    g->tpr = g->opt.threads_per_row;
    g->path = MIS_PATH_CSR;
    g->grid = pick_grid(g);
    if (g->grid <= 0) return set_error(MIS_EDEVICE, "no co-resident blocks for the round kernel");
    int32_t thr[4];
    thresholds_for(g->tpr, thr);
    if (!g->own_stream) {
        e = cudaStreamCreateWithFlags(&g->own_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return set_cuda_error(e, "stream");
    }
    StageLog lg;
    lg.mark("workspace", g->own_stream);
    if (order) {
        e = cudaMemsetAsync(d.col_sel, 0, sizeof(int32_t) * (size_t)col_alloc, g->own_stream);
        if (e == cudaSuccess)
            e = g->opt.order_rows == 2
                    ? build_degree_order(d.rp, d.col, d.n, d.arcs, seg_of(d), d.col_sel, d.split,
                                         g->own_stream)
                    : build_row_partition(d.rp, d.col, d.n, d.arcs, seg_of(d), d.col_sel,
                                          d.split, g->own_stream);
        lg.mark("row ordering", g->own_stream);
        if (e == cudaSuccess)
            e = build_round0_classes(d.rp, d.col_sel, d.split, d.n, seg_of(d), d.r0class,
                                     g->own_stream);
        lg.mark("round-0 classes", g->own_stream);
        // the tested subgraph, when it holds at most half of the arcs
        int64_t s0_arcs = 0;
        if (e == cudaSuccess)
            e = build_s0_graph(d.rp, d.col_sel, d.split, d.r0class, d.n, d.arcs / 2, &d.s0_rp,
                               &d.s0_col, &d.s0_pre, &s0_arcs, g->own_stream);
        if (e == cudaSuccess && d.s0_rp) {
            e = dalloc(&d.order0_s0, d.n, &d.footprint);
            d.s0_arcs = s0_arcs;
            d.s0_bytes = 4 * (2 * (int64_t)d.n + 1) + 4 * (((s0_arcs + 3) / 4) * 4 + 4);
            d.footprint += d.s0_bytes;
        }
        lg.mark("tested subgraph", g->own_stream);
        if (e == cudaSuccess && d.s0_col && d.count == 0) {
            e = build_keyed(d.rp, d.col_sel, d.split, d.r0class, d.n, &d.keyed, &d.n_keyed,
                            &d.out0, &d.n_tested, &d.tested_prefix_arcs, g->own_stream);
            d.footprint += 8 * ((int64_t)d.n_keyed + 1) + ((int64_t)d.n + 15) / 16 * 16;
        }
        if (e != cudaSuccess) return set_cuda_error(e, "degree ordering");
    }
    lg.mark("keyed list", g->own_stream);
    // AUTO: the autotuner's cached choice for the graph's class, if any; a
    // CSR choice takes the place of the default degree bins
    TuneChoice* cached = nullptr;
    bool cached_csr = false;
    if (g->opt.path == MIS_PATH_AUTO && g->opt.threads_per_row == 0)
        cached_choice(g, &cached, &cached_csr);
    lg.mark("tuning lookup", g->own_stream);
    int brc = MIS_OK;
    if (!cached_csr) brc = rebin(g, thr, g->own_stream);
    lg.mark("degree bins", g->own_stream);
    if (brc == MIS_OK && cached) brc = apply_cached(g, cached);
    lg.mark("tuned choice", g->own_stream);
    drop_choice(cached);
    if (brc != MIS_OK) return brc;
    if (g->opt.build_tiles == 1 || g->opt.path == MIS_PATH_TILE || g->opt.path == MIS_PATH_TILE_TC) {
        const int rc = use_tiles(g, g->opt.path == MIS_PATH_AUTO || g->opt.path == MIS_PATH_CSR
                                        ? MIS_PATH_TILE : g->opt.path, 16);
        if (rc != MIS_OK) return rc;
        if (g->opt.path == MIS_PATH_AUTO || g->opt.path == MIS_PATH_CSR) g->path = MIS_PATH_CSR;
    }
    return MIS_OK;
}

// flag word (padded to 8 bytes), the two 64-bit sums of the symmetry check,
// and the two 64-bit counters of the tile-density sample (estimate_arcs_per_tile)
constexpr size_t kFlagsBytes = 40;
constexpr size_t kSampleAccOffset = 24;

int validate_device(mis_graph* g, cudaStream_t s) {
    GraphData& d = g->d;
    // d.flags: the flag word, then (8-byte aligned) the two symmetry sums
    unsigned long long* sym = reinterpret_cast<unsigned long long*>(d.flags) + 1;
    cudaError_t e = cudaMemsetAsync(d.flags, 0, kFlagsBytes, s);
    if (e == cudaSuccess)
        e = launch_validate(d.rp, d.col, d.n, d.arcs, g->opt.check_symmetry, d.flags, sym, s);
    unsigned long long hb[3] = {0, 0, 0};  // the flag word and the two sums
    static_assert(sizeof(hb) == kSampleAccOffset, "flag word and sums");
    if (e == cudaSuccess) e = cudaMemcpyAsync(hb, d.flags, sizeof(hb), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(e, "graph validation");
    unsigned f = (unsigned)(hb[0] & 0xFFFFFFFFull);
    if (g->opt.check_symmetry && (hb[1] | hb[2]) && !(f & kBadRowPtr)) f |= kBadSymmetry;
    if (f) {
        std::string why;
        if (f & kBadRowPtr) why += " row_ptr not monotone from 0 to arcs;";
        if (f & kBadColRange) why += " col_idx out of [0, n);";
        if (f & kBadSelfLoop) why += " self-loop;";
        if (f & kBadOrder) why += " row not strictly increasing (unsorted or duplicate);";
        if (f & kBadSymmetry) why += " not symmetric;";
        return set_error(MIS_EINVAL, "invalid graph:" + why);
    }
    return MIS_OK;
}

// Host CSR without the symmetry check: col_idx goes up in pieces on the
// handle's own stream, all enqueued at once, while row_ptr is checked and
// then each landed piece is checked on `s`, so the checks hide behind the
// copy (host-to-device bandwidth bounds a create).
constexpr int64_t kUploadPiece = 4 << 20;  // arcs per piece

int upload_checked(mis_graph* g, const int32_t* col_idx, cudaStream_t s) {
    GraphData& d = g->d;
    cudaError_t e = cudaSuccess;
    if (!g->own_stream) e = cudaStreamCreateWithFlags(&g->own_stream, cudaStreamNonBlocking);
    std::vector<cudaEvent_t> evs;
    for (int64_t a0 = 0; a0 < d.arcs && e == cudaSuccess; a0 += kUploadPiece) {
        const int64_t a1 = std::min(d.arcs, a0 + kUploadPiece);
        cudaEvent_t ev = nullptr;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) break;
        evs.push_back(ev);
        e = cudaMemcpyAsync(d.col + a0, col_idx + a0, sizeof(int32_t) * (size_t)(a1 - a0),
                            cudaMemcpyHostToDevice, g->own_stream);
        if (e == cudaSuccess) e = cudaEventRecord(ev, g->own_stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(d.flags, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = launch_validate_rowptr(d.rp, d.n, d.arcs, d.flags, s);
    unsigned f = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&f, d.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the arc checks trust row_ptr
    if (e == cudaSuccess && f) e = cudaErrorInvalidValue;
    for (size_t k = 0; k < evs.size() && e == cudaSuccess; ++k) {
        const int64_t a0 = (int64_t)k * kUploadPiece, a1 = std::min(d.arcs, a0 + kUploadPiece);
        e = cudaStreamWaitEvent(s, evs[k], 0);
        // the order check of the first arc of a piece reads the previous
        // piece's last arc, which the copy stream has landed before
        if (e == cudaSuccess)
            e = launch_validate_arcs(d.rp, d.col, d.n, a0, a1, 0, d.flags, nullptr, s);
    }
    if (f) {
        // the copies still run: they finish before the caller frees the graph
        cudaStreamSynchronize(g->own_stream);
        for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
        return set_error(MIS_EINVAL, "invalid graph: row_ptr not monotone from 0 to arcs;");
    }
    f = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&f, d.flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    const cudaError_t se = cudaStreamSynchronize(s);
    const cudaError_t ce = cudaStreamSynchronize(g->own_stream);  // nothing may still run
    for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
    if (e == cudaSuccess) e = se != cudaSuccess ? se : ce;
    if (e != cudaSuccess) return set_cuda_error(e, "graph upload");
    if (f) {
        std::string why;
        if (f & kBadColRange) why += " col_idx out of [0, n);";
        if (f & kBadSelfLoop) why += " self-loop;";
        if (f & kBadOrder) why += " row not strictly increasing (unsorted or duplicate);";
        return set_error(MIS_EINVAL, "invalid graph:" + why);
    }
    return MIS_OK;
}

SolveArgs make_args(mis_graph* g, Workspace& w) {
    GraphData& d = g->d;
    SolveArgs a;
    a.rp = d.rp;
    a.col = d.col;
    a.n = d.n;
    a.word = w.word;
    a.wl0 = w.wl0;
    a.wl1 = w.wl1;
    a.wlp = w.wlp;
    a.col_sel = d.col_sel ? d.col_sel : d.col;
    a.split = d.split;
    a.order0 = d.order0;
    for (int j = 0; j < 6; ++j) a.bin_off[j] = d.bin_off[j];
    a.n_isolated = d.n_isolated;
    a.r0class = d.r0class;
    a.sure_out = d.sure_out;
    a.col_s0 = d.s0_col ? d.s0_col : a.col_sel;
    a.order0_s0 = d.s0_col ? d.order0_s0 : nullptr;
    a.direct = d.count == 0 ? 1 : 0;
    a.keyed = d.keyed;
    a.out0 = d.out0;
    a.n_keyed = d.n_keyed;
    a.n_sure_in = d.n_sure_in;
    a.n_sure_out = d.n_sure_out;
    a.pending = g->csr_pending;
    a.range0_max = (g->csr_range0 && !d.r0class && d.thr[0] >= 1) ? d.thr[0] : 0;
    for (int j = 0; j < 4; ++j) a.thr[j] = d.thr[j];
    a.priority = g->opt.priority;
    a.ctl = w.ctl;
    a.times = w.times;
    a.seg = seg_of(d);
    a.seg.seed = w.seeds;
    a.spin_cap = g->opt.spin_cap > 0 ? g->opt.spin_cap : kDefaultSpinCap;
    a.max_rounds = d.n + 2;
    a.trp = d.tiles.trp;
    a.tcol = d.tiles.tcol;
    a.tbits = d.tiles.tbits;
    a.tpay = d.tpay;
    a.nrb = d.tiles.nrb;
    a.inbits = w.inbits;
    a.rbl0 = w.rbl0;
    a.rbl1 = w.rbl1;
    return a;
}

}  // namespace

void free_graph(mis_graph* g) {
    if (!g) return;
    GraphData& d = g->d;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(d.device);
    if (g->own_stream) cudaStreamSynchronize(g->own_stream);
    if (g->last_stream) cudaStreamSynchronize(g->last_stream);
    dfree(d.rp);
    dfree(d.col);
    dfree(d.blk_seg);
    dfree(d.voff);
    dfree(d.nv);
    dfree(d.garcs);
    dfree(d.roff);
    host_small_free(d.seeds_host);
    free_tiles(d);
    dfree(d.order0);
    dfree(d.word8);
    dfree(d.inb8);
    dfree(d.r0class);
    dfree(d.sure_out);
    dfree(d.s0_rp);
    dfree(d.s0_col);
    dfree(d.s0_pre);
    dfree(d.order0_s0);
    dfree(d.dyn_mark);
    dfree(d.dyn_cnt);
    dfree(d.keyed);
    dfree(d.out0);
    dfree(d.col_sel);
    dfree(d.split);
    ws_free(d.ws);
    host_small_free(d.ctl_host);
    host_small_free(d.times_host);
    dfree(d.flags);
    if (g->own_stream) cudaStreamDestroy(g->own_stream);
    cudaSetDevice(prev);
    delete g;
}

int solve_in(mis_graph* g, Workspace& w, const uint64_t* seeds, uint64_t* seeds_pinned,
             uint8_t* out_dev, cudaStream_t s, int blocks) {
    const bool single_block = blocks == 1;
    GraphData& d = g->d;
    cudaError_t e = cudaSetDevice(d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    SolveArgs a = make_args(g, w);
    a.out = out_dev;
    if (d.count == 0) {
        a.seed0 = seeds[0];
    } else {
        std::memcpy(seeds_pinned, seeds, sizeof(uint64_t) * (size_t)d.count);
        e = cudaMemcpyAsync(w.seeds, seeds_pinned, sizeof(uint64_t) * (size_t)d.count,
                            cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return set_cuda_error(e, "seed upload");
    }
    // the cluster kernel writes every reported field of the control block
    // and the phase times itself
    if (d.n == 0 || g->path != MIS_PATH_CLUSTER) e = reset_control(w, s);
    if (e != cudaSuccess) return set_cuda_error(e, "control reset");
    if (d.n > 0) {
        const bool tile = g->path == MIS_PATH_TILE || g->path == MIS_PATH_TILE_TC;
        if (g->path == MIS_PATH_CLUSTER) {
            e = launch_cluster_solve(a, g->cluster, s);
        } else if (g->path == MIS_PATH_PUSH) {
            const int maxb = push_max_coresident_blocks(d.device);
            if (maxb <= 0) return set_error(MIS_EDEVICE, "no co-resident blocks for the push kernel");
            long long grid = std::min<long long>(maxb, std::max<long long>(1, (d.n + 255) / 256));
            if (blocks > 0) grid = std::min<long long>(grid, blocks);
            e = launch_push_solve(a, (int)grid, s);
        } else if (tile)
            e = launch_tile_solve(a, d.tiles.T, g->tile_slots,
                                  g->path == MIS_PATH_TILE_TC ? g->tile_payload : -1,
                                  blocks > 0 ? std::min(blocks, g->tile_grid) : g->tile_grid, s);
        else if (single_block)
            e = launch_csr_solve_single(a, s);
        else
            e = launch_csr_solve(a, blocks > 0 ? std::min(blocks, g->grid) : g->grid, s);
        if (e != cudaSuccess) return set_cuda_error(e, "round kernel launch");
    }
    return MIS_OK;
}

// Enqueue one solve on stream s in the handle's own workspace.
int solve_multi_in(mis_graph* g, Workspace& w, uint32_t* word8, int k, const uint64_t* seeds,
                   uint8_t* out_dev, cudaStream_t s, int blocks) {
    GraphData& d = g->d;
    cudaError_t e = cudaSetDevice(d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    MultiSeeds ms{};
    for (int i = 0; i < k; ++i) ms.seed[i] = seeds[i];
    SolveArgs a = make_args(g, w);
    a.out = out_dev;
    e = reset_control(w, s);
    if (e != cudaSuccess) return set_cuda_error(e, "control reset");
    if (d.n > 0) {
        const int maxb = multi_max_coresident_blocks(d.device);
        if (maxb <= 0) return set_error(MIS_EDEVICE, "no co-resident blocks for the multi kernel");
        long long grid = ((long long)d.n + 255) / 256;
        if (blocks > 0) grid = std::min<long long>(grid, blocks);
        grid = std::max<long long>(1, std::min<long long>(grid, maxb));
        e = launch_multi_solve(a, word8, k, ms, (int)grid, s);
        if (e != cudaSuccess) return set_cuda_error(e, "multi-seed kernel launch");
    }
    return MIS_OK;
}

int solve_async(mis_graph* g, const uint64_t* seeds, uint8_t* out_dev, cudaStream_t s) {
    const int rc = solve_in(g, g->d.ws, seeds, g->d.seeds_host, out_dev, s, 0);
    if (rc != MIS_OK) return rc;
    g->last_stream = s;
    g->last_path = g->path;
    return MIS_OK;
}

// ---------------------------------------------------------------- autotuner
//
// Chooses, per density class, the round kernel (CSR or tile), its lanes-per-
// row bins or tile size, and the persistent grid, by timing candidate
// configurations on the graph itself (median of a few solves, CUDA events).
// Choices are cached per class (average-degree bucket, size bucket, tile
// locality bucket, device name) in the process and, when TCMIS_TUNE_CACHE
// names a file, on disk.

namespace {

struct TuneChoice {
    int32_t path = MIS_PATH_CSR;
    int32_t param = 0;   // CSR: forced lanes per row (0 = bins); tile: tile size
    int32_t bounds[4] = {8, 4096, 4096, 65536};
    int32_t grid = 0;    // CSR grid request (0 = default)
    float ms = 0.f;
    int32_t pending = 0; // CSR: Phase 1 lists its non-candidates for Phase 2
    int32_t range0 = 1;  // CSR: round 0 takes bin 0 by vertex ranges
    int32_t payload = 0; // tensor-core tile path: MIS_TILE_* form
};

std::mutex g_tune_mu;
std::map<std::string, TuneChoice> g_tune_cache;
bool g_tune_loaded = false;

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* f = std::getenv("TCMIS_TUNE_CACHE");
    if (!f) return;
    std::ifstream in(f);
    std::string line;
    while (std::getline(in, line)) {
        std::istringstream ss(line);
        std::string key;
        TuneChoice c;
        if (ss >> key >> c.path >> c.param >> c.bounds[0] >> c.bounds[1] >> c.bounds[2] >>
            c.bounds[3] >> c.grid >> c.ms) {
            if (!(ss >> c.pending)) c.pending = 0;  // lines written before the field
            if (!(ss >> c.range0)) c.range0 = 1;
            if (!(ss >> c.payload)) c.payload = 0;
            g_tune_cache[key] = c;
        }
    }
}

void tune_save_locked() {
    const char* f = std::getenv("TCMIS_TUNE_CACHE");
    if (!f) return;
    std::ofstream out(f, std::ios::trunc);
    for (const auto& kv : g_tune_cache) {
        const TuneChoice& c = kv.second;
        out << kv.first << ' ' << c.path << ' ' << c.param << ' ' << c.bounds[0] << ' '
            << c.bounds[1] << ' ' << c.bounds[2] << ' ' << c.bounds[3] << ' ' << c.grid << ' '
            << c.ms << ' ' << c.pending << ' ' << c.range0 << ' ' << c.payload << '\n';
    }
}

// Distinct 8-column blocks of 8-row block rb: an 8-way merge of its sorted
// rows, stopped after kSampleArcs arcs (a hub row would make one thread walk
// it all); the tiles of the rest are extrapolated at the same rate.
constexpr int kSampleArcs = 64;

__global__ void tile_sample_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                   int32_t n, int32_t nrb, int count,
                                   unsigned long long* __restrict__ acc) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const int rb = (int)((long long)k * nrb / count);
    int cur[8], end[8];
    long long arcs = 0;
    for (int i = 0; i < 8; ++i) {
        const int v = rb * 8 + i;
        cur[i] = v < n ? rp[v] : 0;
        end[i] = v < n ? rp[v + 1] : 0;
        arcs += end[i] - cur[i];
    }
    // the column block of each row's next arc, kept in registers (one load
    // per arc consumed)
    int head[8];
    for (int i = 0; i < 8; ++i) head[i] = cur[i] < end[i] ? (col[cur[i]] >> 3) : INT32_MAX;
    long long tiles = 0, seen = 0;
    while (seen < kSampleArcs) {
        int cb = INT32_MAX;
        for (int i = 0; i < 8; ++i) cb = min(cb, head[i]);
        if (cb == INT32_MAX) break;
        ++tiles;
        for (int i = 0; i < 8; ++i)
            while (head[i] == cb) {
                ++cur[i];
                ++seen;
                head[i] = cur[i] < end[i] ? (col[cur[i]] >> 3) : INT32_MAX;
            }
    }
    if (seen > 0 && seen < arcs) tiles = (tiles * arcs + seen - 1) / seen;
    atomicAdd(&acc[0], (unsigned long long)arcs);
    atomicAdd(&acc[1], (unsigned long long)tiles);
}

// Estimated arcs per non-empty 8 x 8 tile, from up to 4096 row blocks spread
// evenly over the graph.
double estimate_arcs_per_tile(mis_graph* g) {
    GraphData& d = g->d;
    const int32_t nrb = (d.n + 7) / 8;
    if (nrb == 0 || d.arcs == 0) return 0.0;
    const int count = std::min<int32_t>(nrb, 4096);
    // the counters live in the graph's flag buffer: no allocation here
    unsigned long long* d_acc =
        reinterpret_cast<unsigned long long*>(reinterpret_cast<unsigned char*>(d.flags) +
                                              kSampleAccOffset);
    unsigned long long h[2] = {0, 0};
    cudaStream_t s = g->own_stream;
    cudaError_t e = cudaMemsetAsync(d_acc, 0, 16, s);
    if (e == cudaSuccess) {
        tile_sample_kernel<<<(count + 127) / 128, 128, 0, s>>>(d.rp, d.col, d.n, nrb, count, d_acc);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d_acc, 16, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || h[1] == 0) {
        cudaGetLastError();
        return 0.0;
    }
    return (double)h[0] / (double)h[1];
}

// The device's name with blanks as underscores, looked up once per device
// (cudaGetDeviceProperties takes hundreds of microseconds).
std::string device_name(int device) {
    static std::mutex mu;
    static std::map<int, std::string> names;
    std::lock_guard<std::mutex> lk(mu);
    auto it = names.find(device);
    if (it != names.end()) return it->second;
    cudaDeviceProp prop;
    std::string dev = "gpu";
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) dev = prop.name;
    for (char& c : dev)
        if (c == ' ') c = '_';
    names[device] = dev;
    return dev;
}

std::string density_class(mis_graph* g, double apt) {
    const GraphData& d = g->d;
    const double avg = d.n ? (double)d.arcs / d.n : 0.0;
    int deg_b = 0;
    while (deg_b < 20 && (1 << deg_b) <= avg) ++deg_b;
    int size_b = 0;
    while (size_b < 31 && (1ll << size_b) <= (long long)d.n) ++size_b;
    const char loc = apt < 1.5 ? 's' : (apt < 3.0 ? 'm' : 'd');
    const std::string dev = device_name(d.device);
    // graphs with create-time round-0 structures solve a different problem
    // size than graphs scanned from their full rows: tuned apart
    const int order = d.col_sel ? g->opt.order_rows : 0;
    return dev + ":d" + std::to_string(deg_b) + ":n" + std::to_string(size_b / 2) + ":" + loc +
           ":o" + std::to_string(order) + (d.s0_col ? "s" : "") + (d.count ? ":batch" : "") +
           (g->opt.priority ? ":p" + std::to_string(g->opt.priority) : std::string());
}

int apply_choice(mis_graph* g, const TuneChoice& c) {
    if (c.path == MIS_PATH_TILE_TC) g->tile_payload = c.payload;
    if (c.path == MIS_PATH_TILE || c.path == MIS_PATH_TILE_TC) return use_tiles(g, c.path, c.param);
    if (c.path == MIS_PATH_CLUSTER) {
        if (g->d.count != 0 || !cluster_plan(g->d.rp, g->d.n, &g->cluster))
            return set_error(MIS_EINVAL, "graph too large for one thread-block cluster");
        g->path = MIS_PATH_CLUSTER;
        return MIS_OK;
    }
    if (c.path == MIS_PATH_PUSH) {
        g->path = MIS_PATH_PUSH;
        return MIS_OK;
    }
    g->path = MIS_PATH_CSR;
    int32_t thr[4];
    if (c.param) {
        thresholds_for(c.param, thr);
    } else {
        for (int k = 0; k < 4; ++k) thr[k] = c.bounds[k];
    }
    g->tpr = c.param;
    g->csr_pending = c.pending;
    g->csr_range0 = c.range0;
    if (g->last_stream) cudaStreamSynchronize(g->last_stream);
    const int rc = rebin(g, thr, g->own_stream);
    if (rc != MIS_OK) return rc;
    g->grid = pick_grid(g, c.grid);
    return g->grid > 0 ? MIS_OK : set_error(MIS_EDEVICE, "no co-resident blocks");
}

// Median device time of `reps` solves (after one warm-up) in the handle's
// own workspace, in ms; negative on error.
float time_solves(mis_graph* g, int reps) {
    std::vector<uint64_t> seeds((size_t)std::max(1, g->d.count), 1);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    std::vector<float> ts;
    for (int i = 0; i <= reps; ++i) {
        cudaEventRecord(e0, g->own_stream);
        if (solve_async(g, seeds.data(), g->d.ws.out, g->own_stream) != MIS_OK) break;
        cudaEventRecord(e1, g->own_stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (i > 0) ts.push_back(ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaMemcpy(g->d.ctl_host, g->d.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    if ((int)ts.size() != reps || g->d.ctl_host->err != 0) return -1.f;
    std::sort(ts.begin(), ts.end());
    return ts[ts.size() / 2];
}

}  // namespace

int autotune(mis_graph* g, int reps, mis_tuning* out) {
    if (reps < 1) reps = 3;
    const double apt = estimate_arcs_per_tile(g);
    std::vector<TuneChoice> cands;
    auto bins = [&](int a, int b, int c, int d, int grid) {
        TuneChoice t;
        t.bounds[0] = a;
        t.bounds[1] = b;
        t.bounds[2] = c;
        t.bounds[3] = d;
        t.grid = grid;
        for (int pending : {0, 1}) {
            t.pending = pending;
            cands.push_back(t);
        }
    };
    const int maxg = csr_max_coresident_blocks(g->d.device);
    bins(8, 4096, 4096, 65536, 0);
    bins(8, 4096, 4096, 65536, maxg);
    bins(4, 64, 1024, 65536, 0);
    bins(16, 256, 4096, 65536, 0);
    bins(12, 48, 256, 4096, 0);
    bins(INT32_MAX - 1, INT32_MAX - 1, INT32_MAX - 1, INT32_MAX - 1, 0);  // one lane per row
    // smaller grids: fewer arrivals per grid barrier, for barrier-bound solves
    // (two and one blocks per SM at the kernel's three)
    if (maxg >= 3) {
        bins(8, 4096, 4096, 65536, maxg * 2 / 3);
        bins(8, 4096, 4096, 65536, maxg / 3);
        bins(INT32_MAX - 1, INT32_MAX - 1, INT32_MAX - 1, INT32_MAX - 1, maxg * 2 / 3);
    }
    bins(-1, 65536, 65536, 65536, 0);                                     // four lanes per row
    // without round-0 classes, round 0 can take bin 0 by vertex ranges (the
    // candidates above) or from its list
    if (!g->d.r0class) {
        const size_t k0 = cands.size();
        bins(8, 4096, 4096, 65536, 0);
        bins(4, 64, 1024, 65536, 0);
        bins(16, 256, 4096, 65536, 0);
        bins(32, 4096, 4096, 65536, 0);
        for (size_t k = k0; k < cands.size(); ++k) cands[k].range0 = 0;
        if (maxg >= 3) bins(8, 4096, 4096, 65536, maxg * 2 / 3);
    }
    if (g->d.n <= 65536) bins(8, 4096, 4096, 65536, std::max(1, (g->d.n + 1023) / 1024));
    {
        TuneChoice t;
        t.path = MIS_PATH_PUSH;
        cands.push_back(t);
    }
    if (g->d.count == 0 && g->d.n <= cluster_max_vertices()) {
        TuneChoice t;
        t.path = MIS_PATH_CLUSTER;
        cands.push_back(t);
    }
    if (apt >= 2.5) {
        for (int T : {8, 16}) {
            TuneChoice t;
            t.path = MIS_PATH_TILE;
            t.param = T;
            cands.push_back(t);
        }
        // the tensor-core forms; a stored payload only while it stays within
        // a quarter of the free device memory
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const int64_t est_tiles = (int64_t)((double)g->d.arcs / std::max(apt, 1.0));
        for (int pay : {MIS_TILE_BITS, MIS_TILE_BITS_B1, MIS_TILE_INT8, MIS_TILE_FP16}) {
            if ((pay == MIS_TILE_INT8 || pay == MIS_TILE_FP16) &&
                tile_payload_bytes(est_tiles, pay) > (int64_t)(free_b / 4))
                continue;
            TuneChoice t;
            t.path = MIS_PATH_TILE_TC;
            t.param = 16;
            t.payload = pay;
            cands.push_back(t);
        }
    }
    TuneChoice best;
    best.ms = -1.f;
    // TCMIS_TUNE_LOG set: every candidate's time on stderr
    const bool log = std::getenv("TCMIS_TUNE_LOG") != nullptr;
    for (TuneChoice& c : cands) {
        if (apply_choice(g, c) != MIS_OK) continue;
        c.ms = time_solves(g, reps);
        if (log)
            std::fprintf(stderr,
                         "tcmis tune: path %d param %d bounds %d %d %d %d grid %d pending %d "
                         "range0 %d payload %d: %.4f ms\n",
                         c.path, c.param, c.bounds[0], c.bounds[1], c.bounds[2], c.bounds[3],
                         c.path == MIS_PATH_CSR ? g->grid : g->tile_grid, c.pending, c.range0,
                         c.payload, c.ms);
        if (c.ms > 0.f && (best.ms < 0.f || c.ms < best.ms)) best = c;
    }
    if (best.ms < 0.f) return set_error(MIS_EINTERNAL, "autotuner found no working configuration");
    const int rc = apply_choice(g, best);
    if (rc != MIS_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        g_tune_cache[density_class(g, apt)] = best;
        tune_save_locked();
    }
    if (out) {
        out->path = best.path;
        out->param = best.param;
        for (int k = 0; k < 4; ++k) out->bounds[k] = best.bounds[k];
        out->grid = g->path == MIS_PATH_CSR ? g->grid : g->tile_grid;
        out->ms = best.ms;
        out->csr_pending = best.path == MIS_PATH_CSR ? best.pending : 0;
        out->csr_range0 = (best.path == MIS_PATH_CSR && !g->d.r0class) ? best.range0 : 0;
        out->tile_payload = best.path == MIS_PATH_TILE_TC ? best.payload : -1;
        out->arcs_per_tile = apt;
        out->candidates = (int32_t)cands.size();
    }
    return MIS_OK;
}

// AUTO at create: the cached choice of the graph's class, if any.
bool cached_choice(mis_graph* g, TuneChoice** out, bool* is_csr) {
    *out = nullptr;
    *is_csr = false;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load_locked();
        if (g_tune_cache.empty()) return false;
    }
    const std::string key = density_class(g, estimate_arcs_per_tile(g));
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it == g_tune_cache.end()) return false;
    *out = new TuneChoice(it->second);
    *is_csr = it->second.path == MIS_PATH_CSR;
    return true;
}

int apply_cached(mis_graph* g, TuneChoice* c) { return apply_choice(g, *c); }

void drop_choice(TuneChoice* c) { delete c; }

}  // namespace tcmis

using namespace tcmis;

extern "C" {

void mis_options_init(mis_options* opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->path = MIS_PATH_AUTO;
    opt->threads_per_row = 0;
    opt->check_symmetry = 1;
    opt->build_tiles = -1;
    opt->spin_cap = 0;
    opt->device = 0;
    opt->max_slots = 0;
    opt->hbm_budget = 0;
    opt->serve_blocks = 0;
    opt->order_rows = 1;
    opt->priority = MIS_PRIORITY_EQ1;
}

int mis_last_error(const char** msg) {
    if (msg) *msg = t_err_msg.c_str();
    return t_err_code;
}

const char* mis_version(void) { return "tcmis-gb300 0.1 (sm_103a)"; }

static bool valid_tpr(int t) {
    return t == 0 || t == 1 || t == 4 || t == 16 || t == 32 || t == 512;
}

mis_graph* mis_create_ex(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                         int32_t on_device, const mis_options* opt, void* stream) {
    clear_error();
    if (n < 0 || (n > 0 && !row_ptr)) {
        set_error(MIS_EINVAL, "n must be >= 0 and row_ptr non-null");
        return nullptr;
    }
    mis_options o;
    mis_options_init(&o);
    if (opt) o = *opt;
    if (!valid_tpr(o.threads_per_row)) {
        set_error(MIS_EINVAL, "threads_per_row must be 0, 1, 4, 16, 32 or 512");
        return nullptr;
    }
    if (o.priority < MIS_PRIORITY_EQ1 || o.priority > MIS_PRIORITY_EQ1_Q8) {
        set_error(MIS_EINVAL, "priority must be MIS_PRIORITY_EQ1, _HASH or _EQ1_Q8");
        return nullptr;
    }
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaSetDevice");
        return nullptr;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int64_t arcs = 0;
    if (n > 0) {
        int32_t last = 0;
        if (on_device) {
            e = cudaMemcpyAsync(&last, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                set_cuda_error(e, "reading row_ptr[n]");
                return nullptr;
            }
        } else {
            last = row_ptr[n];
        }
        arcs = last;
        if (arcs < 0) {
            set_error(MIS_EINVAL, "row_ptr[n] must be >= 0");
            return nullptr;
        }
        if (arcs > 0 && !col_idx) {
            set_error(MIS_EINVAL, "col_idx is null");
            return nullptr;
        }
    }
    mis_graph* g = new mis_graph();
    g->opt = o;
    GraphData& d = g->d;
    d.device = o.device;
    d.n = n;
    d.arcs = arcs;
    d.result_bytes = n;
    const int64_t col_alloc = ((arcs + 3) / 4) * 4 + 4;
    if ((e = dalloc(&d.rp, (int64_t)n + 1, &d.footprint)) != cudaSuccess ||
        (e = dalloc(&d.col, col_alloc, &d.footprint)) != cudaSuccess ||
        (e = dalloc(&d.flags, kFlagsBytes / sizeof(unsigned), &d.footprint)) != cudaSuccess) {
        set_cuda_error(e, "graph allocation");
        free_graph(g);
        return nullptr;
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    // only the padding after the last arc needs zeros (int4 loads read it)
    e = cudaMemsetAsync(d.col + arcs, 0, sizeof(int32_t) * (size_t)(col_alloc - arcs), s);
    if (e == cudaSuccess && n > 0)
        e = cudaMemcpyAsync(d.rp, row_ptr, sizeof(int32_t) * ((size_t)n + 1), kind, s);
    if (e == cudaSuccess && n == 0) e = cudaMemsetAsync(d.rp, 0, sizeof(int32_t), s);
    if (e != cudaSuccess) {
        set_cuda_error(e, "graph upload");
        free_graph(g);
        return nullptr;
    }
    StageLog lg;
    lg.mark("allocation", s);
    const bool pipelined = !on_device && !o.check_symmetry && arcs >= kUploadPiece;
    if (pipelined) {
        if (upload_checked(g, col_idx, s) != MIS_OK) {
            free_graph(g);
            return nullptr;
        }
    } else {
        if (arcs > 0)
            e = cudaMemcpyAsync(d.col, col_idx, sizeof(int32_t) * (size_t)arcs, kind, s);
        if (e != cudaSuccess) {
            set_cuda_error(e, "graph upload");
            free_graph(g);
            return nullptr;
        }
        lg.mark("upload", s);
        if (n > 0 && validate_device(g, s) != MIS_OK) {
            free_graph(g);
            return nullptr;
        }
        lg.mark("validation", s);
    }
    if (finish_create(g) != MIS_OK) {
        free_graph(g);
        return nullptr;
    }
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
        set_cuda_error(e, "create");
        free_graph(g);
        return nullptr;
    }
    return g;
}

mis_graph* mis_create(int32_t n, const int32_t* row_ptr, const int32_t* col_idx) {
    return mis_create_ex(n, row_ptr, col_idx, 0, nullptr, nullptr);
}

mis_graph* mis_create_batch(int32_t count, const int32_t* ns, const int32_t* const* row_ptrs,
                            const int32_t* const* col_idxs, const mis_options* opt) {
    clear_error();
    if (count < 1 || !ns || !row_ptrs || !col_idxs) {
        set_error(MIS_EINVAL, "count must be >= 1 with non-null arrays");
        return nullptr;
    }
    mis_options o;
    mis_options_init(&o);
    if (opt) o = *opt;
    if (!valid_tpr(o.threads_per_row)) {
        set_error(MIS_EINVAL, "threads_per_row must be 0, 1, 4, 16, 32 or 512");
        return nullptr;
    }
    if (o.priority < MIS_PRIORITY_EQ1 || o.priority > MIS_PRIORITY_EQ1_Q8) {
        set_error(MIS_EINVAL, "priority must be MIS_PRIORITY_EQ1, _HASH or _EQ1_Q8");
        return nullptr;
    }
    std::vector<int32_t> voff(count), nv(count), garcs(count);
    std::vector<int64_t> roff(count);
    int64_t N = 0, A = 0, R = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (ns[i] < 0 || (ns[i] > 0 && !row_ptrs[i])) {
            set_error(MIS_EINVAL, "graph " + std::to_string(i) + ": bad n or row_ptr");
            return nullptr;
        }
        const int64_t a = ns[i] ? row_ptrs[i][ns[i]] : 0;
        if (a < 0 || (a > 0 && !col_idxs[i]) || (ns[i] > 0 && row_ptrs[i][0] != 0)) {
            set_error(MIS_EINVAL, "graph " + std::to_string(i) + ": bad row_ptr or col_idx");
            return nullptr;
        }
        voff[i] = (int32_t)N;
        nv[i] = ns[i];
        garcs[i] = (int32_t)a;
        roff[i] = R;
        N += ((int64_t)ns[i] + 15) / 16 * 16;
        A += a;
        R += ns[i];
        if (N > INT32_MAX - 16 || A > INT32_MAX - 16) {
            set_error(MIS_EINVAL, "batch exceeds 2^31 vertices or arcs");
            return nullptr;
        }
    }
    cudaError_t e = cudaSetDevice(o.device);
    if (e != cudaSuccess) {
        set_cuda_error(e, "cudaSetDevice");
        return nullptr;
    }
    mis_graph* g = new mis_graph();
    g->opt = o;
    GraphData& d = g->d;
    d.device = o.device;
    d.n = (int32_t)N;
    d.arcs = A;
    d.count = count;
    d.result_bytes = R;
    d.h_nv = nv;
    if ((e = cudaStreamCreateWithFlags(&g->own_stream, cudaStreamNonBlocking)) != cudaSuccess) {
        set_cuda_error(e, "stream");
        free_graph(g);
        return nullptr;
    }
    cudaStream_t s = g->own_stream;
    const int64_t col_alloc = ((A + 3) / 4) * 4 + 4;
    const int64_t nblk = N / 16;
    if ((e = dalloc(&d.rp, N + 1, &d.footprint)) != cudaSuccess ||
        (e = dalloc(&d.col, col_alloc, &d.footprint)) != cudaSuccess ||
        (e = dalloc(&d.flags, kFlagsBytes / sizeof(unsigned), &d.footprint)) != cudaSuccess ||
        (e = dalloc(&d.blk_seg, nblk, &d.footprint)) != cudaSuccess ||
        (e = dalloc(&d.voff, count, &d.footprint)) != cudaSuccess ||
        (e = dalloc(&d.nv, count, &d.footprint)) != cudaSuccess ||
        (e = dalloc(&d.garcs, count, &d.footprint)) != cudaSuccess ||
        (e = dalloc(&d.roff, count, &d.footprint)) != cudaSuccess ||
        !(d.seeds_host = static_cast<uint64_t*>(host_small_alloc(sizeof(uint64_t) * (size_t)count)))) {
        if (e == cudaSuccess) e = cudaErrorMemoryAllocation;
        set_cuda_error(e, "batch allocation");
        free_graph(g);
        return nullptr;
    }
    e = cudaMemsetAsync(d.col, 0, sizeof(int32_t) * (size_t)col_alloc, s);
    int64_t aoff = 0;
    for (int32_t i = 0; i < count && e == cudaSuccess; ++i) {
        const int32_t ni = ns[i];
        const int32_t ai = garcs[i];
        if (ni > 0)
            e = cudaMemcpyAsync(d.rp + voff[i], row_ptrs[i], sizeof(int32_t) * (size_t)ni,
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && ai > 0)
            e = cudaMemcpyAsync(d.col + aoff, col_idxs[i], sizeof(int32_t) * (size_t)ai,
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = launch_relocate(d.rp + voff[i], d.col + aoff, ni, ai, voff[i], (int32_t)aoff, s);
        const int32_t pad_to = (i + 1 < count) ? voff[i + 1] : (int32_t)N;
        if (e == cudaSuccess)
            e = launch_pad_rows(d.rp, voff[i] + ni, pad_to + (i + 1 == count ? 1 : 0),
                                (int32_t)(aoff + ai), s);
        aoff += ai;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.voff, voff.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.nv, nv.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.garcs, garcs.data(), sizeof(int32_t) * count,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.roff, roff.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice,
                            s);
    if (e == cudaSuccess) e = launch_fill_seg(d.blk_seg, d.voff, count, (int32_t)nblk, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        set_cuda_error(e, "batch upload");
        free_graph(g);
        return nullptr;
    }
    // each graph must stay inside its own vertex range
    for (int32_t i = 0; i < count; ++i) {
        const int32_t* rp = row_ptrs[i];
        const int32_t* col = col_idxs[i];
        for (int32_t v = 0; v < ns[i]; ++v)
            if (rp[v] > rp[v + 1]) {
                set_error(MIS_EINVAL, "graph " + std::to_string(i) + ": row_ptr not monotone");
                free_graph(g);
                return nullptr;
            }
        for (int32_t p = 0; p < garcs[i]; ++p)
            if (col[p] < 0 || col[p] >= ns[i]) {
                set_error(MIS_EINVAL, "graph " + std::to_string(i) + ": col_idx out of range");
                free_graph(g);
                return nullptr;
            }
    }
    if (N > 0 && validate_device(g, s) != MIS_OK) {
        free_graph(g);
        return nullptr;
    }
    if (finish_create(g) != MIS_OK) {
        free_graph(g);
        return nullptr;
    }
    return g;
}

int32_t mis_graph_count(const mis_graph* g) { return g ? (g->d.count ? g->d.count : 1) : 0; }

int64_t mis_result_size(const mis_graph* g) { return g ? g->d.result_bytes : 0; }

int64_t mis_footprint(const mis_graph* g) { return g ? g->d.footprint : 0; }

int mis_set_path(mis_graph* g, int32_t path, int32_t threads_per_row) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    if ((path == MIS_PATH_CSR || path == MIS_PATH_AUTO) && !valid_tpr(threads_per_row))
        return set_error(MIS_EINVAL, "bad threads_per_row");
    if (path < MIS_PATH_AUTO || path > MIS_PATH_CLUSTER)
        return set_error(MIS_EINVAL, "unknown path");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    if (path == MIS_PATH_TILE || path == MIS_PATH_TILE_TC)
        return use_tiles(g, path, threads_per_row ? threads_per_row : 16);
    if (path == MIS_PATH_PUSH) {
        g->path = MIS_PATH_PUSH;
        return MIS_OK;
    }
    if (path == MIS_PATH_CLUSTER) {
        if (g->d.count != 0) return set_error(MIS_EINVAL, "the cluster path takes a single graph");
        if (!cluster_plan(g->d.rp, g->d.n, &g->cluster))
            return set_error(MIS_EINVAL, "graph too large for one thread-block cluster");
        g->path = MIS_PATH_CLUSTER;
        return MIS_OK;
    }
    g->path = MIS_PATH_CSR;
    if (threads_per_row == g->tpr) return MIS_OK;
    g->tpr = threads_per_row;
    int32_t thr[4];
    thresholds_for(g->tpr, thr);
    if (g->last_stream) cudaStreamSynchronize(g->last_stream);
    return rebin(g, thr, g->own_stream);
}

int mis_set_csr_bins(mis_graph* g, const int32_t* bounds) {
    clear_error();
    if (!g || !bounds) return set_error(MIS_EINVAL, "null argument");
    if (!(bounds[0] <= bounds[1] && bounds[1] <= bounds[2] && bounds[2] <= bounds[3]))
        return set_error(MIS_EINVAL, "bin bounds must be non-decreasing");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    if (g->last_stream) cudaStreamSynchronize(g->last_stream);
    g->tpr = 0;
    g->path = MIS_PATH_CSR;
    return rebin(g, bounds, g->own_stream);
}

int mis_set_csr_pending(mis_graph* g, int32_t pending) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    if (pending != 0 && pending != 1) return set_error(MIS_EINVAL, "pending must be 0 or 1");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    g->csr_pending = pending;
    return MIS_OK;
}

int mis_tile_payload_ex(mis_graph* g, int32_t payload, void* out, void* stream) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    if (payload < MIS_TILE_BITS || payload > MIS_TILE_FP16)
        return set_error(MIS_EINVAL, "unknown tile payload");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    GraphData& d = g->d;
    cudaError_t e = cudaSetDevice(d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    if (d.tiles.T != 16) {
        const int32_t keep = g->path;
        const int rc = use_tiles(g, MIS_PATH_TILE, 16);
        if (rc != MIS_OK) return rc;
        g->path = keep;
    }
    const bool stored = payload == MIS_TILE_INT8 || payload == MIS_TILE_FP16;
    if (stored && d.tpay_kind != payload) {
        if (g->last_stream) cudaStreamSynchronize(g->last_stream);
        free_payload(d);
        void* p = nullptr;
        e = build_tile_payload(d.tiles, payload, &p, g->own_stream);
        if (e != cudaSuccess) return set_cuda_error(e, "tile payload");
        d.tpay = p;
        d.tpay_kind = payload;
        d.footprint += tile_payload_bytes(d.tiles.ntiles, payload);
    }
    if (!out) return MIS_OK;
    const int64_t bytes = stored ? tile_payload_bytes(d.tiles.ntiles, payload) : 32 * d.tiles.ntiles;
    if (bytes > 0)
        e = cudaMemcpyAsync(out, stored ? d.tpay : (const void*)d.tiles.tbits, (size_t)bytes,
                            cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_cuda_error(e, "tile payload copy");
    return MIS_OK;
}

int mis_set_tile_payload(mis_graph* g, int32_t payload) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    if (payload < MIS_TILE_BITS || payload > MIS_TILE_FP16)
        return set_error(MIS_EINVAL, "unknown tile payload");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    g->tile_payload = payload;
    // a graph already on the tensor-core path switches now (and builds the
    // stored payload if the form reads one)
    if (g->path == MIS_PATH_TILE_TC) return use_tiles(g, MIS_PATH_TILE_TC, 16);
    return MIS_OK;
}

int mis_set_multi_form(mis_graph* g, int32_t form) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    if (form != MIS_MULTI_ROWS && form != MIS_MULTI_ROWS_TC)
        return set_error(MIS_EINVAL, "unknown multi-seed form");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    if (form == MIS_MULTI_ROWS_TC && (g->d.count != 0 || g->d.r0class || g->d.out0 || g->d.s0_col))
        return set_error(MIS_EINVAL,
                         "the tensor-core multi-seed form takes a single graph created "
                         "without round-0 structures (order_rows = 0)");
    g->multi_form = form;
    g->multi_tc_fill = 32;
    return MIS_OK;
}

int mis_autotune_multi(mis_graph* g, int32_t k, int32_t reps, int32_t* form) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    if (k < 1 || k > kMaxMulti) return set_error(MIS_EINVAL, "k must be in [1, 8]");
    if (g->d.count != 0) return set_error(MIS_EINVAL, "multi-seed solves take a single graph");
    if (reps <= 0) reps = 3;
    GraphData& d = g->d;
    bool tc_ok;
    {
        std::lock_guard<std::mutex> lk(g->mu);
        if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
        tc_ok = d.n > 0 && !d.r0class && !d.out0 && !d.s0_col && g->path != MIS_PATH_TILE_TC &&
                !(g->path == MIS_PATH_TILE && d.tiles.T != 16);
        if (!tc_ok) g->multi_form = MIS_MULTI_ROWS;
    }
    if (!tc_ok) {
        if (form) *form = MIS_MULTI_ROWS;
        return MIS_OK;
    }
    cudaError_t e = cudaSetDevice(d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    int64_t scratch_bytes = 0;
    uint8_t* out = nullptr;
    if ((e = dalloc(&out, (int64_t)k * d.n, &scratch_bytes)) != cudaSuccess)
        return set_cuda_error(e, "autotune output");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    uint64_t seeds[kMaxMulti];
    for (int i = 0; i < kMaxMulti; ++i) seeds[i] = (uint64_t)i + 1;
    const cudaStream_t s = g->own_stream;
    // the CSR rows, then the tensor-core form with its switch at three fills:
    // while 1/8, 3/8 or 25/32 of the listed entries are undecided (the last
    // is in practice round 0 only)
    const int32_t forms[4] = {MIS_MULTI_ROWS, MIS_MULTI_ROWS_TC, MIS_MULTI_ROWS_TC,
                              MIS_MULTI_ROWS_TC};
    const int32_t fills[4] = {32, 32, 96, 200};
    float best_ms = 0.f;
    int32_t best = MIS_MULTI_ROWS, best_fill = 32;
    int rc = MIS_OK;
    for (int f = 0; f < 4 && rc == MIS_OK; ++f) {
        {
            std::lock_guard<std::mutex> lk(g->mu);
            g->multi_form = forms[f];
            g->multi_tc_fill = fills[f];
        }
        // the first solve builds what the form needs (tiles, bit vectors)
        rc = mis_solve_multi_ex(g, k, seeds, out, s);
        std::vector<float> ms;
        for (int r = 0; r < reps && rc == MIS_OK; ++r) {
            cudaEventRecord(e0, s);
            rc = mis_solve_multi_ex(g, k, seeds, out, s);
            cudaEventRecord(e1, s);
            if ((e = cudaEventSynchronize(e1)) != cudaSuccess) {
                rc = set_cuda_error(e, "autotune timing");
                break;
            }
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            ms.push_back(t);
        }
        if (rc != MIS_OK) break;
        std::sort(ms.begin(), ms.end());
        const float med = ms[ms.size() / 2];
        if (f == 0 || med < best_ms) {
            best_ms = med;
            best = forms[f];
            best_fill = fills[f];
        }
    }
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    dfree(out);
    {
        std::lock_guard<std::mutex> lk(g->mu);
        g->multi_form = rc == MIS_OK ? best : MIS_MULTI_ROWS;
        g->multi_tc_fill = rc == MIS_OK ? best_fill : 32;
    }
    if (rc != MIS_OK) return rc;
    if (form) *form = best;
    return MIS_OK;
}

int mis_set_csr_range0(mis_graph* g, int32_t on) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    if (on != 0 && on != 1) return set_error(MIS_EINVAL, "range0 must be 0 or 1");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    g->csr_range0 = on;
    return MIS_OK;
}

int mis_autotune(mis_graph* g, int32_t reps, mis_tuning* chosen) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    if (g->d.n == 0) return MIS_OK;
    return autotune(g, reps, chosen);
}

int mis_set_grid(mis_graph* g, int32_t blocks) {
    clear_error();
    if (!g || blocks < 0) return set_error(MIS_EINVAL, "null graph or negative block count");
    std::lock_guard<std::mutex> lk(g->mu);
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    g->grid = pick_grid(g, blocks);
    return g->grid > 0 ? MIS_OK : set_error(MIS_EDEVICE, "no co-resident blocks");
}

int32_t mis_get_grid(const mis_graph* g) { return g ? g->grid : 0; }

int32_t mis_cluster_max_vertices(void) {
    clear_error();
    return cluster_max_vertices();
}

int mis_tiles_ex(mis_graph* g, int32_t* trp, int32_t* tcol, uint64_t* tbits, void* stream) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    std::lock_guard<std::mutex> lk(g->mu);
    const TileCsr& t = g->d.tiles;
    if (t.T == 0) return set_error(MIS_EINVAL, "no tile-CSR built (select a tile path first)");
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e == cudaSuccess && trp)
        e = cudaMemcpyAsync(trp, t.trp, 4 * ((size_t)t.nrb + 1), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && tcol && t.ntiles)
        e = cudaMemcpyAsync(tcol, t.tcol, 4 * (size_t)t.ntiles, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && tbits && t.ntiles)
        e = cudaMemcpyAsync(tbits, t.tbits, 8 * (size_t)(t.T * t.T / 64) * (size_t)t.ntiles,
                            cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return set_cuda_error(e, "tile export");
    return MIS_OK;
}

int mis_solve_ex(mis_graph* g, const uint64_t* seeds, uint8_t* out_status, void* stream) {
    clear_error();
    if (!g || !seeds) return set_error(MIS_EINVAL, "null graph or seeds");
    if (g->d.result_bytes > 0 && !out_status) return set_error(MIS_EINVAL, "null out_status");
    std::lock_guard<std::mutex> lk(g->mu);
    return solve_async(g, seeds, out_status, (cudaStream_t)stream);
}

int mis_solve(mis_graph* g, uint64_t seed, uint8_t* out_status) {
    clear_error();
    if (!g) return set_error(MIS_EINVAL, "null graph");
    if (g->d.result_bytes > 0 && !out_status) return set_error(MIS_EINVAL, "null out_status");
    std::lock_guard<std::mutex> lk(g->mu);
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    if (!g->own_stream) {
        e = cudaStreamCreateWithFlags(&g->own_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return set_cuda_error(e, "stream");
    }
    std::vector<uint64_t> seeds((size_t)std::max(1, g->d.count));
    for (size_t i = 0; i < seeds.size(); ++i) seeds[i] = seed + i;
    int rc = solve_async(g, seeds.data(), g->d.ws.out, g->own_stream);
    if (rc != MIS_OK) return rc;
    if (g->d.result_bytes > 0) {
        e = cudaMemcpyAsync(out_status, g->d.ws.out, (size_t)g->d.result_bytes,
                            cudaMemcpyDeviceToHost, g->own_stream);
        if (e != cudaSuccess) return set_cuda_error(e, "result download");
    }
    e = cudaMemcpyAsync(g->d.ctl_host, g->d.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                        g->own_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(g->own_stream);
    if (e != cudaSuccess) return set_cuda_error(e, "solve");
    if (g->d.ctl_host->err == kErrTimedOut)
        return set_error(MIS_ETIMEDOUT, "device barrier wait exceeded its spin limit");
    if (g->d.ctl_host->err != 0)
        return set_error(MIS_EINTERNAL, "round cap exceeded");
    return MIS_OK;
}

int mis_get_stats(mis_graph* g, mis_stats* st) {
    clear_error();
    if (!g || !st) return set_error(MIS_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(g->mu);
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e == cudaSuccess && g->last_stream) e = cudaStreamSynchronize(g->last_stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d.ctl_host, g->d.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(g->d.times_host, g->d.ws.times, sizeof(PhaseTimes), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return set_cuda_error(e, "stats");
    const Ctl& c = *g->d.ctl_host;
    const PhaseTimes& tm = *g->d.times_host;
    std::memset(st, 0, sizeof(*st));
    st->rounds = c.rounds;
    st->path = g->last_path;
    st->threads_per_row = g->tpr;
    st->tile = g->d.tiles.T;
    st->csr_pending = g->csr_pending;
    st->tile_payload = g->last_path == MIS_PATH_TILE_TC ? g->tile_payload : -1;
    const bool csr = g->last_path == MIS_PATH_CSR;
    st->sure_in = csr ? g->d.n_sure_in : 0;
    st->sure_out = csr ? g->d.n_sure_out : 0;
    st->tested_arcs = !csr ? 0 : g->d.s0_col ? g->d.s0_arcs : -1;
    st->keyed = !csr ? 0 : g->d.out0 ? g->d.n_keyed : -1;
    st->tested_rows = !csr ? 0 : g->d.out0 ? g->d.n_tested : -1;
    st->tested_prefix_arcs = !csr ? 0 : g->d.out0 ? g->d.tested_prefix_arcs : -1;
    st->ntiles = g->d.tiles.ntiles;
    st->alive_sum = (int64_t)c.alive_sum;
    st->mis_size = (int64_t)c.mis_size;
    for (int r = 0; r < 64 && r < kStatRounds; ++r) st->alive_per_round[r] = c.alive[r];
    auto span = [&](int a, int b) -> int64_t {
        return (tm.t[a] && tm.t[b] && tm.t[b] >= tm.t[a]) ? (int64_t)(tm.t[b] - tm.t[a]) : 0;
    };
    st->init_ns = span(0, 1);
    for (int r = 0; r < 64 && r < kStatRounds && r < c.rounds; ++r) {
        const int start = r == 0 ? 1 : 2 + kStatRounds + r - 1;
        st->select_ns[r] = span(start, 2 + r);
        st->exclude_ns[r] = span(2 + r, 2 + kStatRounds + r);
    }
    st->status = c.err == 0 ? MIS_OK : (c.err == kErrTimedOut ? MIS_ETIMEDOUT : MIS_EINTERNAL);
    if (st->status != MIS_OK)
        return set_error(st->status, st->status == MIS_ETIMEDOUT
                                         ? "device barrier wait exceeded its spin limit"
                                         : "round cap exceeded");
    return MIS_OK;
}

int mis_keys_ex(mis_graph* g, const uint64_t* seeds, uint32_t* out_key, void* stream) {
    clear_error();
    if (!g || !seeds || (g->d.result_bytes > 0 && !out_key))
        return set_error(MIS_EINVAL, "null argument");
    std::lock_guard<std::mutex> lk(g->mu);
    GraphData& d = g->d;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSetDevice(d.device);
    SolveArgs a = make_args(g, d.ws);
    if (d.count == 0) {
        a.seed0 = seeds[0];
    } else if (e == cudaSuccess) {
        std::memcpy(d.seeds_host, seeds, sizeof(uint64_t) * (size_t)d.count);
        e = cudaMemcpyAsync(d.ws.seeds, d.seeds_host, sizeof(uint64_t) * (size_t)d.count,
                            cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) e = launch_keys(a, out_key, s);
    if (e != cudaSuccess) return set_cuda_error(e, "keys");
    g->last_stream = s;
    return MIS_OK;
}

int mis_solve_multi_ex(mis_graph* g, int32_t k, const uint64_t* seeds, uint8_t* out_status,
                       void* stream) {
    clear_error();
    if (!g || !seeds) return set_error(MIS_EINVAL, "null graph or seeds");
    if (k < 1 || k > kMaxMulti) return set_error(MIS_EINVAL, "k must be in [1, 8]");
    if (g->d.count != 0) return set_error(MIS_EINVAL, "multi-seed solves take a single graph");
    if (g->d.n > 0 && !out_status) return set_error(MIS_EINVAL, "null out_status");
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    GraphData& d = g->d;
    cudaError_t e = cudaSetDevice(d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    if (!d.word8) {
        if (g->last_stream) cudaStreamSynchronize(g->last_stream);
        const int64_t cap = (d.n + 15) / 16 * 16;
        if ((e = dalloc(&d.word8, (int64_t)kMaxMulti * cap, &d.footprint)) != cudaSuccess)
            return set_cuda_error(e, "multi-seed workspace");
    }
    if (g->path == MIS_PATH_TILE_TC) {
        // the solves as right-hand sides of the tensor-core exclusion
        const int32_t words = tile_multi_bitvector_words(d.tiles.nrb);
        if (!d.inb8) {
            if (g->last_stream) cudaStreamSynchronize(g->last_stream);
            if ((e = dalloc(&d.inb8, (int64_t)kMaxMulti * words, &d.footprint)) != cudaSuccess)
                return set_cuda_error(e, "multi-seed workspace");
        }
        MultiSeeds ms{};
        for (int i = 0; i < k; ++i) ms.seed[i] = seeds[i];
        SolveArgs a = make_args(g, d.ws);
        a.out = out_status;
        cudaStream_t s = (cudaStream_t)stream;
        e = reset_control(d.ws, s);
        if (e != cudaSuccess) return set_cuda_error(e, "control reset");
        if (d.n > 0) {
            const int maxb = tile_multi_max_coresident_blocks(g->tile_payload, d.device);
            if (maxb <= 0) return set_error(MIS_EDEVICE, "no co-resident blocks for the kernel");
            const long long want = std::max<long long>(1, ((long long)d.tiles.nrb + 63) / 64);
            e = launch_tile_multi_solve(a, d.word8, d.inb8, k, ms, g->tile_payload,
                                        (int)std::min<long long>(want, maxb), s);
            if (e != cudaSuccess) return set_cuda_error(e, "multi-seed tile kernel launch");
        }
        g->last_stream = s;
        g->last_path = MIS_PATH_TILE_TC;
        return MIS_OK;
    }
    if (g->multi_form == MIS_MULTI_ROWS_TC) {
        // selection on the CSR rows, exclusion on the 16 x 16 bitmask tiles
        // with the solves as the single-bit MMA's right-hand sides
        if (g->path == MIS_PATH_TILE && d.tiles.T != 16)
            return set_error(MIS_EINVAL, "the graph's single solves use 8 x 8 tiles; "
                                         "set another path before this multi-seed form");
        if (d.tiles.T != 16) {
            if (g->last_stream) cudaStreamSynchronize(g->last_stream);
            free_tiles(d);
            e = build_tiles(d.rp, d.col, d.n, d.arcs, 16, &d.tiles, g->own_stream);
            if (e != cudaSuccess) {
                free_tiles(d);
                return set_cuda_error(e, "tile-CSR conversion");
            }
            d.tile_footprint = 4 * ((int64_t)d.tiles.nrb + 1) + 4 * d.tiles.ntiles +
                               32 * (int64_t)d.tiles.ntiles;
            d.footprint += d.tile_footprint;
        }
        const int32_t words = tile_multi_bitvector_words(d.tiles.nrb);  // 8 * words >= 4 * nrb
        if (!d.inb8) {
            if (g->last_stream) cudaStreamSynchronize(g->last_stream);
            if ((e = dalloc(&d.inb8, (int64_t)kMaxMulti * words, &d.footprint)) != cudaSuccess)
                return set_cuda_error(e, "multi-seed workspace");
        }
        MultiSeeds ms{};
        for (int i = 0; i < k; ++i) ms.seed[i] = seeds[i];
        SolveArgs a = make_args(g, d.ws);
        a.out = out_status;
        cudaStream_t s = (cudaStream_t)stream;
        e = reset_control(d.ws, s);
        if (e != cudaSuccess) return set_cuda_error(e, "control reset");
        if (d.n > 0) {
            const int maxb = multi_rows_tc_max_coresident_blocks(d.device);
            if (maxb <= 0) return set_error(MIS_EDEVICE, "no co-resident blocks for the kernel");
            const long long want = std::max<long long>(1, ((long long)d.n + 255) / 256);
            // the sparse-tile split pays only where a row block's tiles
            // take more than one MMA (more than eight tiles on average)
            const bool split = d.tiles.ntiles > 8LL * d.tiles.nrb;
            e = launch_multi_rows_tc_solve(a, d.word8, d.inb8, k, ms, g->multi_tc_fill, split,
                                           (int)std::min<long long>(want, maxb), s);
            if (e != cudaSuccess) return set_cuda_error(e, "multi-seed rows-tc kernel launch");
        }
        g->last_stream = s;
        g->last_path = MIS_PATH_ROWS_TC;
        return MIS_OK;
    }
    const int rc = solve_multi_in(g, d.ws, d.word8, k, seeds, out_status, (cudaStream_t)stream, 0);
    if (rc != MIS_OK) return rc;
    g->last_stream = (cudaStream_t)stream;
    g->last_path = MIS_PATH_CSR;
    return MIS_OK;
}

int mis_capture(mis_graph* g, const uint64_t* seeds, uint8_t* out_status, mis_replay** replay) {
    clear_error();
    if (!g || !seeds || !replay) return set_error(MIS_EINVAL, "null argument");
    if (g->d.result_bytes > 0 && !out_status) return set_error(MIS_EINVAL, "null out_status");
    *replay = nullptr;
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    auto* r = new (std::nothrow) mis_replay();
    if (!r) return set_error(MIS_ENOMEM, "replay");
    r->g = g;
    r->path = g->path;
    const int count = std::max(1, g->d.count);
    cudaStream_t cs = nullptr;
    e = cudaMallocHost((void**)&r->seeds_pinned, sizeof(uint64_t) * (size_t)count);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        mis_replay_destroy(r);
        return set_cuda_error(e, "capture setup");
    }
    // the graph's memcpy node reads this private pinned copy at every replay
    std::memcpy(r->seeds_pinned, seeds, sizeof(uint64_t) * (size_t)count);
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc = MIS_OK;
    if (e == cudaSuccess) {
        rc = solve_in(g, g->d.ws, r->seeds_pinned, r->seeds_pinned, out_status, cs, 0);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
        r->graph = graph;
        if (rc == MIS_OK && ee != cudaSuccess) rc = set_cuda_error(ee, "stream capture");
    } else {
        rc = set_cuda_error(e, "stream capture");
    }
    if (rc == MIS_OK) {
        e = cudaGraphInstantiate(&r->exec, r->graph, 0);
        if (e != cudaSuccess) rc = set_cuda_error(e, "graph instantiation");
    }
    cudaStreamDestroy(cs);
    if (rc != MIS_OK) {
        mis_replay_destroy(r);
        return rc;
    }
    r->counted = true;
    g->replays.fetch_add(1);
    *replay = r;
    return MIS_OK;
}

int mis_replay_launch(mis_replay* r, void* stream) {
    clear_error();
    if (!r || !r->exec) return set_error(MIS_EINVAL, "null replay");
    mis_graph* g = r->g;
    std::lock_guard<std::mutex> lk(g->mu);
    if (g->inflight.load() > 0) return set_error(MIS_EBUSY, "served requests in flight");
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e == cudaSuccess) e = cudaGraphLaunch(r->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_cuda_error(e, "graph launch");
    g->last_stream = (cudaStream_t)stream;
    g->last_path = r->path;
    return MIS_OK;
}

void mis_replay_destroy(mis_replay* r) {
    if (!r) return;
    if (r->g) cudaSetDevice(r->g->d.device);
    if (r->exec) cudaGraphExecDestroy(r->exec);
    if (r->graph) cudaGraphDestroy(r->graph);
    if (r->seeds_pinned) cudaFreeHost(r->seeds_pinned);
    if (r->counted && r->g) r->g->replays.fetch_sub(1);
    delete r;
}

void mis_destroy(mis_graph* g) {
    if (!g) return;
    serve_release_graph(g);  // frees now, or after its last served request
}

}  // extern "C"
