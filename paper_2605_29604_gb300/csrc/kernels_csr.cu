// kernels_csr.cu -- the CSR round kernel on CUDA cores (the plain GPU form).
//
// One cooperative, persistent launch runs a whole solve:
//
//   init      Eq. 1 priority of every vertex into its packed word (Sec. 2:
//             priorities assigned once and reused every round)
//   rounds    Algorithm 2's while-loop; each round has two phases over the
//             worklist W_r of undecided vertices, separated by grid barriers:
//               Phase 1  selection test: v is a candidate when no undecided
//                        neighbour outranks it (C(v) = [P(v) > Max_Np(v)]);
//                        candidates are marked in the MIS in place.
//               Phase 2+3 exclusion test and state update: an undecided
//                        non-candidate with a candidate neighbour (N_c(v) > 0)
//                        is marked out; the others form W_{r+1} (compaction).
//             Both phases read only what the round-start snapshot fixes (see
//             common.cuh), so rounds and alive-set sizes match Algorithm 2.
//   output    result bytes out[v] = [v in the MIS].
//
// Worklists hold row records {v, row begin, end of the selection prefix, row
// end} and are split into degree bins (fixed at create time, degrees do not
// change): bin j holds the vertices with deg in (thr[j-1], thr[j]].  Bins 0..3
// are scanned by groups of 1, 4, 16 and 32 lanes (a lane of a 1-lane group
// scans several rows at once), bin 4 (hubs) by a whole block.  Each warp
// takes its first chunk of a bin by its index and further chunks through the
// bin's counter.  Phase 2 either scans a pending list of Phase 1's
// non-candidates or triages W_r one vertex per lane (candidates need no scan);
// survivors are staged in shared memory and appended to the next list with
// one atomic per chunk.  Lanes load 16-byte aligned int4 slices of col_idx
// and gather the four neighbour words; scans stop at the first neighbour that
// decides the test.
#include <algorithm>

#include <cub/cub.cuh>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "init.cuh"
#include "internal.h"
#include "worklist.cuh"

namespace tcmis {

constexpr int kCsrBlock = 512;
constexpr int kCsrMinBlocksPerSm = 3;
// Rows scanned at once by one lane when a row has one lane (the scans are
// bound by load latency, so independent rows per lane add loads in flight).
constexpr int kRowsPerLane = 2;
constexpr int kWarps = kCsrBlock / 32;
// A worklist of at most this many rows (after round 0) is finished by one
// block: its rounds then cost two block-wide barriers instead of two grid
// barriers, which on a grid of hundreds of blocks take microseconds each.
constexpr int kSoloRows = 512;
// ... in the triage form of the kernel; the pending form keeps the grid (at
// its register budget the switch costs it spills in the scans).
template <bool kPending>
constexpr bool kSoloPath = !kPending;

// Most rows per chunk taken by one warp, per bin (bin 4 is taken a row at a
// time by a whole block).  A bin of up to nwarps * CH rows is split into equal
// static chunks, one per warp, with no counter atomics; larger bins hand out
// further chunks through the bin's counter.  Same-address atomics serialise in
// L2, so few large chunks beat many small ones here.
constexpr int kChunk0 = 1024, kChunk1 = 512, kChunk2 = 256, kChunk3 = 128;
constexpr int kScanMax = 256;   // rows triaged at once in Phase 2

// Does u outrank v in the selection test?  `wu` is u's word, `wv` v's
// (undecided, so wv is v's key): out words never outrank, undecided ones
// compare by key then id, an in word (a candidate of this round) always does.
__device__ __forceinline__ bool outranks(uint32_t wu, int u, uint32_t wv, int v) {
    return wu > wv || (wu == wv && u > v);
}

// Neighbour words as they stand (through L1: see ld_word_l1).
struct LiveWords {
    const uint32_t* word;
    __device__ __forceinline__ uint32_t operator()(int u) const { return ld_word_l1(word + u); }
};

// Scan of the row [b, e) of v by the group of TPR lanes of this lane; kSelect:
// is there a neighbour that outranks v, else: is there an in neighbour.
// Warp-uniform loop: every lane of the warp iterates until no group has work.
template <int TPR, bool kSelect, class Words>
__device__ __forceinline__ bool group_scan(const int32_t* __restrict__ col, Words nbw, int b,
                                           int e, int v, uint32_t wv, unsigned glane,
                                           unsigned gshift) {
    constexpr unsigned gbits = (TPR == 32) ? 0xFFFFFFFFu : ((1u << TPR) - 1u);
    bool found = false;
    int p0 = (b & ~3) + 4 * (int)glane;
    for (;;) {
        bool hit = false;
        if (!found && p0 < e) {
            const int4 c = __ldg(reinterpret_cast<const int4*>(col + p0));
            const uint32_t w0 = (p0 >= b) ? nbw(c.x) : 0u;
            const uint32_t w1 = (p0 + 1 >= b && p0 + 1 < e) ? nbw(c.y) : 0u;
            const uint32_t w2 = (p0 + 2 >= b && p0 + 2 < e) ? nbw(c.z) : 0u;
            const uint32_t w3 = (p0 + 3 >= b && p0 + 3 < e) ? nbw(c.w) : 0u;
            if (kSelect) {
                hit = outranks(w0, c.x, wv, v) | outranks(w1, c.y, wv, v) |
                      outranks(w2, c.z, wv, v) | outranks(w3, c.w, wv, v);
            } else {
                hit = max(max(w0, w1), max(w2, w3)) >= kWordInMin;
            }
        }
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, hit);
        found = found || ((bal >> gshift) & gbits) != 0u;
        p0 += 4 * TPR;
        const bool more = !found && (p0 - 4 * (int)glane) < e;
        if (!__any_sync(0xFFFFFFFFu, more)) break;
    }
    return found;
}

// Scans of R rows at once by one lane: the records list[idx[i]], i < R, of
// the valid rows.  kSelect: flag[i] = some neighbour outranks the row's vertex
// (only the prefix [b, es) of the row is read), else: flag[i] = some
// neighbour is in the MIS.  All loads of one step are issued before any
// test, so each lane keeps up to R gathers in flight.
template <int R, bool kSelect, class Words>
__device__ __forceinline__ void lane_rows(const int32_t* __restrict__ col, Words nbw,
                                          const int4 (&rec)[R], const bool (&valid)[R],
                                          const uint32_t (&wv)[R], bool (&flag)[R]) {
    int p[R], e[R];
#pragma unroll
    for (int i = 0; i < R; ++i) {
        e[i] = valid[i] ? (kSelect ? rec[i].z : rec[i].w) : 0;
        p[i] = rec[i].y & ~3;
        flag[i] = false;
    }
    for (;;) {
        bool act[R];
        bool any = false;
#pragma unroll
        for (int i = 0; i < R; ++i) {
            act[i] = !flag[i] && p[i] < e[i];
            any |= act[i];
        }
        if (!any) break;
        int4 c[R];
#pragma unroll
        for (int i = 0; i < R; ++i)
            c[i] = act[i] ? __ldg(reinterpret_cast<const int4*>(col + p[i])) : make_int4(0, 0, 0, 0);
        uint32_t w[R][4];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int q = p[i], b = rec[i].y;
            w[i][0] = (act[i] && q >= b) ? nbw(c[i].x) : 0u;
            w[i][1] = (act[i] && q + 1 >= b && q + 1 < e[i]) ? nbw(c[i].y) : 0u;
            w[i][2] = (act[i] && q + 2 >= b && q + 2 < e[i]) ? nbw(c[i].z) : 0u;
            w[i][3] = (act[i] && q + 3 >= b && q + 3 < e[i]) ? nbw(c[i].w) : 0u;
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const int v = rec[i].x;
            bool hit;
            if (kSelect)
                hit = outranks(w[i][0], c[i].x, wv[i], v) | outranks(w[i][1], c[i].y, wv[i], v) |
                      outranks(w[i][2], c[i].z, wv[i], v) | outranks(w[i][3], c[i].w, wv[i], v);
            else
                hit = max(max(w[i][0], w[i][1]), max(w[i][2], w[i][3])) >= kWordInMin;
            flag[i] = flag[i] || (act[i] && hit);
            p[i] += 4;
        }
    }
}

// The adjacency the scans read.  Round 0's selection test reads the full
// rows (col_sel); every other scan reads col_s0 (the tested subgraph's rows
// where the graph has one, else col_sel).  Both come from the kernel
// parameters, so they cost no registers across a phase.
__device__ __forceinline__ const int32_t* select_col(const SolveArgs& a, bool late) {
    return late ? a.col_s0 : a.col_sel;
}
__device__ __forceinline__ const int32_t* exclude_col(const SolveArgs& a) { return a.col_s0; }
// The records of Phase 2 for the rows of `list` (a slice of W_r): in round 0
// with a tested subgraph, the same rows of order0_s0.
__device__ __forceinline__ const int4* pending_view(const SolveArgs& a, const int4* list,
                                                    bool late) {
    return (!late && a.order0_s0) ? a.order0_s0 + (list - a.order0) : list;
}

// Warps taking part in the rounds: the grid's, or block 0's once it finishes
// the rounds alone (kept in shared memory so that the switch costs the
// scans no register).
__shared__ int s_nwarps;

// Static first chunks of each bin, one per warp, rotating over the warps
// from bin to bin (the chunk plan of the worklists), over s_nwarps warps.
struct RoundSched {
    int gw;    // this warp's index among the warps taking part
    int base;  // first warp of the next bin
    __device__ __forceinline__ int nwarps() const { return s_nwarps; }
    __device__ __forceinline__ int first(int total) {
        const int n = nwarps();
        int k = gw - base;
        if (k < 0) k += n;
        base += total < n ? total : 0;
        if (base >= n) base -= n;
        return k;
    }
};

// Candidates this block selected (with a.direct: the MIS size is counted as
// vertices are selected, there is no output pass).
__shared__ unsigned s_selected;
// 1 while block 0 finishes a small worklist alone (its hub bin then takes
// every row itself)
__shared__ int s_solo;

// Puts v (a Phase 1 candidate, word already marked) in the result.
__device__ __forceinline__ void mark_selected(const SolveArgs& a, int v) {
    if (a.direct) {
        if (a.out) a.out[v] = 1;
        atomicAdd(&s_selected, 1u);
    }
}

// Phase 1, bins 0..3: selection test of every row of the bin's list W_r.
// Candidates are marked in the MIS.  kPending: the others form the pending
// list P_r of Phase 2 (appended to pdst, counted in *pnext), each entry the
// row's record in the adjacency Phase 2 scans.
template <int TPR, int CH, bool kPending>
__device__ __forceinline__ void select_bin(const SolveArgs& a, const int4* __restrict__ list,
                                           int cnt, RoundSched& ws, unsigned* grab, int* pnext,
                                           int4* __restrict__ pdst, int32_t* wbuf, bool late) {
    constexpr int G = 32 / TPR;
    constexpr int kPass = TPR == 1 ? 32 * kRowsPerLane : G;  // rows of one warp pass
    static_assert(kPass <= kStageMax, "a warp pass exceeds the staging buffer");
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const unsigned glane = lane % TPR;
    const unsigned gid = lane / TPR;
    const unsigned gshift = gid * TPR;
    const ChunkPlan plan = plan_of<G, CH>(cnt, ws.nwarps());
    int fill = 0;
    for (int k = ws.first(plan.total); k < plan.total; k = next_chunk(plan.total, ws.nwarps(), grab)) {
        int c0, c1;
        plan.range(k, cnt, c0, c1, G);
        for (int base = c0; base < c1; base += kPass) {
            if constexpr (TPR == 1) {
                int4 rec[kRowsPerLane];
                bool valid[kRowsPerLane], blocked[kRowsPerLane];
                uint32_t wv[kRowsPerLane];
#pragma unroll
                for (int i = 0; i < kRowsPerLane; ++i) {
                    const int item = base + (int)lane + 32 * i;
                    valid[i] = item < c1;
                    rec[i] = valid[i] ? list[item] : make_int4(0, 0, 0, 0);
                }
                // every vertex of W_r is undecided and nothing else writes its
                // word in this phase, so it may be read through L1
#pragma unroll
                for (int i = 0; i < kRowsPerLane; ++i)
                    wv[i] = valid[i] ? ld_word_l1(a.word + rec[i].x) : 0u;
                lane_rows<kRowsPerLane, true>(select_col(a, late), LiveWords{a.word}, rec, valid, wv, blocked);
#pragma unroll
                for (int i = 0; i < kRowsPerLane; ++i) {
                    if (valid[i] && !blocked[i]) {
                        a.word[rec[i].x] = wv[i] | kWordInSet;
                        mark_selected(a, rec[i].x);
                    }
                    if (kPending)
                        fill = stage_keep(valid[i] && blocked[i], base + (int)lane + 32 * i, wbuf,
                                          fill);
                }
            } else {
                const int item = base + (int)gid;
                const bool valid = item < c1;
                const int4 rec = valid ? list[item] : make_int4(0, 0, 0, 0);
                const uint32_t wv = valid ? ld_word_l1(a.word + rec.x) : 0u;
                const int e = valid ? rec.z : 0;
                const bool blocked =
                    group_scan<TPR, true>(select_col(a, late), LiveWords{a.word}, rec.y, e, rec.x, wv, glane, gshift);
                const bool lead = glane == 0;
                if (valid && !blocked && lead) {
                    a.word[rec.x] = wv | kWordInSet;
                    mark_selected(a, rec.x);
                }
                if (kPending) fill = stage_keep(valid && blocked && lead, item, wbuf, fill);
            }
            if (kPending)
                fill = flush_if_full(wbuf, fill, kPass, pending_view(a, list, late), pnext, pdst);
        }
    }
    if (kPending) flush_stage(wbuf, fill, pending_view(a, list, late), pnext, pdst);
}

// Phase 2+3, bins 0..3: exclusion test, state update, compaction into
// W_{r+1}.  kPending: `list` is the pending list P_r (undecided
// non-candidates only); else it is W_r, and each chunk (at most kScanMax
// rows) is first triaged one vertex per lane (Phase 1 candidates need no
// scan) into `wscan`.
template <int TPR, int CH, bool kPending>
__device__ __forceinline__ void exclude_bin(const SolveArgs& a, const int4* __restrict__ list,
                                            int cnt, RoundSched& ws, unsigned* grab, int* next,
                                            int4* __restrict__ dst, int32_t* wbuf,
                                            int32_t* wscan) {
    constexpr int G = 32 / TPR;
    constexpr int kPass = TPR == 1 ? 32 * kRowsPerLane : G;
    static_assert(kPass <= kStageMax, "a warp pass exceeds the staging buffer");
    static_assert(kPending || CH <= kScanMax, "a chunk exceeds the triage buffer");
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const unsigned glane = lane % TPR;
    const unsigned gid = lane / TPR;
    const unsigned gshift = gid * TPR;
    const LiveWords nbw{a.word};
    const ChunkPlan plan = plan_of<G, CH>(cnt, ws.nwarps());
    int fill = 0;
    for (int k = ws.first(plan.total); k < plan.total; k = next_chunk(plan.total, ws.nwarps(), grab)) {
        int c0, c1;
        plan.range(k, cnt, c0, c1, G);
        if (!kPending) {
            // triage: wscan gets the list indices of the undecided rows
            __syncwarp();  // the previous chunk is done with wscan
            int nscan = 0;
            for (int base = c0; base < c1; base += 32) {
                const int item = base + (int)lane;
                const bool scan = item < c1 && ld_word_l1(a.word + list[item].x) < kWordInMin;
                nscan = stage_keep(scan, item, wscan, nscan);
            }
            __syncwarp();
            c0 = 0;
            c1 = nscan;
        }
        // row i of the chunk: list[kPending ? i : wscan[i]]
        for (int base = c0; base < c1; base += kPass) {
            if constexpr (TPR == 1) {
                int4 rec[kRowsPerLane];
                int idx[kRowsPerLane];
                bool valid[kRowsPerLane], excl[kRowsPerLane];
                const uint32_t unused[kRowsPerLane] = {};
#pragma unroll
                for (int i = 0; i < kRowsPerLane; ++i) {
                    const int item = base + (int)lane + 32 * i;
                    valid[i] = item < c1;
                    idx[i] = valid[i] ? (kPending ? item : wscan[item]) : 0;
                    rec[i] = valid[i] ? list[idx[i]] : make_int4(0, 0, 0, 0);
                }
                lane_rows<kRowsPerLane, false>(exclude_col(a), nbw, rec, valid, unused, excl);
#pragma unroll
                for (int i = 0; i < kRowsPerLane; ++i) {
                    if (valid[i] && excl[i]) a.word[rec[i].x] = kWordOut;
                    fill = stage_keep(valid[i] && !excl[i], idx[i], wbuf, fill);
                }
            } else {
                const int item = base + (int)gid;
                const bool valid = item < c1;
                const int idx = valid ? (kPending ? item : wscan[item]) : 0;
                const int4 rec = valid ? list[idx] : make_int4(0, 0, 0, 0);
                const int e = valid ? rec.w : 0;
                const bool excl =
                    group_scan<TPR, false>(exclude_col(a), nbw, rec.y, e, rec.x, 0u, glane, gshift);
                const bool lead = glane == 0;
                if (valid && excl && lead) a.word[rec.x] = kWordOut;
                fill = stage_keep(valid && !excl && lead, idx, wbuf, fill);
            }
            fill = flush_if_full(wbuf, fill, kPass, list, next, dst);
        }
    }
    flush_stage(wbuf, fill, list, next, dst);
}

// Round 0 of bin 0 without its list (a.range0_max > 0; graphs with no
// create-time round-0 classes): the warps split the vertex range [0, n) into
// contiguous slices and each lane takes kRowsPerLane vertices of a 64-vertex
// pass, reading row_ptr in sequence instead of 16-byte row records.  Lanes
// whose vertex is isolated or heavier than the bin (degree > range0_max) sit
// the pass out; those rows are in the lists of bins 1..4.
__device__ __forceinline__ void range0_slice(const SolveArgs& a, const RoundSched& ws, int& v0,
                                             int& v1) {
    constexpr int kPass = 32 * kRowsPerLane;
    const int nw = ws.nwarps();
    int per = (int)(((long long)a.n + nw - 1) / nw);
    per = (int)(((long long)per + kPass - 1) / kPass * kPass);
    const long long b = (long long)ws.gw * per;
    v0 = (int)min(b, (long long)a.n);
    v1 = (int)min(b + per, (long long)a.n);
}

// The record {v, row begin, prefix end, row end} of vertex v < n, and
// whether v is a light row (1 <= degree <= range0_max).  Graphs without
// round-0 classes have no selection prefixes either (both come with Eq. 1's
// degree-ordered rows), so the prefix is the whole row.
__device__ __forceinline__ bool range0_record(const SolveArgs& a, int v, int4& rec) {
    const int b = __ldg(a.rp + v);
    const int e = __ldg(a.rp + v + 1);
    rec = make_int4(v, b, e, e);
    return (unsigned)(e - b - 1) < (unsigned)a.range0_max;
}

// Appends the staged vertices' records to `dst` with one atomic on `next`.
__device__ __forceinline__ void flush_stage_v(const SolveArgs& a, const int32_t* wbuf, int fill,
                                              int* next, int4* __restrict__ dst) {
    __syncwarp();
    if (fill) {
        const unsigned lane = lane_id();
        int o = 0;
        if (lane == 0) o = atomicAdd(next, fill);
        o = __shfl_sync(0xFFFFFFFFu, o, 0);
        for (int i = (int)lane; i < fill; i += 32) {
            int4 rec;
            range0_record(a, wbuf[i], rec);
            dst[o + i] = rec;
        }
    }
    __syncwarp();
}

// Phase 1 of round 0, bin 0, by vertex ranges.  Candidates are marked in the
// MIS; the non-candidates are found again by Phase 2's range pass (no
// pending list).
__device__ __forceinline__ void select_range0(const SolveArgs& a, const RoundSched& ws) {
    constexpr int R = kRowsPerLane;
    const unsigned lane = lane_id();
    int v0, v1;
    range0_slice(a, ws, v0, v1);
    for (int base = v0; base < v1; base += 32 * R) {
        int4 rec[R];
        bool valid[R], blocked[R];
        uint32_t wv[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const unsigned v = (unsigned)base + lane + 32u * i;  // no overflow: base < 2^31
            valid[i] = v < (unsigned)v1 && range0_record(a, (int)v, rec[i]);
            if (!valid[i]) rec[i] = make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int i = 0; i < R; ++i) wv[i] = valid[i] ? ld_word_l1(a.word + rec[i].x) : 0u;
        lane_rows<R, true>(a.col_sel, LiveWords{a.word}, rec, valid, wv, blocked);
#pragma unroll
        for (int i = 0; i < R; ++i)
            if (valid[i] && !blocked[i]) {
                a.word[rec[i].x] = wv[i] | kWordInSet;
                mark_selected(a, rec[i].x);
            }
    }
}

// Phase 2+3 of round 0, bin 0, by vertex ranges: the light rows still
// undecided after Phase 1 are tested for a selected neighbour; the others
// are staged and appended to bin 0 of W_1 as records.
__device__ __forceinline__ void exclude_range0(const SolveArgs& a, const RoundSched& ws,
                                               int* next, int4* __restrict__ dst,
                                               int32_t* wbuf) {
    constexpr int R = kRowsPerLane;
    constexpr int kPass = 32 * R;
    const unsigned lane = lane_id();
    int v0, v1;
    range0_slice(a, ws, v0, v1);
    const uint32_t unused[R] = {};
    int fill = 0;
    for (int base = v0; base < v1; base += kPass) {
        int4 rec[R];
        bool valid[R], excl[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
            const unsigned v = (unsigned)base + lane + 32u * i;  // no overflow: base < 2^31
            valid[i] = v < (unsigned)v1 && range0_record(a, (int)v, rec[i]);
            if (!valid[i]) rec[i] = make_int4(0, 0, 0, 0);
        }
#pragma unroll
        for (int i = 0; i < R; ++i)  // undecided non-candidates only
            valid[i] = valid[i] && (ld_word_l1(a.word + rec[i].x) >> 29) == 1u;
        lane_rows<R, false>(exclude_col(a), LiveWords{a.word}, rec, valid, unused, excl);
#pragma unroll
        for (int i = 0; i < R; ++i) {
            if (valid[i] && excl[i]) a.word[rec[i].x] = kWordOut;
            fill = stage_keep(valid[i] && !excl[i], rec[i].x, wbuf, fill);
        }
        if (fill > kStageMax - kPass) {
            flush_stage_v(a, wbuf, fill, next, dst);
            fill = 0;
        }
    }
    flush_stage_v(a, wbuf, fill, next, dst);
}

// Bin 4 (hubs): the whole block scans one row at a time.  kSelect: Phase 1
// (kPending: non-candidates appended to the pending list), else Phase 2+3
// (survivors appended to W_{r+1}); hub rows are few, so entries are appended
// one by one.
template <bool kSelect, bool kPending>
__device__ __forceinline__ void block_bin(const SolveArgs& a, const int4* __restrict__ list,
                                          int cnt, unsigned* grab, int* next,
                                          int4* __restrict__ dst, bool late) {
    const int32_t* __restrict__ col = kSelect ? select_col(a, late) : exclude_col(a);
    __shared__ int s_row;
    if ((int)blockIdx.x >= cnt) return;  // no row left for this block
    int item = (int)blockIdx.x;          // first row: no atomic
    for (;;) {
        if (item >= cnt) break;
        const int4 rec = list[item];
        const int v = rec.x;
        // the word of v does not change during this row's scan in either phase
        const uint32_t wv = ld_word_l1(a.word + v);
        const bool skip = !kSelect && !kPending && wv >= kWordInMin;  // a candidate
        const int b = rec.y;
        const int e = skip ? b : kSelect ? rec.z : rec.w;
        bool found = false;
        for (int base = b & ~3; base < e; base += 4 * (int)blockDim.x) {
            const int p0 = base + 4 * (int)threadIdx.x;
            bool hit = false;
            if (p0 < e) {
                const int4 c = __ldg(reinterpret_cast<const int4*>(col + p0));
                const uint32_t w0 = (p0 >= b) ? ld_word_l1(a.word + c.x) : 0u;
                const uint32_t w1 = (p0 + 1 >= b && p0 + 1 < e) ? ld_word_l1(a.word + c.y) : 0u;
                const uint32_t w2 = (p0 + 2 >= b && p0 + 2 < e) ? ld_word_l1(a.word + c.z) : 0u;
                const uint32_t w3 = (p0 + 3 >= b && p0 + 3 < e) ? ld_word_l1(a.word + c.w) : 0u;
                if (kSelect)
                    hit = outranks(w0, c.x, wv, v) | outranks(w1, c.y, wv, v) |
                          outranks(w2, c.z, wv, v) | outranks(w3, c.w, wv, v);
                else
                    hit = max(max(w0, w1), max(w2, w3)) >= kWordInMin;
            }
            if (__syncthreads_or(hit)) {
                found = true;
                break;
            }
        }
        if (threadIdx.x == 0 && !skip) {
            if (kSelect) {
                if (!found) {
                    a.word[v] = wv | kWordInSet;
                    mark_selected(a, v);
                }
                else if (kPending) dst[atomicAdd(next, 1)] = pending_view(a, list, late)[item];
            } else if (found) {
                a.word[v] = kWordOut;
            } else {
                dst[atomicAdd(next, 1)] = rec;
            }
        }
        const int nb = (kSoloPath<kPending> && s_solo) ? 1 : (int)gridDim.x;
        if (cnt <= nb) break;  // every row was a first row
        __syncthreads();
        if (threadIdx.x == 0) s_row = nb + (int)atomicAdd(grab, 1u);
        __syncthreads();
        item = s_row;
    }
}

// Lanes per row of a bin whose base width is BASE: in rounds after the first
// (`late`) the rows are the survivors of earlier rounds, which need the
// longest scans, and there are few of them, so a bin takes the widest group
// (up to a warp) at which all its rows still fit in one pass of the grid's
// lanes: latency, not throughput.
template <int BASE>
__device__ __forceinline__ int lanes_per_row(int cnt, bool late, int nwarps) {
    if (!late) return BASE;
    const long long lanes = 32LL * nwarps;
    if (BASE < 32 && 32LL * cnt <= lanes) return 32;
    if (BASE < 16 && 16LL * cnt <= lanes) return 16;
    if (BASE < 4 && 4LL * cnt <= lanes) return 4;
    return BASE;
}

// Phase 1 of bin j (base width BASE, chunk CH) at the width lanes_per_row picks.
template <int BASE, int CH, bool kPending>
__device__ __forceinline__ void select_bin_at(const SolveArgs& a, const int4* list, int cnt,
                                              bool late, RoundSched& ws, unsigned* grab,
                                              int* pnext, int4* pend, int32_t* wbuf) {
    switch (lanes_per_row<BASE>(cnt, late, ws.nwarps())) {
        case 32:
            select_bin<32, kChunk3, kPending>(a, list, cnt, ws, grab, pnext, pend, wbuf, late);
            break;
        case 16:
            select_bin<16, kChunk2, kPending>(a, list, cnt, ws, grab, pnext, pend, wbuf, late);
            break;
        case 4: select_bin<4, kChunk1, kPending>(a, list, cnt, ws, grab, pnext, pend, wbuf, late); break;
        default: select_bin<BASE, CH, kPending>(a, list, cnt, ws, grab, pnext, pend, wbuf, late);
    }
}

// Phase 2+3 of one bin, likewise.  A triaged chunk must fit the triage buffer.
template <int BASE, int CH, bool kPending>
__device__ __forceinline__ void exclude_bin_at(const SolveArgs& a, const int4* list, int cnt,
                                               bool late, RoundSched& ws, unsigned* grab,
                                               int* next, int4* dst, int32_t* wbuf,
                                               int32_t* wscan) {
    constexpr int kX3 = (kPending || kChunk3 <= kScanMax) ? kChunk3 : kScanMax;
    constexpr int kX2 = (kPending || kChunk2 <= kScanMax) ? kChunk2 : kScanMax;
    constexpr int kX1 = (kPending || kChunk1 <= kScanMax) ? kChunk1 : kScanMax;
    constexpr int kX = (kPending || CH <= kScanMax) ? CH : kScanMax;
    switch (lanes_per_row<BASE>(cnt, late, ws.nwarps())) {
        case 32: exclude_bin<32, kX3, kPending>(a, list, cnt, ws, grab, next, dst, wbuf, wscan); break;
        case 16: exclude_bin<16, kX2, kPending>(a, list, cnt, ws, grab, next, dst, wbuf, wscan); break;
        case 4: exclude_bin<4, kX1, kPending>(a, list, cnt, ws, grab, next, dst, wbuf, wscan); break;
        default: exclude_bin<BASE, kX, kPending>(a, list, cnt, ws, grab, next, dst, wbuf, wscan);
    }
}

// Phase 1 over the bins of one worklist: hubs first, then the bins of longer
// rows.
template <bool kPending, bool kRange0>
__device__ __forceinline__ void select_phase(const SolveArgs& a, const int4* src, const int* cnt,
                                             bool late, RoundSched& ws, unsigned* grab,
                                             int* pnext, int4* pend, int32_t* wbuf) {
    const int* off = a.bin_off;
    block_bin<true, kPending>(a, src + off[4], cnt[4], &grab[4], &pnext[4], pend + off[4], late);
    select_bin_at<32, kChunk3, kPending>(a, src + off[3], cnt[3], late, ws, &grab[3], &pnext[3],
                                         pend + off[3], wbuf);
    select_bin_at<16, kChunk2, kPending>(a, src + off[2], cnt[2], late, ws, &grab[2], &pnext[2],
                                         pend + off[2], wbuf);
    select_bin_at<4, kChunk1, kPending>(a, src + off[1], cnt[1], late, ws, &grab[1], &pnext[1],
                                        pend + off[1], wbuf);
    if (kRange0 && !late)
        select_range0(a, ws);
    else
        select_bin_at<1, kChunk0, kPending>(a, src + off[0], cnt[0], late, ws, &grab[0],
                                            &pnext[0], pend + off[0], wbuf);
}

// Phase 2+3 over the bins of `list` (W_r, or P_r when kPending).
template <bool kPending, bool kRange0>
__device__ __forceinline__ void exclude_phase(const SolveArgs& a, const int4* list,
                                              const int* cnt, bool late, RoundSched& ws,
                                              unsigned* grab, int* next, int4* dst,
                                              int32_t* wbuf, int32_t* wscan) {
    const int* off = a.bin_off;
    block_bin<false, kPending>(a, list + off[4], cnt[4], &grab[4], &next[4], dst + off[4], late);
    exclude_bin_at<32, kChunk3, kPending>(a, list + off[3], cnt[3], late, ws, &grab[3],
                                          &next[3], dst + off[3], wbuf, wscan);
    exclude_bin_at<16, kChunk2, kPending>(a, list + off[2], cnt[2], late, ws, &grab[2],
                                          &next[2], dst + off[2], wbuf, wscan);
    exclude_bin_at<4, kChunk1, kPending>(a, list + off[1], cnt[1], late, ws, &grab[1],
                                         &next[1], dst + off[1], wbuf, wscan);
    if (kRange0 && !late)
        exclude_range0(a, ws, &next[0], dst + off[0], wbuf);
    else
        exclude_bin_at<1, kChunk0, kPending>(a, list + off[0], cnt[0], late, ws, &grab[0],
                                             &next[0], dst + off[0], wbuf, wscan);
}

// Initialisation with the keyed list (a.out0 set): the result starts as the
// create-time bytes out0 (16-byte copies where out is aligned) and only the
// keyed vertices get their Eq. 1 words; no other word is read by any test.
__device__ __forceinline__ void init_keyed(const SolveArgs& a) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    if (a.out) {
        long long done = 0;
        if (((uintptr_t)a.out & 15) == 0) {
            const long long nq = n / 16;
            const uint4* src = reinterpret_cast<const uint4*>(a.out0);
            uint4* dst = reinterpret_cast<uint4*>(a.out);
            for (long long i = tid; i < nq; i += nthreads) dst[i] = __ldg(src + i);
            done = nq * 16;
        }
        for (long long v = done + tid; v < n; v += nthreads) a.out[v] = a.out0[v];
    }
    const int mode = a.priority;
    const float dbar = average_degree(a.rp[n], n);
    const uint64_t smix = mix64(a.seed0);
    for (long long i = tid; i < a.n_keyed; i += nthreads) {
        const int2 k = __ldg(a.keyed + i);
        a.word[k.x] = undecided_word(mode, priority_key(mode, dbar, k.y, smix, (uint32_t)k.x));
    }
}

// The barrier of a block finishing the rounds alone: the same hooks as
// grid_barrier (leader bookkeeping, then `after`), run by thread 0 between
// two block-wide barriers, which also order the block's global writes.
template <class Leader, class After>
__device__ __forceinline__ void block_sync(Leader leader, After after) {
    __syncthreads();
    if (threadIdx.x == 0) {
        leader();
        after();
    }
    __syncthreads();
}

// Writes out[v] = [v in the MIS] and adds the MIS size to ctl->mis_size.
__device__ __forceinline__ void output_pass(const SolveArgs& a) {
    const int32_t n = a.n;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    unsigned in_cnt = 0;
    if (a.seg.count == 0 && ((uintptr_t)a.out & 3) == 0) {
        // four vertices per thread: 16-byte word loads, 4-byte result stores
        for (long long v = 4 * tid; v < n; v += 4 * nthreads) {
            const uint4 q = *reinterpret_cast<const uint4*>(a.word + v);
            const uint32_t b0 = q.x >= kWordInMin, b1 = q.y >= kWordInMin;
            const uint32_t b2 = q.z >= kWordInMin, b3 = q.w >= kWordInMin;
            if (v + 4 <= n) {
                *reinterpret_cast<uint32_t*>(a.out + v) = b0 | (b1 << 8) | (b2 << 16) | (b3 << 24);
                in_cnt += b0 + b1 + b2 + b3;
            } else {
                const uint32_t bb[4] = {b0, b1, b2, b3};
                for (int k = 0; k < 4 && v + k < n; ++k) {
                    a.out[v + k] = (uint8_t)bb[k];
                    in_cnt += bb[k];
                }
            }
        }
    } else {
        for (long long v = tid; v < n; v += nthreads) {
            const bool in = ld_word(a.word + v) >= kWordInMin;
            in_cnt += in;
            if (a.seg.count == 0) {
                a.out[v] = in;
            } else {
                const int g = a.seg.blk_seg[v >> 4];
                const int local = (int)v - a.seg.voff[g];
                if (local < a.seg.nv[g]) a.out[a.seg.roff[g] + local] = in;
            }
        }
    }
    for (int o = 16; o; o >>= 1) in_cnt += __shfl_xor_sync(0xFFFFFFFFu, in_cnt, o);
    if (lane_id() == 0 && in_cnt) atomicAdd(&a.ctl->mis_size, (unsigned long long)in_cnt);
}

// per-bin sizes of W_r and of P_r, copied once per block after each barrier
// (kept in shared memory, out of the scans' registers)
__shared__ int s_cnt[kBins];
__shared__ int s_pcnt[kBins];

// The barrier of a round: the grid's, or block 0's alone once it finishes
// the rounds by itself (s_solo).  The round's bookkeeping (`book`: stats,
// timestamps, resetting the ring counters of the round after next) is done
// by block 0 once past the barrier, not by the last block to arrive, so
// block 0 is the only block that ever writes those counters outside a
// phase -- which is what lets it carry on alone at any round.
template <bool kPending, class Book, class After>
__device__ __forceinline__ bool round_barrier(const SolveArgs& a, Book book, After after) {
    if (kSoloPath<kPending> && s_solo) {
        block_sync(book, after);
        return true;
    }
    return grid_barrier(a.ctl, gridDim.x, a.spin_cap, NoLeader(), [&]() {
        if (blockIdx.x == 0) book();
        after();
    });
}

// kRange0: round 0 takes bin 0 by vertex ranges (a.range0_max > 0); a
// separate instance, so that the list form keeps its register budget.
template <bool kPending, bool kRange0>
__global__ void __launch_bounds__(kCsrBlock, kCsrMinBlocksPerSm)
    csr_solve_kernel(const SolveArgs a) {
    __shared__ int32_t s_stage[kWarps][kStageMax];
    __shared__ int32_t s_scan[kPending ? 1 : kWarps][kPending ? 1 : kScanMax];
    const unsigned nblocks = gridDim.x;
    Ctl* ctl = a.ctl;
    PhaseTimes* times = a.times;
    int32_t* wbuf = s_stage[threadIdx.x / 32];
    int32_t* wscan = kPending ? nullptr : &s_scan[kPending ? 0 : threadIdx.x / 32][0];
    grid_barrier_start();
    if (threadIdx.x < kBins) s_cnt[threadIdx.x] = a.bin_off[threadIdx.x + 1] - a.bin_off[threadIdx.x];
    if (threadIdx.x == 0) {
        s_selected = 0;
        s_solo = 0;
        s_nwarps = (int)(nblocks * (blockDim.x / 32));
    }
    if (times && blockIdx.x == 0 && threadIdx.x == 0) times->t[0] = global_ns();

    // ---- init: Eq. 1 priorities (and, direct, the create-time result bytes)
    if (a.out0) init_keyed(a);
    else init_words(a, (a.n + 15) / 16 * 16, true, a.direct ? a.out : nullptr);  // padded to 16
    if (!round_barrier<kPending>(
            a,
            [times]() {
                if (times) times->t[1] = global_ns();
            },
            []() {}))
        return;

    // vertices decided without a test (isolated ones and sure candidates at
    // init, sure exclusions in round 0's Phase 2) belong to round 0's alive set
    const int decided0 = a.n_isolated + a.n_sure_in + a.n_sure_out;
    RoundSched ws;
    ws.gw = (int)(blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32);
    ws.base = 0;
    for (int r = 0;; ++r) {
        int total = 0;
        for (int j = 0; j < kBins; ++j) total += s_cnt[j];
        if (!(total > 0 || (r == 0 && decided0 > 0))) break;
        if (r >= a.max_rounds) {
            if (threadIdx.x == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            return;
        }
        // A small worklist is finished by block 0 alone, with block-level
        // barriers: every block reads the same total, so all see the switch;
        // the others are done (the result is written as vertices are
        // decided).  Block 0 keeps the ring counters, which it alone resets,
        // and its warps keep their indices.  Worklists only shrink, so once
        // switched every later round switches again (idempotent).
        if constexpr (kSoloPath<kPending>) {
            if (a.direct && r > 0 && total <= kSoloRows) {
                if (blockIdx.x != 0) break;
                __syncthreads();  // every thread has read the shared state of the last round
                if (threadIdx.x == 0) {
                    s_solo = 1;
                    s_nwarps = (int)(blockDim.x / 32);
                }
                __syncthreads();
                ws.base = 0;  // first() needs base < nwarps
            }
        }
        const int4* src = (r == 0) ? a.order0 : ((r & 1) ? a.wl1 : a.wl0);
        int4* dst = ((r + 1) & 1) ? a.wl1 : a.wl0;
        int* next = ctl->bcnt[(r + 1) & 3];
        int* pnext = ctl->pcnt[r & 3];
        const int rr = r;

        // ---- Phase 1: selection test
        select_phase<kPending, kRange0>(a, src, s_cnt, r > 0, ws, ctl->grab[(2 * r) & 3], pnext, a.wlp,
                               wbuf);
        if (!round_barrier<kPending>(
                a,
                [ctl, times, rr]() {
                    if (times && rr < kStatRounds) times->t[2 + rr] = global_ns();
                    for (int j = 0; j < kBins; ++j) ctl->grab[(2 * rr + 2) & 3][j] = 0;
                },
                [pnext]() {
                    if (kPending)
                        for (int j = 0; j < kBins; ++j) s_pcnt[j] = __ldcg(pnext + j);
                }))
            return;

        // ---- Phase 2+3: exclusion test, state update, compaction
        if (r == 0 && !a.out0) {
            // the sure exclusions: neighbours of sure candidates (with the
            // keyed list no test reads their words, and out0 has them out)
            const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
            const long long nthreads = (long long)nblocks * blockDim.x;
            for (long long i = tid; i < a.n_sure_out; i += nthreads) a.word[a.sure_out[i]] = kWordOut;
        }
        if (kPending)
            exclude_phase<true, kRange0>(a, a.wlp, s_pcnt, r > 0, ws, ctl->grab[(2 * r + 1) & 3], next,
                                dst, wbuf, wscan);
        else  // W_r's rows in the adjacency Phase 2 scans
            exclude_phase<false, kRange0>(a, pending_view(a, src, r > 0), s_cnt, r > 0, ws,
                                 ctl->grab[(2 * r + 1) & 3], next, dst, wbuf, wscan);
        const int cur = total + (r == 0 ? decided0 : 0);
        if (!round_barrier<kPending>(
                a,
                [ctl, times, rr, cur]() {
                    if (times && rr < kStatRounds) times->t[2 + kStatRounds + rr] = global_ns();
                    if (rr < kStatRounds) ctl->alive[rr] = cur;
                    ctl->alive_sum += (unsigned long long)cur;
                    ctl->rounds = rr + 1;
                    for (int j = 0; j < kBins; ++j) {
                        ctl->grab[(2 * rr + 3) & 3][j] = 0;
                        ctl->bcnt[(rr + 2) & 3][j] = 0;
                        ctl->pcnt[(rr + 2) & 3][j] = 0;
                    }
                },
                [next]() {
                    for (int j = 0; j < kBins; ++j) s_cnt[j] = __ldcg(next + j);
                }))
            return;
    }

    // ---- output
    if (!a.direct) {
        if (a.out) output_pass(a);
        return;
    }
    // the result is complete; the MIS size is the create-time part plus the
    // candidates every block selected
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long c = s_selected;
        if (blockIdx.x == 0) c += (unsigned long long)a.n_isolated + (unsigned long long)a.n_sure_in;
        if (c) atomicAdd(&ctl->mis_size, c);
    }
}

const void* csr_kernel_fn(const SolveArgs& a) {
    const bool range0 = a.range0_max > 0;
    if (a.pending)
        return range0 ? (const void*)csr_solve_kernel<true, true>
                      : (const void*)csr_solve_kernel<true, false>;
    return range0 ? (const void*)csr_solve_kernel<false, true>
                  : (const void*)csr_solve_kernel<false, false>;
}

cudaError_t launch_csr_solve(const SolveArgs& a, int grid, cudaStream_t s) {
    void* args[] = {const_cast<SolveArgs*>(&a)};
    return cudaLaunchCooperativeKernel(csr_kernel_fn(a), dim3(grid), dim3(kCsrBlock), args, 0, s);
}

cudaError_t launch_csr_solve_single(const SolveArgs& a, cudaStream_t s) {
    void* args[] = {const_cast<SolveArgs*>(&a)};
    return cudaLaunchKernel(csr_kernel_fn(a), dim3(1), dim3(kCsrBlock), args, 0, s);
}

int csr_block_size() { return kCsrBlock; }

int csr_max_coresident_blocks(int device) {
    // every form: the grid must fit whichever one a solve launches
    const void* fns[] = {(const void*)csr_solve_kernel<false, false>,
                         (const void*)csr_solve_kernel<true, false>,
                         (const void*)csr_solve_kernel<false, true>,
                         (const void*)csr_solve_kernel<true, true>};
    int per_sm = 1 << 30, sms = 0;
    for (const void* fn : fns) {
        int p = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, fn, kCsrBlock, 0) != cudaSuccess)
            return 0;
        per_sm = std::min(per_sm, p);
    }
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

// ---------------------------------------------------------------- degree bins
//
// order0 = the round-0 records: every real vertex of degree >= 1 (batch
// padding excluded) that round 0 has to test, grouped by bin, ascending id
// inside a bin; sure_out = the sure round-0 exclusions, ascending.  Two
// kernels: per-block class counts, then (after the host turns the counts into
// offsets) a stable scatter.  Blocks own contiguous vertex ranges.

// classes: bins 0..4, then isolated, sure candidates, sure exclusions
constexpr int kIsolated = kBins, kSureIn = kBins + 1, kSureOut = kBins + 2;
constexpr int kClasses = kBins + 3;

struct BinThr {
    int32_t t[kBins - 1];
};

__device__ __forceinline__ int bin_of(int deg, const BinThr& thr) {
    int j = 0;
#pragma unroll
    for (int k = 0; k < kBins - 1; ++k) j += deg > thr.t[k];
    return j;
}

__device__ __forceinline__ bool is_real(const SegTable& seg, long long v) {
    if (seg.count == 0) return true;
    const int g = seg.blk_seg[v >> 4];
    return (int)v - seg.voff[g] < seg.nv[g];
}

// Class of vertex v (-1 for batch padding).
__device__ __forceinline__ int class_of(const SegTable& seg, const int32_t* rp,
                                        const uint8_t* r0class, long long v, const BinThr& thr) {
    if (!is_real(seg, v)) return -1;
    const int deg = rp[v + 1] - rp[v];
    if (deg == 0) return kIsolated;
    if (r0class && r0class[v] == 1) return kSureIn;
    if (r0class && r0class[v] == 2) return kSureOut;
    return bin_of(deg, thr);
}

__global__ void bin_count_kernel(const int32_t* __restrict__ rp, const uint8_t* __restrict__ r0class,
                                 int32_t n, const SegTable seg, const BinThr thr,
                                 int32_t* __restrict__ blkcnt) {
    __shared__ int c[kClasses];
    if (threadIdx.x < kClasses) c[threadIdx.x] = 0;
    __syncthreads();
    const long long v0 = (long long)n * blockIdx.x / gridDim.x;
    const long long v1 = (long long)n * (blockIdx.x + 1) / gridDim.x;
    for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        const int j = class_of(seg, rp, r0class, v, thr);
        if (j >= 0) atomicAdd(&c[j], 1);
    }
    __syncthreads();
    if (threadIdx.x < kClasses) blkcnt[blockIdx.x * kClasses + threadIdx.x] = c[threadIdx.x];
}

// blockDim.x must be 256
__global__ void bin_scatter_kernel(const int32_t* __restrict__ rp,
                                   const int32_t* __restrict__ split,
                                   const uint8_t* __restrict__ r0class, int32_t n,
                                   const SegTable seg, const BinThr thr,
                                   const int32_t* __restrict__ blkoff,
                                   int4* __restrict__ order0, int32_t* __restrict__ sure_out,
                                   const int32_t* __restrict__ s0_rp,
                                   const int32_t* __restrict__ s0_pre,
                                   int4* __restrict__ order0_s0) {
    __shared__ int wsum[8][kClasses];
    __shared__ int run[kClasses];
    const unsigned lane = lane_id();
    const int w = threadIdx.x / 32;
    if (threadIdx.x < kClasses) run[threadIdx.x] = blkoff[blockIdx.x * kClasses + threadIdx.x];
    __syncthreads();
    const long long v0 = (long long)n * blockIdx.x / gridDim.x;
    const long long v1 = (long long)n * (blockIdx.x + 1) / gridDim.x;
    for (long long c0 = v0; c0 < v1; c0 += blockDim.x) {
        const long long v = c0 + threadIdx.x;
        const int j = v < v1 ? class_of(seg, rp, r0class, v, thr) : -1;
        int rank = 0;
        for (int b = 0; b < kClasses; ++b) {
            const unsigned m = __ballot_sync(0xFFFFFFFFu, j == b);
            if (j == b) rank = __popc(m & lanemask_lt());
            if (lane == 0) wsum[w][b] = __popc(m);
        }
        __syncthreads();
        if (j >= 0 && (j < kBins || j == kSureOut)) {
            int off = run[j];
            for (int x = 0; x < w; ++x) off += wsum[x][j];
            if (j == kSureOut) {
                sure_out[off + rank] = (int32_t)v;
            } else {
                const int b = rp[v], e = rp[v + 1];
                order0[off + rank] = make_int4((int)v, b, split ? b + split[v] : e, e);
                if (order0_s0)  // the same row in the tested subgraph
                    order0_s0[off + rank] =
                        make_int4((int)v, s0_rp[v], s0_rp[v] + s0_pre[v], s0_rp[v + 1]);
            }
        }
        __syncthreads();
        if (threadIdx.x < kClasses) {
            int t = 0;
            for (int x = 0; x < 8; ++x) t += wsum[x][threadIdx.x];
            run[threadIdx.x] += t;
        }
        __syncthreads();
    }
}

cudaError_t build_bins(const int32_t* rp, const int32_t* split, const uint8_t* r0class,
                       int32_t n, const SegTable& seg, const int32_t thr[4], int4* order0,
                       int32_t* sure_out, const int32_t* s0_rp, const int32_t* s0_pre,
                       int4* order0_s0, Round0Plan* plan, cudaStream_t s) {
    *plan = Round0Plan{};
    if (n == 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>(1024, ((long long)n + 255) / 256);
    BinThr t;
    for (int k = 0; k < kBins - 1; ++k) t.t[k] = thr[k];
    int32_t* d_cnt = nullptr;
    cudaError_t e = dev_alloc((void**)&d_cnt, sizeof(int32_t) * blocks * kClasses);
    if (e != cudaSuccess) return e;
    std::vector<int32_t> h((size_t)blocks * kClasses);
    bin_count_kernel<<<blocks, 256, 0, s>>>(rp, r0class, n, seg, t, d_cnt);
    e = cudaGetLastError();
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_cnt, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        int64_t tot[kClasses] = {};
        for (int b = 0; b < blocks; ++b)
            for (int j = 0; j < kClasses; ++j) tot[j] += h[(size_t)b * kClasses + j];
        int64_t acc = 0;
        for (int j = 0; j < kBins; ++j) {
            plan->bin_off[j] = (int32_t)acc;
            acc += tot[j];
        }
        plan->bin_off[kBins] = (int32_t)acc;
        plan->n_isolated = (int32_t)tot[kIsolated];
        plan->n_sure_in = (int32_t)tot[kSureIn];
        plan->n_sure_out = (int32_t)tot[kSureOut];
        // running offsets per block: bins into order0, sure exclusions into
        // sure_out (isolated vertices and sure candidates are not listed)
        int64_t run[kClasses] = {};
        for (int j = 0; j < kBins; ++j) run[j] = plan->bin_off[j];
        for (int b = 0; b < blocks; ++b)
            for (int j = 0; j < kClasses; ++j) {
                const int32_t c = h[(size_t)b * kClasses + j];
                h[(size_t)b * kClasses + j] = (int32_t)run[j];
                run[j] += c;
            }
        e = cudaMemcpyAsync(d_cnt, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) {
        bin_scatter_kernel<<<blocks, 256, 0, s>>>(rp, split, r0class, n, seg, t, d_cnt, order0,
                                                  sure_out, s0_rp, s0_pre, order0_s0);
        e = cudaGetLastError();
    }
    const cudaError_t se = cudaStreamSynchronize(s);  // also on error: nothing may still run
    if (e == cudaSuccess) e = se;
    dev_free(d_cnt);
    return e;
}

// ---------------------------------------------------------------- round-0 classes
//
// Eq. 1 ranks a vertex of degree <= deg(v) - 2 strictly above v for every
// seed (the order kept by the degree-ordered rows, see kernels_order.cu).
// So a vertex whose selection prefix is empty outranks all its neighbours: it
// is a candidate of round 0 whatever the seed (class 1).  A vertex of another
// class with a class-1 neighbour is outranked by it and has a candidate
// neighbour: it is excluded in round 0 (class 2).  Such a neighbour has degree
// <= deg(v) - 2, so it lies in v's selection prefix; a warp scans the prefix
// and stops at the first one.  Round counts and alive sets are unchanged:
// these vertices are decided in round 0 exactly as the tests would decide
// them, only without running the tests.

__global__ void round0_class_kernel(const int32_t* __restrict__ rp,
                                    const int32_t* __restrict__ col_sel,
                                    const int32_t* __restrict__ split, int32_t n,
                                    const SegTable seg, uint8_t* __restrict__ r0class) {
    const long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const unsigned lane = lane_id();
    if (v >= n) return;
    const int b = rp[v];
    const int deg = rp[v + 1] - b;
    const int pre = split[v];
    uint8_t c = 0;
    if (deg > 0 && is_real(seg, v)) {
        if (pre == 0) {
            c = 1;
        } else {
            for (int p0 = b; p0 < b + pre; p0 += 32) {
                const int p = p0 + (int)lane;
                bool hit = false;
                if (p < b + pre) {
                    const int u = col_sel[p];
                    hit = split[u] == 0 && rp[u + 1] > rp[u];
                }
                if (__any_sync(0xFFFFFFFFu, hit)) {
                    c = 2;
                    break;
                }
            }
        }
    }
    if (lane == 0) r0class[v] = c;
}

cudaError_t build_round0_classes(const int32_t* rp, const int32_t* col_sel, const int32_t* split,
                                 int32_t n, const SegTable& seg, uint8_t* r0class,
                                 cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const long long threads = 32LL * n;
    round0_class_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(rp, col_sel, split, n,
                                                                         seg, r0class);
    cudaError_t e = cudaGetLastError();
    const cudaError_t se = cudaStreamSynchronize(s);
    return e != cudaSuccess ? e : se;
}

// ---------------------------------------------------------------- the tested subgraph
//
// S0 = the vertices of degree >= 1 that round 0 has to test (class 0).  An S0
// vertex has no class-1 neighbour (else it would be class 2), so in round 0
// its exclusion test can only be decided by an S0 candidate; and after round
// 0 every vertex outside S0 is decided (class 1 in, class 2 out), so in every
// later round both tests only need the S0 neighbours.  Round 0's selection
// test is the one exception (class-2 neighbours are still undecided then) and
// keeps the full rows.  Where S0 is small (power-law graphs), its internal
// adjacency -- each row in col_sel's order, selection prefix first -- makes
// those scans short.

__device__ __forceinline__ bool in_s0(const uint8_t* r0class, const int32_t* rp, long long v) {
    return r0class[v] == 0 && rp[v + 1] > rp[v];
}

// One warp per vertex: S0 neighbours of an S0 row, in its selection prefix
// (pre) and in all (tot); 0 for the other vertices.
__global__ void s0_count_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col_sel,
                                const int32_t* __restrict__ split,
                                const uint8_t* __restrict__ r0class, int32_t n,
                                int32_t* __restrict__ tot, int32_t* __restrict__ pre) {
    const long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const unsigned lane = lane_id();
    if (v >= n) return;
    int ct = 0, cp = 0;
    if (in_s0(r0class, rp, v)) {
        const int b = rp[v], e = rp[v + 1], es = b + split[v];
        for (int p = b + (int)lane; p < e; p += 32) {
            const bool hit = in_s0(r0class, rp, col_sel[p]);
            ct += hit;
            cp += hit && p < es;
        }
        for (int o = 16; o; o >>= 1) {
            ct += __shfl_xor_sync(0xFFFFFFFFu, ct, o);
            cp += __shfl_xor_sync(0xFFFFFFFFu, cp, o);
        }
    }
    if (lane == 0) {
        tot[v] = ct;
        pre[v] = cp;
    }
}

// One warp per S0 row: its S0 neighbours, in order, to s0_col[s0_rp[v] ...].
__global__ void s0_scatter_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col_sel,
                                  const uint8_t* __restrict__ r0class, int32_t n,
                                  const int32_t* __restrict__ s0_rp, int32_t* __restrict__ s0_col) {
    const long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const unsigned lane = lane_id();
    if (v >= n || !in_s0(r0class, rp, v)) return;
    const int b = rp[v], e = rp[v + 1];
    int out = s0_rp[v];
    for (int p0 = b; p0 < e; p0 += 32) {
        const int p = p0 + (int)lane;
        const int u = p < e ? col_sel[p] : 0;
        const bool hit = p < e && in_s0(r0class, rp, u);
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, hit);
        if (hit) s0_col[out + __popc(bal & lanemask_lt())] = u;
        out += __popc(bal);
    }
}

cudaError_t build_s0_graph(const int32_t* rp, const int32_t* col_sel, const int32_t* split,
                           const uint8_t* r0class, int32_t n, int64_t max_arcs, int32_t** s0_rp,
                           int32_t** s0_col, int32_t** s0_pre, int64_t* s0_arcs,
                           cudaStream_t s) {
    *s0_rp = *s0_col = *s0_pre = nullptr;
    *s0_arcs = 0;
    if (n == 0) return cudaSuccess;
    int32_t *tot = nullptr, *rpo = nullptr, *pre = nullptr, *colo = nullptr;
    void* temp = nullptr;
    size_t temp_bytes = 0;
    const unsigned blocks = (unsigned)((32LL * n + 255) / 256);
    cudaError_t e = dev_alloc((void**)&tot, sizeof(int32_t) * ((size_t)n + 1));
    if (e == cudaSuccess) e = dev_alloc((void**)&rpo, sizeof(int32_t) * ((size_t)n + 1));
    if (e == cudaSuccess) e = dev_alloc((void**)&pre, sizeof(int32_t) * (size_t)n);
    if (e == cudaSuccess) e = cudaMemsetAsync(tot + n, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) {
        s0_count_kernel<<<blocks, 256, 0, s>>>(rp, col_sel, split, r0class, n, tot, pre);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cub::DeviceScan::ExclusiveSum(nullptr, temp_bytes, tot, rpo, n + 1, s);
    if (e == cudaSuccess) e = dev_alloc(&temp, temp_bytes ? temp_bytes : 1);
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(temp, temp_bytes, tot, rpo, n + 1, s);
    int32_t total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, rpo + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const bool worth = e == cudaSuccess && (int64_t)total <= max_arcs;
    if (worth) {
        // padded like col_idx: 16-byte slices may read up to 3 entries past a row
        const size_t alloc = ((size_t)total + 3) / 4 * 4 + 4;
        e = dev_alloc((void**)&colo, sizeof(int32_t) * alloc);
        if (e == cudaSuccess) e = cudaMemsetAsync(colo, 0, sizeof(int32_t) * alloc, s);
        if (e == cudaSuccess) {
            s0_scatter_kernel<<<blocks, 256, 0, s>>>(rp, col_sel, r0class, n, rpo, colo);
            e = cudaGetLastError();
        }
    }
    const cudaError_t se = cudaStreamSynchronize(s);  // also on error: nothing may still run
    if (e == cudaSuccess) e = se;
    dev_free(tot);
    dev_free(temp);
    if (e != cudaSuccess || !worth) {
        dev_free(rpo);
        dev_free(pre);
        dev_free(colo);
        return e;
    }
    *s0_rp = rpo;
    *s0_col = colo;
    *s0_pre = pre;
    *s0_arcs = total;
    return cudaSuccess;
}

// ---- the keyed vertices and the create-time result bytes
//
// With the tested subgraph, a solve only ever reads the words of two sets of
// vertices: those of S0 (every scan) and the vertices in an S0 row's
// selection prefix (round 0's selection test; they are S0 or class-2
// vertices, since class 1 has no S0 neighbour).  Every other vertex is
// decided before any test and no scan reads its word: isolated vertices and
// class 1 are in the MIS, class 2 is out.  So the solve computes keys for the
// keyed list alone (sorted by vertex, with each degree), copies the result
// bytes of the vertices decided at create time from out0 (1: isolated or
// class 1), and marks its own candidates in the result as it selects them.

// One warp per vertex: flag an S0 vertex and every vertex of its selection
// prefix (benign duplicate writes of 1); count S0 rows and prefix arcs.
__global__ void keyed_mark_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col_sel,
                                  const int32_t* __restrict__ split,
                                  const uint8_t* __restrict__ r0class, int32_t n,
                                  int32_t* __restrict__ need,
                                  unsigned long long* __restrict__ sums) {
    const long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    const unsigned lane = lane_id();
    if (v >= n || !in_s0(r0class, rp, v)) return;
    if (lane == 0) {
        need[v] = 1;
        atomicAdd(&sums[0], 1ull);
        atomicAdd(&sums[1], (unsigned long long)split[v]);
    }
    const int b = rp[v], es = b + split[v];
    for (int p = b + (int)lane; p < es; p += 32) need[col_sel[p]] = 1;
}

// keyed[pos[v]] = {v, degree of v} for every flagged v; out0[v] = 1 for the
// isolated vertices and class 1.
__global__ void keyed_pack_kernel(const int32_t* __restrict__ rp,
                                  const uint8_t* __restrict__ r0class, int32_t n,
                                  const int32_t* __restrict__ need,
                                  const int32_t* __restrict__ pos, int2* __restrict__ keyed,
                                  uint8_t* __restrict__ out0) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int deg = rp[v + 1] - rp[v];
    if (need[v]) keyed[pos[v]] = make_int2((int)v, deg);
    out0[v] = (deg == 0 || r0class[v] == 1) ? 1 : 0;
}

cudaError_t build_keyed(const int32_t* rp, const int32_t* col_sel, const int32_t* split,
                        const uint8_t* r0class, int32_t n, int2** keyed, int32_t* n_keyed,
                        uint8_t** out0, int32_t* n_tested, int64_t* prefix_arcs,
                        cudaStream_t s) {
    *keyed = nullptr;
    *out0 = nullptr;
    *n_keyed = 0;
    *n_tested = 0;
    *prefix_arcs = 0;
    if (n == 0) return cudaSuccess;
    int32_t *need = nullptr, *pos = nullptr;
    unsigned long long* sums = nullptr;
    unsigned long long hsums[2] = {0, 0};
    int2* kd = nullptr;
    uint8_t* o0 = nullptr;
    void* temp = nullptr;
    size_t temp_bytes = 0;
    cudaError_t e = dev_alloc((void**)&need, sizeof(int32_t) * ((size_t)n + 1));
    if (e == cudaSuccess) e = dev_alloc((void**)&pos, sizeof(int32_t) * ((size_t)n + 1));
    // result bytes padded to 16 for the solve's 16-byte copies
    if (e == cudaSuccess) e = dev_alloc((void**)&o0, ((size_t)n + 15) / 16 * 16);
    if (e == cudaSuccess) e = dev_alloc((void**)&sums, sizeof(hsums));
    if (e == cudaSuccess) e = cudaMemsetAsync(need, 0, sizeof(int32_t) * ((size_t)n + 1), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o0, 0, ((size_t)n + 15) / 16 * 16, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sums, 0, sizeof(hsums), s);
    if (e == cudaSuccess) {
        keyed_mark_kernel<<<(unsigned)((32LL * n + 255) / 256), 256, 0, s>>>(
            rp, col_sel, split, r0class, n, need, sums);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cub::DeviceScan::ExclusiveSum(nullptr, temp_bytes, need, pos, n + 1, s);
    if (e == cudaSuccess) e = dev_alloc(&temp, temp_bytes ? temp_bytes : 1);
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(temp, temp_bytes, need, pos, n + 1, s);
    int32_t total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&total, pos + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hsums, sums, sizeof(hsums), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = dev_alloc((void**)&kd, sizeof(int2) * ((size_t)total + 1));
    if (e == cudaSuccess) {
        keyed_pack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rp, r0class, n, need, pos,
                                                                      kd, o0);
        e = cudaGetLastError();
    }
    const cudaError_t se = cudaStreamSynchronize(s);  // also on error: nothing may still run
    if (e == cudaSuccess) e = se;
    dev_free(need);
    dev_free(pos);
    dev_free(temp);
    dev_free(sums);
    if (e != cudaSuccess) {
        dev_free(kd);
        dev_free(o0);
        return e;
    }
    *keyed = kd;
    *n_keyed = total;
    *out0 = o0;
    *n_tested = (int32_t)hsums[0];
    *prefix_arcs = (int64_t)hsums[1];
    return cudaSuccess;
}

}  // namespace tcmis
