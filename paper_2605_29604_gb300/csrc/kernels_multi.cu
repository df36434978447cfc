// kernels_multi.cu -- K <= 8 solves of one graph in one persistent launch.
//
// The solves differ only in their seed, so they share the graph, its
// degree-ordered rows, its round-0 classes (which do not depend on the seed)
// and one worklist: a vertex stays on it while any solve has it undecided.
// Each vertex holds one packed word per solve (the layout of common.cuh),
// the K words of a vertex side by side in one 32-byte sector, so a neighbour
// gather fetches the state of every solve at once and one row scan decides
// the selection test (Phase 1) or the exclusion test (Phase 2) of Algorithm 2
// for all solves that still have the vertex undecided.  Rounds run in lock
// step; a solve that has finished has no undecided vertex and drops out of
// every test.  The result of each solve is the one a single solve with its
// seed gives (the rounds of each solve are exactly its own).
//
// With the tested subgraph and the keyed vertices of a single graph (see
// kernels_csr.cu), the launch works as the single-solve kernel does: the
// words of the keyed vertices only (one 32-byte sector each), round 0's
// exclusion test and every later round on the tested subgraph, and results
// written as vertices are decided (from the create-time bytes out0), with no
// output pass.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tile_tc.cuh"
#include "worklist.cuh"

namespace tcmis {

namespace {

constexpr int kMultiBlock = 512;
constexpr int kMultiMinBlocksPerSm = 2;
constexpr int kMultiWarps = kMultiBlock / 32;
// Schedule of a bin's rows: warp passes of G = 32 / TPR rows, pass k taken
// by warp k mod nwarps (counted from the bin's first warp), so at any moment
// the grid works on a window of about nwarps * G consecutive rows.  On a
// graph with local rows the neighbours' eight-word records (32 bytes per
// vertex, more than L2 holds at 4 M vertices) are then re-read from L2
// rather than DRAM; contiguous chunks per warp spread the window over the
// whole list.

// The eight words of vertex v (solves beyond K hold "out" and never count).
__device__ __forceinline__ void load8(const uint32_t* word8, int v, uint32_t (&w)[kMaxMulti]) {
    const uint4* p = reinterpret_cast<const uint4*>(word8 + (size_t)kMaxMulti * v);
    const uint4 a = p[0], b = p[1];
    w[0] = a.x; w[1] = a.y; w[2] = a.z; w[3] = a.w;
    w[4] = b.x; w[5] = b.y; w[6] = b.z; w[7] = b.w;
}

__device__ __forceinline__ void store8(uint32_t* word8, int v, const uint32_t (&w)[kMaxMulti]) {
    uint4* p = reinterpret_cast<uint4*>(word8 + (size_t)kMaxMulti * v);
    p[0] = make_uint4(w[0], w[1], w[2], w[3]);
    p[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// Solves with v undecided.
__device__ __forceinline__ unsigned undecided_mask(const uint32_t (&w)[kMaxMulti]) {
    unsigned m = 0;
#pragma unroll
    for (int s = 0; s < kMaxMulti; ++s) m |= ((w[s] >> 29) == 1u ? 1u : 0u) << s;
    return m;
}

// Solves in which u (words wu) decides v's test: kSelect: u outranks v
// (words wv; out words never do, in words always do), else: u is in the MIS.
template <bool kSelect>
__device__ __forceinline__ unsigned decides(const uint32_t (&wu)[kMaxMulti], int u,
                                            const uint32_t (&wv)[kMaxMulti], int v) {
    unsigned m = 0;
#pragma unroll
    for (int s = 0; s < kMaxMulti; ++s) {
        const bool hit = kSelect ? (wu[s] > wv[s] || (wu[s] == wv[s] && u > v))
                                 : wu[s] >= kWordInMin;
        m |= (hit ? 1u : 0u) << s;
    }
    return m;
}

// Scan of the row [b, e) of v by the group of TPR lanes of this lane, for the
// solves in `act` (the same for the whole group).  Returns the solves in
// which some neighbour decides the test.  Warp-uniform loop.
template <int TPR, bool kSelect>
__device__ __forceinline__ unsigned group_scan8(const int32_t* __restrict__ col,
                                                const uint32_t* __restrict__ word8, int b, int e,
                                                int v, const uint32_t (&wv)[kMaxMulti],
                                                unsigned act, unsigned glane) {
    unsigned found = 0;
    int p0 = (b & ~3) + 4 * (int)glane;
    for (;;) {
        unsigned hit = 0;
        if ((act & ~found) != 0u && p0 < e) {
            const int4 c = __ldg(reinterpret_cast<const int4*>(col + p0));
            const int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (p0 + q >= b && p0 + q < e) {
                    uint32_t wu[kMaxMulti];
                    load8(word8, cc[q], wu);
                    hit |= decides<kSelect>(wu, cc[q], wv, v);
                }
            }
        }
#pragma unroll
        for (int o = 1; o < TPR; o <<= 1) hit |= __shfl_xor_sync(0xFFFFFFFFu, hit, o);
        found |= hit & act;
        p0 += 4 * TPR;
        const bool more = (act & ~found) != 0u && (p0 - 4 * (int)glane) < e;
        if (!__any_sync(0xFFFFFFFFu, more)) break;
    }
    return found;
}

struct MultiCtx {
    const SolveArgs& a;
    uint32_t* word8;
    int32_t* wbuf;
    int k;                     // solves in the launch
    uint32_t* inb4 = nullptr;  // in-set bits of the tensor-core form (see select_bin8)
};

// Candidates marked in the results by this block (with the keyed vertices).
__shared__ unsigned s_msel;

// Phase 1 over one bin at TPR lanes per row: for every row, the selection
// test in each solve that has the row undecided; candidates are marked in.
// Counts the undecided (vertex, solve) pairs into *alive.
// kRowsTc (the kernel with the exclusion on tensor cores, below): each
// candidate also sets its bits in the in-set bits `x.inb4` (while non-null).
template <int TPR, bool kRowsTc = false>
__device__ __forceinline__ void select_bin8(const MultiCtx& x, const int4* __restrict__ list,
                                            int cnt, WarpSched& ws, unsigned long long* alive,
                                            bool late) {
    constexpr int G = 32 / TPR;
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const unsigned glane = lane % TPR;
    const unsigned gid = lane / TPR;
    const int total = (cnt + G - 1) / G;
    unsigned count = 0;
    for (int k = ws.first(total); k < total; k += ws.nwarps) {
        const int c0 = k * G, c1 = min(c0 + G, cnt);
        for (int base = c0; base < c1; base += G) {
            const int item = base + (int)gid;
            const bool valid = item < c1;
            const int4 rec = valid ? list[item] : make_int4(0, 0, 0, 0);
            uint32_t wv[kMaxMulti];
            unsigned act = 0;
            if (valid) {
                load8(x.word8, rec.x, wv);
                act = undecided_mask(wv);
            } else {
#pragma unroll
                for (int s = 0; s < kMaxMulti; ++s) wv[s] = 0u;
            }
            // round 0 reads the full selection prefixes, later rounds the
            // tested subgraph's rows (col_s0 is col_sel without one)
            const unsigned blocked =
                group_scan8<TPR, true>(late ? x.a.col_s0 : x.a.col_sel, x.word8, rec.y,
                                       valid ? rec.z : 0, rec.x, wv, act, glane);
            const unsigned cand = act & ~blocked;
            if (glane == 0 && valid) {
                count += __popc(act);
                if (cand) {
#pragma unroll
                    for (int s = 0; s < kMaxMulti; ++s)
                        if ((cand >> s) & 1u) wv[s] |= kWordInSet;
                    store8(x.word8, rec.x, wv);
                    if (x.a.out0) {  // results written as decided
                        if (x.a.out)
                            for (int s = 0; s < x.k; ++s)
                                if ((cand >> s) & 1u) x.a.out[(long long)s * x.a.n + rec.x] = 1;
                        atomicAdd(&s_msel, (unsigned)__popc(cand));
                    }
                    if (kRowsTc && x.inb4) {
                        // solve s's bit of v: word 4 (v / 16) + s / 2, bit v % 16 + 16 (s & 1)
                        const int sh = rec.x & 15;
                        uint32_t* wb = x.inb4 + 4LL * (rec.x >> 4);
#pragma unroll
                        for (int j = 0; j < kMaxMulti / 2; ++j) {
                            const uint32_t bits = (((cand >> (2 * j)) & 1u) << sh) |
                                                  (((cand >> (2 * j + 1)) & 1u) << (sh + 16));
                            if (bits) atomicOr(wb + j, bits);
                        }
                    }
                }
            }
        }
    }
    for (int o = 16; o; o >>= 1) count += __shfl_xor_sync(0xFFFFFFFFu, count, o);
    if (lane == 0 && count) atomicAdd(alive, (unsigned long long)count);
}

// Phase 2+3 over one bin: in each solve that still has the row undecided (a
// non-candidate), the exclusion test; the row stays on the worklist while
// some solve keeps it undecided.
template <int TPR>
__device__ __forceinline__ void exclude_bin8(const MultiCtx& x, const int4* __restrict__ list,
                                             int cnt, WarpSched& ws, int* next,
                                             int4* __restrict__ dst) {
    constexpr int G = 32 / TPR;
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const unsigned glane = lane % TPR;
    const unsigned gid = lane / TPR;
    const int total = (cnt + G - 1) / G;
    int fill = 0;
    for (int k = ws.first(total); k < total; k += ws.nwarps) {
        const int c0 = k * G, c1 = min(c0 + G, cnt);
        for (int base = c0; base < c1; base += G) {
            const int item = base + (int)gid;
            const bool valid = item < c1;
            const int4 rec = valid ? list[item] : make_int4(0, 0, 0, 0);
            uint32_t wv[kMaxMulti];
            unsigned und = 0;
            if (valid) {
                load8(x.word8, rec.x, wv);
                und = undecided_mask(wv);
            } else {
#pragma unroll
                for (int s = 0; s < kMaxMulti; ++s) wv[s] = 0u;
            }
            const unsigned excl = group_scan8<TPR, false>(x.a.col_s0, x.word8, rec.y,
                                                          valid ? rec.w : 0, rec.x, wv, und, glane);
            const bool lead = glane == 0 && valid;
            if (lead && excl) {
#pragma unroll
                for (int s = 0; s < kMaxMulti; ++s)
                    if ((excl >> s) & 1u) wv[s] = kWordOut;
                store8(x.word8, rec.x, wv);
            }
            fill = stage_keep(lead && (und & ~excl) != 0u, item, x.wbuf, fill);
            fill = flush_if_full(x.wbuf, fill, G, list, next, dst);
        }
    }
    flush_stage(x.wbuf, fill, list, next, dst);
}

// Lanes per row of a bin of base width BASE (as in the single-solve kernel:
// from round 1 on, the widest group at which the bin fits one grid pass).
template <int BASE>
__device__ __forceinline__ int multi_lanes(int cnt, bool late, int nwarps) {
    if (!late) return BASE;
    const long long lanes = 32LL * nwarps;
    if (BASE < 32 && 32LL * cnt <= lanes) return 32;
    if (BASE < 16 && 16LL * cnt <= lanes) return 16;
    if (BASE < 4 && 4LL * cnt <= lanes) return 4;
    return BASE;
}

template <int BASE, bool kRowsTc = false>
__device__ __forceinline__ void select_at8(const MultiCtx& x, const int4* list, int cnt, bool late,
                                           WarpSched& ws, unsigned long long* alive) {
    switch (multi_lanes<BASE>(cnt, late, ws.nwarps)) {
        case 32: select_bin8<32, kRowsTc>(x, list, cnt, ws, alive, late); break;
        case 16: select_bin8<16, kRowsTc>(x, list, cnt, ws, alive, late); break;
        case 4: select_bin8<4, kRowsTc>(x, list, cnt, ws, alive, late); break;
        default: select_bin8<BASE, kRowsTc>(x, list, cnt, ws, alive, late);
    }
}

template <int BASE>
__device__ __forceinline__ void exclude_at8(const MultiCtx& x, const int4* list, int cnt,
                                            bool late, WarpSched& ws, int* next, int4* dst) {
    switch (multi_lanes<BASE>(cnt, late, ws.nwarps)) {
        case 32: exclude_bin8<32>(x, list, cnt, ws, next, dst); break;
        case 16: exclude_bin8<16>(x, list, cnt, ws, next, dst); break;
        case 4: exclude_bin8<4>(x, list, cnt, ws, next, dst); break;
        default: exclude_bin8<BASE>(x, list, cnt, ws, next, dst);
    }
}

// Eq. 1 words of every vertex for the K seeds (solves beyond K: out); the
// round-0 decisions known at create time are written here too (isolated and
// sure candidates: in, in every solve).
__device__ __forceinline__ void init_words8(const SolveArgs& a, uint32_t* word8, int k,
                                            const uint64_t (&smix)[kMaxMulti]) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    const int32_t n_words = (n + 15) / 16 * 16;
    const float dbar = n > 0 ? average_degree(a.rp[n], n) : 0.f;
    for (long long v = tid; v < n_words; v += nthreads) {
        uint32_t w[kMaxMulti];
        const int deg = v < n ? a.rp[v + 1] - a.rp[v] : 0;
        // in at init in every solve: an in word blocks and excludes whatever
        // its key bits, so these words need no key
        const bool in0 = v < n && (deg == 0 || (a.r0class && a.r0class[v] == 1));
#pragma unroll
        for (int s = 0; s < kMaxMulti; ++s) {
            if (v >= n || s >= k) w[s] = kWordOut;
            else if (in0) w[s] = kWordInMin;
            else w[s] = undecided_word(a.priority, priority_key(a.priority, dbar, deg, smix[s], (uint32_t)v));
        }
        store8(word8, (int)v, w);
    }
}

// With the keyed vertices: their eight words only (the only words any test
// reads), and each solve's result started from the create-time bytes out0.
__device__ __forceinline__ void init_keyed8(const SolveArgs& a, uint32_t* word8, int k,
                                            const uint64_t (&smix)[kMaxMulti]) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    if (a.out) {
        for (int s = 0; s < k; ++s) {
            uint8_t* out = a.out + (long long)s * n;
            long long done = 0;
            if (((uintptr_t)out & 15) == 0) {
                const long long nq = n / 16;
                const uint4* src = reinterpret_cast<const uint4*>(a.out0);
                for (long long i = tid; i < nq; i += nthreads)
                    reinterpret_cast<uint4*>(out)[i] = __ldg(src + i);
                done = nq * 16;
            }
            for (long long v = done + tid; v < n; v += nthreads) out[v] = a.out0[v];
        }
    }
    const float dbar = average_degree(a.rp[n], n);
    for (long long i = tid; i < a.n_keyed; i += nthreads) {
        const int2 kv = __ldg(a.keyed + i);
        uint32_t w[kMaxMulti];
#pragma unroll
        for (int s = 0; s < kMaxMulti; ++s)
            w[s] = s < k ? undecided_word(a.priority, priority_key(a.priority, dbar, kv.y, smix[s],
                                                                   (uint32_t)kv.x))
                         : kWordOut;
        store8(word8, kv.x, w);
    }
}

__global__ void __launch_bounds__(kMultiBlock, kMultiMinBlocksPerSm)
    multi_solve_kernel(const SolveArgs a, uint32_t* word8, int k, const MultiSeeds seeds) {
    __shared__ int32_t s_stage[kMultiWarps][kStageMax];
    __shared__ int s_cnt[kBins];
    const unsigned nblocks = gridDim.x;
    Ctl* ctl = a.ctl;
    PhaseTimes* times = a.times;
    const MultiCtx x{a, word8, s_stage[threadIdx.x / 32], k};
    grid_barrier_start();
    if (threadIdx.x < kBins) s_cnt[threadIdx.x] = a.bin_off[threadIdx.x + 1] - a.bin_off[threadIdx.x];
    if (threadIdx.x == 0) s_msel = 0;
    if (times && blockIdx.x == 0 && threadIdx.x == 0) times->t[0] = global_ns();

    // ---- init: Eq. 1 priorities of every solve
    {
        uint64_t smix[kMaxMulti];
#pragma unroll
        for (int s = 0; s < kMaxMulti; ++s) smix[s] = mix64(seeds.seed[s]);
        if (a.out0) init_keyed8(a, word8, k, smix);
        else init_words8(a, word8, k, smix);
    }
    if (!grid_barrier(ctl, nblocks, a.spin_cap, [times]() {
            if (times) times->t[1] = global_ns();
        }))
        return;

    const int decided0 = a.n_isolated + a.n_sure_in + a.n_sure_out;
    WarpSched ws;
    ws.gw = (int)(blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32);
    ws.nwarps = (int)(nblocks * (blockDim.x / 32));
    ws.base = 0;
    const int* off = a.bin_off;
    for (int r = 0;; ++r) {
        int total = 0;
        for (int j = 0; j < kBins; ++j) total += s_cnt[j];
        if (!(total > 0 || (r == 0 && decided0 > 0))) break;
        if (r >= a.max_rounds) {
            if (threadIdx.x == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            return;
        }
        const int4* src = (r == 0) ? a.order0 : ((r & 1) ? a.wl1 : a.wl0);
        int4* dst = ((r + 1) & 1) ? a.wl1 : a.wl0;
        int* next = ctl->bcnt[(r + 1) & 3];
        unsigned long long* acc = &ctl->alive_acc64[r & 3];
        const int rr = r;
        const bool late = r > 0;

        // ---- Phase 1: selection test of every solve; hubs take a warp per row
        select_at8<32>(x, src + off[4], s_cnt[4], late, ws, acc);
        select_at8<32>(x, src + off[3], s_cnt[3], late, ws, acc);
        select_at8<16>(x, src + off[2], s_cnt[2], late, ws, acc);
        select_at8<4>(x, src + off[1], s_cnt[1], late, ws, acc);
        select_at8<1>(x, src + off[0], s_cnt[0], late, ws, acc);
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [times, rr]() {
                if (times && rr < kStatRounds) times->t[2 + rr] = global_ns();
            }))
            return;

        // ---- Phase 2+3: exclusion test, state update, compaction
        if (r == 0 && !a.out0) {  // (no test reads these words with the keyed vertices)
            const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
            const long long nthreads = (long long)nblocks * blockDim.x;
            const uint4 out4 = make_uint4(kWordOut, kWordOut, kWordOut, kWordOut);
            for (long long i = tid; i < a.n_sure_out; i += nthreads) {
                uint4* p = reinterpret_cast<uint4*>(word8 + (size_t)kMaxMulti * a.sure_out[i]);
                p[0] = out4;
                p[1] = out4;
            }
        }
        // round 0's rows in the tested subgraph, where the graph has one
        if (r == 0 && a.order0_s0) src = a.order0_s0;
        exclude_at8<32>(x, src + off[4], s_cnt[4], late, ws, &next[4], dst + off[4]);
        exclude_at8<32>(x, src + off[3], s_cnt[3], late, ws, &next[3], dst + off[3]);
        exclude_at8<16>(x, src + off[2], s_cnt[2], late, ws, &next[2], dst + off[2]);
        exclude_at8<4>(x, src + off[1], s_cnt[1], late, ws, &next[1], dst + off[1]);
        exclude_at8<1>(x, src + off[0], s_cnt[0], late, ws, &next[0], dst + off[0]);
        const long long extra = r == 0 ? (long long)k * decided0 : 0;
        if (!grid_barrier(
                ctl, nblocks, a.spin_cap,
                [ctl, times, rr, extra]() {
                    // Phase 1 of this round summed its undecided pairs into
                    // alive_acc64[rr & 3] before the previous barrier
                    const unsigned long long cur = ctl->alive_acc64[rr & 3] + (unsigned long long)extra;
                    ctl->alive_acc64[(rr + 2) & 3] = 0;
                    if (times && rr < kStatRounds) times->t[2 + kStatRounds + rr] = global_ns();
                    if (rr < kStatRounds) ctl->alive[rr] = (int)cur;
                    ctl->alive_sum += cur;
                    ctl->rounds = rr + 1;
                    for (int j = 0; j < kBins; ++j) ctl->bcnt[(rr + 2) & 3][j] = 0;
                },
                [next]() {
                    for (int j = 0; j < kBins; ++j) s_cnt[j] = __ldcg(next + j);
                }))
            return;
    }

    // ---- with the keyed vertices the results are complete: the MIS sizes are
    // the create-time part of each solve plus the candidates marked
    if (a.out0) {
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned long long c = s_msel;
            if (blockIdx.x == 0)
                c += (unsigned long long)k * ((unsigned long long)a.n_isolated + a.n_sure_in);
            if (c) atomicAdd(&ctl->mis_size, c);
        }
        return;
    }
    // ---- output: out[s * n + v] = [v in the MIS of solve s]
    if (a.out) {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        unsigned in_cnt = 0;
        for (long long v = tid; v < a.n; v += nthreads) {
            uint32_t w[kMaxMulti];
            load8(word8, (int)v, w);
#pragma unroll
            for (int s = 0; s < kMaxMulti; ++s) {
                if (s < k) {
                    const bool in = w[s] >= kWordInMin;
                    a.out[(long long)s * a.n + v] = in;
                    in_cnt += in;
                }
            }
        }
        for (int o = 16; o; o >>= 1) in_cnt += __shfl_xor_sync(0xFFFFFFFFu, in_cnt, o);
        if (lane_id() == 0 && in_cnt) atomicAdd(&ctl->mis_size, (unsigned long long)in_cnt);
    }
}

// ---------------------------------------------------------------- rows + tensor cores
//
// The same k solves with Phase 2 as the product N_c = A x [C_1 .. C_k] over
// the graph's 16 x 16 bitmask tiles on the single-bit MMA (Sec. 3.1 Phase 2,
// Sec. 3.2), and Phase 1 as above on the CSR rows with per-vertex worklists.
// (On tiles alone, Phase 1 keeps a row block on its list while any of its
// 16 x k entries is undecided and scans no faster than the rows; the product
// is where the tiles pay.)  Per round:
//
//   Phase 1  selection test over the vertex lists (select_bin8<kRowsTc>):
//            candidates are marked in their words and set their bits in the
//            in-set bits inb4 (4 words per row block: solve s's 16 bits of
//            row block b at word 4 b + s / 2, bits 16 (s & 1) ..).
//   Phase 2  exclusion test over the row-block list: D = A x C with C the
//            in-set bits of every round so far.  That equals this round's
//            product on the entries it decides: a vertex undecided at a
//            round's start has no neighbour in the set (it would have been
//            excluded), so its in-set neighbours are this round's candidates.
//            Undecided entries with D > 0 are out.  A row block stays on the
//            row-block list while it keeps an undecided entry, and each row
//            that keeps one goes on the next vertex list, in its degree bin,
//            with its record rebuilt from row_ptr (a graph without
//            create-time structures has no selection prefixes).
//
// The product costs the same for a listed row block however few of its
// 16 x k entries are still undecided, and the scans of the CSR form shrink
// with them.  So after each Phase 1 the kernel compares the round's undecided
// pairs with the entries of the listed row blocks: from the first round where
// fewer than tc_fill / 256 of them are undecided, Phase 2 is the CSR form's
// exclusion scan over the (exact) vertex lists for the rest of the solve, and
// the loop ends when those are empty; until then it ends when the row-block
// list is empty.  (Where the break-even lies depends on the graph's degree and
// tile density; the host's autotuner times a few fills.)  Either way every
// entry of every solve is decided at the end, and the round count is
// Algorithm 2's.  Graphs with create-time round-0 structures do not take this
// kernel (the host checks).
//
// A warp takes row blocks gw, gw + W, ... of the list; each tile of a row
// block goes to one lane, whose bits arrive by cp.async a row block ahead.
// Where only one degree bin is in use, survivors are staged without their
// row degrees.

constexpr int kRbKeep = 64;   // row blocks staged per warp before an append
constexpr int kSvMax = 48;    // survivors staged per warp and bin before an append
// shared words per warp: two buffers of 32 tiles' bits (8 words each), the
// listed tiles' C segments and slots, the staged row blocks, the staged
// survivors of each bin
constexpr int kRtBits = 2 * 32 * 8;
constexpr int kRtWords = kRtBits + 128 + 32 + 16 + kRbKeep + kBins * kSvMax;  // + 16 row masks
constexpr int kRtSmemBytes = kMultiWarps * kRtWords * 4;

__device__ __forceinline__ uint2 ld_pair8(const uint32_t* word8, int v, int q) {
    return *reinterpret_cast<const uint2*>(word8 + (size_t)kMaxMulti * v + 2 * q);
}

__device__ __forceinline__ void st_pair8(uint32_t* word8, int v, int q, uint2 w) {
    *reinterpret_cast<uint2*>(word8 + (size_t)kMaxMulti * v + 2 * q) = w;
}

// Lane l starts the copy of tile t0 + l of a row block (its 32 bytes of bits)
// into slot l of `buf` and returns the tile's column block (-1: no tile);
// commits one copy group either way.
__device__ __forceinline__ int rb_copy(const SolveArgs& a, int t0, int t1, uint32_t* buf) {
    const int t = t0 + (int)lane_id();
    int cb = -1;
    if (t < t1) {
        cb = __ldg(a.tcol + t);
        const uint64_t* src = a.tbits + 4LL * t;
        cp_async16(buf + 8 * lane_id(), src);
        cp_async16(buf + 8 * lane_id() + 4, src + 2);
    }
    cp_async_commit();
    return cb;
}

// Appends a warp's staged survivors of bin j (vertex ids) to the bin's list
// as row records {v, row begin, row end, row end}.
__device__ __forceinline__ void flush_survivors(const SolveArgs& a, const int32_t* sv, int cnt,
                                                int* next, int4* __restrict__ dst) {
    __syncwarp();
    const unsigned lane = lane_id();
    int o = 0;
    if (lane == 0) o = atomicAdd(next, cnt);
    o = __shfl_sync(0xFFFFFFFFu, o, 0);
    for (int i = (int)lane; i < cnt; i += 32) {
        const int v = sv[i];
        const int b = __ldg(a.rp + v), e = __ldg(a.rp + v + 1);
        dst[o + i] = make_int4(v, b, e, e);
    }
    __syncwarp();
}

__device__ __forceinline__ void flush_blocks(const int32_t* keep, int cnt, int* next,
                                             int32_t* __restrict__ dst) {
    __syncwarp();
    const unsigned lane = lane_id();
    int o = 0;
    if (lane == 0) o = atomicAdd(next, cnt);
    o = __shfl_sync(0xFFFFFFFFu, o, 0);
    for (int k = (int)lane; k < cnt; k += 32) dst[o + k] = keep[k];
    __syncwarp();
}

// Phases 2 and 3 over the row-block list `list` (cnt entries).  Lane (g, q)
// owns rows g and g + 8 in solves 2q and 2q + 1 (the MMA's D fragment).
// `sw`: the warp's kRtWords words of shared memory.  next_rb / dst_rb: the
// next row-block list; next_v / dst_v: the next vertex lists, per bin;
// one_bin: the bin of every row of degree >= 1 when only one bin is in use,
// else -1.
//
// Warp gw takes list entries gw, gw + W, ... (W warps).  While it multiplies
// one row block, the next one's bits are on their way into the other shared
// buffer (cp.async), its words and column blocks into registers, the tile
// range of the one after and the list entry of the third: each load has a
// whole row block's work to arrive in.
template <bool kSplit>
__device__ __forceinline__ void rows_tc_exclude(const SolveArgs& a, uint32_t* word8,
                                                const uint32_t* inb4,
                                                const int32_t* __restrict__ list, int cnt,
                                                int* next_rb, int32_t* __restrict__ dst_rb,
                                                int* next_v, int4* __restrict__ dst_v,
                                                uint32_t* sw, int one_bin) {
    const unsigned lane = lane_id();
    const int g = (int)(lane >> 2), q = (int)(lane & 3);
    const long long nw = (long long)gridDim.x * (blockDim.x / 32);
    const long long gw = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (gw >= cnt) return;
    uint32_t* cs = sw + kRtBits;
    int32_t* idx = reinterpret_cast<int32_t*>(cs + 128);
    uint32_t* sd = reinterpret_cast<uint32_t*>(idx + 32);  // 16 row masks
    int32_t* keep = reinterpret_cast<int32_t*>(sd + 16);
    int32_t* sv = keep + kRbKeep;  // kBins x kSvMax
    int nkeep = 0;
    uint32_t nsv = 0;  // survivors staged per bin, 6 bits each (at most kSvMax)
    const int32_t* off = a.bin_off;
    // the in-set bits were written in Phase 1 of this launch: read through L2
    auto cseg4 = [inb4](int cb) -> uint4 {
        return cb >= 0 ? __ldcg(reinterpret_cast<const uint4*>(inb4 + 4LL * cb))
                       : make_uint4(0u, 0u, 0u, 0u);
    };
    // stage 0: the current row block; 1: the next; 2: the one after
    int rb0 = list[gw];
    int t00 = a.trp[rb0], t10 = a.trp[rb0 + 1];
    const int cb0 = rb_copy(a, t00, t10, sw);
    uint2 w0 = ld_pair8(word8, rb0 * 16 + g, q), w1 = ld_pair8(word8, rb0 * 16 + g + 8, q);
    int rb1 = -1, t01 = 0, t11 = 0, rb2 = -1;
    if (gw + nw < cnt) {
        rb1 = list[gw + nw];
        t01 = a.trp[rb1];
        t11 = a.trp[rb1 + 1];
    }
    if (gw + 2 * nw < cnt) rb2 = list[gw + 2 * nw];
    uint4 c = cseg4(cb0);
    int it = 0;
    for (long long item = gw; item < cnt; item += nw, ++it) {
        uint32_t* bits = sw + 256 * (it & 1);
        // ---- the next row block's bits, words and column blocks; the tile
        // range of the one after; the list entry of the third
        int cb1 = -1;
        uint2 w0n = make_uint2(0u, 0u), w1n = w0n;
        if (rb1 >= 0) {
            cb1 = rb_copy(a, t01, t11, sw + 256 * ((it + 1) & 1));
            w0n = ld_pair8(word8, rb1 * 16 + g, q);
            w1n = ld_pair8(word8, rb1 * 16 + g + 8, q);
        } else {
            cp_async_commit();  // one group per row block, for the count below
        }
        int t02 = 0, t12 = 0;
        if (rb2 >= 0) {
            t02 = a.trp[rb2];
            t12 = a.trp[rb2 + 1];
        }
        const int rb3 = item + 3 * nw < cnt ? list[item + 3 * nw] : -1;
        const int rb = rb0;
        const int rpv = one_bin >= 0 ? 0 : __ldg(a.rp + min(rb * 16 + (int)min(lane, 16u), a.n));

        // undecided entries after Phase 1 (the non-candidates): a row block
        // without any needs no product and leaves the list
        const int v0 = rb * 16 + g, v1 = v0 + 8;
        const unsigned und = ((w0.x >> 29) == 1u ? 1u : 0u) | ((w0.y >> 29) == 1u ? 2u : 0u) |
                             ((w1.x >> 29) == 1u ? 4u : 0u) | ((w1.y >> 29) == 1u ? 8u : 0u);
        const bool work = __any_sync(0xFFFFFFFFu, und != 0u);

        // ---- D = A x C of this row block: its bits are the older copy group
        cp_async_wait<1>();
        if (kSplit && lane < 16) sd[lane] = 0u;
        __syncwarp();
        int acc[4] = {0, 0, 0, 0};
        if (work) b1_pass<kSplit>(bits, c, cs, idx, sd, acc);
        for (int tb = t00 + 32; work && tb < t10; tb += 32) {  // row blocks of > 32 tiles
            const int t = tb + (int)lane;
            uint4 cc = make_uint4(0u, 0u, 0u, 0u);
            if (t < t10) {
                const uint4* bp = reinterpret_cast<const uint4*>(a.tbits + 4LL * t);
                *reinterpret_cast<uint4*>(bits + 8 * lane) = __ldg(bp);
                *reinterpret_cast<uint4*>(bits + 8 * lane + 4) = __ldg(bp + 1);
                cc = cseg4(__ldg(a.tcol + t));
            }
            __syncwarp();
            b1_pass<kSplit>(bits, cc, cs, idx, sd, acc);
        }
        uint32_t sd0 = 0, sd8 = 0;
        if (kSplit) {
            __syncwarp();  // the sparse tiles' row masks
            sd0 = sd[g] >> (2 * q);
            sd8 = sd[g + 8] >> (2 * q);
        }
        const uint4 c_n = cseg4(cb1);  // the next row block's C segments

        // ---- update: undecided entries (the non-candidates) with D > 0 are out
        const unsigned out = und & ((acc[0] > 0 || (sd0 & 1u) ? 1u : 0u) |
                                    (acc[1] > 0 || (sd0 & 2u) ? 2u : 0u) |
                                    (acc[2] > 0 || (sd8 & 1u) ? 4u : 0u) |
                                    (acc[3] > 0 || (sd8 & 2u) ? 8u : 0u));
        if (out & 3u) {
            if (out & 1u) w0.x = kWordOut;
            if (out & 2u) w0.y = kWordOut;
            st_pair8(word8, v0, q, w0);
        }
        if (out & 12u) {
            if (out & 4u) w1.x = kWordOut;
            if (out & 8u) w1.y = kWordOut;
            st_pair8(word8, v1, q, w1);
        }
        const unsigned rem = und & ~out;
        if (__any_sync(0xFFFFFFFFu, rem != 0u)) {
            if (lane == 0) keep[nkeep] = rb;
            if (++nkeep == kRbKeep) {
                flush_blocks(keep, nkeep, next_rb, dst_rb);
                nkeep = 0;
            }
            // rows with an undecided entry in some solve: onto the next vertex
            // list, in their degree bin; lane (g, 0) takes rows g and g + 8,
            // which keep an entry iff some lane (g, q) does
            const unsigned k0 = __ballot_sync(0xFFFFFFFFu, (rem & 3u) != 0u);
            const unsigned k1 = __ballot_sync(0xFFFFFFFFu, (rem & 12u) != 0u);
            const bool r0 = q == 0 && ((k0 >> (lane & ~3u)) & 0xFu) != 0u;
            const bool r1 = q == 0 && ((k1 >> (lane & ~3u)) & 0xFu) != 0u;
            int j0 = -1, j1 = -1;
            if (one_bin >= 0) {
                // every row of degree >= 1 in one bin: no degrees needed
                j0 = r0 ? one_bin : -1;
                j1 = r1 ? one_bin : -1;
            } else {
                const int b0 = __shfl_sync(0xFFFFFFFFu, rpv, g);
                const int bm = __shfl_sync(0xFFFFFFFFu, rpv, g + 1);
                const int b8 = __shfl_sync(0xFFFFFFFFu, rpv, g + 8);
                const int be = __shfl_sync(0xFFFFFFFFu, rpv, g + 9);
                if (r0) {
                    j0 = 0;
#pragma unroll
                    for (int t = 0; t < kBins - 1; ++t) j0 += bm - b0 > a.thr[t];
                }
                if (r1) {
                    j1 = 0;
#pragma unroll
                    for (int t = 0; t < kBins - 1; ++t) j1 += be - b8 > a.thr[t];
                }
            }
            // one bin for every kept row (the usual case): one pass of staging
            int jr = one_bin;
            bool single = one_bin >= 0;
            if (!single) {
                jr = __shfl_sync(0xFFFFFFFFu, j0 >= 0 ? j0 : j1,
                                 __ffs(__ballot_sync(0xFFFFFFFFu, j0 >= 0 || j1 >= 0)) - 1);
                single = !__any_sync(0xFFFFFFFFu, (j0 >= 0 && j0 != jr) || (j1 >= 0 && j1 != jr));
            }
#pragma unroll
            for (int bj = 0; bj < kBins; ++bj) {
                if (single && bj != jr) continue;
                const unsigned m0 = __ballot_sync(0xFFFFFFFFu, j0 == bj);
                const unsigned m1 = __ballot_sync(0xFFFFFFFFu, j1 == bj);
                if ((m0 | m1) == 0u) continue;
                const int have = (int)((nsv >> (6 * bj)) & 63u);
                int32_t* dst = sv + bj * kSvMax + have;
                if (j0 == bj) dst[__popc(m0 & lanemask_lt())] = v0;
                if (j1 == bj) dst[__popc(m0) + __popc(m1 & lanemask_lt())] = v1;
                const int now = have + __popc(m0) + __popc(m1);
                nsv = (nsv & ~(63u << (6 * bj))) | ((uint32_t)now << (6 * bj));
                if (now > kSvMax - 16) {
                    flush_survivors(a, sv + bj * kSvMax, now, &next_v[bj], dst_v + off[bj]);
                    nsv &= ~(63u << (6 * bj));
                }
            }
        }
        // ---- shift the stages
        rb0 = rb1;
        t00 = t01;
        t10 = t11;
        w0 = w0n;
        w1 = w1n;
        c = c_n;
        rb1 = rb2;
        t01 = t02;
        t11 = t12;
        rb2 = rb3;
    }
    cp_async_wait<0>();
    if (nkeep) flush_blocks(keep, nkeep, next_rb, dst_rb);
#pragma unroll
    for (int bj = 0; bj < kBins; ++bj) {
        const int have = (int)((nsv >> (6 * bj)) & 63u);
        if (have) flush_survivors(a, sv + bj * kSvMax, have, &next_v[bj], dst_v + off[bj]);
    }
}

// kSplit: the exclusion passes take sparse tiles on CUDA cores where that
// saves an MMA (row blocks of more than eight tiles; the host picks the form
// from the graph's tiles per row block).
template <bool kSplit>
__global__ void __launch_bounds__(kMultiBlock, kMultiMinBlocksPerSm)
    multi_rows_tc_kernel(const SolveArgs a, uint32_t* word8, uint32_t* inb4, int k,
                         const MultiSeeds seeds, int tc_fill) {
    // kRtSmemBytes of dynamic shared memory: kRtWords words per warp
    extern __shared__ __align__(16) uint32_t s_rt[];
    __shared__ int s_cnt[kBins];
    __shared__ int s_rbcnt;
    __shared__ int s_tc;  // Phase 2 of this round on tensor cores
    const unsigned nblocks = gridDim.x;
    Ctl* ctl = a.ctl;
    PhaseTimes* times = a.times;
    uint32_t* sw = s_rt + (threadIdx.x / 32) * kRtWords;
    // the one degree bin in use, if there is only one (-1: several)
    int one_bin = -1;
    for (int j = 0; j < kBins; ++j)
        if (a.bin_off[j + 1] > a.bin_off[j]) one_bin = one_bin == -1 ? j : -2;
    if (one_bin < 0) one_bin = -1;
    // the CSR form's Phase 2 stages its survivors in the same shared words
    MultiCtx x{a, word8, reinterpret_cast<int32_t*>(sw), k};
    x.inb4 = inb4;
    bool tc = true;
    grid_barrier_start();
    if (threadIdx.x < kBins) s_cnt[threadIdx.x] = a.bin_off[threadIdx.x + 1] - a.bin_off[threadIdx.x];
    if (threadIdx.x == 0) s_rbcnt = a.nrb;
    if (times && blockIdx.x == 0 && threadIdx.x == 0) times->t[0] = global_ns();

    // ---- init: Eq. 1 priorities of every solve, no vertex in the set, every
    // row block on the list
    {
        uint64_t smix[kMaxMulti];
#pragma unroll
        for (int s = 0; s < kMaxMulti; ++s) smix[s] = mix64(seeds.seed[s]);
        init_words8(a, word8, k, smix);
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        for (long long i = tid; i < (long long)a.nrb; i += nthreads) {
            reinterpret_cast<uint4*>(inb4)[i] = make_uint4(0u, 0u, 0u, 0u);
            a.rbl0[i] = (int32_t)i;
        }
    }
    if (!grid_barrier(ctl, nblocks, a.spin_cap, [times]() {
            if (times) times->t[1] = global_ns();
        }))
        return;

    const int decided0 = a.n_isolated;
    WarpSched ws;
    ws.gw = (int)(blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32);
    ws.nwarps = (int)(nblocks * (blockDim.x / 32));
    ws.base = 0;
    const int* off = a.bin_off;
    for (int r = 0;; ++r) {
        if (tc) {
            if (s_rbcnt == 0) break;
        } else {
            int total = 0;
            for (int j = 0; j < kBins; ++j) total += s_cnt[j];
            if (total == 0) break;
        }
        if (r >= a.max_rounds) {
            if (threadIdx.x == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            return;
        }
        const int4* src = (r == 0) ? a.order0 : ((r & 1) ? a.wl1 : a.wl0);
        int4* dst = ((r + 1) & 1) ? a.wl1 : a.wl0;
        int* next = ctl->bcnt[(r + 1) & 3];
        unsigned long long* acc = &ctl->alive_acc64[r & 3];
        const int rr = r;
        const bool late = r > 0;

        // ---- Phase 1: selection test of every solve on the CSR rows
        select_at8<32, true>(x, src + off[4], s_cnt[4], late, ws, acc);
        select_at8<32, true>(x, src + off[3], s_cnt[3], late, ws, acc);
        select_at8<16, true>(x, src + off[2], s_cnt[2], late, ws, acc);
        select_at8<4, true>(x, src + off[1], s_cnt[1], late, ws, acc);
        select_at8<1, true>(x, src + off[0], s_cnt[0], late, ws, acc);
        // every block decides the form of Phase 2 from the same counts
        const int rbcnt = s_rbcnt;
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [times, rr]() {
                if (times && rr < kStatRounds) times->t[2 + rr] = global_ns();
            },
            [ctl, rr, rbcnt, k, tc, tc_fill]() {
                const unsigned long long und = __ldcg(&ctl->alive_acc64[rr & 3]);
                s_tc = tc && und * 256ull >= (unsigned long long)rbcnt * 16ull * k * tc_fill;
            }))
            return;
        if (tc && !s_tc) {
            tc = false;  // for the rest of the solve
            x.inb4 = nullptr;
        }

        // ---- Phases 2 and 3: exclusion test, update, compaction
        if (tc) {
            rows_tc_exclude<kSplit>(a, word8, inb4, (r & 1) ? a.rbl1 : a.rbl0, rbcnt,
                            &ctl->cnt[(r + 1) & 3], (r & 1) ? a.rbl0 : a.rbl1, next, dst, sw,
                            one_bin);
        } else {
            exclude_at8<32>(x, src + off[4], s_cnt[4], late, ws, &next[4], dst + off[4]);
            exclude_at8<32>(x, src + off[3], s_cnt[3], late, ws, &next[3], dst + off[3]);
            exclude_at8<16>(x, src + off[2], s_cnt[2], late, ws, &next[2], dst + off[2]);
            exclude_at8<4>(x, src + off[1], s_cnt[1], late, ws, &next[1], dst + off[1]);
            exclude_at8<1>(x, src + off[0], s_cnt[0], late, ws, &next[0], dst + off[0]);
        }
        const long long extra = r == 0 ? (long long)k * decided0 : 0;
        if (!grid_barrier(
                ctl, nblocks, a.spin_cap,
                [ctl, times, rr, extra]() {
                    const unsigned long long cur = ctl->alive_acc64[rr & 3] + (unsigned long long)extra;
                    ctl->alive_acc64[(rr + 2) & 3] = 0;
                    if (times && rr < kStatRounds) times->t[2 + kStatRounds + rr] = global_ns();
                    if (rr < kStatRounds) ctl->alive[rr] = (int)cur;
                    ctl->alive_sum += cur;
                    ctl->rounds = rr + 1;
                    for (int j = 0; j < kBins; ++j) ctl->bcnt[(rr + 2) & 3][j] = 0;
                    ctl->cnt[(rr + 2) & 3] = 0;
                },
                [ctl, next, rr]() {
                    for (int j = 0; j < kBins; ++j) s_cnt[j] = __ldcg(next + j);
                    s_rbcnt = __ldcg(&ctl->cnt[(rr + 1) & 3]);
                }))
            return;
    }

    // ---- output: out[s * n + v] = [v in the MIS of solve s]
    if (a.out) {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        unsigned in_cnt = 0;
        for (long long v = tid; v < a.n; v += nthreads) {
            uint32_t w[kMaxMulti];
            load8(word8, (int)v, w);
#pragma unroll
            for (int s = 0; s < kMaxMulti; ++s) {
                if (s < k) {
                    const bool in = w[s] >= kWordInMin;
                    a.out[(long long)s * a.n + v] = in;
                    in_cnt += in;
                }
            }
        }
        for (int o = 16; o; o >>= 1) in_cnt += __shfl_xor_sync(0xFFFFFFFFu, in_cnt, o);
        if (lane_id() == 0 && in_cnt) atomicAdd(&ctl->mis_size, (unsigned long long)in_cnt);
    }
}

}  // namespace

cudaError_t launch_multi_solve(const SolveArgs& a, uint32_t* word8, int k,
                               const MultiSeeds& seeds, int grid, cudaStream_t s) {
    void* args[] = {const_cast<SolveArgs*>(&a), &word8, &k, const_cast<MultiSeeds*>(&seeds)};
    return cudaLaunchCooperativeKernel((const void*)multi_solve_kernel, dim3(grid),
                                       dim3(kMultiBlock), args, 0, s);
}

cudaError_t launch_multi_rows_tc_solve(const SolveArgs& a, uint32_t* word8, uint32_t* inb4, int k,
                                      const MultiSeeds& seeds, int tc_fill, bool split, int grid,
                                      cudaStream_t s) {
    void* args[] = {const_cast<SolveArgs*>(&a), &word8, &inb4, &k,
                    const_cast<MultiSeeds*>(&seeds), &tc_fill};
    const void* fn = split ? (const void*)multi_rows_tc_kernel<true>
                           : (const void*)multi_rows_tc_kernel<false>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kMultiBlock), args, kRtSmemBytes, s);
}

int multi_rows_tc_max_coresident_blocks(int device) {
    int per_sm = 1 << 30, sms = 0;
    // above the default 48 KB of dynamic shared memory per block; the grid
    // must fit either form
    const void* fns[] = {(const void*)multi_rows_tc_kernel<false>,
                         (const void*)multi_rows_tc_kernel<true>};
    for (const void* fn : fns) {
        int p = 0;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kRtSmemBytes) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, fn, kMultiBlock, kRtSmemBytes) !=
                cudaSuccess)
            return 0;
        per_sm = std::min(per_sm, p);
    }
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

int multi_max_coresident_blocks(int device) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)multi_solve_kernel,
                                                      kMultiBlock, 0) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

}  // namespace tcmis
