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
// Worklists are split into degree bins (fixed at create time, degrees do not
// change): bin j holds the vertices with deg in (thr[j-1], thr[j]].  Bins 0..3
// are scanned by groups of 1, 4, 16 and 32 lanes, bin 4 (hubs) by a whole
// block.  Warps take chunks of a bin's list through an atomic counter (heavy
// bins first; the chunk shrinks when a bin is small so that the chunks spread
// over all warps).  In Phase 2 a chunk is first triaged one vertex per lane
// (candidates need no scan), the remaining vertices are scanned by groups,
// and survivors are staged in shared memory and appended to the next list
// with one atomic per chunk.  Each lane loads 16-byte aligned int4 slices of
// col_idx and gathers the four neighbour words; scans stop at the first
// neighbour that decides the test.
#include <algorithm>
#include <cstdio>
#include <vector>

#include "common.cuh"
#include "init.cuh"
#include "internal.h"

namespace tcmis {

constexpr int kCsrBlock = 512;
constexpr int kCsrMinBlocksPerSm = 3;
constexpr int kWarps = kCsrBlock / 32;

// Rows per chunk taken by one warp, per bin (bin 4 is taken a row at a time
// by a whole block).
constexpr int kChunk0 = 256, kChunk1 = 128, kChunk2 = 64, kChunk3 = 32;
constexpr int kStageMax = 256;

// Does u outrank v in the selection test?  `wu` is u's word, `wv` v's
// (undecided, so wv is v's key): out words never outrank, undecided ones
// compare by key then id, an in word (a candidate of this round) always does.
__device__ __forceinline__ bool outranks(uint32_t wu, int u, uint32_t wv, int v) {
    return wu > wv || (wu == wv && u > v);
}

// Scan of the row [b, e) of v by the group of TPR lanes of this lane; kSelect:
// is there a neighbour that outranks v, else: is there an in neighbour.
// Warp-uniform loop: every lane of the warp iterates until no group has work.
template <int TPR, bool kSelect>
__device__ __forceinline__ bool group_scan(const int32_t* __restrict__ col,
                                           const uint32_t* __restrict__ word, int b, int e,
                                           int v, uint32_t wv, unsigned glane, unsigned gshift) {
    constexpr unsigned gbits = (TPR == 32) ? 0xFFFFFFFFu : ((1u << TPR) - 1u);
    bool found = false;
    int p0 = (b & ~3) + 4 * (int)glane;
    for (;;) {
        bool hit = false;
        if (!found && p0 < e) {
            const int4 c = __ldg(reinterpret_cast<const int4*>(col + p0));
            const uint32_t w0 = (p0 >= b) ? ld_word_l1(word + c.x) : 0u;
            const uint32_t w1 = (p0 + 1 >= b && p0 + 1 < e) ? ld_word_l1(word + c.y) : 0u;
            const uint32_t w2 = (p0 + 2 >= b && p0 + 2 < e) ? ld_word_l1(word + c.z) : 0u;
            const uint32_t w3 = (p0 + 3 >= b && p0 + 3 < e) ? ld_word_l1(word + c.w) : 0u;
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

// Work split of a bin of `cnt` rows into chunks taken through one counter:
// `nbig` chunks of `ch` rows (at most CH, fewer when the bin is small so that
// the chunks spread over all warps) cover most of the bin, then chunks of one
// warp pass (G rows) finish it, so that the last warps of a phase do not
// wait long for a straggler.
struct ChunkPlan {
    int ch;
    int nbig;
    int total;  // chunks in all
    __device__ __forceinline__ void range(int k, int cnt, int& c0, int& c1, int G) const {
        if (k < nbig) {
            c0 = k * ch;
            c1 = c0 + ch;
        } else {
            c0 = nbig * ch + (k - nbig) * G;
            c1 = min(c0 + G, cnt);
        }
    }
};

template <int G, int CH>
__device__ __forceinline__ ChunkPlan plan_of(int cnt) {
    const long long nwarps = (long long)gridDim.x * (blockDim.x / 32);
    long long per = (cnt + nwarps - 1) / nwarps;
    per = ((per + G - 1) / G) * G;
    if (per < G) per = G;
    ChunkPlan p;
    p.ch = per < CH ? (int)per : CH;
    p.nbig = (int)((long long)cnt * 7 / 8 / p.ch);
    p.total = p.nbig + (cnt - p.nbig * p.ch + G - 1) / G;
    return p;
}

__device__ __forceinline__ long long global_warp() {
    return (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
}

// Phase 1, bins 0..3: selection test of every row of the bin's list.
template <int TPR, int CH>
__device__ __forceinline__ void select_bin(const SolveArgs& a, const int32_t* __restrict__ list,
                                           int cnt, unsigned* grab) {
    constexpr int G = 32 / TPR;
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const unsigned glane = lane % TPR;
    const unsigned gid = lane / TPR;
    const unsigned gshift = gid * TPR;
    const ChunkPlan plan = plan_of<G, CH>(cnt);
    if (global_warp() >= plan.total) return;
    for (;;) {
        int k = 0;
        if (lane == 0) k = (int)atomicAdd(grab, 1u);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (k >= plan.total) break;
        int c0, c1;
        plan.range(k, cnt, c0, c1, G);
        for (int base = c0; base < c1; base += G) {
            const int item = base + (int)gid;
            const bool valid = item < c1;
            const int v = valid ? list[item] : 0;
            // every vertex of W_r is undecided and nothing else writes its
            // word in this phase, so each lane may load it
            const uint32_t wv = valid ? ld_word_l1(a.word + v) : 0u;
            const int b = valid ? a.rp[v] : 0;
            // only neighbours of degree <= deg(v) + 1 can outrank v
            const int e = valid ? (a.split ? b + a.split[v] : a.rp[v + 1]) : 0;
            const bool blocked =
                group_scan<TPR, true>(a.col_sel, a.word, b, e, v, wv, glane, gshift);
            if (valid && !blocked && glane == 0) a.word[v] = wv | kWordInSet;
        }
    }
}

// Phase 2+3, bins 0..3: triage, exclusion test, compaction.
template <int TPR, int CH>
__device__ __forceinline__ void exclude_bin(const SolveArgs& a, const int32_t* __restrict__ list,
                                            int cnt, unsigned* grab, int* next,
                                            int32_t* __restrict__ dst, int32_t* wscan,
                                            int32_t* wkeep) {
    static_assert(CH <= kStageMax, "chunk exceeds the staging buffers");
    constexpr int G = 32 / TPR;
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const unsigned glane = lane % TPR;
    const unsigned gid = lane / TPR;
    const unsigned gshift = gid * TPR;
    const ChunkPlan plan = plan_of<G, CH>(cnt);
    if (global_warp() >= plan.total) return;
    for (;;) {
        int k = 0;
        if (lane == 0) k = (int)atomicAdd(grab, 1u);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        if (k >= plan.total) break;
        int c0, c1;
        plan.range(k, cnt, c0, c1, G);
        // triage, one vertex per lane: candidates of Phase 1 are done
        int nscan = 0;
        for (int base = c0; base < c1; base += 32) {
            const int item = base + (int)lane;
            const int v = item < c1 ? list[item] : -1;
            const bool scan = v >= 0 && ld_word_l1(a.word + v) < kWordInMin;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, scan);
            if (scan) wscan[nscan + __popc(bal & lanemask_lt())] = v;
            nscan += __popc(bal);
        }
        __syncwarp();
        // exclusion test of the remaining (undecided) vertices
        int nkeep = 0;
        for (int base = 0; base < nscan; base += G) {
            const int item = base + (int)gid;
            const bool valid = item < nscan;
            const int v = valid ? wscan[item] : 0;
            const int b = valid ? a.rp[v] : 0;
            const int e = valid ? a.rp[v + 1] : 0;
            const bool excl = group_scan<TPR, false>(a.col_sel, a.word, b, e, v, 0u, glane, gshift);
            const bool lead = glane == 0;
            if (valid && excl && lead) a.word[v] = kWordOut;
            const bool keep = valid && !excl && lead;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
            if (keep) wkeep[nkeep + __popc(bal & lanemask_lt())] = v;
            nkeep += __popc(bal);
        }
        __syncwarp();
        if (nkeep) {
            int o = 0;
            if (lane == 0) o = atomicAdd(next, nkeep);
            o = __shfl_sync(0xFFFFFFFFu, o, 0);
            for (int i = (int)lane; i < nkeep; i += 32) dst[o + i] = wkeep[i];
        }
        __syncwarp();
    }
}

// Bin 4 (hubs): the whole block scans one row at a time.  kSelect: Phase 1,
// else Phase 2+3 (survivors appended one by one: hub rows are few).
template <bool kSelect>
__device__ __forceinline__ void block_bin(const SolveArgs& a, const int32_t* __restrict__ list,
                                          int cnt, unsigned* grab, int* next,
                                          int32_t* __restrict__ dst) {
    __shared__ int s_row;
    if ((int)blockIdx.x >= cnt) return;  // no row left for this block
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_row = (int)atomicAdd(grab, 1u);
        __syncthreads();
        const int item = s_row;
        if (item >= cnt) break;
        const int v = list[item];
        // the word of v does not change during this row's scan in either phase
        const uint32_t wv = ld_word_l1(a.word + v);
        if (!kSelect && wv >= kWordInMin) continue;  // a candidate: nothing to do
        const int b = a.rp[v];
        const int e = (kSelect && a.split) ? b + a.split[v] : a.rp[v + 1];
        bool found = false;
        for (int base = b & ~3; base < e; base += 4 * (int)blockDim.x) {
            const int p0 = base + 4 * (int)threadIdx.x;
            bool hit = false;
            if (p0 < e) {
                const int4 c = __ldg(reinterpret_cast<const int4*>(a.col_sel + p0));
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
        if (threadIdx.x == 0) {
            if (kSelect) {
                if (!found) a.word[v] = wv | kWordInSet;
            } else if (found) {
                a.word[v] = kWordOut;
            } else {
                dst[atomicAdd(next, 1)] = v;
            }
        }
    }
}

__global__ void __launch_bounds__(kCsrBlock, kCsrMinBlocksPerSm)
    csr_solve_kernel(const SolveArgs a) {
    __shared__ int32_t s_scan[kWarps][kStageMax];
    __shared__ int32_t s_keep[kWarps][kStageMax];
    const unsigned lane = lane_id();
    const unsigned nblocks = gridDim.x;
    Ctl* ctl = a.ctl;
    PhaseTimes* times = a.times;
    const int32_t n = a.n;
    int32_t* wscan = s_scan[threadIdx.x / 32];
    int32_t* wkeep = s_keep[threadIdx.x / 32];
    if (times && blockIdx.x == 0 && threadIdx.x == 0) times->t[0] = global_ns();

    // ---- init: Eq. 1 priorities
    init_words(a, (a.n + 15) / 16 * 16, true);  // words are padded to 16
    if (!grid_barrier(ctl, nblocks, a.spin_cap, [times]() {
            if (times) times->t[1] = global_ns();
        }))
        return;

    int cnt[kBins];
    int total = 0;
    for (int j = 0; j < kBins; ++j) {
        cnt[j] = a.bin_off[j + 1] - a.bin_off[j];
        total += cnt[j];
    }
    // isolated vertices were decided at init but belong to round 0's alive set
    const int iso = a.n_isolated;
    const int* off = a.bin_off;
    // in rounds after the first, a bin with no more rows than warps gets one
    // warp (or 4 lanes for short rows) per row: latency, not throughput
    const int nwarps_all = (int)(nblocks * (blockDim.x / 32));
    for (int r = 0; total > 0 || (r == 0 && iso > 0); ++r) {
        const int32_t* src = (r == 0) ? a.order0 : ((r & 1) ? a.wl1 : a.wl0);
        int32_t* dst = ((r + 1) & 1) ? a.wl1 : a.wl0;
        int* next = ctl->bcnt[(r + 1) & 3];

        // ---- Phase 1: selection test.  Round 0 scans most rows only up to
        // their first few arcs (a blocker turns up early); later rounds keep
        // the rows that need long scans, so a small bin gets wider groups.
        unsigned* grab = ctl->grab[(2 * r) & 3];
        block_bin<true>(a, src + off[4], cnt[4], &grab[4], nullptr, nullptr);
        if (r == 0) {
            select_bin<32, kChunk3>(a, src + off[3], cnt[3], &grab[3]);
            select_bin<16, kChunk2>(a, src + off[2], cnt[2], &grab[2]);
            select_bin<4, kChunk1>(a, src + off[1], cnt[1], &grab[1]);
            select_bin<1, kChunk0>(a, src + off[0], cnt[0], &grab[0]);
        } else {
            select_bin<32, kChunk3>(a, src + off[3], cnt[3], &grab[3]);
            if (cnt[2] <= nwarps_all) select_bin<32, kChunk3>(a, src + off[2], cnt[2], &grab[2]);
            else select_bin<16, kChunk2>(a, src + off[2], cnt[2], &grab[2]);
            if (cnt[1] <= nwarps_all) select_bin<32, kChunk3>(a, src + off[1], cnt[1], &grab[1]);
            else select_bin<4, kChunk1>(a, src + off[1], cnt[1], &grab[1]);
            if (cnt[0] <= nwarps_all) select_bin<4, kChunk1>(a, src + off[0], cnt[0], &grab[0]);
            else select_bin<1, kChunk0>(a, src + off[0], cnt[0], &grab[0]);
        }
        const int rr = r;
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [ctl, times, rr]() {
                if (times && rr < kStatRounds) times->t[2 + rr] = global_ns();
                for (int j = 0; j < kBins; ++j) ctl->grab[(2 * rr + 2) & 3][j] = 0;
            }))
            return;

        // ---- Phase 2+3: exclusion test, state update, compaction
        grab = ctl->grab[(2 * r + 1) & 3];
        block_bin<false>(a, src + off[4], cnt[4], &grab[4], &next[4], dst + off[4]);
        if (r == 0) {
            exclude_bin<32, kChunk3>(a, src + off[3], cnt[3], &grab[3], &next[3], dst + off[3],
                                     wscan, wkeep);
            exclude_bin<16, kChunk2>(a, src + off[2], cnt[2], &grab[2], &next[2], dst + off[2],
                                     wscan, wkeep);
            exclude_bin<4, kChunk1>(a, src + off[1], cnt[1], &grab[1], &next[1], dst + off[1],
                                    wscan, wkeep);
            exclude_bin<1, kChunk0>(a, src + off[0], cnt[0], &grab[0], &next[0], dst + off[0],
                                    wscan, wkeep);
        } else {
            exclude_bin<32, kChunk3>(a, src + off[3], cnt[3], &grab[3], &next[3], dst + off[3],
                                     wscan, wkeep);
            if (cnt[2] <= nwarps_all)
                exclude_bin<32, kChunk3>(a, src + off[2], cnt[2], &grab[2], &next[2],
                                         dst + off[2], wscan, wkeep);
            else
                exclude_bin<16, kChunk2>(a, src + off[2], cnt[2], &grab[2], &next[2],
                                         dst + off[2], wscan, wkeep);
            if (cnt[1] <= nwarps_all)
                exclude_bin<32, kChunk3>(a, src + off[1], cnt[1], &grab[1], &next[1],
                                         dst + off[1], wscan, wkeep);
            else
                exclude_bin<4, kChunk1>(a, src + off[1], cnt[1], &grab[1], &next[1],
                                        dst + off[1], wscan, wkeep);
            if (cnt[0] <= nwarps_all)
                exclude_bin<4, kChunk1>(a, src + off[0], cnt[0], &grab[0], &next[0],
                                        dst + off[0], wscan, wkeep);
            else
                exclude_bin<1, kChunk0>(a, src + off[0], cnt[0], &grab[0], &next[0],
                                        dst + off[0], wscan, wkeep);
        }
        const int cur = total + (r == 0 ? iso : 0);
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [ctl, times, rr, cur]() {
                if (times && rr < kStatRounds) times->t[2 + kStatRounds + rr] = global_ns();
                if (rr < kStatRounds) ctl->alive[rr] = cur;
                ctl->alive_sum += (unsigned long long)cur;
                ctl->rounds = rr + 1;
                for (int j = 0; j < kBins; ++j) {
                    ctl->grab[(2 * rr + 3) & 3][j] = 0;
                    ctl->bcnt[(rr + 2) & 3][j] = 0;
                }
            }))
            return;
        total = 0;
        for (int j = 0; j < kBins; ++j) {
            cnt[j] = ld_acquire_int(&next[j]);
            total += cnt[j];
        }
        if (total > 0 && r + 1 >= a.max_rounds) {
            if (threadIdx.x == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            return;
        }
    }

    // ---- output
    if (a.out) {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
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
        if (lane == 0 && in_cnt) atomicAdd(&ctl->mis_size, (unsigned long long)in_cnt);
    }
}

cudaError_t launch_csr_solve(const SolveArgs& a, int grid, cudaStream_t s) {
    void* args[] = {const_cast<SolveArgs*>(&a)};
    return cudaLaunchCooperativeKernel((const void*)csr_solve_kernel, dim3(grid),
                                       dim3(kCsrBlock), args, 0, s);
}

cudaError_t launch_csr_solve_single(const SolveArgs& a, cudaStream_t s) {
    csr_solve_kernel<<<1, kCsrBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int csr_block_size() { return kCsrBlock; }

int csr_max_coresident_blocks(int device) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)csr_solve_kernel,
                                                      kCsrBlock, 0) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

// ---------------------------------------------------------------- degree bins
//
// order0 = the round-0 list: every real vertex (batch padding excluded),
// grouped by bin, ascending id inside a bin.  Two kernels: per-block bin
// counts, then (after the host turns the counts into offsets) a stable
// scatter.  Blocks own contiguous vertex ranges.

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

// A vertex of the round-0 list: real and not isolated.
__device__ __forceinline__ bool listed(const SegTable& seg, const int32_t* rp, long long v) {
    return is_real(seg, v) && rp[v + 1] > rp[v];
}

__global__ void bin_count_kernel(const int32_t* __restrict__ rp, int32_t n, const SegTable seg,
                                 const BinThr thr, int32_t* __restrict__ blkcnt,
                                 int32_t* __restrict__ n_iso) {
    __shared__ int c[kBins];
    __shared__ int iso;
    if (threadIdx.x < kBins) c[threadIdx.x] = 0;
    if (threadIdx.x == 0) iso = 0;
    __syncthreads();
    const long long v0 = (long long)n * blockIdx.x / gridDim.x;
    const long long v1 = (long long)n * (blockIdx.x + 1) / gridDim.x;
    for (long long v = v0 + threadIdx.x; v < v1; v += blockDim.x) {
        if (!is_real(seg, v)) continue;
        const int deg = rp[v + 1] - rp[v];
        if (deg == 0) atomicAdd(&iso, 1);
        else atomicAdd(&c[bin_of(deg, thr)], 1);
    }
    __syncthreads();
    if (threadIdx.x < kBins) blkcnt[blockIdx.x * kBins + threadIdx.x] = c[threadIdx.x];
    if (threadIdx.x == 0 && iso) atomicAdd(n_iso, iso);
}

// blockDim.x must be 256
__global__ void bin_scatter_kernel(const int32_t* __restrict__ rp, int32_t n, const SegTable seg,
                                   const BinThr thr, const int32_t* __restrict__ blkoff,
                                   int32_t* __restrict__ order0) {
    __shared__ int wsum[8][kBins];
    __shared__ int run[kBins];
    const unsigned lane = lane_id();
    const int w = threadIdx.x / 32;
    if (threadIdx.x < kBins) run[threadIdx.x] = blkoff[blockIdx.x * kBins + threadIdx.x];
    __syncthreads();
    const long long v0 = (long long)n * blockIdx.x / gridDim.x;
    const long long v1 = (long long)n * (blockIdx.x + 1) / gridDim.x;
    for (long long c0 = v0; c0 < v1; c0 += blockDim.x) {
        const long long v = c0 + threadIdx.x;
        int j = -1;
        if (v < v1 && listed(seg, rp, v)) j = bin_of(rp[v + 1] - rp[v], thr);
        int rank = 0;
        for (int b = 0; b < kBins; ++b) {
            const unsigned m = __ballot_sync(0xFFFFFFFFu, j == b);
            if (j == b) rank = __popc(m & lanemask_lt());
            if (lane == 0) wsum[w][b] = __popc(m);
        }
        __syncthreads();
        if (j >= 0) {
            int off = run[j];
            for (int x = 0; x < w; ++x) off += wsum[x][j];
            order0[off + rank] = (int32_t)v;
        }
        __syncthreads();
        if (threadIdx.x < kBins) {
            int t = 0;
            for (int x = 0; x < 8; ++x) t += wsum[x][threadIdx.x];
            run[threadIdx.x] += t;
        }
        __syncthreads();
    }
}

cudaError_t build_bins(const int32_t* rp, int32_t n, const SegTable& seg, const int32_t thr[4],
                       int32_t* order0, int32_t bin_off[6], int32_t* n_isolated,
                       cudaStream_t s) {
    for (int j = 0; j <= kBins; ++j) bin_off[j] = 0;
    *n_isolated = 0;
    if (n == 0) return cudaSuccess;
    const int blocks = (int)std::min<long long>(1024, ((long long)n + 255) / 256);
    BinThr t;
    for (int k = 0; k < kBins - 1; ++k) t.t[k] = thr[k];
    int32_t* d_cnt = nullptr;
    cudaError_t e = dev_alloc((void**)&d_cnt, sizeof(int32_t) * (blocks * kBins + 1));
    if (e != cudaSuccess) return e;
    std::vector<int32_t> h((size_t)blocks * kBins);
    int32_t iso = 0;
    e = cudaMemsetAsync(d_cnt + blocks * kBins, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) {
        bin_count_kernel<<<blocks, 256, 0, s>>>(rp, n, seg, t, d_cnt, d_cnt + blocks * kBins);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h.data(), d_cnt, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&iso, d_cnt + blocks * kBins, sizeof(int32_t), cudaMemcpyDeviceToHost,
                            s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    *n_isolated = iso;
    if (e == cudaSuccess) {
        int64_t tot[kBins] = {};
        for (int b = 0; b < blocks; ++b)
            for (int j = 0; j < kBins; ++j) tot[j] += h[(size_t)b * kBins + j];
        int64_t acc = 0;
        for (int j = 0; j < kBins; ++j) {
            bin_off[j] = (int32_t)acc;
            acc += tot[j];
        }
        bin_off[kBins] = (int32_t)acc;
        int64_t run[kBins];
        for (int j = 0; j < kBins; ++j) run[j] = bin_off[j];
        for (int b = 0; b < blocks; ++b)
            for (int j = 0; j < kBins; ++j) {
                const int32_t c = h[(size_t)b * kBins + j];
                h[(size_t)b * kBins + j] = (int32_t)run[j];
                run[j] += c;
            }
        e = cudaMemcpyAsync(d_cnt, h.data(), sizeof(int32_t) * h.size(), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) {
        bin_scatter_kernel<<<blocks, 256, 0, s>>>(rp, n, seg, t, d_cnt, order0);
        e = cudaGetLastError();
    }
    const cudaError_t se = cudaStreamSynchronize(s);  // also on error: nothing may still run
    if (e == cudaSuccess) e = se;
    dev_free(d_cnt);
    return e;
}

}  // namespace tcmis
