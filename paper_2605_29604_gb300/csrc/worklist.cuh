// worklist.cuh -- how the persistent round kernels split a worklist among
// warps and append to the next one.
#pragma once

#include "common.cuh"

namespace tcmis {

// Finish each bin with chunks of one warp pass (balance at the end of a
// phase, at the price of more counter atomics): measured slower, off.
constexpr bool kTailChunks = false;
constexpr int kStageMax = 512;  // list entries staged per warp before an append

// Work split of a bin of `cnt` rows into chunks: `nbig` chunks of `ch` rows
// (at most CH, fewer when the bin is small so that the chunks spread over all
// warps) cover most of the bin, then chunks of one warp pass (G rows) finish
// it, so that the last warps of a phase do not wait long for a straggler.
struct ChunkPlan {
    int ch;
    int nbig;
    int total;  // chunks in all
    __device__ __forceinline__ void range(int k, int cnt, int& c0, int& c1, int G) const {
        if (k < nbig) {
            c0 = k * ch;
            c1 = min(c0 + ch, cnt);
        } else {
            c0 = nbig * ch + (k - nbig) * G;
            c1 = min(c0 + G, cnt);
        }
    }
};

template <int G, int CH>
__device__ __forceinline__ ChunkPlan plan_of(int cnt, int nwarps) {
    long long per = ((long long)cnt + nwarps - 1) / nwarps;
    per = ((per + G - 1) / G) * G;
    if (per < G) per = G;
    ChunkPlan p;
    p.ch = per < CH ? (int)per : CH;
    if (kTailChunks) {
        p.nbig = (int)((long long)cnt * 7 / 8 / p.ch);
        p.total = p.nbig + (cnt - p.nbig * p.ch + G - 1) / G;
    } else {
        p.nbig = (cnt + p.ch - 1) / p.ch;  // the last one may be short
        p.total = p.nbig;
    }
    return p;
}

// Who takes which chunk.  Warp w of the grid starts on chunk (w - base) mod
// nwarps of a bin (no atomic); the chunks past the first nwarps are handed out
// through the bin's counter.  `base` moves on by each bin's share, so that
// bins smaller than the grid land on different warps.
struct WarpSched {
    int gw;      // this warp's index in the grid
    int nwarps;  // warps in the grid
    int base;    // first warp of the next bin
    __device__ __forceinline__ int first(int total) {
        int k = gw - base;
        if (k < 0) k += nwarps;
        base += total < nwarps ? total : 0;
        if (base >= nwarps) base -= nwarps;
        return k;
    }
};

__device__ __forceinline__ int next_chunk(int total, int nwarps, unsigned* grab) {
    if (total <= nwarps) return total;  // every chunk was a first chunk
    int k = 0;
    if (lane_id() == 0) k = nwarps + (int)atomicAdd(grab, 1u);
    return __shfl_sync(0xFFFFFFFFu, k, 0);
}

// Stages up to 32 list indices per call (the group leaders' `keep` flags) in
// the warp's shared buffer; returns the new fill.
__device__ __forceinline__ int stage_keep(bool keep, int idx, int32_t* wbuf, int fill) {
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
    if (keep) wbuf[fill + __popc(bal & lanemask_lt())] = idx;
    return fill + __popc(bal);
}

// Appends the records list[wbuf[i]] of the warp's staged entries to `dst`
// with one atomic on `next`.
__device__ __forceinline__ void flush_stage(const int32_t* wbuf, int fill, const int4* list,
                                            int* next, int4* __restrict__ dst) {
    __syncwarp();
    if (fill) {
        const unsigned lane = lane_id();
        int o = 0;
        if (lane == 0) o = atomicAdd(next, fill);
        o = __shfl_sync(0xFFFFFFFFu, o, 0);
        for (int i = (int)lane; i < fill; i += 32) dst[o + i] = list[wbuf[i]];
    }
    __syncwarp();
}

// Appends the staged entries when another pass could overflow the buffer.
__device__ __forceinline__ int flush_if_full(const int32_t* wbuf, int fill, int pass_rows,
                                             const int4* list, int* next, int4* dst) {
    if (fill > kStageMax - pass_rows) {
        flush_stage(wbuf, fill, list, next, dst);
        return 0;
    }
    return fill;
}

}  // namespace tcmis
