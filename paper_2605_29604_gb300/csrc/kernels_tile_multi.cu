// kernels_tile_multi.cu -- K <= 8 solves of one graph on its 16 x 16 tiles,
// the exclusion test on tensor cores with K real right-hand sides.
//
// Phase 2 of Algorithm 2 is the product N_c = A x C (Sec. 3.1).  One solve
// fills one column of an m16n8 MMA; K solves of the same graph, run in lock
// step, fill K of its eight: N_c = A x [C_1 .. C_K], one product per tile
// group for all of them (rowblock_nc, tile_tc.cuh, in the graph's payload
// form).  Each solve keeps its own words (the layout of kernels_multi.cu:
// eight words per vertex, side by side) and its own in-set bit vector, the B
// operand: C_s's 16 bits on a tile's column block are one 16-bit load.
//
// A warp takes one row block (16 vertices):
//
//   Phase 1  selection test (CUDA cores): lane (i, h) owns row i in solves
//            4h .. 4h + 3 and scans the row in the CSR, four neighbours per
//            step; each neighbour's four words (16 bytes) are compared with
//            the row's.  Candidates are marked in their words and in C_s.
//            (Visiting the row's neighbours tile by tile costs a step per
//            tile of the row block, also where the row has no bit in it.)
//   Phase 2  exclusion test (tensor cores): D = sum over tiles of A_t x C.
//            Lane (g, q), g = lane / 4 and q = lane % 4, receives the MMA
//            entries D[g][2q], D[g][2q+1], D[g+8][2q], D[g+8][2q+1] and owns
//            those rows and solves: an undecided entry with D > 0 is out.
//   Phase 3  the row block stays on the worklist while any of its 16 x K
//            entries is undecided.
//
// Warp w takes list entries w, w + W, w + 2W, ... (W warps in the grid), so
// the grid works on a window of about W consecutive row blocks at a time and
// the neighbour words of a graph with local rows come from L2.
//
// Every solve sees the round-start snapshot exactly as a single solve does,
// so each solve's set and rounds are those of its single solve.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "tile_tc.cuh"

namespace tcmis {

namespace {

constexpr int kTmBlock = 512;
constexpr int kTmWarps = kTmBlock / 32;
constexpr int kTmChunk = 64;  // survivors staged per warp before an append

__device__ __forceinline__ bool outranks_m(uint32_t wu, int u, uint32_t wv, int v) {
    return wu > wv || (wu == wv && u > v);
}

__device__ __forceinline__ uint2 ld_pair(const uint32_t* word8, int v, int q) {
    return *reinterpret_cast<const uint2*>(word8 + (size_t)kMaxMulti * v + 2 * q);
}

__device__ __forceinline__ void st_pair(uint32_t* word8, int v, int q, uint2 w) {
    *reinterpret_cast<uint2*>(word8 + (size_t)kMaxMulti * v + 2 * q) = w;
}

// Undecided flags of the lane's four entries: bit 0 (row g, solve 2q), bit 1
// (g, 2q+1), bit 2 (g+8, 2q), bit 3 (g+8, 2q+1).
__device__ __forceinline__ unsigned und4(uint2 w0, uint2 w1) {
    return ((w0.x >> 29) == 1u ? 1u : 0u) | ((w0.y >> 29) == 1u ? 2u : 0u) |
           ((w1.x >> 29) == 1u ? 4u : 0u) | ((w1.y >> 29) == 1u ? 8u : 0u);
}

struct TmArgs {
    uint32_t* word8;   // kMaxMulti words per vertex, nrb * 16 vertices
    uint32_t* inb8;    // kMaxMulti bit vectors of nrb * 16 bits, `words` words apart
    int32_t words;     // 32-bit words per bit vector
    int32_t k;         // solves
    MultiSeeds seeds;
};

__device__ __forceinline__ unsigned und_quad(uint4 w) {
    return ((w.x >> 29) == 1u ? 1u : 0u) | ((w.y >> 29) == 1u ? 2u : 0u) |
           ((w.z >> 29) == 1u ? 4u : 0u) | ((w.w >> 29) == 1u ? 8u : 0u);
}

__device__ __forceinline__ unsigned blocks4(uint4 wu, int u, uint4 wv, int v) {
    return (outranks_m(wu.x, u, wv.x, v) ? 1u : 0u) | (outranks_m(wu.y, u, wv.y, v) ? 2u : 0u) |
           (outranks_m(wu.z, u, wv.z, v) ? 4u : 0u) | (outranks_m(wu.w, u, wv.w, v) ? 8u : 0u);
}

// Phase 1 over the row-block list.  Here lane (i, h), i = lane / 2 and
// h = lane % 2, owns row i in solves 4h .. 4h + 3.
__device__ __forceinline__ void tm_select(const SolveArgs& a, const TmArgs& m,
                                          const int32_t* __restrict__ list, int cnt,
                                          unsigned long long& alive) {
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const int i = (int)(lane >> 1), h = (int)(lane & 1);
    // warp gw takes list entries gw, gw + nw, gw + 2 nw, ...: at any moment
    // the warps work on a window of about nw consecutive entries, so the
    // neighbour words of a graph with local rows are re-read from L2
    const long long nw = (long long)gridDim.x * (blockDim.x / 32);
    const long long gw = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    {
        if (gw >= cnt) return;
        int rb_n = list[gw];
        for (long long item = gw; item < cnt; item += nw) {
            const int rb = rb_n;
            if (item + nw < cnt) rb_n = list[item + nw];
            const int v = rb * 16 + i;
            uint4* wp = reinterpret_cast<uint4*>(m.word8 + (size_t)kMaxMulti * v + 4 * h);
            uint4 w = *wp;
            const unsigned und = und_quad(w);
            alive += __popc(und);
            unsigned blocked = ~und & 0xFu;
            const uint32_t* w8 = m.word8 + 4 * h;
            // row v from the CSR, four neighbours per step (one 16-byte load
            // of col_idx), their words in this lane's four solves gathered
            // before any test
            const int rb0 = und ? a.rp[v] : 0;
            const int re0 = und ? a.rp[v + 1] : 0;
            int p0 = rb0 & ~3;
            for (;;) {
                const bool act = blocked != 0xFu && p0 < re0;
                if (!__any_sync(0xFFFFFFFFu, act)) break;
                if (act) {
                    const int4 c = __ldg(reinterpret_cast<const int4*>(a.col + p0));
                    const bool h0 = p0 >= rb0, h1 = p0 + 1 >= rb0 && p0 + 1 < re0,
                               h2 = p0 + 2 >= rb0 && p0 + 2 < re0, h3 = p0 + 3 < re0;
                    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
                    const uint4 q0 = h0 ? *reinterpret_cast<const uint4*>(w8 + (size_t)kMaxMulti * c.x) : z;
                    const uint4 q1 = h1 ? *reinterpret_cast<const uint4*>(w8 + (size_t)kMaxMulti * c.y) : z;
                    const uint4 q2 = h2 ? *reinterpret_cast<const uint4*>(w8 + (size_t)kMaxMulti * c.z) : z;
                    const uint4 q3 = h3 ? *reinterpret_cast<const uint4*>(w8 + (size_t)kMaxMulti * c.w) : z;
                    blocked |= (h0 ? blocks4(q0, c.x, w, v) : 0u) | (h1 ? blocks4(q1, c.y, w, v) : 0u) |
                               (h2 ? blocks4(q2, c.z, w, v) : 0u) | (h3 ? blocks4(q3, c.w, w, v) : 0u);
                }
                p0 += 4;
            }
            const unsigned cand = und & ~blocked;
            if (cand) {
                if (cand & 1u) w.x |= kWordInSet;
                if (cand & 2u) w.y |= kWordInSet;
                if (cand & 4u) w.z |= kWordInSet;
                if (cand & 8u) w.w |= kWordInSet;
                *wp = w;
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if ((cand >> k) & 1u)
                        atomicOr(m.inb8 + (size_t)(4 * h + k) * m.words + (v >> 5), 1u << (v & 31));
            }
        }
    }
}

// Phases 2 and 3 over the row-block list: N_c on tensor cores, state update,
// compaction of the row blocks that keep an undecided entry.
template <int P>
__device__ __forceinline__ void tm_exclude(const SolveArgs& a, const TmArgs& m,
                                           const int32_t* __restrict__ list, int cnt, int* next,
                                           int32_t* __restrict__ dst, int32_t* wkeep) {
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const int g = (int)(lane >> 2), q = (int)(lane & 3);
    // C of solve g (this lane's B column), 16 bits per column block
    const uint16_t* cseg = g < m.k ? reinterpret_cast<const uint16_t*>(m.inb8 + (size_t)g * m.words)
                                   : nullptr;
    // the schedule of tm_select: warp gw takes entries gw, gw + nw, ...
    const long long nw = (long long)gridDim.x * (blockDim.x / 32);
    const long long gw = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    if (gw >= cnt) return;
    int nkeep = 0;
    // survivors are staged per warp and appended kTmChunk at a time
    auto flush = [&]() {
        __syncwarp();
        int o = 0;
        if (lane == 0) o = atomicAdd(next, nkeep);
        o = __shfl_sync(0xFFFFFFFFu, o, 0);
        for (int k = (int)lane; k < nkeep; k += 32) dst[o + k] = wkeep[k];
        __syncwarp();
        nkeep = 0;
    };
    {
        int rb_n = list[gw];
        int t0_n = a.trp[rb_n], t1_n = a.trp[rb_n + 1];
        for (long long item = gw; item < cnt; item += nw) {
            const int rb = rb_n, t0 = t0_n, t1 = t1_n;
            if (item + nw < cnt) {
                rb_n = list[item + nw];
                t0_n = a.trp[rb_n];
                t1_n = a.trp[rb_n + 1];
            }
            int d[4];
            rowblock_nc<P>(a.tbits, a.tpay, t0, t1,
                           [&](int t) -> uint32_t {
                               return cseg ? (uint32_t)cseg[__ldg(a.tcol + t)] : 0u;
                           },
                           d);
            const int v0 = rb * 16 + g, v1 = v0 + 8;
            uint2 w0 = ld_pair(m.word8, v0, q), w1 = ld_pair(m.word8, v1, q);
            const unsigned und = und4(w0, w1);  // after Phase 1: the non-candidates
            const unsigned out = und & ((d[0] > 0 ? 1u : 0u) | (d[1] > 0 ? 2u : 0u) |
                                        (d[2] > 0 ? 4u : 0u) | (d[3] > 0 ? 8u : 0u));
            if (out & 3u) {
                if (out & 1u) w0.x = kWordOut;
                if (out & 2u) w0.y = kWordOut;
                st_pair(m.word8, v0, q, w0);
            }
            if (out & 12u) {
                if (out & 4u) w1.x = kWordOut;
                if (out & 8u) w1.y = kWordOut;
                st_pair(m.word8, v1, q, w1);
            }
            if (__any_sync(0xFFFFFFFFu, (und & ~out) != 0u)) {
                if (lane == 0) wkeep[nkeep] = rb;
                ++nkeep;
                if (nkeep == kTmChunk) flush();
            }
        }
        if (nkeep) flush();
    }
}

template <int P>
__global__ void __launch_bounds__(kTmBlock, 2) tile_multi_kernel(const SolveArgs a, const TmArgs m) {
    __shared__ int32_t s_keep[kTmWarps][kTmChunk];
    __shared__ unsigned long long s_alive;
    __shared__ int s_count;
    const unsigned lane = lane_id();
    const unsigned nblocks = gridDim.x;
    Ctl* ctl = a.ctl;
    PhaseTimes* times = a.times;
    const int32_t n = a.n, nrb = a.nrb;
    int32_t* wkeep = s_keep[threadIdx.x / 32];
    grid_barrier_start();
    if (times && blockIdx.x == 0 && threadIdx.x == 0) times->t[0] = global_ns();

    // ---- init: each solve's priorities (Sec. 2), empty C, all row blocks
    {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        const float dbar = n > 0 ? average_degree(a.rp[n], n) : 0.f;
        const int mode = a.priority;
        uint64_t smix[kMaxMulti];
#pragma unroll
        for (int s = 0; s < kMaxMulti; ++s) smix[s] = mix64(m.seeds.seed[s]);
        for (long long v = tid; v < (long long)nrb * 16; v += nthreads) {
            const int deg = v < n ? a.rp[v + 1] - a.rp[v] : 0;
            uint32_t w[kMaxMulti];
#pragma unroll
            for (int s = 0; s < kMaxMulti; ++s) {
                if (v >= n || s >= m.k) w[s] = kWordOut;
                else w[s] = deg ? undecided_word(mode, priority_key(mode, dbar, deg, smix[s],
                                                                     (uint32_t)v))
                                : kKeyIsolated;
            }
            uint4* p = reinterpret_cast<uint4*>(m.word8 + (size_t)kMaxMulti * v);
            p[0] = make_uint4(w[0], w[1], w[2], w[3]);
            p[1] = make_uint4(w[4], w[5], w[6], w[7]);
        }
        for (long long i = tid; i < (long long)kMaxMulti * m.words; i += nthreads) m.inb8[i] = 0u;
        for (long long rb = tid; rb < nrb; rb += nthreads) a.rbl0[rb] = (int32_t)rb;
    }
    if (threadIdx.x == 0) s_alive = 0;
    if (!grid_barrier(ctl, nblocks, a.spin_cap, [times]() {
            if (times) times->t[1] = global_ns();
        }))
        return;

    int count = nrb;
    for (int r = 0; count > 0; ++r) {
        const int32_t* src = (r & 1) ? a.rbl1 : a.rbl0;
        int32_t* dst = (r & 1) ? a.rbl0 : a.rbl1;
        int* next = &ctl->bcnt[(r + 1) & 3][0];

        // ---- Phase 1: selection test (CUDA cores)
        unsigned long long alive = 0;
        tm_select(a, m, src, count, alive);
        for (int o = 16; o; o >>= 1) alive += __shfl_xor_sync(0xFFFFFFFFu, alive, o);
        if (lane == 0 && alive) atomicAdd(&s_alive, alive);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_alive) atomicAdd(&ctl->alive_acc64[r & 3], s_alive);
            s_alive = 0;
        }
        const int rr = r;
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [times, rr]() {
                if (times && rr < kStatRounds) times->t[2 + rr] = global_ns();
            }))
            return;

        // ---- Phases 2 and 3: exclusion test (tensor cores), update, compaction
        tm_exclude<P>(a, m, src, count, next, dst, wkeep);
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [ctl, times, rr]() {
                const unsigned long long alive = ctl->alive_acc64[rr & 3];
                if (times && rr < kStatRounds) times->t[2 + kStatRounds + rr] = global_ns();
                if (rr < kStatRounds) ctl->alive[rr] = (int)alive;
                ctl->alive_sum += alive;
                if (alive > 0) ctl->rounds = rr + 1;
                ctl->bcnt[(rr + 2) & 3][0] = 0;
                ctl->alive_acc64[(rr + 2) & 3] = 0;
            },
            [next]() { s_count = __ldcg(next); }))
            return;
        count = s_count;
        if (count > 0 && r + 1 >= a.max_rounds) {
            if (threadIdx.x == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            return;
        }
    }

    // ---- output: solve s's result at out + s * n
    if (a.out) {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        unsigned in_cnt = 0;
        for (long long v = tid; v < n; v += nthreads) {
            const uint4* p = reinterpret_cast<const uint4*>(m.word8 + (size_t)kMaxMulti * v);
            const uint4 x = p[0], y = p[1];
            const uint32_t w[kMaxMulti] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w};
            for (int s = 0; s < m.k; ++s) {
                const bool in = w[s] >= kWordInMin;
                in_cnt += in;
                a.out[(size_t)s * n + v] = in;
            }
        }
        for (int o = 16; o; o >>= 1) in_cnt += __shfl_xor_sync(0xFFFFFFFFu, in_cnt, o);
        if (lane == 0 && in_cnt) atomicAdd(&ctl->mis_size, (unsigned long long)in_cnt);
    }
}

const void* tile_multi_fn(int P) {
    switch (P) {
        case kPayBitsF16: return (const void*)tile_multi_kernel<kPayBitsF16>;
        case kPayB1: return (const void*)tile_multi_kernel<kPayB1>;
        case kPayI8: return (const void*)tile_multi_kernel<kPayI8>;
        case kPayF16: return (const void*)tile_multi_kernel<kPayF16>;
        default: return nullptr;
    }
}

}  // namespace

int32_t tile_multi_bitvector_words(int32_t nrb) { return (nrb * 16 + 31) / 32; }

cudaError_t launch_tile_multi_solve(const SolveArgs& a, uint32_t* word8, uint32_t* inb8, int k,
                                    const MultiSeeds& seeds, int payload, int grid,
                                    cudaStream_t s) {
    const void* fn = tile_multi_fn(payload);
    if (!fn || k < 1 || k > kMaxMulti) return cudaErrorInvalidValue;
    TmArgs m;
    m.word8 = word8;
    m.inb8 = inb8;
    m.words = tile_multi_bitvector_words(a.nrb);
    m.k = k;
    m.seeds = seeds;
    void* args[] = {const_cast<SolveArgs*>(&a), &m};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kTmBlock), args, 0, s);
}

int tile_multi_max_coresident_blocks(int payload, int device) {
    const void* fn = tile_multi_fn(payload);
    if (!fn) return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTmBlock, 0) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

}  // namespace tcmis
