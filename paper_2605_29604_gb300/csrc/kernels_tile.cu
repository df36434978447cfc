// kernels_tile.cu -- tile-CSR format and the tile round kernels.
//
// The paper represents the graph as a block-tiled adjacency matrix A that
// keeps only its non-zero tiles, in a compressed block format (Sec. 3.2;
// Algorithm 2, "represent G as tiled A"), and evaluates the neighbour
// interactions of a round on those tiles.  Here:
//
//   format    tile-CSR: row block rb (T consecutive vertices) owns the tiles
//             [trp[rb], trp[rb+1]); tcol[t] is the column block of tile t;
//             tbits holds its T x T 0/1 entries as row-major bits (T = 8: one
//             64-bit word per tile; T = 16: four, i.e. one 16-bit row each).
//   Phase 1   selection test per row block, a group of T lanes (lane i = row
//             i): for each tile, the T words of the tile's column block are
//             one contiguous segment (32 or 64 bytes), compared against the
//             row's key where the row's bit is set.
//   Phase 2   exclusion test N_c = A x C (Algorithm 2), C kept as a bit-packed
//             in-set vector: row i is excluded when (row bits & C segment) != 0.
//             Tiles whose C segment is zero contribute nothing (the early
//             exit of Sec. 3.2).  The tensor-core variant (T = 16) computes
//             the same product with mma.sync m16n8k16: the tile's bits are
//             expanded to an fp16 A fragment in registers, the C segment to
//             the first column of the B fragment, fp32 accumulation (exact:
//             each tile adds at most 16 per row).
//   Phase 3   state update and compaction of the row blocks that still hold
//             an undecided vertex.
//
// Both phases see the round-start snapshot exactly as the CSR kernel does, so
// the tile kernels return the same set and the same rounds as every path.
#include <algorithm>
#include <cstdio>
#include <vector>

#include <cub/cub.cuh>

#include "common.cuh"
#include "init.cuh"
#include "internal.h"
#include "tile_tc.cuh"

namespace tcmis {

// ---------------------------------------------------------------- converter

namespace {

constexpr int kArcsPerThread = 16;

// Sort key of arc (v, u): tile (v / T, u / T) as rb * nrb + cb; value: the
// arc's bit inside the tile, (v % T) * T + (u % T).
__global__ void tile_keys_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 int32_t n, int64_t arcs, int T, int32_t nrb,
                                 uint64_t* __restrict__ keys, uint8_t* __restrict__ vals) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p0 = t * kArcsPerThread;
    if (p0 >= arcs) return;
    const int64_t p1 = (arcs < p0 + kArcsPerThread) ? arcs : p0 + kArcsPerThread;
    int lo = 0, hi = n;  // row of p0: last v with rp[v] <= p0
    while (hi - lo > 1) {
        const int mid = lo + (hi - lo) / 2;
        if ((int64_t)rp[mid] <= p0) lo = mid;
        else hi = mid;
    }
    int v = lo;
    for (int64_t p = p0; p < p1; ++p) {
        while ((int64_t)rp[v + 1] <= p) ++v;
        const int u = col[p];
        keys[p] = (uint64_t)(v / T) * (uint64_t)nrb + (uint64_t)(u / T);
        vals[p] = (uint8_t)((v % T) * T + (u % T));
    }
}

__global__ void tile_flags_kernel(const uint64_t* __restrict__ keys, int64_t arcs,
                                  int32_t* __restrict__ flags) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < arcs) flags[p] = (p == 0 || keys[p] != keys[p - 1]) ? 1 : 0;
}

__global__ void tile_fill_kernel(const uint64_t* __restrict__ keys,
                                 const uint8_t* __restrict__ vals,
                                 const int32_t* __restrict__ flags,
                                 const int32_t* __restrict__ tid, int64_t arcs, int T,
                                 int32_t nrb, int32_t* __restrict__ tcol,
                                 int32_t* __restrict__ trow, uint64_t* __restrict__ tbits) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= arcs) return;
    const int32_t t = tid[p] - 1;
    if (flags[p]) {
        tcol[t] = (int32_t)(keys[p] % (uint64_t)nrb);
        trow[t] = (int32_t)(keys[p] / (uint64_t)nrb);
    }
    const int bit = vals[p];
    const int words = T * T / 64;
    atomicOr((unsigned long long*)&tbits[(int64_t)t * words + bit / 64], 1ull << (bit % 64));
}

// trp[rb] = first tile whose row block is >= rb.
__global__ void tile_rowptr_kernel(const int32_t* __restrict__ trow, int64_t ntiles, int32_t nrb,
                                   int32_t* __restrict__ trp) {
    const long long rb = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (rb > nrb) return;
    int64_t lo = 0, hi = ntiles;
    while (lo < hi) {
        const int64_t mid = lo + (hi - lo) / 2;
        if (trow[mid] < rb) lo = mid + 1;
        else hi = mid;
    }
    trp[rb] = (int32_t)lo;
}

int bits_for(uint64_t x) {
    int b = 1;
    while (b < 64 && (1ull << b) <= x) ++b;
    return b;
}

}  // namespace

cudaError_t build_tiles(const int32_t* rp, const int32_t* col, int32_t n, int64_t arcs, int T,
                        TileCsr* out, cudaStream_t s) {
    *out = TileCsr();
    out->T = T;
    if (T != 8 && T != 16) return cudaErrorInvalidValue;
    const int32_t nrb = (n + T - 1) / T;
    out->nrb = nrb;
    const int words = T * T / 64;
    cudaError_t e = dev_alloc((void**)&out->trp, sizeof(int32_t) * ((size_t)nrb + 1));
    if (e != cudaSuccess) return e;
    if (arcs == 0) {
        e = cudaMemsetAsync(out->trp, 0, sizeof(int32_t) * ((size_t)nrb + 1), s);
        if (e == cudaSuccess) e = dev_alloc((void**)&out->tcol, sizeof(int32_t));
        if (e == cudaSuccess) e = dev_alloc((void**)&out->tbits, sizeof(uint64_t) * words);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    }
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint8_t *v0 = nullptr, *v1 = nullptr;
    int32_t *flags = nullptr, *tid = nullptr, *trow = nullptr;
    void* temp = nullptr;
    size_t temp_bytes = 0, scan_bytes = 0;
    const int key_bits = bits_for((uint64_t)nrb * (uint64_t)nrb);
    auto cleanup = [&]() {
        cudaStreamSynchronize(s);  // no kernel may still use the temporaries
        dev_free(k0);
        dev_free(k1);
        dev_free(v0);
        dev_free(v1);
        dev_free(flags);
        dev_free(tid);
        dev_free(trow);
        dev_free(temp);
    };
    const size_t A = (size_t)arcs;
    if ((e = dev_alloc((void**)&k0, 8 * A)) != cudaSuccess ||
        (e = dev_alloc((void**)&k1, 8 * A)) != cudaSuccess ||
        (e = dev_alloc((void**)&v0, A)) != cudaSuccess ||
        (e = dev_alloc((void**)&v1, A)) != cudaSuccess ||
        (e = dev_alloc((void**)&flags, 4 * A)) != cudaSuccess ||
        (e = dev_alloc((void**)&tid, 4 * A)) != cudaSuccess) {
        cleanup();
        return e;
    }
    {
        const long long work = (arcs + kArcsPerThread - 1) / kArcsPerThread;
        tile_keys_kernel<<<(unsigned)((work + 255) / 256), 256, 0, s>>>(rp, col, n, arcs, T, nrb,
                                                                        k0, v0);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            cleanup();
            return e;
        }
    }
    cub::DoubleBuffer<uint64_t> dk(k0, k1);
    cub::DoubleBuffer<uint8_t> dv(v0, v1);
    e = cub::DeviceRadixSort::SortPairs(nullptr, temp_bytes, dk, dv, arcs, 0, key_bits, s);
    if (e == cudaSuccess)
        e = cub::DeviceScan::InclusiveSum(nullptr, scan_bytes, flags, tid, arcs, s);
    if (e == cudaSuccess) e = dev_alloc(&temp, std::max(temp_bytes, scan_bytes));
    if (e == cudaSuccess)
        e = cub::DeviceRadixSort::SortPairs(temp, temp_bytes, dk, dv, arcs, 0, key_bits, s);
    const unsigned ablocks = (unsigned)((arcs + 255) / 256);
    if (e == cudaSuccess) {
        tile_flags_kernel<<<ablocks, 256, 0, s>>>(dk.Current(), arcs, flags);
        e = cudaGetLastError();
    }
    // tid[p] = (tiles starting at or before arc p); arc p belongs to tile tid[p] - 1
    if (e == cudaSuccess) e = cub::DeviceScan::InclusiveSum(temp, scan_bytes, flags, tid, arcs, s);
    int32_t last_tid = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&last_tid, tid + arcs - 1, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cleanup();
        return e;
    }
    const int64_t ntiles = (int64_t)last_tid;
    out->ntiles = ntiles;
    if ((e = dev_alloc((void**)&out->tcol, 4 * (size_t)ntiles)) != cudaSuccess ||
        (e = dev_alloc((void**)&trow, 4 * (size_t)ntiles)) != cudaSuccess ||
        (e = dev_alloc((void**)&out->tbits, 8 * (size_t)words * (size_t)ntiles)) != cudaSuccess) {
        cleanup();
        return e;
    }
    e = cudaMemsetAsync(out->tbits, 0, 8 * (size_t)words * (size_t)ntiles, s);
    if (e == cudaSuccess) {
        tile_fill_kernel<<<ablocks, 256, 0, s>>>(dk.Current(), dv.Current(), flags, tid, arcs, T,
                                                 nrb, out->tcol, trow, out->tbits);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        tile_rowptr_kernel<<<(unsigned)((nrb + 1 + 255) / 256), 256, 0, s>>>(trow, ntiles, nrb,
                                                                             out->trp);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cleanup();
    return e;
}

// ---------------------------------------------------------------- round kernels

namespace {

constexpr int kTileBlock = 512;
constexpr int kTileWarps = kTileBlock / 32;
constexpr int kTileChunk = 64;  // row blocks per warp chunk (upper bound)

__device__ __forceinline__ bool outranks_t(uint32_t wu, int u, uint32_t wv, int v) {
    return wu > wv || (wu == wv && u > v);
}

// Row i's T bits of tile t.
template <int T>
__device__ __forceinline__ uint32_t tile_row(const uint64_t* __restrict__ tbits, int t, int i) {
    if (T == 8) return (uint32_t)(__ldg(tbits + t) >> (8 * i)) & 0xFFu;
    return (uint32_t)(__ldg(tbits + (int64_t)t * 4 + (i >> 2)) >> (16 * (i & 3))) & 0xFFFFu;
}

// The T in-set bits of column block cb.
template <int T>
__device__ __forceinline__ uint32_t in_segment(const uint32_t* inbits, int cb) {
    if (T == 8) return reinterpret_cast<const uint8_t*>(inbits)[cb];
    return reinterpret_cast<const uint16_t*>(inbits)[cb];
}

template <int G>
__device__ __forceinline__ int tile_chunk(int cnt) {
    const long long nwarps = (long long)gridDim.x * (blockDim.x / 32);
    long long per = (cnt + nwarps - 1) / nwarps;
    per = ((per + G - 1) / G) * G;
    if (per < G) per = G;
    return per < kTileChunk ? (int)per : kTileChunk;
}

__device__ __forceinline__ long long tile_gwarp() {
    return (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
}

// OR of v over the S lanes of this lane's group (S a power of two <= 32).
template <int S>
__device__ __forceinline__ uint32_t group_or(uint32_t v) {
#pragma unroll
    for (int o = S / 2; o > 0; o >>= 1) v |= __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// Row i's T bits of a tile whose payload words are already in registers.
template <int T>
__device__ __forceinline__ uint32_t row_bits(const uint64_t* w, int i) {
    if (T == 8) return (uint32_t)(w[0] >> (8 * i)) & 0xFFu;
    return (uint32_t)(w[i >> 2] >> (16 * (i & 3))) & 0xFFFFu;
}

// The T words of a block of T consecutive vertices (16-byte aligned).
template <int T>
__device__ __forceinline__ void load_block_words(const uint32_t* word, int first, uint32_t* w) {
    const uint4* p = reinterpret_cast<const uint4*>(word + first);
#pragma unroll
    for (int q = 0; q < T / 4; ++q) {
        const uint4 x = p[q];
        w[4 * q] = x.x;
        w[4 * q + 1] = x.y;
        w[4 * q + 2] = x.z;
        w[4 * q + 3] = x.w;
    }
}

// Phase 1 over the row-block list.  A group of S lanes takes one row block;
// each lane evaluates whole tiles (lane k takes tiles t0 + k, t0 + k + S, ...)
// against the T words of the row block and the T words of the tile's column
// block, and the group ORs the per-row "outranked" masks.
template <int T, int S>
__device__ __forceinline__ void tile_select(const SolveArgs& a, const int32_t* __restrict__ list,
                                            int cnt, unsigned* grab, unsigned& alive_cnt) {
    constexpr int G = 32 / S;
    constexpr uint32_t kFull = (T == 32) ? 0xFFFFFFFFu : ((1u << T) - 1u);
    constexpr int W = T * T / 64;
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const int slot = (int)(lane % S);
    const unsigned gid = lane / S;
    const int ch = tile_chunk<G>(cnt);
    if (tile_gwarp() >= (cnt + ch - 1) / ch) return;
    for (;;) {
        int c0 = 0;
        if (lane == 0) c0 = (int)atomicAdd(grab, (unsigned)ch);
        c0 = __shfl_sync(0xFFFFFFFFu, c0, 0);
        if (c0 >= cnt) break;
        const int c1 = min(c0 + ch, cnt);
        for (int base = c0; base < c1; base += G) {
            const int item = base + (int)gid;
            const bool valid = item < c1;
            const int rb = valid ? list[item] : 0;
            uint32_t wr[T];
            load_block_words<T>(a.word, rb * T, wr);
            uint32_t und = 0;
#pragma unroll
            for (int i = 0; i < T; ++i) und |= (uint32_t)((wr[i] >> 29) == 1u) << i;
            if (!valid) und = 0;
            if (slot == 0) alive_cnt += __popc(und);
            uint32_t blocked = ~und & kFull;
            const int t0 = valid ? a.trp[rb] : 0;
            const int t1 = valid ? a.trp[rb + 1] : 0;
            for (int t = t0 + slot;; t += S) {
                uint32_t m = 0;
                if (t < t1 && blocked != kFull) {
                    const int cb = __ldg(a.tcol + t);
                    uint64_t tw[W];
#pragma unroll
                    for (int k = 0; k < W; ++k) tw[k] = __ldg(a.tbits + (int64_t)t * W + k);
#pragma unroll
                    for (int h = 0; h < T / 8; ++h) {
                        uint32_t wc[8];
                        load_block_words<8>(a.word, cb * T + 8 * h, wc);
#pragma unroll
                        for (int i = 0; i < T; ++i) {
                            const uint32_t rbits = row_bits<T>(tw, i) >> (8 * h);
                            bool hit = false;
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                hit |= ((rbits >> j) & 1u) &&
                                       outranks_t(wc[j], cb * T + 8 * h + j, wr[i], rb * T + i);
                            m |= (uint32_t)hit << i;
                        }
                    }
                }
                blocked |= group_or<S>(m);
                const bool more = t - slot + S < t1 && blocked != kFull;
                if (!__any_sync(0xFFFFFFFFu, more)) break;
            }
            const uint32_t cand = und & ~blocked;
            if (slot == 0 && cand) {
                for (int i = 0; i < T; ++i)
                    if ((cand >> i) & 1u) a.word[rb * T + i] = wr[i] | kWordInSet;
                const int first = rb * T;
                atomicOr(a.inbits + (first >> 5), cand << (first & 31));
            }
        }
    }
}

// Phase 2+3 on CUDA cores: per tile, (row bits & C segment) != 0, ORed over
// the group; then state update and compaction of row blocks.
template <int T, int S>
__device__ __forceinline__ void tile_exclude(const SolveArgs& a, const int32_t* __restrict__ list,
                                             int cnt, unsigned* grab, int* next,
                                             int32_t* __restrict__ dst, int32_t* wkeep) {
    constexpr int G = 32 / S;
    constexpr uint32_t kFull = (T == 32) ? 0xFFFFFFFFu : ((1u << T) - 1u);
    constexpr int W = T * T / 64;
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const int slot = (int)(lane % S);
    const unsigned gid = lane / S;
    const int ch = tile_chunk<G>(cnt);
    if (tile_gwarp() >= (cnt + ch - 1) / ch) return;
    for (;;) {
        int c0 = 0;
        if (lane == 0) c0 = (int)atomicAdd(grab, (unsigned)ch);
        c0 = __shfl_sync(0xFFFFFFFFu, c0, 0);
        if (c0 >= cnt) break;
        const int c1 = min(c0 + ch, cnt);
        int nkeep = 0;
        for (int base = c0; base < c1; base += G) {
            const int item = base + (int)gid;
            const bool valid = item < c1;
            const int rb = valid ? list[item] : 0;
            uint32_t wr[T];
            load_block_words<T>(a.word, rb * T, wr);
            uint32_t und = 0;
#pragma unroll
            for (int i = 0; i < T; ++i) und |= (uint32_t)((wr[i] >> 29) == 1u) << i;
            if (!valid) und = 0;
            uint32_t hit = ~und & kFull;
            const int t0 = valid ? a.trp[rb] : 0;
            const int t1 = valid ? a.trp[rb + 1] : 0;
            for (int t = t0 + slot;; t += S) {
                uint32_t m = 0;
                if (t < t1 && hit != kFull) {
                    const uint32_t seg = in_segment<T>(a.inbits, __ldg(a.tcol + t));
                    if (seg) {
                        uint64_t tw[W];
#pragma unroll
                        for (int k = 0; k < W; ++k) tw[k] = __ldg(a.tbits + (int64_t)t * W + k);
#pragma unroll
                        for (int i = 0; i < T; ++i) m |= (uint32_t)((row_bits<T>(tw, i) & seg) != 0u) << i;
                    }
                }
                hit |= group_or<S>(m);
                const bool more = t - slot + S < t1 && hit != kFull;
                if (!__any_sync(0xFFFFFFFFu, more)) break;
            }
            const uint32_t out = und & hit;
            for (int i = slot; i < T; i += S)
                if ((out >> i) & 1u) a.word[rb * T + i] = kWordOut;
            const bool keep = valid && slot == 0 && (und & ~hit) != 0u;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
            if (keep) wkeep[nkeep + __popc(bal & lanemask_lt())] = rb;
            nkeep += __popc(bal);
        }
        __syncwarp();
        if (nkeep) {
            int o = 0;
            if (lane == 0) o = atomicAdd(next, nkeep);
            o = __shfl_sync(0xFFFFFFFFu, o, 0);
            for (int q = (int)lane; q < nkeep; q += 32) dst[o + q] = wkeep[q];
        }
        __syncwarp();
    }
}

// Phase 2+3 on tensor cores (T = 16): one warp per row block; N_c of its 16
// rows by rowblock_nc in payload form P, with C (the in-set bits) as column 0
// of the B operand.
template <int P>
__device__ __forceinline__ void tile_exclude_tc(const SolveArgs& a,
                                                const int32_t* __restrict__ list, int cnt,
                                                unsigned* grab, int* next,
                                                int32_t* __restrict__ dst, int32_t* wkeep) {
    if (cnt <= 0) return;
    const unsigned lane = lane_id();
    const bool col0 = (lane >> 2) == 0;  // this lane's B column is solve 0
    const uint16_t* inseg = reinterpret_cast<const uint16_t*>(a.inbits);
    const int ch = tile_chunk<1>(cnt);
    if (tile_gwarp() >= (cnt + ch - 1) / ch) return;
    for (;;) {
        int c0 = 0;
        if (lane == 0) c0 = (int)atomicAdd(grab, (unsigned)ch);
        c0 = __shfl_sync(0xFFFFFFFFu, c0, 0);
        if (c0 >= cnt) break;
        const int c1 = min(c0 + ch, cnt);
        int nkeep = 0;
        for (int item = c0; item < c1; ++item) {
            const int rb = list[item];
            int d[4];
            rowblock_nc<P>(a.tbits, a.tpay, a.trp[rb], a.trp[rb + 1],
                           [&](int t) -> uint32_t {
                               return col0 ? (uint32_t)inseg[__ldg(a.tcol + t)] : 0u;
                           },
                           d);
            // N_c of rows g (d[0]) and g + 8 (d[2]) sit in column 0, lanes q == 0
            const int nc_lo = __shfl_sync(0xFFFFFFFFu, d[0], (int)(lane & 7) * 4);
            const int nc_hi = __shfl_sync(0xFFFFFFFFu, d[2], (int)(lane & 7) * 4);
            bool keep_row = false;
            if (lane < 16) {
                const int v = rb * 16 + (int)lane;
                const int nc = lane < 8 ? nc_lo : nc_hi;
                const uint32_t wv = ld_word_l1(a.word + v);
                if ((wv >> 29) == 1u) {
                    if (nc > 0) a.word[v] = kWordOut;
                    else keep_row = true;
                }
            }
            if (__any_sync(0xFFFFFFFFu, keep_row)) {
                if (lane == 0) wkeep[nkeep] = rb;
                ++nkeep;
            }
        }
        __syncwarp();
        if (nkeep) {
            int o = 0;
            if (lane == 0) o = atomicAdd(next, nkeep);
            o = __shfl_sync(0xFFFFFFFFu, o, 0);
            for (int k = (int)lane; k < nkeep; k += 32) dst[o + k] = wkeep[k];
        }
        __syncwarp();
    }
}

// P: the tensor-core payload form of Phase 2 (tile_tc.cuh), or -1 for the
// CUDA-core popc form.
template <int T, int S, int P>
__global__ void __launch_bounds__(kTileBlock, 2) tile_solve_kernel(const SolveArgs a) {
    __shared__ int32_t s_keep[kTileWarps][kTileChunk];
    __shared__ unsigned s_alive;
    __shared__ int s_count;  // next worklist size, loaded once per block
    const unsigned lane = lane_id();
    const unsigned nblocks = gridDim.x;
    Ctl* ctl = a.ctl;
    PhaseTimes* times = a.times;
    const int32_t n = a.n;
    const int32_t nrb = a.nrb;
    int32_t* wkeep = s_keep[threadIdx.x / 32];
    grid_barrier_start();
    if (times && blockIdx.x == 0 && threadIdx.x == 0) times->t[0] = global_ns();

    // ---- init: Eq. 1 priorities (tile padding out), empty in-set bits,
    // round-0 row-block list
    init_words(a, nrb * T, false);
    {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        const long long nwords = ((long long)nrb * T + 31) / 32;
        for (long long k = tid; k < nwords; k += nthreads) a.inbits[k] = 0u;
        for (long long rb = tid; rb < nrb; rb += nthreads) a.rbl0[rb] = (int32_t)rb;
    }
    if (threadIdx.x == 0) s_alive = 0;
    if (!grid_barrier(ctl, nblocks, a.spin_cap, [times]() {
            if (times) times->t[1] = global_ns();
        }))
        return;
    (void)n;

    int count = nrb;
    for (int r = 0; count > 0; ++r) {
        const int32_t* src = (r & 1) ? a.rbl1 : a.rbl0;
        int32_t* dst = (r & 1) ? a.rbl0 : a.rbl1;
        int* next = &ctl->bcnt[(r + 1) & 3][0];

        // ---- Phase 1: selection test
        unsigned alive_cnt = 0;
        tile_select<T, S>(a, src, count, &ctl->grab[(2 * r) & 3][0], alive_cnt);
        for (int o = 16; o; o >>= 1) alive_cnt += __shfl_xor_sync(0xFFFFFFFFu, alive_cnt, o);
        if (lane == 0 && alive_cnt) atomicAdd(&s_alive, alive_cnt);
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_alive) atomicAdd(&ctl->alive_acc[r & 3], (int)s_alive);
            s_alive = 0;
        }
        const int rr = r;
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [ctl, times, rr]() {
                if (times && rr < kStatRounds) times->t[2 + rr] = global_ns();
                ctl->grab[(2 * rr + 2) & 3][0] = 0;
            }))
            return;

        // ---- Phase 2+3: exclusion test, state update, compaction
        if constexpr (P >= 0)
            tile_exclude_tc<P>(a, src, count, &ctl->grab[(2 * r + 1) & 3][0], next, dst, wkeep);
        else
            tile_exclude<T, S>(a, src, count, &ctl->grab[(2 * r + 1) & 3][0], next, dst, wkeep);
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [ctl, times, rr]() {
                const int alive = ctl->alive_acc[rr & 3];
                if (times && rr < kStatRounds) times->t[2 + kStatRounds + rr] = global_ns();
                if (rr < kStatRounds) ctl->alive[rr] = alive;
                ctl->alive_sum += (unsigned long long)alive;
                if (alive > 0) ctl->rounds = rr + 1;
                ctl->grab[(2 * rr + 3) & 3][0] = 0;
                ctl->bcnt[(rr + 2) & 3][0] = 0;
                ctl->alive_acc[(rr + 2) & 3] = 0;
            },
            [next]() { s_count = __ldcg(next); }))
            return;
        count = s_count;
        if (count > 0 && r + 1 >= a.max_rounds) {
            if (threadIdx.x == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            return;
        }
    }

    // ---- output
    if (a.out) {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        unsigned in_cnt = 0;
        for (long long v = tid; v < a.n; v += nthreads) {
            const bool in = ld_word(a.word + v) >= kWordInMin;
            in_cnt += in;
            if (a.seg.count == 0) {
                a.out[v] = in;
            } else {
                const int gg = a.seg.blk_seg[v >> 4];
                const int local = (int)v - a.seg.voff[gg];
                if (local < a.seg.nv[gg]) a.out[a.seg.roff[gg] + local] = in;
            }
        }
        for (int o = 16; o; o >>= 1) in_cnt += __shfl_xor_sync(0xFFFFFFFFu, in_cnt, o);
        if (lane == 0 && in_cnt) atomicAdd(&ctl->mis_size, (unsigned long long)in_cnt);
    }
}

const void* tile_kernel_fn(int T, int S, int P) {
    if (P >= 0) {
        if (T != 16) return nullptr;
        switch (P) {
            case kPayBitsF16: return (const void*)tile_solve_kernel<16, 8, kPayBitsF16>;
            case kPayB1: return (const void*)tile_solve_kernel<16, 8, kPayB1>;
            case kPayI8: return (const void*)tile_solve_kernel<16, 8, kPayI8>;
            case kPayF16: return (const void*)tile_solve_kernel<16, 8, kPayF16>;
            default: return nullptr;
        }
    }
    if (T == 8 && S == 1) return (const void*)tile_solve_kernel<8, 1, -1>;
    if (T == 8 && S == 2) return (const void*)tile_solve_kernel<8, 2, -1>;
    if (T == 8 && S == 4) return (const void*)tile_solve_kernel<8, 4, -1>;
    if (T == 16 && S == 1) return (const void*)tile_solve_kernel<16, 1, -1>;
    if (T == 16 && S == 4) return (const void*)tile_solve_kernel<16, 4, -1>;
    if (T == 8 && S == 8) return (const void*)tile_solve_kernel<8, 8, -1>;
    if (T == 8 && S == 32) return (const void*)tile_solve_kernel<8, 32, -1>;
    if (T == 16 && S == 8) return (const void*)tile_solve_kernel<16, 8, -1>;
    if (T == 16 && S == 32) return (const void*)tile_solve_kernel<16, 32, -1>;
    return nullptr;
}

}  // namespace

cudaError_t launch_tile_solve(const SolveArgs& a, int T, int S, int tc_payload, int grid,
                              cudaStream_t s) {
    const void* fn = tile_kernel_fn(T, S, tc_payload);
    if (!fn) return cudaErrorInvalidValue;
    void* args[] = {const_cast<SolveArgs*>(&a)};
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kTileBlock), args, 0, s);
}

int tile_max_coresident_blocks(int T, int S, int tc_payload, int device) {
    const void* fn = tile_kernel_fn(T, S, tc_payload);
    if (!fn) return 0;
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kTileBlock, 0) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

// ---------------------------------------------------------------- stored payloads
//
// The int8 and fp16 payload forms of the tensor-core exclusion, expanded from
// the bitmask: tile t's entry (i, j) at byte (kPayI8) or half (kPayF16)
// offset t * 256 + i * 16 + j.  One thread per tile row.

namespace {

__global__ void expand_payload_kernel(const uint64_t* __restrict__ tbits, int64_t ntiles, int P,
                                      void* __restrict__ out) {
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= ntiles * 16) return;
    const int t = (int)(x >> 4), i = (int)(x & 15);
    const uint32_t r = tile_row16(tbits, t, i);
    if (P == kPayI8) {
        uint4 v;
        v.x = bytes_of4(r & 0xFu);
        v.y = bytes_of4((r >> 4) & 0xFu);
        v.z = bytes_of4((r >> 8) & 0xFu);
        v.w = bytes_of4((r >> 12) & 0xFu);
        reinterpret_cast<uint4*>(out)[x] = v;
    } else {
        uint32_t h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) h[k] = half2_of((r >> (2 * k)) & 1u, (r >> (2 * k + 1)) & 1u);
        uint4* o = reinterpret_cast<uint4*>(out) + 2 * x;
        o[0] = make_uint4(h[0], h[1], h[2], h[3]);
        o[1] = make_uint4(h[4], h[5], h[6], h[7]);
    }
}

}  // namespace

int64_t tile_payload_bytes(int64_t ntiles, int P) {
    return P == kPayI8 ? 256 * ntiles : P == kPayF16 ? 512 * ntiles : 0;
}

cudaError_t build_tile_payload(const TileCsr& tiles, int P, void** out, cudaStream_t s) {
    *out = nullptr;
    if (tiles.T != 16 || (P != kPayI8 && P != kPayF16)) return cudaErrorInvalidValue;
    const int64_t bytes = tile_payload_bytes(tiles.ntiles, P);
    cudaError_t e = dev_alloc(out, (size_t)std::max<int64_t>(bytes, 16));
    if (e != cudaSuccess) return e;
    if (tiles.ntiles > 0) {
        const long long rows = tiles.ntiles * 16;
        expand_payload_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, s>>>(tiles.tbits,
                                                                            tiles.ntiles, P, *out);
        e = cudaGetLastError();
    }
    const cudaError_t se = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = se;
    if (e != cudaSuccess) {
        dev_free(*out);
        *out = nullptr;
    }
    return e;
}

}  // namespace tcmis
