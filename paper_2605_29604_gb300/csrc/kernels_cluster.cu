// kernels_cluster.cu -- one thread-block cluster solves a small graph.
//
// Algorithm 2's rounds need two barriers each; on a grid of hundreds of
// blocks a software grid barrier costs microseconds, which dominates the
// solve of a graph of a few thousand vertices.  Here one cluster of C CTAs
// (C <= 16, one per SM) takes the whole graph:
//
//   state    the packed vertex words (common.cuh) live in the CTAs' shared
//            memory: vertex v in CTA v >> shift at slot v & (chunk - 1), chunk
//            = 2^shift >= n / C; every neighbour word is read through
//            distributed shared memory, never from global memory;
//   barriers the phases are separated by the cluster's hardware barrier
//            (barrier.cluster arrive/wait through cooperative groups), which
//            every CTA reaches the same number of times: the loop exit is
//            decided from counts that all CTAs read after the same barrier;
//   rows     a thread that owns one vertex keeps up to kCached neighbour ids
//            in registers for all rounds; longer rows, and threads with
//            several vertices, read their rows from global memory each round.
//
// Phase 1 (selection test) and Phase 2 (exclusion test, state update) read
// the round-start snapshot exactly as the grid kernel does (see common.cuh),
// so the rounds and alive sets are Algorithm 2's.
#include <algorithm>

#include <cooperative_groups.h>

#include "common.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace tcmis {

namespace {

constexpr int kClusterThreads = 1024;
constexpr int kCached = 10;  // neighbour ids kept in registers per owned vertex

struct ClusterArgs {
    int32_t shift;   // chunk = 1 << shift vertices per CTA
    int32_t ncta;    // CTAs in the cluster
};

__device__ __forceinline__ bool outranks_c(uint32_t wu, int u, uint32_t wv, int v) {
    return wu > wv || (wu == wv && u > v);
}

__global__ void __launch_bounds__(kClusterThreads, 1)
    cluster_solve_kernel(const SolveArgs a, const ClusterArgs c) {
    extern __shared__ uint32_t s_word[];  // this CTA's chunk of vertex words
    __shared__ int s_rem[2];              // this CTA's undecided count, by round parity
    __shared__ unsigned s_sel;            // candidates this CTA selected
    __shared__ int s_total;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int chunk = 1 << c.shift;
    const int32_t n = a.n;
    const int base = rank * chunk;
    const int tid = (int)threadIdx.x;
    const int nth = (int)blockDim.x;
    Ctl* ctl = a.ctl;
    PhaseTimes* times = a.times;
    const int mode = a.priority;
    const uint64_t smix = mix64(a.seed0);
    const float dbar = n > 0 ? average_degree(a.rp[n], n) : 0.f;
    if (tid == 0) {
        s_rem[0] = s_rem[1] = 0;
        s_sel = 0;
        if (rank == 0 && times) times->t[0] = global_ns();
    }
    // the word of vertex u, wherever it lives in the cluster
    auto word_of = [&](int u) -> uint32_t* {
        return cluster.map_shared_rank(s_word + (u & (chunk - 1)), u >> c.shift);
    };

    // ---- init: Eq. 1 priorities; isolated vertices straight into the set
    // (and the result); the owned row cached when a thread has one vertex
    const bool single = chunk <= nth;
    int cached[kCached];
    int my_b = 0, my_deg = 0;
    for (int k = tid; k < chunk; k += nth) {
        const int v = base + k;
        uint32_t w = kWordOut;
        if (v < n) {
            const int b = a.rp[v], deg = a.rp[v + 1] - b;
            w = deg ? undecided_word(mode, priority_key(mode, dbar, deg, smix, (uint32_t)v))
                    : (kKeyIsolated | kWordInSet);
            if (a.out) a.out[v] = deg ? 0 : 1;
            if (single) {
                my_b = b;
                my_deg = deg;
            }
        }
        s_word[k] = w;
    }
    if (single) {
#pragma unroll
        for (int k = 0; k < kCached; ++k) cached[k] = k < my_deg ? __ldg(a.col + my_b + k) : 0;
    }
    cluster.sync();
    if (rank == 0 && tid == 0 && times) times->t[1] = global_ns();

    // Scan of v's row: kSelect: does an undecided or selected neighbour
    // outrank v (word wv), else: is a neighbour in the set.
    auto scan = [&](int v, int b, int deg, bool use_cache, uint32_t wv, bool sel) -> bool {
        int k = 0;
        if (use_cache) {
            // every cached neighbour's word is requested before any is tested
            uint32_t wu[kCached];
#pragma unroll
            for (int q = 0; q < kCached; ++q) wu[q] = q < deg ? *word_of(cached[q]) : 0u;
            bool hit = false;
#pragma unroll
            for (int q = 0; q < kCached; ++q)
                hit |= q < deg && (sel ? outranks_c(wu[q], cached[q], wv, v) : wu[q] >= kWordInMin);
            if (hit) return true;
            k = kCached;
        }
        for (; k < deg; ++k) {
            const int u = __ldg(a.col + b + k);
            const uint32_t wu = *word_of(u);
            if (sel ? outranks_c(wu, u, wv, v) : wu >= kWordInMin) return true;
        }
        return false;
    };

    int alive = n;  // round 0's alive set: every vertex
    for (int r = 0;; ++r) {
        const int par = r & 1;
        // ---- Phase 1: selection test
        unsigned sel = 0;
        for (int k = tid; k < chunk; k += nth) {
            const int v = base + k;
            if (v >= n) break;
            const uint32_t wv = s_word[k];
            if ((wv >> 29) != 1u) continue;  // decided
            const int b = single ? my_b : a.rp[v];
            const int deg = single ? my_deg : a.rp[v + 1] - b;
            if (!scan(v, b, deg, single, wv, true)) {
                s_word[k] = wv | kWordInSet;
                if (a.out) a.out[v] = 1;
                ++sel;
            }
        }
        if (sel) atomicAdd(&s_sel, sel);
        cluster.sync();
        if (rank == 0 && tid == 0 && times && r < kStatRounds) times->t[2 + r] = global_ns();
        // ---- Phases 2 and 3: exclusion test, state update; count the rest
        int rem = 0;
        for (int k = tid; k < chunk; k += nth) {
            const int v = base + k;
            if (v >= n) break;
            const uint32_t wv = s_word[k];
            if ((wv >> 29) != 1u) continue;
            const int b = single ? my_b : a.rp[v];
            const int deg = single ? my_deg : a.rp[v + 1] - b;
            if (scan(v, b, deg, single, wv, false)) s_word[k] = kWordOut;
            else ++rem;
        }
        for (int o = 16; o; o >>= 1) rem += __shfl_xor_sync(0xFFFFFFFFu, rem, o);
        if ((tid & 31) == 0 && rem) atomicAdd(&s_rem[par], rem);
        cluster.sync();
        // every CTA sums the same counts, so all leave the loop together
        if (tid < 32) {
            int total = tid < c.ncta ? *cluster.map_shared_rank(&s_rem[par], tid) : 0;
            for (int o = 16; o; o >>= 1) total += __shfl_xor_sync(0xFFFFFFFFu, total, o);
            if (tid == 0) s_total = total;
            if (rank == 0 && tid == 0) {
                if (times && r < kStatRounds) times->t[2 + kStatRounds + r] = global_ns();
                if (r < kStatRounds) ctl->alive[r] = alive;
                ctl->alive_sum += (unsigned long long)alive;
                ctl->rounds = r + 1;
            }
        }
        __syncthreads();
        const int total = s_total;
        // the other slot, last read (by every CTA) before this round's first
        // barrier, is cleared for the next round's count
        if (tid == 0) s_rem[par ^ 1] = 0;
        if (total == 0) break;
        if (r + 1 >= a.max_rounds) {
            if (rank == 0 && tid == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            break;  // uniform: every CTA saw the same total and round
        }
        alive = total;
        __syncthreads();
    }
    // the MIS size: this CTA's candidates and its isolated vertices (put in
    // the set at init without a test)
    unsigned iso = 0;
    for (int k = tid; k < chunk; k += nth) {
        const int v = base + k;
        if (v >= n) break;
        iso += (a.rp[v + 1] == a.rp[v]) ? 1u : 0u;
    }
    for (int o = 16; o; o >>= 1) iso += __shfl_xor_sync(0xFFFFFFFFu, iso, o);
    if ((tid & 31) == 0 && iso) atomicAdd(&s_sel, iso);
    __syncthreads();
    if (tid == 0 && s_sel) atomicAdd(&ctl->mis_size, (unsigned long long)s_sel);
    // no CTA may leave while another still reads its shared memory
    cluster.sync();
}

// The cluster that takes a graph of n vertices: 16 CTAs where the device can
// co-schedule them, else 8; each CTA holds chunk = 2^shift >= n / ncta words
// in at most kClusterSmem bytes.  Returns false when the graph is too large.
constexpr int kClusterSmem = 128 * 1024;

}  // namespace

bool cluster_plan(int32_t n, int* ncta_out, int* shift_out) {
    for (int ncta : {16, 8}) {
        int shift = 5;
        while ((long long)(1 << shift) * ncta < n) ++shift;
        const size_t smem = sizeof(uint32_t) << shift;
        if (smem > (size_t)kClusterSmem) continue;
        if (ncta > 8 && cudaFuncSetAttribute(cluster_solve_kernel,
                                             cudaFuncAttributeNonPortableClusterSizeAllowed,
                                             1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (cudaFuncSetAttribute(cluster_solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ncta);
        cfg.blockDim = dim3(std::min(kClusterThreads, std::max(32, 1 << shift)));
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = ncta;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, cluster_solve_kernel, &cfg) != cudaSuccess ||
            clusters < 1) {
            cudaGetLastError();
            continue;
        }
        *ncta_out = ncta;
        *shift_out = shift;
        return true;
    }
    return false;
}

int32_t cluster_max_vertices() {
    int ncta = 0, shift = 0;
    // the largest n whose plan fits: one word per vertex within kClusterSmem per CTA
    const int32_t guess = 16 * (kClusterSmem / 4);
    for (int32_t n = guess; n >= 1024; n /= 2)
        if (cluster_plan(n, &ncta, &shift)) return n;
    return 0;
}

cudaError_t launch_cluster_solve(const SolveArgs& a, int ncta, int shift, cudaStream_t s) {
    if (ncta < 1 || ncta > 16 || shift < 5 || (long long)ncta << shift < a.n)
        return cudaErrorInvalidConfiguration;
    const int chunk = 1 << shift;
    ClusterArgs c;
    c.shift = shift;
    c.ncta = ncta;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(ncta);
    cfg.blockDim = dim3(std::min(kClusterThreads, std::max(32, chunk)));
    cfg.dynamicSmemBytes = sizeof(uint32_t) * (size_t)chunk;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, cluster_solve_kernel, a, c);
}

}  // namespace tcmis
