// kernels_cluster.cu -- one thread-block cluster solves a small graph.
//
// Algorithm 2's rounds need two barriers each; on a grid of hundreds of
// blocks a software grid barrier costs microseconds, which dominates the
// solve of a graph of a few thousand vertices.  Here one cluster of C CTAs
// (C <= 16, one per SM) takes the whole graph:
//
//   state    the packed vertex words (common.cuh) live in the CTAs' shared
//            memory.  CTA r owns the vertices of chunk r (chunk = 2^shift >=
//            n / C).  Where a replica of every word fits in each CTA, every
//            scan reads local shared memory and, after each phase's barrier,
//            every CTA reads (pulls) from the others one bit per owned vertex
//            whose state changed; otherwise a CTA holds its own chunk and
//            neighbour words are read through distributed shared memory;
//   barriers the phases are separated by the cluster's hardware barrier
//            (barrier.cluster arrive/wait through cooperative groups), which
//            every CTA reaches the same number of times: the loop exit is
//            decided from counts that all CTAs read after the same barrier;
//   rows     where they fit, each CTA copies its vertices' row offsets and
//            arcs into shared memory once (coalesced loads at init), so every
//            later scan reads its row on chip; otherwise rows are read from
//            global memory.  A scan requests kBatch neighbour words before it
//            tests any of them.
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
constexpr int kBatch = 8;  // neighbour words requested at once by a thread

struct ClusterArgs {
    int32_t shift;      // chunk = 1 << shift vertices per CTA
    int32_t ncta;       // CTAs in the cluster
    int32_t smem_rows;  // 1: each CTA holds its rows (row_ptr and col_idx slices)
                        // in shared memory; 0: rows are read from global memory
};

__device__ __forceinline__ bool outranks_c(uint32_t wu, int u, uint32_t wv, int v) {
    return wu > wv || (wu == wv && u > v);
}

// kRep = false: CTA r holds the words of its own chunk only; neighbour words
// are read through distributed shared memory.  kRep = true: every CTA holds a
// replica of all words, so no scan leaves the SM.  In each phase a CTA
// writes one bit per owned vertex whose state changed (one word per warp,
// from a ballot) into its own part of that phase's bitmask; after the
// cluster barrier every CTA reads the other CTAs' parts (remote loads: a
// pull costs one load latency, where remote stores before the barrier would
// make its release wait for every store to be acknowledged).  Phase 2 tests
// a neighbour's bit in the round's selection bitmask (a vertex still
// undecided at a round's start has no neighbour in the set, so only this
// round's selections can exclude it).  After Phase 2 every CTA ORs the
// round's exclusion bits into its bitmask of excluded vertices; the replica
// keeps every other chunk's initial words, and Phase 1 counts a neighbour
// that outranks v by its word only if its excluded bit is clear (an
// undecided vertex has no neighbour in the set, so the excluded bit is the
// only state change Phase 1 needs).  kRows: the CTA's rows are in shared
// memory.
//
// No store in the round loop goes to global or remote shared memory: the
// undecided counts are read by every CTA from every CTA after the barrier,
// and the statistics (undecided counts, phase end times) stay in rank 0's
// shared memory until the end.
template <bool kRep, bool kRows>
__global__ void __launch_bounds__(kClusterThreads, 1)
    cluster_solve_kernel(const SolveArgs a, const ClusterArgs c) {
    extern __shared__ __align__(16) uint32_t s_dyn[];
    __shared__ int s_cnt[2];     // this CTA's undecided count, by round parity
    __shared__ int s_total;      // the cluster's undecided count
    __shared__ unsigned s_size;  // this CTA's part of the MIS size
    __shared__ int s_err;        // rank 0: the error code
    __shared__ unsigned long long s_t[2 + 2 * kStatRounds];  // rank 0: phase end times
    __shared__ int s_alive[kStatRounds];                     // rank 0: alive set sizes
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int chunk = 1 << c.shift;
    const int32_t n = a.n;
    const int base = rank * chunk;
    const int cnt = max(0, min(chunk, n - base));  // this CTA's vertices
    const int tid = (int)threadIdx.x;
    const int nth = (int)blockDim.x;
    const int lane = tid & 31;
    // shared memory: the words (own chunk, or all chunks), with kRep the two
    // change bitmasks of every chunk and the excluded bitmask, then (kRows)
    // the own rows
    const int nwords = kRep ? c.ncta * chunk : chunk;
    const int mshift = c.shift - 5;  // bitmask words per chunk: 2^mshift
    const int nmask = kRep ? c.ncta << mshift : 0;
    uint32_t* s_word = s_dyn;
    uint32_t* s_new_in = s_dyn + nwords;
    uint32_t* s_new_out = s_new_in + nmask;
    uint32_t* s_gone = s_new_out + nmask;
    int32_t* s_rp = reinterpret_cast<int32_t*>(s_gone + nmask);
    int32_t* s_col = s_rp + chunk + 1;
    uint32_t* s_own = kRep ? s_word + base : s_word;  // the own chunk's words
    const int mode = a.priority;
    const uint64_t smix = mix64(a.seed0);
    // the loads init depends on, issued first: the arc count (for d-bar) and
    // the bounds of the own slice of arcs
    const int32_t arcs_all = n > 0 ? a.rp[n] : 0;
    const int arc0 = kRows && cnt > 0 ? a.rp[base] : 0;
    const int arcs = kRows && cnt > 0 ? a.rp[base + cnt] - arc0 : 0;
    const float dbar = n > 0 ? average_degree(arcs_all, n) : 0.f;
    const bool stats = rank == 0;
    if (tid == 0) {
        s_cnt[0] = s_cnt[1] = 0;
        s_size = 0;
        s_err = 0;
    }
    if (stats) {
        for (int i = tid; i < 2 + 2 * kStatRounds; i += nth) s_t[i] = 0;
        if (tid == 0) s_t[0] = global_ns();
    }
    // the word of vertex u: in this CTA (kRep), else wherever it lives
    auto word_of = [&](int u) -> const uint32_t* {
        if (kRep) return s_word + u;
        return cluster.map_shared_rank(s_word + (u & (chunk - 1)), u >> c.shift);
    };

    // ---- init: the own vertices' Eq. 1 priorities (isolated vertices
    // straight into the set) and row offsets, the CTA's arcs into shared
    // memory (coalesced copies, four loads in flight per thread); after the
    // barrier, with kRep, the other chunks' words into the replica (16-byte
    // remote loads)
    for (int k = tid; k < chunk; k += nth) {
        const int v = base + k;
        uint32_t w = kWordOut;
        if (v < n) {
            const int r0 = a.rp[v];
            const int deg = a.rp[v + 1] - r0;
            if (kRows) s_rp[k] = r0 - arc0;
            w = deg ? undecided_word(mode, priority_key(mode, dbar, deg, smix, (uint32_t)v))
                    : (kKeyIsolated | kWordInSet);
        }
        s_own[k] = w;
    }
    if (kRows && tid == 0) s_rp[cnt] = arcs;
    if (kRows) {
        for (int p0 = tid; p0 < arcs; p0 += 4 * nth) {
            int32_t x[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) x[j] = p0 + j * nth < arcs ? __ldg(a.col + arc0 + p0 + j * nth) : 0;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (p0 + j * nth < arcs) s_col[p0 + j * nth] = x[j];
        }
    }
    for (int j = tid; j < nmask; j += nth) s_gone[j] = 0u;
    cluster.sync();
    if (kRep) {
        // a word pulled while its owner marks it selected in round 0 is
        // either value; both compare the same way in every later test (a
        // candidate outranks each undecided neighbour, and no undecided
        // vertex neighbours a vertex in the set)
        // (four loads in flight per thread before any store)
        const int qshift = c.shift - 2;  // 16-byte quads per chunk: 2^qshift
        const int nquad = c.ncta << qshift;
        for (int p0 = tid; p0 < nquad; p0 += 4 * nth) {
            uint4 x[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = p0 + j * nth, q = p >> qshift;
                if (p < nquad && q != rank)
                    x[j] = *reinterpret_cast<const uint4*>(cluster.map_shared_rank(s_word, q) + 4 * p);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = p0 + j * nth;
                if (p < nquad && (p >> qshift) != rank) reinterpret_cast<uint4*>(s_word)[p] = x[j];
            }
        }
        __syncthreads();
    }
    if (stats && tid == 0) s_t[1] = global_ns();

    // Scan of the row of v (local index k).  sel: does an undecided or
    // selected neighbour outrank v (word wv; kRep: and is it not excluded)?
    // else: is a neighbour in the set (kRep: selected in this round)?
    // kBatch loads are issued before any of them is tested.
    auto scan = [&](int k, int v, uint32_t wv, bool sel, bool late) -> bool {
        const int32_t* row;
        int deg;
        if (kRows) {
            row = s_col + s_rp[k];
            deg = s_rp[k + 1] - s_rp[k];
        } else {
            row = a.col + a.rp[v];
            deg = a.rp[v + 1] - a.rp[v];
        }
        for (int q0 = 0; q0 < deg; q0 += kBatch) {
            int u[kBatch];
            uint32_t x[kBatch];
#pragma unroll
            for (int q = 0; q < kBatch; ++q) u[q] = q0 + q < deg ? row[q0 + q] : 0;
#pragma unroll
            for (int q = 0; q < kBatch; ++q)
                x[q] = q0 + q >= deg ? 0u
                       : (kRep && !sel) ? (s_new_in[u[q] >> 5] >> (u[q] & 31)) & 1u
                                        : *word_of(u[q]);
            bool hit[kBatch];
            bool any = false;
#pragma unroll
            for (int q = 0; q < kBatch; ++q) {
                hit[q] = q0 + q < deg && (sel ? outranks_c(x[q], u[q], wv, v)
                                              : kRep ? x[q] != 0u : x[q] >= kWordInMin);
                any |= hit[q];
            }
            // a neighbour that outranks v by its word counts only if it is
            // not excluded; the bits are read only for such neighbours, and
            // not at all in round 0 (nothing is excluded yet)
            if (kRep && sel && any && late) {
                any = false;
#pragma unroll
                for (int q = 0; q < kBatch; ++q)
                    any |= hit[q] && !((s_gone[u[q] >> 5] >> (u[q] & 31)) & 1u);
            }
            if (any) return true;
        }
        return false;
    };

    int alive = n;  // round 0's alive set: every vertex
    unsigned long long alive_sum = 0;
    int r = 0;
    for (;; ++r) {
        const int par = r & 1;
        // ---- Phase 1: selection test over the own chunk (kRep: every warp
        // covers whole 32-vertex words, so its ballot is the word's bits)
        for (int k = tid; k < (kRep ? chunk : cnt); k += nth) {
            bool cand = false;
            if (k < cnt) {
                const uint32_t wv = s_own[k];
                if ((wv >> 29) == 1u && !scan(k, base + k, wv, true, r > 0)) {
                    s_own[k] = wv | kWordInSet;
                    cand = true;
                }
            }
            if (kRep) {
                const unsigned m = __ballot_sync(0xFFFFFFFFu, cand);
                if (lane == 0) s_new_in[(rank << mshift) + (k >> 5)] = m;
            }
        }
        cluster.sync();
        if (kRep) {
            // the other CTAs' selections of this round
            for (int i = tid; i < nmask; i += nth) {
                const int q = i >> mshift;
                if (q != rank) s_new_in[i] = *cluster.map_shared_rank(s_new_in + i, q);
            }
            __syncthreads();
        }
        if (stats && tid == 0 && r < kStatRounds) s_t[2 + r] = global_ns();
        // ---- Phases 2 and 3: exclusion test, state update; count the rest
        int rem = 0;
        for (int k = tid; k < (kRep ? chunk : cnt); k += nth) {
            bool out = false;
            if (k < cnt) {
                const uint32_t wv = s_own[k];
                if ((wv >> 29) == 1u) {
                    if (scan(k, base + k, wv, false, r > 0)) {
                        s_own[k] = kWordOut;
                        out = true;
                    } else {
                        ++rem;
                    }
                }
            }
            if (kRep) {
                const unsigned m = __ballot_sync(0xFFFFFFFFu, out);
                if (lane == 0) s_new_out[(rank << mshift) + (k >> 5)] = m;
            }
        }
        for (int o = 16; o; o >>= 1) rem += __shfl_xor_sync(0xFFFFFFFFu, rem, o);
        if (lane == 0 && rem) atomicAdd(&s_cnt[par], rem);
        cluster.sync();
        // every CTA's count (the same sum in every CTA, so all leave the loop
        // together) and, with kRep, the round's exclusions of every chunk
        if (tid < 32) {
            int t = lane < c.ncta ? *cluster.map_shared_rank(&s_cnt[par], lane) : 0;
            for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
            if (lane == 0) s_total = t;
        }
        if (kRep) {
            for (int i = tid; i < nmask; i += nth) {
                const int q = i >> mshift;
                s_gone[i] |= q == rank ? s_new_out[i] : *cluster.map_shared_rank(s_new_out + i, q);
            }
        }
        if (stats && tid == 0) {
            if (r < kStatRounds) {
                s_t[2 + kStatRounds + r] = global_ns();
                s_alive[r] = alive;
            }
            alive_sum += (unsigned long long)alive;
        }
        __syncthreads();
        const int total = s_total;
        // the other count, last read by the other CTAs before this round's
        // first barrier, is cleared for round r + 1
        if (tid == 0) s_cnt[par ^ 1] = 0;
        if (total == 0) break;
        if (r + 1 >= a.max_rounds) {
            if (stats && tid == 0) s_err = kErrInternal;
            break;  // uniform: every CTA saw the same total and round
        }
        alive = total;
        __syncthreads();
    }
    // this CTA's part of the MIS size (isolated vertices included); rank 0
    // reads every CTA's after the barrier
    unsigned in_cnt = 0;
    for (int k = tid; k < cnt; k += nth) in_cnt += s_own[k] >= kWordInMin ? 1u : 0u;
    for (int o = 16; o; o >>= 1) in_cnt += __shfl_xor_sync(0xFFFFFFFFu, in_cnt, o);
    if (lane == 0 && in_cnt) atomicAdd(&s_size, in_cnt);
    cluster.sync();
    unsigned long long mis_size = 0;
    if (stats && tid < 32) {
        unsigned long long t = lane < c.ncta ? *cluster.map_shared_rank(&s_size, lane) : 0ull;
        for (int o = 16; o; o >>= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
        mis_size = t;
    }
    // no CTA leaves while another may still read its shared memory
    cluster.sync();
    // the result of the own vertices: global stores only after the last
    // barrier, whose release would otherwise wait for them
    if (a.out)
        for (int k = tid; k < cnt; k += nth) a.out[base + k] = s_own[k] >= kWordInMin ? 1 : 0;
    // rank 0 writes every field of the control block and of the phase times
    // that a solve reports, so the launch needs no reset before it
    if (stats) {
        const int rounds = r + 1;
        if (tid == 0) {
            a.ctl->err = s_err;
            a.ctl->mis_size = mis_size;
            a.ctl->rounds = rounds;
            a.ctl->alive_sum = alive_sum;
        }
        for (int i = tid; i < kStatRounds; i += nth) a.ctl->alive[i] = i < rounds ? s_alive[i] : 0;
        if (a.times)
            for (int i = tid; i < 2 + 2 * kStatRounds; i += nth) a.times->t[i] = s_t[i];
    }
}

// static shared memory of the kernel (counters, rank 0's statistics) and a
// margin, kept out of the dynamic budget
constexpr size_t kStaticSmem = 2048;

const void* cluster_fn(int replicated, int smem_rows) {
    if (replicated)
        return smem_rows ? (const void*)cluster_solve_kernel<true, true>
                         : (const void*)cluster_solve_kernel<true, false>;
    return smem_rows ? (const void*)cluster_solve_kernel<false, true>
                     : (const void*)cluster_solve_kernel<false, false>;
}

}  // namespace

// The cluster that takes a graph of n vertices: 16 CTAs where the device can
// co-schedule them, else 8; each CTA holds chunk = 2^shift >= n / ncta words
// and, where they fit too, its rows.  Reads row_ptr at the CTAs' boundaries
// (d_rp on the device) to size the largest slice of arcs.
bool cluster_plan(const int32_t* d_rp, int32_t n, ClusterPlan* plan) {
    int max_optin = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t budget = (size_t)max_optin > kStaticSmem ? (size_t)max_optin - kStaticSmem : 0;
    for (int ncta : {16, 8}) {
        int shift = 5;
        while ((long long)(1 << shift) * ncta < n) ++shift;
        const int chunk = 1 << shift;
        // the largest slice of arcs a CTA owns
        long long max_slice = 0;
        int32_t prev = 0;
        for (int k = 1; k <= ncta; ++k) {
            const long long vb = std::min<long long>((long long)k * chunk, n);
            int32_t x = 0;
            if (n > 0 && cudaMemcpy(&x, d_rp + vb, sizeof(int32_t), cudaMemcpyDeviceToHost) !=
                             cudaSuccess)
                return false;
            max_slice = std::max<long long>(max_slice, (long long)x - prev);
            prev = x;
        }
        const size_t rows = sizeof(int32_t) * ((size_t)chunk + 1 + (size_t)max_slice);
        // a replica of every word (and the three bitmasks) if it fits,
        // else the own chunk's words; the rows on chip if they fit as well
        const size_t rep = sizeof(uint32_t) * ((size_t)ncta * chunk + 3 * ((size_t)ncta * chunk / 32));
        const size_t own = sizeof(uint32_t) * (size_t)chunk;
        int replicated, smem_rows;
        if (rep + rows <= budget) {
            replicated = 1;
            smem_rows = 1;
        } else if (own + rows <= budget) {
            replicated = 0;
            smem_rows = 1;
        } else if (rep <= budget) {
            replicated = 1;
            smem_rows = 0;
        } else if (own <= budget) {
            replicated = 0;
            smem_rows = 0;
        } else {
            continue;
        }
        const size_t smem = (replicated ? rep : own) + (smem_rows ? rows : 0);
        const void* fn = cluster_fn(replicated, smem_rows);
        if (ncta > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed,
                                             1) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(ncta);
        cfg.blockDim = dim3(std::min(kClusterThreads, std::max(32, chunk)));
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = ncta;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess || clusters < 1) {
            cudaGetLastError();
            continue;
        }
        plan->ncta = ncta;
        plan->shift = shift;
        plan->smem_rows = smem_rows;
        plan->replicated = replicated;
        plan->smem_bytes = (int64_t)smem;
        return true;
    }
    return false;
}

int32_t cluster_max_vertices() {
    int max_optin = 0, dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&max_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
        return 0;
    // the vertex words alone in 16 CTAs (the rows may then stay in global memory)
    const long long words = ((long long)max_optin - (long long)kStaticSmem) / 4;
    int shift = 5;
    while ((2LL << shift) <= words) ++shift;
    return (int32_t)std::min<long long>(16LL << shift, 1LL << 30);
}

cudaError_t launch_cluster_solve(const SolveArgs& a, const ClusterPlan& p, cudaStream_t s) {
    if (p.ncta < 1 || p.ncta > 16 || p.shift < 5 || ((long long)p.ncta << p.shift) < a.n)
        return cudaErrorInvalidConfiguration;
    const int chunk = 1 << p.shift;
    ClusterArgs c;
    c.shift = p.shift;
    c.ncta = p.ncta;
    c.smem_rows = p.smem_rows;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(p.ncta);
    cfg.blockDim = dim3(std::min(kClusterThreads, std::max(32, chunk)));
    cfg.dynamicSmemBytes = (size_t)p.smem_bytes;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = p.ncta;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.replicated)
        return p.smem_rows ? cudaLaunchKernelEx(&cfg, cluster_solve_kernel<true, true>, a, c)
                           : cudaLaunchKernelEx(&cfg, cluster_solve_kernel<true, false>, a, c);
    return p.smem_rows ? cudaLaunchKernelEx(&cfg, cluster_solve_kernel<false, true>, a, c)
                       : cudaLaunchKernelEx(&cfg, cluster_solve_kernel<false, false>, a, c);
}

}  // namespace tcmis
