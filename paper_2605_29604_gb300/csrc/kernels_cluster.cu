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
//            scan reads local shared memory and the CTAs exchange, after each
//            phase, one bit per owned vertex whose state changed; otherwise a
//            CTA holds its own chunk and neighbour words are read through
//            distributed shared memory;
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
// replica of all words, so every scan reads local shared memory; in each
// phase a CTA publishes one bit per owned vertex whose state changed (one
// word per warp, from a ballot), storing it into every CTA's copy of the
// change bitmask, and after the cluster barrier every CTA folds the bits it
// received into its replica.  Two bitmasks (selected, excluded) keep a
// phase's bits until every CTA has folded them.
template <bool kRep>
__global__ void __launch_bounds__(kClusterThreads, 1)
    cluster_solve_kernel(const SolveArgs a, const ClusterArgs c) {
    extern __shared__ uint32_t s_dyn[];
    __shared__ int s_rem[2];  // this CTA's undecided count, by round parity
    __shared__ unsigned s_sel;
    __shared__ int s_total;
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int chunk = 1 << c.shift;
    const int32_t n = a.n;
    const int base = rank * chunk;
    const int cnt = max(0, min(chunk, n - base));  // this CTA's vertices
    const int tid = (int)threadIdx.x;
    const int nth = (int)blockDim.x;
    // shared memory: the words (own chunk, or all chunks), with kRep the two
    // change bitmasks of the own chunk, then (smem_rows) the own rows
    const int nwords = kRep ? c.ncta * chunk : chunk;
    const int nmask = kRep ? c.ncta * (chunk / 32) : 0;  // change bits of every chunk
    uint32_t* s_word = s_dyn;
    uint32_t* s_new_in = s_dyn + nwords;
    uint32_t* s_new_out = s_new_in + nmask;
    int32_t* s_rp = reinterpret_cast<int32_t*>(s_new_out + nmask);
    int32_t* s_col = s_rp + chunk + 1;
    uint32_t* s_own = kRep ? s_word + base : s_word;  // the own chunk's words
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
    // the word of vertex u: in this CTA (kRep), else wherever it lives
    auto word_of = [&](int u) -> const uint32_t* {
        if (kRep) return s_word + u;
        return cluster.map_shared_rank(s_word + (u & (chunk - 1)), u >> c.shift);
    };

    // ---- init: the CTA's rows into shared memory (coalesced copies), then
    // Eq. 1 priorities (of all vertices with kRep); isolated vertices straight
    // into the set, and the own vertices' result bytes
    const int arc0 = cnt > 0 ? a.rp[base] : 0;
    if (c.smem_rows && cnt > 0) {
        const int arc1 = a.rp[base + cnt];
        for (int k = tid; k <= cnt; k += nth) s_rp[k] = a.rp[base + k] - arc0;
        for (int p = tid; p < arc1 - arc0; p += nth) s_col[p] = __ldg(a.col + arc0 + p);
    }
    for (int i = tid; i < nwords; i += nth) {
        const int v = kRep ? i : base + i;
        uint32_t w = kWordOut;
        if (v < n) {
            const int deg = a.rp[v + 1] - a.rp[v];
            w = deg ? undecided_word(mode, priority_key(mode, dbar, deg, smix, (uint32_t)v))
                    : (kKeyIsolated | kWordInSet);
        }
        s_word[i] = w;
    }
    cluster.sync();
    if (rank == 0 && tid == 0 && times) times->t[1] = global_ns();

    // Scan of the row of v (local index k): sel: does an undecided or
    // selected neighbour outrank v (word wv); else: is a neighbour in the set.
    // kBatch neighbour words are requested before any of them is tested.
    auto scan = [&](int k, int v, uint32_t wv, bool sel) -> bool {
        const int32_t* row;
        int deg;
        if (c.smem_rows) {
            row = s_col + s_rp[k];
            deg = s_rp[k + 1] - s_rp[k];
        } else {
            row = a.col + a.rp[v];
            deg = a.rp[v + 1] - a.rp[v];
        }
        for (int q0 = 0; q0 < deg; q0 += kBatch) {
            int u[kBatch];
            uint32_t wu[kBatch];
#pragma unroll
            for (int q = 0; q < kBatch; ++q) u[q] = q0 + q < deg ? row[q0 + q] : 0;
#pragma unroll
            for (int q = 0; q < kBatch; ++q) wu[q] = q0 + q < deg ? *word_of(u[q]) : 0u;
            bool hit = false;
#pragma unroll
            for (int q = 0; q < kBatch; ++q)
                hit |= q0 + q < deg && (sel ? outranks_c(wu[q], u[q], wv, v) : wu[q] >= kWordInMin);
            if (hit) return true;
        }
        return false;
    };
    // kRep: a warp's change word of the own chunk, stored into every CTA's
    // copy of the bitmask (remote stores, made visible by the next barrier)
    auto publish = [&](uint32_t* mask, int k, unsigned m) {
        const int lane = tid & 31;
        if (lane < c.ncta) *cluster.map_shared_rank(mask + rank * (chunk / 32) + (k >> 5), lane) = m;
    };
    // kRep: fold the other CTAs' changes, received in local shared memory,
    // into the replica (in: OR the set bits, else: out)
    auto fold = [&](const uint32_t* mask, bool in) {
        const int per = chunk / 32;
        for (int i = tid; i < c.ncta * per; i += nth) {
            const int q = i / per, j = i - q * per;
            if (q == rank) continue;
            uint32_t bits = mask[i];
            while (bits) {
                const int b = __ffs(bits) - 1;
                bits &= bits - 1;
                uint32_t* w = s_word + q * chunk + 32 * j + b;
                *w = in ? (*w | kWordInSet) : kWordOut;
            }
        }
    };

    int alive = n;  // round 0's alive set: every vertex
    for (int r = 0;; ++r) {
        const int par = r & 1;
        // ---- Phase 1: selection test over the own chunk (kRep: every warp
        // covers whole 32-vertex words, so its ballot is the word's bits)
        unsigned sel = 0;
        for (int k = tid; k < (kRep ? chunk : cnt); k += nth) {
            bool cand = false;
            if (k < cnt) {
                const uint32_t wv = s_own[k];
                if ((wv >> 29) == 1u && !scan(k, base + k, wv, true)) {
                    s_own[k] = wv | kWordInSet;
                    cand = true;
                    ++sel;
                }
            }
            if (kRep) publish(s_new_in, k, __ballot_sync(0xFFFFFFFFu, cand));
        }
        if (sel) atomicAdd(&s_sel, sel);
        cluster.sync();
        if (rank == 0 && tid == 0 && times && r < kStatRounds) times->t[2 + r] = global_ns();
        if (kRep) {
            fold(s_new_in, true);
            __syncthreads();
        }
        // ---- Phases 2 and 3: exclusion test, state update; count the rest
        int rem = 0;
        for (int k = tid; k < (kRep ? chunk : cnt); k += nth) {
            bool out = false;
            if (k < cnt) {
                const uint32_t wv = s_own[k];
                if ((wv >> 29) == 1u) {
                    if (scan(k, base + k, wv, false)) {
                        s_own[k] = kWordOut;
                        out = true;
                    } else {
                        ++rem;
                    }
                }
            }
            if (kRep) publish(s_new_out, k, __ballot_sync(0xFFFFFFFFu, out));
        }
        for (int o = 16; o; o >>= 1) rem += __shfl_xor_sync(0xFFFFFFFFu, rem, o);
        if ((tid & 31) == 0 && rem) atomicAdd(&s_rem[par], rem);
        cluster.sync();
        if (kRep) fold(s_new_out, false);
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
    // the result of the own vertices, written once after the rounds (so that
    // no phase has global stores for the cluster barrier's fence to wait on),
    // and the MIS size: this CTA's candidates and its isolated vertices (put
    // in the set at init without a test)
    unsigned iso = 0;
    for (int k = tid; k < cnt; k += nth) {
        if (a.out) a.out[base + k] = s_own[k] >= kWordInMin ? 1 : 0;
        iso += (a.rp[base + k + 1] == a.rp[base + k]) ? 1u : 0u;
    }
    for (int o = 16; o; o >>= 1) iso += __shfl_xor_sync(0xFFFFFFFFu, iso, o);
    if ((tid & 31) == 0 && iso) atomicAdd(&s_sel, iso);
    __syncthreads();
    if (tid == 0 && s_sel) atomicAdd(&ctl->mis_size, (unsigned long long)s_sel);
    // no CTA may leave while another still reads its shared memory
    cluster.sync();
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
    const size_t budget = (size_t)max_optin > 1024 ? (size_t)max_optin - 1024 : 0;
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
        // a replica of every word (and the two change bitmasks) if it fits,
        // else the own chunk's words; the rows on chip if they fit as well
        const size_t rep = sizeof(uint32_t) * ((size_t)ncta * chunk + (size_t)ncta * chunk / 16);
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
        const void* fn = replicated ? (const void*)cluster_solve_kernel<true>
                                    : (const void*)cluster_solve_kernel<false>;
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
    const long long words = ((long long)max_optin - 1024) / 4;
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
    if (p.replicated) return cudaLaunchKernelEx(&cfg, cluster_solve_kernel<true>, a, c);
    return cudaLaunchKernelEx(&cfg, cluster_solve_kernel<false>, a, c);
}

}  // namespace tcmis
