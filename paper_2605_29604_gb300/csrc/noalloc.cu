// noalloc.cu -- a solve entry point that allocates no memory at all.
//
// Some callers cannot call cudaMalloc: code running inside a custom
// allocator or memory pool that must not recurse into the CUDA allocator,
// processes whose device memory is fully reserved up front by a framework,
// or real-time loops where an allocation's implicit synchronisation and
// latency are not acceptable.  mis_solve_noalloc serves them: the caller
// passes the graph and the result buffer (device memory it already owns),
// and the solve's scratch -- the packed per-vertex words, two worklists and
// the control block of the persistent kernel -- lives in one file-scope
// __device__ array of fixed size.  Every GPU that loads this library holds
// that array until the process exits.
//
// The kernel here is a separate variant of the CSR round kernel: it loads
// col_idx one element at a time (the caller's buffer need not be padded or
// 16-byte aligned) and clamps every index it reads, so a graph that breaks
// the input contract yields an unspecified set but no out-of-bounds access.
// The graph is not validated.
#include <cstddef>

#include "common.cuh"
#include "graph.h"
#include "internal.h"
#include "tcmis.h"

namespace tcmis {

namespace {

constexpr int32_t kNoAllocMaxVertices = 262144;  // 2^18 vertices
constexpr int kNoAllocTpr = 8;
constexpr int kNoAllocBlock = 512;
constexpr size_t kCtlBytes = 1024;
constexpr size_t kVecBytes = sizeof(int32_t) * (size_t)kNoAllocMaxVertices;
// layout: control block, words, worklist 0, worklist 1
constexpr size_t kScratchBytes = kCtlBytes + 3 * kVecBytes;  // 3 MiB + 1 KiB
static_assert(sizeof(Ctl) <= kCtlBytes, "control block does not fit");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

template <bool kSelect>
__device__ __forceinline__ bool scan_scalar(const int32_t* __restrict__ col,
                                            const uint32_t* __restrict__ word, int b, int e,
                                            int v, uint32_t wv, int n, unsigned glane,
                                            unsigned gshift) {
    constexpr unsigned gbits = (1u << kNoAllocTpr) - 1u;
    bool found = false;
    int p = b + (int)glane;
    for (;;) {
        bool hit = false;
        if (!found && p < e) {
            const int u = __ldg(col + p);
            if ((unsigned)u < (unsigned)n) {
                const uint32_t wu = ld_word(word + u);
                hit = kSelect ? (wu > wv || (wu == wv && u > v)) : (wu >= kWordInMin);
            }
        }
        const unsigned bal = __ballot_sync(0xFFFFFFFFu, hit);
        found = found || ((bal >> gshift) & gbits) != 0u;
        p += kNoAllocTpr;
        const bool more = !found && (p - (int)glane) < e;
        if (!__any_sync(0xFFFFFFFFu, more)) break;
    }
    return found;
}

__global__ void __launch_bounds__(kNoAllocBlock, 2)
    noalloc_solve_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                         int32_t n, uint64_t seed, uint8_t* __restrict__ out, long long spin_cap) {
    constexpr int G = 32 / kNoAllocTpr;
    Ctl* ctl = reinterpret_cast<Ctl*>(g_noalloc_scratch);
    uint32_t* word = reinterpret_cast<uint32_t*>(g_noalloc_scratch + kCtlBytes);
    int32_t* wl0 = reinterpret_cast<int32_t*>(g_noalloc_scratch + kCtlBytes + kVecBytes);
    int32_t* wl1 = reinterpret_cast<int32_t*>(g_noalloc_scratch + kCtlBytes + 2 * kVecBytes);
    const unsigned lane = lane_id();
    const unsigned glane = lane % kNoAllocTpr;
    const unsigned gid = lane / kNoAllocTpr;
    const unsigned gshift = gid * kNoAllocTpr;
    const unsigned nblocks = gridDim.x;
    const int wpb = blockDim.x / 32;
    const long long gwarp = (long long)blockIdx.x * wpb + threadIdx.x / 32;
    const long long nwarps = (long long)nblocks * wpb;
    grid_barrier_start();
    __shared__ int s_count;        // next worklist size, loaded once per block
    // a null col_idx reads as a graph without arcs (the host rejects it when
    // row_ptr[n] > 0), so no scan ever dereferences it
    const int arcs = col ? max(0, rp[n]) : 0;
    auto row = [&](int v, int& b, int& e) {
        b = min(max(rp[v], 0), arcs);
        e = min(max(rp[v + 1], b), arcs);
    };

    // init: Eq. 1 priorities
    {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        const float dbar = average_degree(arcs, n);
        const uint64_t smix = mix64(seed);
        for (long long v = tid; v < n; v += nthreads) {
            int b, e;
            row((int)v, b, e);
            const int deg = e - b;
            word[v] = deg ? eq1_key(dbar, deg, smix, (uint32_t)v) : kKeyIsolated;
        }
    }
    if (!grid_barrier(ctl, nblocks, spin_cap, NoLeader())) return;

    int count = n;
    for (int r = 0;; ++r) {
        const int32_t* wl_in = (r == 0) ? nullptr : ((r & 1) ? wl1 : wl0);
        int32_t* wl_out = ((r + 1) & 1) ? wl1 : wl0;
        int* next_cnt = &ctl->cnt[(r + 1) & 3];
        // Phase 1: selection test
        for (long long pass = gwarp; pass * G < count; pass += nwarps) {
            const long long item = pass * G + gid;
            const bool valid = item < count;
            const int v = valid ? (wl_in ? wl_in[item] : (int)item) : 0;
            const uint32_t wv = valid ? ld_word(word + v) : 0u;
            const bool und = valid && (wv >> 29) == 1u;
            int b = 0, e = 0;
            if (und) row(v, b, e);
            const bool blocked = scan_scalar<true>(col, word, b, e, v, wv, n, glane, gshift);
            if (und && !blocked && glane == 0) word[v] = wv | kWordInSet;
        }
        if (!grid_barrier(ctl, nblocks, spin_cap, NoLeader())) return;
        // Phase 2+3: exclusion test, state update, compaction
        for (long long pass = gwarp; pass * G < count; pass += nwarps) {
            const long long item = pass * G + gid;
            const bool valid = item < count;
            const int v = valid ? (wl_in ? wl_in[item] : (int)item) : 0;
            const uint32_t wv = valid ? ld_word(word + v) : 0u;
            const bool und = valid && (wv >> 29) == 1u;
            int b = 0, e = 0;
            if (und) row(v, b, e);
            const bool excl = scan_scalar<false>(col, word, b, e, v, wv, n, glane, gshift);
            const bool lead = glane == 0;
            if (und && excl && lead) word[v] = kWordOut;
            const bool keep = und && !excl && lead;
            const unsigned bal = __ballot_sync(0xFFFFFFFFu, keep);
            if (bal) {
                int base = 0;
                if (lane == 0) base = atomicAdd(next_cnt, __popc(bal));
                base = __shfl_sync(0xFFFFFFFFu, base, 0);
                if (keep) wl_out[base + __popc(bal & lanemask_lt())] = v;
            }
        }
        const int rr = r;
        const int cur = count;
        if (!grid_barrier(ctl, nblocks, spin_cap, [ctl, rr, cur]() {
                if (rr < kStatRounds) ctl->alive[rr] = cur;
                ctl->alive_sum += (unsigned long long)cur;
                ctl->rounds = rr + 1;
                ctl->cnt[(rr + 2) & 3] = 0;
            },
            [next_cnt]() { s_count = __ldcg(next_cnt); }))
            return;
        count = s_count;
        if (count == 0) break;
        if (r + 1 >= n + 2) {
            if (threadIdx.x == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            return;
        }
    }
    // output
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)nblocks * blockDim.x;
    for (long long v = tid; v < n; v += nthreads) out[v] = ld_word(word + v) >= kWordInMin;
}

}  // namespace

}  // namespace tcmis

using namespace tcmis;

extern "C" int mis_solve_noalloc(int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                 uint64_t seed, uint8_t* out_status, void* stream) {
    clear_error();
    if (n < 0 || n > kNoAllocMaxVertices)
        return set_error(MIS_EINVAL, "mis_solve_noalloc: n must be in [0, 262144] (the size of "
                                     "its fixed scratch array)");
    if (n > 0 && (!row_ptr || !out_status))
        return set_error(MIS_EINVAL, "mis_solve_noalloc: null row_ptr or out_status");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_cuda_error(e, "mis_solve_noalloc: cudaGetDevice");
    // The scratch array's address as the current device sees it, looked up on
    // every call: the first lookup on a device loads the module there, later
    // ones are table lookups.  Not cached, because a context that is torn
    // down and created again (cudaDeviceReset) may place the array elsewhere.
    void* base = nullptr;
    e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
    if (e != cudaSuccess || !base)
        return set_cuda_error(e == cudaSuccess ? cudaErrorInvalidSymbol : e,
                              "mis_solve_noalloc: cudaGetSymbolAddress");
    if (n == 0) return MIS_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (!col_idx) {
        // col_idx may be null only for a graph without arcs
        int32_t arcs = 0;
        e = cudaMemcpyAsync(&arcs, row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return set_cuda_error(e, "mis_solve_noalloc: read row_ptr[n]");
        if (arcs != 0)
            return set_error(MIS_EINVAL, "mis_solve_noalloc: null col_idx with row_ptr[n] > 0");
    }
    // the control block must start at zero; words and worklists are written
    // before they are read
    e = cudaMemsetAsync(base, 0, kCtlBytes, s);
    if (e != cudaSuccess) return set_cuda_error(e, "mis_solve_noalloc: control reset");
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, noalloc_solve_kernel,
                                                      kNoAllocBlock, 0);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || per_sm * sms <= 0)
        return set_cuda_error(e == cudaSuccess ? cudaErrorLaunchOutOfResources : e,
                              "mis_solve_noalloc: occupancy");
    const int rows_per_pass = (kNoAllocBlock / 32) * (32 / kNoAllocTpr);
    int grid = (int)((n + 2LL * rows_per_pass - 1) / (2LL * rows_per_pass));
    grid = grid < 1 ? 1 : (grid > per_sm * sms ? per_sm * sms : grid);
    long long spin_cap = 20000000;
    void* args[] = {(void*)&row_ptr, (void*)&col_idx, (void*)&n, (void*)&seed,
                    (void*)&out_status, (void*)&spin_cap};
    e = cudaLaunchCooperativeKernel((const void*)noalloc_solve_kernel, dim3(grid),
                                    dim3(kNoAllocBlock), args, 0, s);
    if (e != cudaSuccess) return set_cuda_error(e, "mis_solve_noalloc: launch");
    int err = 0;
    e = cudaMemcpyAsync(&err, (const char*)base + offsetof(Ctl, err), sizeof(int),
                        cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return set_cuda_error(e, "mis_solve_noalloc: solve");
    if (err == kErrTimedOut)
        return set_error(MIS_ETIMEDOUT, "mis_solve_noalloc: device barrier wait gave up");
    if (err != 0) return set_error(MIS_EINTERNAL, "mis_solve_noalloc: round cap exceeded");
    return MIS_OK;
}
