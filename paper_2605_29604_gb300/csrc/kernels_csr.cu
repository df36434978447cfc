// kernels_csr.cu -- the CSR round kernel on CUDA cores (the plain GPU form).
//
// One cooperative, persistent launch runs a whole solve:
//
//   init      Eq. 1 priority of every vertex into its packed word (Sec. 2:
//             priorities assigned once and reused every round)
//   rounds    Algorithm 2's while-loop.  Each round has two phases separated
//             by a grid barrier, both over the worklist of undecided vertices:
//               Phase 1  selection test: v is a candidate when no undecided
//                        neighbour outranks it (C(v) = [P(v) > Max_Np(v)]);
//                        candidates are marked in the MIS in place.
//               Phase 2+3 exclusion test and state update: an undecided
//                        non-candidate with a candidate neighbour
//                        (N_c(v) > 0) is marked out; the rest are appended to
//                        the next round's worklist (compaction).
//             Both phases read only what the round-start snapshot fixes (see
//             common.cuh), so the rounds match Algorithm 2 exactly.
//   output    result bytes out[v] = [v in the MIS].
//
// Rows are scanned by groups of TPR lanes (4, 8, 16 or 32), each lane
// loading 16-byte aligned int4 slices of col_idx and gathering the four
// neighbour words; a group stops at the first neighbour that decides its
// test (a blocker in Phase 1, a candidate in Phase 2).
#include <cstdio>

#include "common.cuh"
#include "internal.h"

namespace tcmis {

constexpr int kCsrBlock = 512;

// Any neighbour of the row [b, e) satisfying the phase's test, for the group
// of TPR lanes this lane belongs to.  Warp-uniform control flow: every lane of
// the warp runs the loop until no group in the warp has work left.
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
            const uint32_t w0 = (p0 >= b) ? ld_word(word + c.x) : 0u;
            const uint32_t w1 = (p0 + 1 >= b && p0 + 1 < e) ? ld_word(word + c.y) : 0u;
            const uint32_t w2 = (p0 + 2 >= b && p0 + 2 < e) ? ld_word(word + c.z) : 0u;
            const uint32_t w3 = (p0 + 3 >= b && p0 + 3 < e) ? ld_word(word + c.w) : 0u;
            if (kSelect) {
                hit = (w0 > wv) | (w1 > wv) | (w2 > wv) | (w3 > wv) |
                      ((w0 == wv) & (c.x > v)) | ((w1 == wv) & (c.y > v)) |
                      ((w2 == wv) & (c.z > v)) | ((w3 == wv) & (c.w > v));
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

template <int TPR>
__global__ void __launch_bounds__(kCsrBlock, 2) csr_solve_kernel(const SolveArgs a) {
    constexpr int G = 32 / TPR;  // rows per warp pass
    const unsigned lane = lane_id();
    const unsigned glane = lane % TPR;
    const unsigned gid = lane / TPR;
    const unsigned gshift = gid * TPR;
    const unsigned nblocks = gridDim.x;
    const int wpb = blockDim.x / 32;
    const long long gwarp = (long long)blockIdx.x * wpb + threadIdx.x / 32;
    const long long nwarps = (long long)nblocks * wpb;
    Ctl* ctl = a.ctl;
    const int32_t n = a.n;

    // ---- init: Eq. 1 priorities
    {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        float dbar0 = 0.f;
        uint64_t smix0 = 0;
        if (a.seg.count == 0 && n > 0) {
            dbar0 = average_degree(a.rp[n], n);
            smix0 = mix64(a.seed0);
        }
        for (long long v = tid; v < n; v += nthreads) {
            const int deg = a.rp[v + 1] - a.rp[v];
            uint32_t w;
            if (a.seg.count == 0) {
                w = deg ? eq1_key(dbar0, deg, smix0, (uint32_t)v) : kKeyIsolated;
            } else {
                const int g = a.seg.blk_seg[v >> 4];
                const int local = (int)v - a.seg.voff[g];
                if (local >= a.seg.nv[g]) {
                    w = kWordOut;  // padding vertex between two graphs
                } else if (deg == 0) {
                    w = kKeyIsolated;
                } else {
                    const float dbar = average_degree(a.seg.arcs[g], a.seg.nv[g]);
                    w = eq1_key(dbar, deg, mix64(a.seg.seed[g]), (uint32_t)local);
                }
            }
            a.word[v] = w;
        }
    }
    if (!grid_barrier(ctl, nblocks, a.spin_cap, NoLeader())) return;

    int count = n;  // round 0 works on the identity list
    for (int r = 0;; ++r) {
        const int32_t* wl_in = (r == 0) ? nullptr : ((r & 1) ? a.wl1 : a.wl0);
        int32_t* wl_out = ((r + 1) & 1) ? a.wl1 : a.wl0;
        int* next_cnt = &ctl->cnt[(r + 1) & 3];

        // ---- Phase 1: selection test
        for (long long pass = gwarp; pass * G < count; pass += nwarps) {
            const long long item = pass * G + gid;
            const bool valid = item < count;
            const int v = valid ? (wl_in ? wl_in[item] : (int)item) : 0;
            const uint32_t wv = valid ? ld_word(a.word + v) : 0u;
            const bool und = valid && (wv >> 29) == 1u;
            const int b = und ? a.rp[v] : 0;
            const int e = und ? a.rp[v + 1] : 0;
            const bool blocked = group_scan<TPR, true>(a.col, a.word, b, e, v, wv, glane, gshift);
            if (und && !blocked && glane == 0) a.word[v] = wv | kWordInSet;
        }
        if (!grid_barrier(ctl, nblocks, a.spin_cap, NoLeader())) return;

        // ---- Phase 2+3: exclusion test, state update, compaction
        for (long long pass = gwarp; pass * G < count; pass += nwarps) {
            const long long item = pass * G + gid;
            const bool valid = item < count;
            const int v = valid ? (wl_in ? wl_in[item] : (int)item) : 0;
            const uint32_t wv = valid ? ld_word(a.word + v) : 0u;
            const bool und = valid && (wv >> 29) == 1u;
            const int b = und ? a.rp[v] : 0;
            const int e = und ? a.rp[v + 1] : 0;
            const bool excl = group_scan<TPR, false>(a.col, a.word, b, e, v, wv, glane, gshift);
            const bool lead = glane == 0;
            if (und && excl && lead) a.word[v] = kWordOut;
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
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [ctl, rr, cur]() {
                if (rr < kStatRounds) ctl->alive[rr] = cur;
                ctl->alive_sum += (unsigned long long)cur;
                ctl->rounds = rr + 1;
                ctl->cnt[(rr + 2) & 3] = 0;
            }))
            return;
        count = ld_acquire_int(next_cnt);
        if (count == 0) break;
        if (r + 1 >= a.max_rounds) {
            if (threadIdx.x == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            return;
        }
    }

    // ---- output
    if (a.out) {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        unsigned in_cnt = 0;
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
        for (int o = 16; o; o >>= 1) in_cnt += __shfl_xor_sync(0xFFFFFFFFu, in_cnt, o);
        if (lane == 0 && in_cnt) atomicAdd(&ctl->mis_size, (unsigned long long)in_cnt);
    }
}

template <int TPR>
static cudaError_t launch_t(const SolveArgs& a, int grid, cudaStream_t s) {
    void* args[] = {const_cast<SolveArgs*>(&a)};
    return cudaLaunchCooperativeKernel((const void*)csr_solve_kernel<TPR>, dim3(grid),
                                       dim3(kCsrBlock), args, 0, s);
}

cudaError_t launch_csr_solve(const SolveArgs& a, int tpr, int grid, cudaStream_t s) {
    switch (tpr) {
        case 4: return launch_t<4>(a, grid, s);
        case 8: return launch_t<8>(a, grid, s);
        case 16: return launch_t<16>(a, grid, s);
        case 32: return launch_t<32>(a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

int csr_block_size() { return kCsrBlock; }

int csr_max_coresident_blocks(int tpr, int device) {
    int per_sm = 0, sms = 0;
    const void* fn = nullptr;
    switch (tpr) {
        case 4: fn = (const void*)csr_solve_kernel<4>; break;
        case 8: fn = (const void*)csr_solve_kernel<8>; break;
        case 16: fn = (const void*)csr_solve_kernel<16>; break;
        case 32: fn = (const void*)csr_solve_kernel<32>; break;
        default: return 0;
    }
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kCsrBlock, 0) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

}  // namespace tcmis
