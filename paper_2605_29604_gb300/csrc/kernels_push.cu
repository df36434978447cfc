// kernels_push.cu -- the work-efficient push/decrement form of the rounds.
//
// The same rounds as Algorithm 2, reached without re-scanning rows: each
// vertex keeps cnt[v], the number of its undecided neighbours that outrank
// it (computed once; only the selection prefix of a row can hold them).  A
// vertex is a candidate of round r exactly when cnt[v] = 0 at the start of
// the round (Phase 1, C(v) = [P(v) > Max_Np(v)]).  Then:
//
//   Phase 1   the ready list R_r (vertices whose count reached 0) goes in;
//   Phase 2   each candidate pushes its undecided neighbours out (N_c > 0),
//             each exclusion taken once (compare-and-swap on the word);
//   Phase 3   each newly excluded vertex x decrements cnt[w] of every
//             undecided neighbour w that x outranks; a count that reaches 0
//             puts w on R_{r+1}.
//
// Invariant: at the start of a round, cnt[v] of an undecided v counts its
// undecided higher neighbours (a higher neighbour cannot have gone in, else v
// was excluded with it), so R_r is exactly the candidate set of Algorithm 2
// and the rounds, alive sets and result are the same.  Every arc is read a
// bounded number of times: once to count, once from a candidate, once from
// an excluded vertex.
//
// An excluded vertex keeps the low 29 bits of its key in its word (state 000,
// still below every undecided word and never "in"), so Phase 3 can restore
// its key.  Short rows are scanned by one lane, rows longer than a warp by
// the whole warp.
#include <algorithm>

#include "common.cuh"
#include "init.cuh"
#include "internal.h"

namespace tcmis {

namespace {

constexpr int kPushBlock = 512;
constexpr int kPushMinBlocksPerSm = 3;
constexpr int kShortRow = 32;  // rows up to this length are scanned by one lane

__device__ __forceinline__ bool outranks_p(uint32_t wu, int u, uint32_t wv, int v) {
    return wu > wv || (wu == wv && u > v);
}

__device__ __forceinline__ bool undecided(uint32_t w) { return (w >> 29) == 1u; }

// Warp-aggregated append of v (where `take`) to list[*next ...].
__device__ __forceinline__ void append(bool take, int v, int* next, int32_t* list) {
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, take);
    if (!bal) return;
    int base = 0;
    if (lane_id() == 0) base = atomicAdd(next, __popc(bal));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    if (take) list[base + __popc(bal & lanemask_lt())] = v;
}

struct PushLists {
    int32_t* ready;      // R_r
    int32_t* ready_nx;   // R_{r+1}
    int32_t* excluded;   // X_r
    int32_t* cnt;        // undecided higher neighbours
};

// The count of vertex v (deg >= 1): neighbours at positions [b, e) of
// col_sel (its selection prefix, where all those able to outrank v sit) that
// outrank it.  One lane (kWarp false) or the whole warp.
template <bool kWarp>
__device__ __forceinline__ int count_higher(const SolveArgs& a, int v, uint32_t wv, int b, int e) {
    int c = 0;
    const int lane = kWarp ? (int)lane_id() : 0;
    const int step = kWarp ? 32 : 1;
    for (int p = b + lane; p < e; p += step) {
        const int u = __ldg(a.col_sel + p);
        c += outranks_p(ld_word(a.word + u), u, wv, v) ? 1 : 0;
    }
    if (kWarp)
        for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    return c;
}

__global__ void __launch_bounds__(kPushBlock, kPushMinBlocksPerSm)
    push_solve_kernel(const SolveArgs a, const PushLists pl) {
    __shared__ int s_cnt[2];
    __shared__ unsigned long long s_alive0;
    const unsigned nblocks = gridDim.x;
    Ctl* ctl = a.ctl;
    PhaseTimes* times = a.times;
    const unsigned lane = lane_id();
    const long long gwarp = (long long)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
    const long long nwarps = (long long)nblocks * (blockDim.x / 32);
    grid_barrier_start();
    if (times && blockIdx.x == 0 && threadIdx.x == 0) times->t[0] = global_ns();

    // ---- init: keys (isolated vertices in), then the counts and R_0
    init_words(a, (a.n + 15) / 16 * 16, true);
    if (!grid_barrier(ctl, nblocks, a.spin_cap, NoLeader())) return;
    int* r_next0 = &ctl->bcnt[0][0];
    unsigned long long alive_local = 0;
    for (long long base = gwarp * 32; base < a.n; base += nwarps * 32) {
        const long long v = base + lane;
        bool live = false;
        uint32_t wv = 0;
        int b = 0, e = 0;
        if (v < a.n) {
            wv = ld_word(a.word + v);
            live = undecided(wv);  // real, deg >= 1 (isolated ones are in, padding out)
            b = a.rp[v];
            e = a.split ? b + a.split[v] : a.rp[v + 1];
        }
        alive_local += live ? 1 : 0;
        bool zero = false;
        if (live && e - b <= kShortRow) {
            const int c = count_higher<false>(a, (int)v, wv, b, e);
            pl.cnt[v] = c;
            zero = c == 0;
        }
        unsigned longs = __ballot_sync(0xFFFFFFFFu, live && e - b > kShortRow);
        while (longs) {
            const int src = __ffs(longs) - 1;
            longs &= longs - 1;
            const int lv = __shfl_sync(0xFFFFFFFFu, (int)v, src);
            const uint32_t lw = __shfl_sync(0xFFFFFFFFu, wv, src);
            const int lb = __shfl_sync(0xFFFFFFFFu, b, src);
            const int le = __shfl_sync(0xFFFFFFFFu, e, src);
            const int c = count_higher<true>(a, lv, lw, lb, le);
            if ((int)lane == src) {
                pl.cnt[v] = c;
                zero = c == 0;
            }
        }
        append(zero, (int)v, r_next0, pl.ready);
    }
    // vertices decided at init (isolated ones) are candidates of round 0: in
    // its alive set, and among the vertices it decides
    unsigned iso_local = 0;
    {
        const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
        const long long nthreads = (long long)nblocks * blockDim.x;
        for (long long v = tid; v < a.n; v += nthreads)
            if (ld_word(a.word + v) >= kWordInMin) ++iso_local;  // (in at init)
    }
    alive_local += iso_local;
    for (int o = 16; o; o >>= 1) {
        alive_local += __shfl_xor_sync(0xFFFFFFFFu, alive_local, o);
        iso_local += __shfl_xor_sync(0xFFFFFFFFu, iso_local, o);
    }
    if (lane == 0 && alive_local) atomicAdd(&ctl->alive_acc64[0], alive_local);
    if (lane == 0 && iso_local) atomicAdd(&ctl->alive_acc[0], (int)iso_local);
    if (!grid_barrier(
            ctl, nblocks, a.spin_cap,
            [times]() {
                if (times) times->t[1] = global_ns();
            },
            [r_next0, ctl]() {
                s_cnt[0] = __ldcg(r_next0);
                s_alive0 = __ldcg(&ctl->alive_acc64[0]);
            }))
        return;

    int nready = s_cnt[0];
    // round 0 runs whenever a vertex is alive (isolated ones alone included:
    // they were decided at init and make up round 0's alive set)
    const bool any_alive = s_alive0 > 0;
    int32_t* ready = pl.ready;
    int32_t* ready_nx = pl.ready_nx;
    for (int r = 0; nready > 0 || (r == 0 && any_alive); ++r) {
        if (r >= a.max_rounds) {
            if (threadIdx.x == 0) atomicCAS(&ctl->err, 0, kErrInternal);
            return;
        }
        const int rr = r;
        int* x_next = &ctl->pcnt[r & 3][0];
        int* r_next = &ctl->bcnt[(r + 1) & 3][0];

        // ---- Phase 1: the ready vertices are the candidates: in
        {
            const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
            const long long nthreads = (long long)nblocks * blockDim.x;
            for (long long i = tid; i < nready; i += nthreads) {
                const int v = ready[i];
                a.word[v] = ld_word(a.word + v) | kWordInSet;
            }
        }
        if (!grid_barrier(ctl, nblocks, a.spin_cap, [times, rr]() {
                if (times && rr < kStatRounds) times->t[2 + rr] = global_ns();
            }))
            return;

        // ---- Phase 2: every candidate pushes its undecided neighbours out
        for (long long base = gwarp * 32; base < nready; base += nwarps * 32) {
            const long long i = base + lane;
            const int c = i < nready ? ready[i] : 0;
            const int b = i < nready ? a.rp[c] : 0;
            const int e = i < nready ? a.rp[c + 1] : 0;
            const bool shortrow = e - b <= kShortRow;
            // one lane per short row ...
            for (int k = 0; k < kShortRow; ++k) {
                const int p = b + k;
                bool take = false;
                int u = 0;
                if (shortrow && p < e) {
                    u = __ldg(a.col_sel + p);
                    const uint32_t wu = ld_word(a.word + u);
                    take = undecided(wu) && atomicCAS(a.word + u, wu, wu & 0x1FFFFFFFu) == wu;
                }
                append(take, u, x_next, pl.excluded);
                if (!__any_sync(0xFFFFFFFFu, shortrow && p + 1 < e)) break;
            }
            // ... the whole warp per long row
            unsigned longs = __ballot_sync(0xFFFFFFFFu, i < nready && !shortrow);
            while (longs) {
                const int src = __ffs(longs) - 1;
                longs &= longs - 1;
                const int lb = __shfl_sync(0xFFFFFFFFu, b, src);
                const int le = __shfl_sync(0xFFFFFFFFu, e, src);
                for (int p0 = lb; p0 < le; p0 += 32) {
                    const int p = p0 + (int)lane;
                    bool take = false;
                    int u = 0;
                    if (p < le) {
                        u = __ldg(a.col_sel + p);
                        const uint32_t wu = ld_word(a.word + u);
                        take = undecided(wu) && atomicCAS(a.word + u, wu, wu & 0x1FFFFFFFu) == wu;
                    }
                    append(take, u, x_next, pl.excluded);
                }
            }
        }
        if (!grid_barrier(
                ctl, nblocks, a.spin_cap, NoLeader(),
                [x_next]() {
                    s_cnt[1] = __ldcg(x_next);
                }))
            return;
        const int nx = s_cnt[1];

        // ---- Phase 3: every excluded vertex releases the neighbours it outranked
        for (long long base = gwarp * 32; base < nx; base += nwarps * 32) {
            const long long i = base + lane;
            const int x = i < nx ? pl.excluded[i] : 0;
            const uint32_t kx = i < nx ? (ld_word(a.word + x) | 0x20000000u) : 0u;  // its key
            const int b = i < nx ? a.rp[x] : 0;
            const int e = i < nx ? a.rp[x + 1] : 0;
            const bool shortrow = e - b <= kShortRow;
            for (int k = 0; k < kShortRow; ++k) {
                const int p = b + k;
                bool ready_w = false;
                int w = 0;
                if (shortrow && p < e) {
                    w = __ldg(a.col_sel + p);
                    const uint32_t ww = ld_word(a.word + w);
                    if (undecided(ww) && outranks_p(kx, x, ww, w))
                        ready_w = atomicSub(pl.cnt + w, 1) == 1;
                }
                append(ready_w, w, r_next, ready_nx);
                if (!__any_sync(0xFFFFFFFFu, shortrow && p + 1 < e)) break;
            }
            unsigned longs = __ballot_sync(0xFFFFFFFFu, i < nx && !shortrow);
            while (longs) {
                const int src = __ffs(longs) - 1;
                longs &= longs - 1;
                const int lx = __shfl_sync(0xFFFFFFFFu, x, src);
                const uint32_t lk = __shfl_sync(0xFFFFFFFFu, kx, src);
                const int lb = __shfl_sync(0xFFFFFFFFu, b, src);
                const int le = __shfl_sync(0xFFFFFFFFu, e, src);
                for (int p0 = lb; p0 < le; p0 += 32) {
                    const int p = p0 + (int)lane;
                    bool ready_w = false;
                    int w = 0;
                    if (p < le) {
                        w = __ldg(a.col_sel + p);
                        const uint32_t ww = ld_word(a.word + w);
                        if (undecided(ww) && outranks_p(lk, lx, ww, w))
                            ready_w = atomicSub(pl.cnt + w, 1) == 1;
                    }
                    append(ready_w, w, r_next, ready_nx);
                }
            }
        }
        const int cur_ready = nready;
        if (!grid_barrier(
                ctl, nblocks, a.spin_cap,
                [ctl, times, rr, cur_ready, nx]() {
                    // alive at the start of round rr, then minus C_rr and X_rr
                    const unsigned long long alive = ctl->alive_acc64[rr & 3];
                    if (times && rr < kStatRounds) times->t[2 + kStatRounds + rr] = global_ns();
                    if (rr < kStatRounds) ctl->alive[rr] = (int)alive;
                    ctl->alive_sum += alive;
                    ctl->rounds = rr + 1;
                    const unsigned long long iso =
                        rr == 0 ? (unsigned long long)ctl->alive_acc[0] : 0ull;
                    ctl->alive_acc64[(rr + 1) & 3] =
                        alive - (unsigned long long)cur_ready - (unsigned long long)nx - iso;
                    ctl->pcnt[(rr + 2) & 3][0] = 0;
                    ctl->bcnt[(rr + 2) & 3][0] = 0;
                },
                [r_next]() {
                    s_cnt[0] = __ldcg(r_next);
                }))
            return;
        nready = s_cnt[0];
        int32_t* t = ready;
        ready = ready_nx;
        ready_nx = t;
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
                const int g = a.seg.blk_seg[v >> 4];
                const int local = (int)v - a.seg.voff[g];
                if (local < a.seg.nv[g]) a.out[a.seg.roff[g] + local] = in;
            }
        }
        for (int o = 16; o; o >>= 1) in_cnt += __shfl_xor_sync(0xFFFFFFFFu, in_cnt, o);
        if (lane == 0 && in_cnt) atomicAdd(&ctl->mis_size, (unsigned long long)in_cnt);
    }
}

}  // namespace

cudaError_t launch_push_solve(const SolveArgs& a, int grid, cudaStream_t s) {
    // the lists live in the worklist buffers (int4[n] each, so 4n int32 each)
    PushLists pl;
    pl.ready = reinterpret_cast<int32_t*>(a.wl0);
    pl.ready_nx = reinterpret_cast<int32_t*>(a.wl1);
    pl.excluded = reinterpret_cast<int32_t*>(a.wlp);
    pl.cnt = reinterpret_cast<int32_t*>(a.wlp) + 2 * (((int64_t)a.n + 15) / 16 * 16);
    SolveArgs b = a;
    b.r0class = nullptr;  // every vertex is counted: no create-time shortcuts
    void* args[] = {&b, &pl};
    return cudaLaunchCooperativeKernel((const void*)push_solve_kernel, dim3(grid),
                                       dim3(kPushBlock), args, 0, s);
}

int push_max_coresident_blocks(int device) {
    int per_sm = 0, sms = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void*)push_solve_kernel,
                                                      kPushBlock, 0) != cudaSuccess)
        return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess)
        return 0;
    return per_sm * sms;
}

}  // namespace tcmis
