// common.cuh -- device-side building blocks shared by the round kernels.
//
// Per-vertex state is one packed 32-bit word, read by every neighbour test:
//
//   bits 31..29  state    001 = undecided (alive), 111 = in the MIS, 000 = out
//   bits 28..0   the low 29 bits of the priority key
//
// The priority key is the bit pattern of the binary32 priority P of Eq. 1.
// For any valid graph P lies in [1/(n+1), 1], so its exponent field is in
// [95, 127]: bits 31 and 30 of the key are 0 and bit 29 is 1.  An undecided
// word is therefore exactly the key, an out word is any value below 2^29 (we
// store 0) and an in word is the key with bits 31..30 set.  One unsigned
// compare then decides both neighbour tests of a round:
//
//   selection test (Phase 1, Algorithm 2): u blocks v when
//       word(u) > word(v)  or  (word(u) == word(v) and u > v)
//     out words never block; undecided words compare by key then id; an in
//     word (a candidate chosen earlier in the same phase) always blocks, which
//     is exactly what the round-start snapshot says, because a candidate
//     outranks every undecided neighbour.
//   exclusion test (Phase 2): v has a candidate neighbour when word(u) >= 0xE0000000.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace tcmis {

constexpr uint32_t kWordInMin = 0xE0000000u;  // words >= this are in the MIS
constexpr uint32_t kWordInSet = 0xC0000000u;  // OR'd into an undecided word
constexpr uint32_t kWordOut = 0u;             // out of the MIS
constexpr uint32_t kKeyIsolated = 0x3F800000u; // key used for deg-0 vertices (P = 1)

// error codes written by kernels into Ctl::err (match the MIS_E* values)
constexpr int kErrTimedOut = -4;
constexpr int kErrInternal = -6;

constexpr int kStatRounds = 64;
constexpr int kBins = 5;  // degree bins of the CSR round kernel

// Control block of one solve in device memory; zeroed before every launch.
struct Ctl {
    unsigned long long bar_arrivals;  // grid barrier: block arrivals in this launch
    int err;              // first error (0 = none)
    int rounds;           // rounds completed
    int cnt[4];           // worklist sizes, ring indexed by round & 3
    unsigned long long alive_sum;
    unsigned long long mis_size;
    int alive[kStatRounds];
    unsigned grab[4][kBins];  // per-bin work counters, ring indexed by round & 3
    int bcnt[4][kBins];       // per-bin worklist sizes, ring indexed by round & 3
    int pcnt[4][kBins];       // per-bin pending-list sizes, ring indexed by round & 3
    int alive_acc[4];         // |A| at round start, ring indexed by round & 3
    unsigned long long alive_acc64[4];  // the same, summed over the solves of a
                                        // multi-seed launch, ring indexed
};

// Phase timestamps of one solve (device %globaltimer, ns), written by the
// last block to reach each grid barrier: t[0] kernel start, t[1] end of the
// priority init, t[2 + r] end of Phase 1 of round r, t[2 + kStatRounds + r]
// end of Phases 2+3 of round r (rounds beyond kStatRounds are not recorded).
struct PhaseTimes {
    unsigned long long t[2 * kStatRounds + 2];
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- Eq. 1

// splitmix64 finaliser (Steele, Lea, Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 30;
    z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z;
}

// Average degree d of Eq. 1: arcs / n in binary32, round-to-nearest.
__device__ __forceinline__ float average_degree(int32_t arcs, int32_t n) {
    return __fdiv_rn(__int2float_rn(arcs), __int2float_rn(n));
}

// Eq. 1 key of a vertex with deg >= 1: bits of d / ((d + deg) - eps), each
// operation binary32 round-to-nearest (explicit intrinsics: no contraction).
// seed_mix = mix64(seed); eps = (hi32(mix64(seed_mix ^ id)) >> 8) * 2^-24.
__device__ __forceinline__ uint32_t eq1_key(float dbar, int32_t deg, uint64_t seed_mix,
                                            uint32_t local_id) {
    const uint32_t h = (uint32_t)(mix64(seed_mix ^ (uint64_t)local_id) >> 32);
    const float eps = __fmul_rn(__uint2float_rn(h >> 8), 0x1p-24f);
    const float den = __fsub_rn(__fadd_rn(dbar, __int2float_rn(deg)), eps);
    return __float_as_uint(__fdiv_rn(dbar, den));
}

// Priority heuristics of Sec. 3.3 (values of mis_options.priority): H2/H3 =
// Eq. 1 above; H1 = random priority hash(v); Eq. 1 discretised to 8 bits.
constexpr int kPrioEq1 = 0, kPrioHash = 1, kPrioEq1Q8 = 2;

// Key of a vertex of degree >= 1 under heuristic `mode`: Eq. 1's bits;
// H1: 2^29 + (hi32(mix64(seed_mix ^ id)) >> 3), the hash's high 29 bits;
// 8-bit: trunc(255 * P) with P Eq. 1's binary32 value (product round-to-
// nearest, then truncation).
__device__ __forceinline__ uint32_t priority_key(int mode, float dbar, int32_t deg,
                                                 uint64_t seed_mix, uint32_t local_id) {
    if (mode == kPrioHash)
        return 0x20000000u + ((uint32_t)(mix64(seed_mix ^ (uint64_t)local_id) >> 32) >> 3);
    const uint32_t k = eq1_key(dbar, deg, seed_mix, local_id);
    if (mode == kPrioEq1Q8) return __float2uint_rz(__fmul_rn(__uint_as_float(k), 255.0f));
    return k;
}

// The undecided word of a key (bits 31..29 = 001, order kept): Eq. 1 and H1
// keys already have that form; an 8-bit key is placed in the low bits.
__device__ __forceinline__ uint32_t undecided_word(int mode, uint32_t key) {
    return mode == kPrioEq1Q8 ? (0x20000000u | key) : key;
}

// ---------------------------------------------------------------- memory helpers

__device__ __forceinline__ uint32_t ld_word(const uint32_t* p) { return __ldcg(p); }

// Word load through L1.  Safe for the round kernels: the L1 is invalidated by
// the acquire in every grid barrier, and inside one round a stale copy can only
// hide a change that does not alter any test of that round (see the state
// notes of the CSR kernel).
__device__ __forceinline__ uint32_t ld_word_l1(const uint32_t* p) { return *p; }

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_acquire_int(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}


// ---------------------------------------------------------------- grid barrier
//
// Software barrier over all blocks of a cooperative launch (co-residency is
// guaranteed by the launch).  Ctl::bar_arrivals counts block arrivals over the
// whole launch and is never reset: the k-th barrier of a launch is complete
// once it reaches k * nblocks, so a block arrives with one atomic and waits by
// polling that same counter (no generation flag, no reset, no release step).
// The count of barriers a block has passed sits in shared memory (thread 0
// alone uses it); a kernel calls grid_barrier_start() once before its first
// barrier.
//
// The last block to arrive runs `leader` (one thread) but nobody waits for
// it, so a leader may only write what other blocks read after the NEXT
// barrier or after the launch (the round kernels' ring-indexed counters are
// laid out for that).  After the wait, thread 0 of every block runs `after`
// (e.g. to copy counters written before the barrier into shared memory, one
// load per block instead of one per warp).
//
// Every wait is bounded: after `spin_cap` polls the block records
// kErrTimedOut and leaves; a block that sees an error while waiting leaves
// too, so a failed barrier never hangs the device.  Returns false when the
// launch must stop.
__shared__ unsigned s_bar_epoch;

__device__ __forceinline__ void grid_barrier_start() {
    if (threadIdx.x == 0) s_bar_epoch = 0;
}

template <class Leader, class After>
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, unsigned nblocks, long long spin_cap,
                                             Leader leader, After after) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned epoch = ++s_bar_epoch;
        const unsigned long long target = (unsigned long long)epoch * nblocks;
        int ok = 1;
        __threadfence();  // the block's writes before its arrival
        const unsigned long long arrived = atomicAdd(&ctl->bar_arrivals, 1ull) + 1ull;
        if (arrived >= target) {
            __threadfence();  // acquire: the other blocks' writes before theirs
            leader();
        } else {
            long long polls = 0;
            while (ld_acquire_u64(&ctl->bar_arrivals) < target) {
                if (++polls > spin_cap) {
                    atomicCAS(&ctl->err, 0, kErrTimedOut);
                    ok = 0;
                    break;
                }
                if ((polls & 63) == 0 && ld_acquire_int(&ctl->err) != 0) {
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
        }
        if (ok) after();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

struct NoLeader {
    __device__ void operator()() const {}
};

template <class Leader>
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, unsigned nblocks, long long spin_cap,
                                             Leader leader) {
    return grid_barrier(ctl, nblocks, spin_cap, leader, NoLeader());
}

// ---------------------------------------------------------------- warp helpers

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

}  // namespace tcmis
