// tile_tc.cuh -- the exclusion product of one 16-row block on tensor cores.
//
// Phase 2 of Algorithm 2 is the product N_c = A x C of the 0/1 adjacency A
// with the 0/1 vector C of the round's candidates (Sec. 3.1); the paper runs
// it as 16 x 16 fp16 tiles with fp32 accumulation (Listing 1).  With several
// solves of one graph in one launch, C becomes [C_1 .. C_8] and the product
// fills the eight columns of an m16n8 MMA.  rowblock_nc computes, for one
// block of 16 rows and its non-empty tiles [t0, t1):
//
//   D[i][s] = sum over tiles t, columns j of A_t(i, j) * C_s(16 * tcol[t] + j)
//
// for 16 rows i and 8 right-hand sides s, in one of four payload forms:
//
//   kPayBitsF16  the tile's bitmask expanded to fp16 A fragments in registers,
//                m16n8k16, one tile per MMA;
//   kPayB1       the bitmask itself on the single-bit MMA (AND, then POPC,
//                accumulated in int32), m16n8k128, eight tiles per MMA;
//   kPayI8       stored 16 x 16 int8 0/1 tiles, m16n8k32 s8, two tiles per MMA;
//   kPayF16      stored 16 x 16 fp16 0/1 tiles (the paper's format), m16n8k16.
//
// Every form is exact: entries are 0/1 and a row of one launch's product is at
// most the row's degree (< 2^24, exact in fp32; int32 for the integer forms).
// Fragment coordinates of a lane: g = lane / 4 (A rows g and g + 8, B and D
// column g), q = lane % 4; the lane receives D[g][2q], D[g][2q + 1],
// D[g + 8][2q], D[g + 8][2q + 1].  Groups of tiles whose C segments are zero
// in every column add nothing and are skipped (the early exit of Sec. 3.2).
#pragma once

#include <cstdint>

#include "common.cuh"

namespace tcmis {

constexpr int kPayBitsF16 = 0;
constexpr int kPayB1 = 1;
constexpr int kPayI8 = 2;
constexpr int kPayF16 = 3;

// Row i's 16 bits of tile t (bit j = entry (i, j)); four 64-bit words per tile.
__device__ __forceinline__ uint32_t tile_row16(const uint64_t* __restrict__ tbits, int t, int i) {
    return (uint32_t)(__ldg(tbits + (long long)t * 4 + (i >> 2)) >> (16 * (i & 3))) & 0xFFFFu;
}

// fp16 pair {lo, hi} of two 0/1 values (1.0 = 0x3C00).
__device__ __forceinline__ uint32_t half2_of(uint32_t lo, uint32_t hi) {
    return (lo ? 0x3C00u : 0u) | (hi ? 0x3C000000u : 0u);
}

// Four int8 0/1 values from the low four bits (bit b -> byte b).
__device__ __forceinline__ uint32_t bytes_of4(uint32_t bits) {
    return (bits & 1u) | ((bits & 2u) << 7) | ((bits & 4u) << 14) | ((bits & 8u) << 21);
}

__device__ __forceinline__ void mma_f16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                        uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_s8(int (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                       uint32_t a3, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k32.row.col.s32.s8.s8.s32 "
        "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void mma_b1(int (&c)[4], uint32_t a0, uint32_t a1, uint32_t b0) {
    asm volatile(
        "mma.sync.aligned.m16n8k128.row.col.s32.b1.b1.s32.and.popc "
        "{%0, %1, %2, %3}, {%4, %5}, {%6}, {%0, %1, %2, %3};\n"
        : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
        : "r"(a0), "r"(a1), "r"(b0));
}

// D of one row block (see above).  seg(t): the 16 C bits of this lane's
// column g on tile t's column block (0 for columns beyond the solves).
// pay: the stored int8 (256 bytes per tile) or fp16 (512 bytes per tile)
// payload for kPayI8 / kPayF16, unused otherwise.  Warp-uniform: every lane
// of the warp calls it for the same row block.
template <int P, class Seg>
__device__ __forceinline__ void rowblock_nc(const uint64_t* __restrict__ tbits,
                                            const void* __restrict__ pay, int t0, int t1,
                                            Seg seg, int (&d)[4]) {
    const unsigned lane = lane_id();
    const int g = (int)(lane >> 2), q = (int)(lane & 3);
    if constexpr (P == kPayB1) {
        int acc[4] = {0, 0, 0, 0};
        for (int tb = t0; tb < t1; tb += 8) {
            // this lane's 32 k-slots are tiles tb + 2q and tb + 2q + 1
            const int ta = tb + 2 * q, tc = ta + 1;
            uint32_t b0 = 0;
            if (ta < t1) b0 = seg(ta);
            if (tc < t1) b0 |= seg(tc) << 16;
            if (!__any_sync(0xFFFFFFFFu, b0 != 0u)) continue;
            uint32_t a0 = 0, a1 = 0;
            if (ta < t1) {
                a0 = tile_row16(tbits, ta, g);
                a1 = tile_row16(tbits, ta, g + 8);
            }
            if (tc < t1) {
                a0 |= tile_row16(tbits, tc, g) << 16;
                a1 |= tile_row16(tbits, tc, g + 8) << 16;
            }
            mma_b1(acc, a0, a1, b0);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = acc[k];
    } else if constexpr (P == kPayI8) {
        const uint32_t* p8 = reinterpret_cast<const uint32_t*>(pay);  // 64 words per tile
        int acc[4] = {0, 0, 0, 0};
        for (int tb = t0; tb < t1; tb += 2) {
            const bool two = tb + 1 < t1;
            const uint32_t s0 = seg(tb), s1 = two ? seg(tb + 1) : 0u;
            if (!__any_sync(0xFFFFFFFFu, (s0 | s1) != 0u)) continue;
            const uint32_t* pa = p8 + (long long)tb * 64;
            const uint32_t a0 = __ldg(pa + g * 4 + q), a1 = __ldg(pa + (g + 8) * 4 + q);
            uint32_t a2 = 0, a3 = 0;
            if (two) {
                a2 = __ldg(pa + 64 + g * 4 + q);
                a3 = __ldg(pa + 64 + (g + 8) * 4 + q);
            }
            mma_s8(acc, a0, a1, a2, a3, bytes_of4((s0 >> (4 * q)) & 0xFu),
                   bytes_of4((s1 >> (4 * q)) & 0xFu));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = acc[k];
    } else {
        const uint32_t* p16 = reinterpret_cast<const uint32_t*>(pay);  // 128 words per tile
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int t = t0; t < t1; ++t) {
            const uint32_t s = seg(t);
            if (!__any_sync(0xFFFFFFFFu, s != 0u)) continue;
            uint32_t a0, a1, a2, a3;
            if constexpr (P == kPayF16) {
                const uint32_t* pt = p16 + (long long)t * 128;
                a0 = __ldg(pt + g * 8 + q);
                a1 = __ldg(pt + (g + 8) * 8 + q);
                a2 = __ldg(pt + g * 8 + q + 4);
                a3 = __ldg(pt + (g + 8) * 8 + q + 4);
            } else {
                const uint32_t r0 = tile_row16(tbits, t, g), r8 = tile_row16(tbits, t, g + 8);
                a0 = half2_of((r0 >> (2 * q)) & 1u, (r0 >> (2 * q + 1)) & 1u);
                a1 = half2_of((r8 >> (2 * q)) & 1u, (r8 >> (2 * q + 1)) & 1u);
                a2 = half2_of((r0 >> (2 * q + 8)) & 1u, (r0 >> (2 * q + 9)) & 1u);
                a3 = half2_of((r8 >> (2 * q + 8)) & 1u, (r8 >> (2 * q + 9)) & 1u);
            }
            mma_f16(acc, a0, a1, a2, a3, half2_of((s >> (2 * q)) & 1u, (s >> (2 * q + 1)) & 1u),
                    half2_of((s >> (2 * q + 8)) & 1u, (s >> (2 * q + 9)) & 1u));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = (int)acc[k];
    }
}

// Asynchronous 16-byte copy global -> shared (L2 only) and its groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// Waits until at most N of this thread's committed groups are pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Tiles with at most this many arcs are multiplied on CUDA cores (an arc
// (i, j) adds C_s(j) to row i for every solve s), the rest on the MMA: a
// sparse tile costs the MMA as much as a dense one.
constexpr int kSparseTileArcs = 2;

// One pass of up to 32 tiles of a row block.  The tiles' bits sit in the
// warp's shared buffer `bits` (tile slot l at words 8 l .. 8 l + 7: row i at
// word i / 2, bits 16 (i & 1) ..), and lane l holds `c`, the C segments of
// slot l's column block for all eight solves (16 bytes: solve s's 16 bits at
// word s / 2, bits 16 (s & 1) ..; zero for a slot without a tile).  Tiles
// whose segments are zero in every solve add nothing and are dropped (the
// early exit of Sec. 3.2).  With kSplit, where it lowers the pass's MMA
// count, tiles of at most kSparseTileArcs arcs are taken by their lane on CUDA
// cores: for each arc (i, j) the solves s with j in C_s are ORed into the
// warp's row masks `sd[i]` (bit s).  The others are listed
// in `idx` with their segments in `cs` (4 words each) and fed to m16n8k128
// eight at a time, accumulating into `acc` (the D fragment of rowblock_nc).
// Row (i, s) has a neighbour in C iff acc's entry > 0 or bit s of sd[i] is
// set.  Warp-uniform; every lane's part of `bits` must be visible
// (__syncwarp), and sd is cleared by the caller once per row block.
template <bool kSplit>
__device__ __forceinline__ void b1_pass(const uint32_t* bits, const uint4& c, uint32_t* cs,
                                        int32_t* idx, uint32_t* sd, int (&acc)[4]) {
    const unsigned lane = lane_id();
    const int g = (int)(lane >> 2), q = (int)(lane & 3);
    const bool nz = (c.x | c.y | c.z | c.w) != 0u;
    // the split only where it saves an MMA (a warp-uniform choice): never
    // with at most eight tiles
    const int n_nz = kSplit ? __popc(__ballot_sync(0xFFFFFFFFu, nz)) : 0;
    uint4 lo = make_uint4(0u, 0u, 0u, 0u), hi = lo;
    int arcs = 0;
    if (n_nz > 8 && nz) {
        lo = *reinterpret_cast<const uint4*>(bits + 8 * lane);
        hi = *reinterpret_cast<const uint4*>(bits + 8 * lane + 4);
        arcs = __popc(lo.x) + __popc(lo.y) + __popc(lo.z) + __popc(lo.w) + __popc(hi.x) +
               __popc(hi.y) + __popc(hi.z) + __popc(hi.w);
    }
    const int n_dense =
        n_nz > 8 ? __popc(__ballot_sync(0xFFFFFFFFu, nz && arcs > kSparseTileArcs)) : n_nz;
    const bool split = (n_dense + 7) / 8 < (n_nz + 7) / 8;
    const bool dense = nz && (!kSplit || !split || arcs > kSparseTileArcs);
    if (kSplit && nz && !dense) {
        const uint32_t w[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            uint32_t x = w[k];
            while (x) {
                const int bit = 32 * k + __ffs(x) - 1;
                x &= x - 1u;
                const int i = bit >> 4, j = bit & 15;
                // bit s of m: column j of solve s's segment
                const uint32_t t0 = (c.x >> j) & 0x10001u, t1 = (c.y >> j) & 0x10001u;
                const uint32_t t2 = (c.z >> j) & 0x10001u, t3 = (c.w >> j) & 0x10001u;
                const uint32_t m = ((t0 | (t0 >> 15)) & 3u) | (((t1 | (t1 >> 15)) & 3u) << 2) |
                                   (((t2 | (t2 >> 15)) & 3u) << 4) |
                                   (((t3 | (t3 >> 15)) & 3u) << 6);
                if (m) atomicOr(sd + i, m);
            }
        }
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, dense);
    const int m = __popc(bal);
    if (m == 0) return;
    if (dense) {
        const int p = __popc(bal & lanemask_lt());
        idx[p] = (int32_t)lane;
        *reinterpret_cast<uint4*>(cs + 4 * p) = c;
    }
    __syncwarp();
    const int sh = 16 * (g & 1);
    for (int k = 0; k < m; k += 8) {
        // this lane's 32 k-slots: listed tiles k + 2q (bits 0..15) and
        // k + 2q + 1 (bits 16..31)
        const int ta = k + 2 * q, tc = ta + 1;
        uint32_t a0 = 0, a1 = 0, b0 = 0;
        if (ta < m) {
            const uint32_t* s = bits + 8 * idx[ta];
            a0 = (s[g >> 1] >> sh) & 0xFFFFu;
            a1 = (s[(g + 8) >> 1] >> sh) & 0xFFFFu;
            b0 = (cs[4 * ta + (g >> 1)] >> sh) & 0xFFFFu;
        }
        if (tc < m) {
            const uint32_t* s = bits + 8 * idx[tc];
            a0 |= ((s[g >> 1] >> sh) & 0xFFFFu) << 16;
            a1 |= ((s[(g + 8) >> 1] >> sh) & 0xFFFFu) << 16;
            b0 |= ((cs[4 * tc + (g >> 1)] >> sh) & 0xFFFFu) << 16;
        }
        mma_b1(acc, a0, a1, b0);
    }
    __syncwarp();
}

}  // namespace tcmis
