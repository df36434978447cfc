// init.cuh -- the priority initialisation shared by the round kernels.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace tcmis {

// Priority (Eq. 1, or the heuristic a.priority selects, Sec. 3.3) of every
// vertex v < n_words into its packed word (Sec. 2: assigned once per solve).  Vertices at or beyond a.n (tile padding) and
// batch padding vertices are out.  Isolated vertices have no neighbour to
// compare with, so every round-0 selection test accepts them: with
// isolated_in they are written in the MIS right away (the CSR kernel keeps
// them out of its worklists), and so are the sure round-0 candidates of
// a.r0class (class 1); else isolated vertices get a fixed key and are decided
// in round 0 like every other vertex.  With `out` (a single graph), the
// result byte of every vertex < n is written too: 1 for those put in the MIS
// here, 0 for the rest until a round selects them.  Grid-stride over the
// whole launch.
__device__ __forceinline__ void init_words(const SolveArgs& a, int32_t n_words,
                                           bool isolated_in, uint8_t* out = nullptr) {
    const uint8_t* r0class = isolated_in ? a.r0class : nullptr;
    const int mode = a.priority;
    const uint32_t iso = isolated_in ? (kKeyIsolated | kWordInSet) : kKeyIsolated;
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    float dbar0 = 0.f;
    uint64_t smix0 = 0;
    if (a.seg.count == 0 && n > 0) {
        dbar0 = average_degree(a.rp[n], n);
        smix0 = mix64(a.seed0);
    }
    if ((n_words & 3) == 0) {
        // four vertices per thread: 16-byte loads of row_ptr, stores of words.
        // In a batch the four share one 16-vertex block, hence one graph
        // (offsets are multiples of 16): its parameters are looked up once.
        for (long long v = 4 * tid; v < n_words; v += 4 * nthreads) {
            float dbar = dbar0;
            uint64_t smix = smix0;
            long long first = 0;  // the graph's first vertex in the union
            long long limit = n;  // its vertices
            if (a.seg.count != 0 && v < n) {
                const int g = a.seg.blk_seg[v >> 4];
                first = a.seg.voff[g];
                limit = a.seg.nv[g];
                dbar = average_degree(a.seg.arcs[g], a.seg.nv[g]);
                smix = mix64(a.seg.seed[g]);
            }
            int r[5];
            if (v + 4 <= n) {
                const int4 q = *reinterpret_cast<const int4*>(a.rp + v);
                r[0] = q.x;
                r[1] = q.y;
                r[2] = q.z;
                r[3] = q.w;
                r[4] = a.rp[v + 4];
            } else {
                for (int k = 0; k < 5; ++k) r[k] = (v + k <= n) ? a.rp[v + k] : 0;
            }
            // class-1 flags of the four vertices (bytes of one aligned word)
            uint32_t sure = 0;
            if (r0class) {
                if (v + 4 <= n) {
                    sure = *reinterpret_cast<const uint32_t*>(r0class + v);
                } else {
                    for (int k = 0; k < 4; ++k)
                        if (v + k < n) sure |= (uint32_t)r0class[v + k] << (8 * k);
                }
            }
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const long long u = v + k;
                const long long local = u - first;
                const int deg = r[k + 1] - r[k];
                if (u >= n || local >= limit) {
                    w[k] = kWordOut;  // beyond n, or padding between two graphs
                } else {
                    w[k] = deg ? undecided_word(mode, priority_key(mode, dbar, deg, smix,
                                                                   (uint32_t)local))
                               : iso;
                    if (((sure >> (8 * k)) & 0xFFu) == 1u) w[k] |= kWordInSet;
                }
            }
            *reinterpret_cast<uint4*>(a.word + v) = make_uint4(w[0], w[1], w[2], w[3]);
            if (out && v < n) {
                uint32_t b = 0;
#pragma unroll
                for (int k = 0; k < 4; ++k) b |= (uint32_t)(w[k] >= kWordInMin) << (8 * k);
                if (v + 4 <= n && ((uintptr_t)(out + v) & 3) == 0) {
                    *reinterpret_cast<uint32_t*>(out + v) = b;
                } else {
                    for (int k = 0; k < 4 && v + k < n; ++k) out[v + k] = (uint8_t)(b >> (8 * k));
                }
            }
        }
        return;
    }
    for (long long v = tid; v < n_words; v += nthreads) {
        uint32_t w;
        if (v >= n) {
            w = kWordOut;
        } else {
            const int deg = a.rp[v + 1] - a.rp[v];
            if (a.seg.count == 0) {
                w = deg ? undecided_word(mode, priority_key(mode, dbar0, deg, smix0, (uint32_t)v))
                        : iso;
            } else {
                const int g = a.seg.blk_seg[v >> 4];
                const int local = (int)v - a.seg.voff[g];
                if (local >= a.seg.nv[g]) {
                    w = kWordOut;  // padding vertex between two graphs
                } else if (deg == 0) {
                    w = iso;
                } else {
                    const float dbar = average_degree(a.seg.arcs[g], a.seg.nv[g]);
                    w = undecided_word(mode, priority_key(mode, dbar, deg, mix64(a.seg.seed[g]),
                                                          (uint32_t)local));
                }
            }
            if (r0class && r0class[v] == 1) w |= kWordInSet;
            if (out) out[v] = w >= kWordInMin;
        }
        a.word[v] = w;
    }
}

}  // namespace tcmis
