// kernels_util.cu -- input validation, key export and batch packing kernels.
#include "common.cuh"
#include "internal.h"

namespace tcmis {

// ---------------------------------------------------------------- validation
//
// The input contract of the C ABI: row_ptr[0] = 0, non-decreasing,
// row_ptr[n] = arcs; col in [0, n); no self-loop; rows strictly increasing;
// symmetric.  Two kernels: row pointers first (the arc kernel trusts them).

__global__ void validate_rowptr_kernel(const int32_t* __restrict__ rp, int32_t n, int64_t arcs,
                                       unsigned* flags) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    unsigned bad = 0;
    if (tid == 0 && (rp[0] != 0 || (int64_t)rp[n] != arcs)) bad |= kBadRowPtr;
    for (long long v = tid; v < n; v += nthreads)
        if (rp[v] > rp[v + 1]) bad |= kBadRowPtr;
    if (bad) atomicOr(flags, bad);
}

// Each thread checks a run of consecutive arcs: it finds the row of its first
// arc by binary search over row_ptr and walks forward from there.
constexpr int kArcsPerThread = 16;

// Symmetry as equality of two arc sets: with rows strictly increasing (no
// duplicate arcs, checked on the way), the graph is symmetric exactly when
// its arc set equals the set of reversed arcs.  Each set is summarised by the
// sums (mod 2^64) of two fixed 64-bit hashes of its ordered pairs; every arc
// (v, u) adds h(v, u) - h(u, v) to each running sum, so equal sets leave both
// sums at zero.  Unequal sets leave both at zero only if two independent
// 64-bit sums cancel by accident.  One pass over the arcs with no search,
// where the previous check binary-searched v in row u for every arc.
__device__ __forceinline__ unsigned long long arc_hash(uint32_t a, uint32_t b, uint64_t salt) {
    return mix64((((uint64_t)a << 32) | b) ^ salt);
}
constexpr uint64_t kSymSalt0 = 0x6A09E667F3BCC908ull;  // fractional bits of sqrt(2)
constexpr uint64_t kSymSalt1 = 0xBB67AE8584CAA73Bull;  // fractional bits of sqrt(3)

// Checks the arcs [a0, a1) (all of them: a0 = 0, a1 = arcs).
__global__ void validate_arcs_kernel(const int32_t* __restrict__ rp,
                                     const int32_t* __restrict__ col, int32_t n, int64_t a0,
                                     int64_t a1, int check_symmetry, unsigned* flags,
                                     unsigned long long* sym) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p0 = a0 + t * kArcsPerThread;
    // threads past the end check nothing but still join the warp's sums
    const int64_t p1 = p0 >= a1 ? p0 : ((a1 < p0 + kArcsPerThread) ? a1 : p0 + kArcsPerThread);
    // row = last v with rp[v] <= p0
    int lo = 0, hi = p0 < a1 ? n : 1;  // invariant rp[lo] <= p0 < rp[hi]
    while (hi - lo > 1) {
        const int mid = lo + (hi - lo) / 2;
        if ((int64_t)rp[mid] <= p0) lo = mid;
        else hi = mid;
    }
    int v = lo;
    unsigned bad = 0;
    unsigned long long s0 = 0, s1 = 0;
    for (int64_t p = p0; p < p1; ++p) {
        while ((int64_t)rp[v + 1] <= p) ++v;
        const int u = col[p];
        if (u < 0 || u >= n) {
            bad |= kBadColRange;
            continue;
        }
        if (u == v) bad |= kBadSelfLoop;
        if (p > rp[v] && col[p - 1] >= u) bad |= kBadOrder;
        if (check_symmetry) {
            s0 += arc_hash((uint32_t)v, (uint32_t)u, kSymSalt0) -
                  arc_hash((uint32_t)u, (uint32_t)v, kSymSalt0);
            s1 += arc_hash((uint32_t)v, (uint32_t)u, kSymSalt1) -
                  arc_hash((uint32_t)u, (uint32_t)v, kSymSalt1);
        }
    }
    if (bad) atomicOr(flags, bad);
    if (check_symmetry && sym) {
        for (int o = 16; o; o >>= 1) {
            s0 += __shfl_xor_sync(0xFFFFFFFFu, s0, o);
            s1 += __shfl_xor_sync(0xFFFFFFFFu, s1, o);
        }
        if ((threadIdx.x & 31) == 0 && (s0 | s1)) {
            atomicAdd(sym, s0);
            atomicAdd(sym + 1, s1);
        }
    }
}

cudaError_t launch_validate(const int32_t* rp, const int32_t* col, int32_t n, int64_t arcs,
                            int check_symmetry, unsigned* d_flags, unsigned long long* d_sym,
                            cudaStream_t s) {
    // row pointers (host reads the flags before the arc pass)
    const int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    if (blocks < 1) blocks = 1;
    if (blocks > 65535) blocks = 65535;
    validate_rowptr_kernel<<<(unsigned)blocks, threads, 0, s>>>(rp, n, arcs, d_flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    unsigned hflags = 0;
    e = cudaMemcpyAsync(&hflags, d_flags, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess || hflags || arcs == 0) return e;
    return launch_validate_arcs(rp, col, n, 0, arcs, check_symmetry, d_flags, d_sym, s);
}

cudaError_t launch_validate_rowptr(const int32_t* rp, int32_t n, int64_t arcs, unsigned* d_flags,
                                   cudaStream_t s) {
    const int threads = 256;
    long long blocks = (n + threads - 1) / threads;
    if (blocks < 1) blocks = 1;
    if (blocks > 65535) blocks = 65535;
    validate_rowptr_kernel<<<(unsigned)blocks, threads, 0, s>>>(rp, n, arcs, d_flags);
    return cudaGetLastError();
}

cudaError_t launch_validate_arcs(const int32_t* rp, const int32_t* col, int32_t n, int64_t a0,
                                 int64_t a1, int check_symmetry, unsigned* d_flags,
                                 unsigned long long* d_sym, cudaStream_t s) {
    if (a1 <= a0) return cudaSuccess;
    const int threads = 256;
    const long long work = (a1 - a0 + kArcsPerThread - 1) / kArcsPerThread;
    const long long ablocks = (work + threads - 1) / threads;
    validate_arcs_kernel<<<(unsigned)ablocks, threads, 0, s>>>(rp, col, n, a0, a1,
                                                                check_symmetry, d_flags, d_sym);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- key export

__global__ void keys_kernel(const SolveArgs a, uint32_t* __restrict__ out_key) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    const int32_t n = a.n;
    float dbar0 = 0.f;
    uint64_t smix0 = 0;
    if (a.seg.count == 0 && n > 0) {
        dbar0 = average_degree(a.rp[n], n);
        smix0 = mix64(a.seed0);
    }
    for (long long v = tid; v < n; v += nthreads) {
        const int deg = a.rp[v + 1] - a.rp[v];
        if (a.seg.count == 0) {
            out_key[v] = deg ? priority_key(a.priority, dbar0, deg, smix0, (uint32_t)v) : 0xFFFFFFFFu;
        } else {
            const int g = a.seg.blk_seg[v >> 4];
            const int local = (int)v - a.seg.voff[g];
            if (local >= a.seg.nv[g]) continue;
            const float dbar = average_degree(a.seg.arcs[g], a.seg.nv[g]);
            out_key[a.seg.roff[g] + local] =
                deg ? priority_key(a.priority, dbar, deg, mix64(a.seg.seed[g]), (uint32_t)local)
                    : 0xFFFFFFFFu;
        }
    }
}

cudaError_t launch_keys(const SolveArgs& a, uint32_t* out_key, cudaStream_t s) {
    if (a.n == 0) return cudaSuccess;
    const int threads = 256;
    long long blocks = (a.n + threads - 1) / threads;
    if (blocks > 4096) blocks = 4096;
    keys_kernel<<<(unsigned)blocks, threads, 0, s>>>(a, out_key);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- batch packing

// blk_seg[j] = the graph whose vertex range holds 16-vertex block j.
__global__ void fill_seg_kernel(int32_t* __restrict__ blk_seg, const int32_t* __restrict__ voff,
                                int32_t count, int32_t nblk) {
    const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nblk) return;
    const long long first = j * 16;
    int lo = 0, hi = count;  // last g with voff[g] <= first
    while (hi - lo > 1) {
        const int mid = lo + (hi - lo) / 2;
        if (voff[mid] <= first) lo = mid;
        else hi = mid;
    }
    blk_seg[j] = lo;
}

cudaError_t launch_fill_seg(int32_t* blk_seg, const int32_t* voff, int32_t count, int32_t nblk,
                            cudaStream_t s) {
    if (nblk == 0) return cudaSuccess;
    fill_seg_kernel<<<(nblk + 255) / 256, 256, 0, s>>>(blk_seg, voff, count, nblk);
    return cudaGetLastError();
}

// In-place relocation of one graph copied into the union: row pointers gain
// the arc offset, neighbour ids gain the vertex offset.
__global__ void relocate_kernel(int32_t* __restrict__ rp, int32_t* __restrict__ col, int32_t n,
                                int32_t arcs, int32_t voff, int32_t aoff) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    for (long long i = tid; i < n; i += nthreads) rp[i] += aoff;
    for (long long p = tid; p < arcs; p += nthreads) col[p] += voff;
}

cudaError_t launch_relocate(int32_t* rp, int32_t* col, int32_t n, int32_t arcs, int32_t voff,
                            int32_t aoff, cudaStream_t s) {
    const long long work = n > arcs ? n : arcs;
    if (work == 0) return cudaSuccess;
    long long blocks = (work + 255) / 256;
    if (blocks > 2048) blocks = 2048;
    relocate_kernel<<<(unsigned)blocks, 256, 0, s>>>(rp, col, n, arcs, voff, aoff);
    return cudaGetLastError();
}

__global__ void fill_kernel(int32_t* __restrict__ p, int32_t count, int32_t value) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) p[i] = value;
}

cudaError_t launch_pad_rows(int32_t* dst_rp, int32_t from, int32_t to, int32_t value,
                            cudaStream_t s) {
    const int32_t cnt = to - from;
    if (cnt <= 0) return cudaSuccess;
    fill_kernel<<<(cnt + 255) / 256, 256, 0, s>>>(dst_rp + from, cnt, value);
    return cudaGetLastError();
}

}  // namespace tcmis
