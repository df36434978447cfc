// kernels_order.cu -- degree-ordered adjacency for the CSR round kernel.
//
// Eq. 1 gives lower priorities to higher degrees: in exact arithmetic
// deg(u) >= deg(v) + 2 implies P(u) < d/(d + deg(v) + 1) < P(v), because the
// perturbation eps lies in [0, 1).  Each binary32 operation of the key adds a
// relative error of at most 2^-24, so the strict order survives rounding as
// long as d + deg(v) < 2^20 (the gap 1/(d + deg(v)) then exceeds the summed
// rounding error several times over).  Hence the selection test of Phase 1
// only needs the neighbours of degree <= deg(v) + 1: no other neighbour can
// outrank v, whatever the seed.
//
// At create time each row is reordered so that the neighbours of degree
// <= deg(v) + 1 come first; split[v] counts them (vertices with
// d + deg(v) >= 2^19 keep their whole row as the prefix).  Two modes:
//   partition  a stable partition (one flag pass, one scan, one scatter);
//   sort       a stable sort of each row by neighbour degree, which also
//              brings the low-degree neighbours -- the likely candidates that
//              exclude a vertex in Phase 2 -- to the front of every row.
// None of this depends on the seed.
#include <cub/cub.cuh>

#include "common.cuh"
#include "internal.h"

namespace tcmis {

namespace {

__global__ void neighbour_degree_kernel(const int32_t* __restrict__ rp,
                                        const int32_t* __restrict__ col, int64_t arcs,
                                        int32_t* __restrict__ ndeg) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= arcs) return;
    const int u = col[p];
    ndeg[p] = rp[u + 1] - rp[u];
}

__global__ void split_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ ndeg,
                             int32_t n, const SegTable seg, double dbar0,
                             int32_t* __restrict__ split) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n) return;
    const int b = rp[v], e = rp[v + 1];
    const int deg = e - b;
    double dbar = dbar0;
    if (seg.count) {
        const int g = seg.blk_seg[v >> 4];
        dbar = seg.nv[g] ? (double)seg.arcs[g] / seg.nv[g] : 0.0;
    }
    if (dbar + deg >= (double)(1 << 19)) {
        split[v] = deg;
        return;
    }
    // first position whose neighbour degree exceeds deg + 1
    int lo = b, hi = e;
    while (lo < hi) {
        const int mid = lo + (hi - lo) / 2;
        if (ndeg[mid] <= deg + 1) lo = mid + 1;
        else hi = mid;
    }
    split[v] = lo - b;
}

constexpr int kArcsPerThread = 16;

// Per-thread run of consecutive arcs: the row of the first by binary search.
__device__ __forceinline__ int row_of(const int32_t* __restrict__ rp, int32_t n, int64_t p0) {
    int lo = 0, hi = n;  // last v with rp[v] <= p0
    while (hi - lo > 1) {
        const int mid = lo + (hi - lo) / 2;
        if ((int64_t)rp[mid] <= p0) lo = mid;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ bool whole_row(const SegTable& seg, double dbar0, int v, int deg) {
    double dbar = dbar0;
    if (seg.count) {
        const int g = seg.blk_seg[v >> 4];
        dbar = seg.nv[g] ? (double)seg.arcs[g] / seg.nv[g] : 0.0;
    }
    return dbar + deg >= (double)(1 << 19);
}

// flag[p] = 1 when arc p's neighbour belongs to the selection prefix of its row.
__global__ void prefix_flag_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                   int32_t n, int64_t arcs, const SegTable seg, double dbar0,
                                   int32_t* __restrict__ flag) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p0 = t * kArcsPerThread;
    if (p0 >= arcs) return;
    const int64_t p1 = (arcs < p0 + kArcsPerThread) ? arcs : p0 + kArcsPerThread;
    int v = row_of(rp, n, p0);
    for (int64_t p = p0; p < p1; ++p) {
        while ((int64_t)rp[v + 1] <= p) ++v;
        const int deg = rp[v + 1] - rp[v];
        const int u = col[p];
        flag[p] = (whole_row(seg, dbar0, v, deg) || rp[u + 1] - rp[u] <= deg + 1) ? 1 : 0;
    }
}

// Stable partition of each row by flag, from the exclusive scan `pos` of the
// flags (pos has arcs + 1 entries).
__global__ void prefix_scatter_kernel(const int32_t* __restrict__ rp,
                                      const int32_t* __restrict__ col, int32_t n, int64_t arcs,
                                      const int32_t* __restrict__ flag,
                                      const int32_t* __restrict__ pos,
                                      int32_t* __restrict__ col_sel, int32_t* __restrict__ split) {
    const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t p0 = t * kArcsPerThread;
    if (p0 >= arcs) return;
    const int64_t p1 = (arcs < p0 + kArcsPerThread) ? arcs : p0 + kArcsPerThread;
    int v = row_of(rp, n, p0);
    for (int64_t p = p0; p < p1; ++p) {
        while ((int64_t)rp[v + 1] <= p) ++v;
        const int b = rp[v], e = rp[v + 1];
        const int low = pos[e] - pos[b];
        const int before = pos[p] - pos[b];  // prefix arcs of this row before p
        const int64_t dst = flag[p] ? b + before : b + low + (p - b - before);
        col_sel[dst] = col[p];
        if (p == b) split[v] = low;
    }
}

__global__ void split_zero_rows_kernel(const int32_t* __restrict__ rp, int32_t n,
                                       int32_t* __restrict__ split) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n && rp[v] == rp[v + 1]) split[v] = 0;
}

}  // namespace

cudaError_t build_row_partition(const int32_t* rp, const int32_t* col, int32_t n, int64_t arcs,
                                const SegTable& seg, int32_t* col_sel, int32_t* split,
                                cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaSuccess;
    int32_t *flag = nullptr, *pos = nullptr;
    void* temp = nullptr;
    size_t temp_bytes = 0;
    const double dbar0 = (double)arcs / (double)n;
    const unsigned rows = (unsigned)((n + 255) / 256);
    if (arcs > 0) {
        const long long work = (arcs + kArcsPerThread - 1) / kArcsPerThread;
        const unsigned blocks = (unsigned)((work + 255) / 256);
        if ((e = dev_alloc((void**)&flag, 4 * ((size_t)arcs + 1))) == cudaSuccess &&
            (e = dev_alloc((void**)&pos, 4 * ((size_t)arcs + 1))) == cudaSuccess &&
            (e = cudaMemsetAsync(flag + arcs, 0, 4, s)) == cudaSuccess) {
            prefix_flag_kernel<<<blocks, 256, 0, s>>>(rp, col, n, arcs, seg, dbar0, flag);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cub::DeviceScan::ExclusiveSum(nullptr, temp_bytes, flag, pos, (int)arcs + 1, s);
        if (e == cudaSuccess) e = dev_alloc(&temp, temp_bytes ? temp_bytes : 1);
        if (e == cudaSuccess)
            e = cub::DeviceScan::ExclusiveSum(temp, temp_bytes, flag, pos, (int)arcs + 1, s);
        if (e == cudaSuccess) {
            prefix_scatter_kernel<<<blocks, 256, 0, s>>>(rp, col, n, arcs, flag, pos, col_sel,
                                                         split);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        split_zero_rows_kernel<<<rows, 256, 0, s>>>(rp, n, split);
        e = cudaGetLastError();
    }
    const cudaError_t se = cudaStreamSynchronize(s);  // also on error: nothing may still run
    if (e == cudaSuccess) e = se;
    dev_free(flag);
    dev_free(pos);
    dev_free(temp);
    return e;
}

cudaError_t build_degree_order(const int32_t* rp, const int32_t* col, int32_t n, int64_t arcs,
                               const SegTable& seg, int32_t* col_sel, int32_t* split,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    if (arcs == 0) {
        cudaError_t e = cudaMemsetAsync(split, 0, sizeof(int32_t) * (size_t)n, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        return e;
    }
    int32_t *k0 = nullptr, *k1 = nullptr;
    void* temp = nullptr;
    size_t temp_bytes = 0;
    cudaError_t e = dev_alloc((void**)&k0, 4 * (size_t)arcs);
    if (e == cudaSuccess) e = dev_alloc((void**)&k1, 4 * (size_t)arcs);
    if (e == cudaSuccess) {
        neighbour_degree_kernel<<<(unsigned)((arcs + 255) / 256), 256, 0, s>>>(rp, col, arcs, k0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cub::DeviceSegmentedSort::StableSortPairs(nullptr, temp_bytes, k0, k1, col, col_sel,
                                                     (int)arcs, n, rp, rp + 1, s);
    if (e == cudaSuccess) e = dev_alloc(&temp, temp_bytes ? temp_bytes : 1);
    if (e == cudaSuccess)
        e = cub::DeviceSegmentedSort::StableSortPairs(temp, temp_bytes, k0, k1, col, col_sel,
                                                     (int)arcs, n, rp, rp + 1, s);
    const double dbar0 = (double)arcs / (double)n;
    if (e == cudaSuccess) {
        split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rp, k1, n, seg, dbar0, split);
        e = cudaGetLastError();
    }
    const cudaError_t se = cudaStreamSynchronize(s);  // also on error: nothing may still run
    if (e == cudaSuccess) e = se;
    dev_free(k0);
    dev_free(k1);
    dev_free(temp);
    return e;
}

}  // namespace tcmis
