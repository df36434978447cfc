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
// At create time each row is sorted by neighbour degree (stable, so ties keep
// ascending ids) and split[v] counts the neighbours of degree <= deg(v) + 1;
// vertices with d + deg(v) >= 2^19 keep their whole row (split[v] = deg(v)).
// The exclusion test scans the same ordered rows: the candidates that exclude
// a vertex are local maxima of the priority, i.e. mostly low-degree
// neighbours, which now come first.  None of this depends on the seed.
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

}  // namespace

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
    cudaError_t e = cudaMalloc((void**)&k0, 4 * (size_t)arcs);
    if (e == cudaSuccess) e = cudaMalloc((void**)&k1, 4 * (size_t)arcs);
    if (e == cudaSuccess) {
        neighbour_degree_kernel<<<(unsigned)((arcs + 255) / 256), 256, 0, s>>>(rp, col, arcs, k0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess)
        e = cub::DeviceSegmentedSort::StableSortPairs(nullptr, temp_bytes, k0, k1, col, col_sel,
                                                     (int)arcs, n, rp, rp + 1, s);
    if (e == cudaSuccess) e = cudaMalloc(&temp, temp_bytes ? temp_bytes : 1);
    if (e == cudaSuccess)
        e = cub::DeviceSegmentedSort::StableSortPairs(temp, temp_bytes, k0, k1, col, col_sel,
                                                     (int)arcs, n, rp, rp + 1, s);
    const double dbar0 = (double)arcs / (double)n;
    if (e == cudaSuccess) {
        split_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(rp, k1, n, seg, dbar0, split);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(k0);
    cudaFree(k1);
    cudaFree(temp);
    return e;
}

}  // namespace tcmis
