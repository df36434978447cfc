// mem.cu -- device memory for the library: the stream-ordered pool allocator.
//
// Graph handles, workspaces and create-time temporaries come from the
// device's default memory pool with its release threshold raised, so memory
// freed by one create or destroy is reused by the next without returning to
// the driver.  Allocations are stream-ordered on the legacy default stream and
// made visible to every stream before the call returns.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "internal.h"

namespace tcmis {

namespace {
std::mutex g_pool_mu;
bool g_pool_ready[64] = {};
}  // namespace

static cudaError_t prepare_pool() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaSuccess;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (g_pool_ready[dev]) return cudaSuccess;
    cudaMemPool_t pool;
    e = cudaDeviceGetDefaultMemPool(&pool, dev);
    if (e != cudaSuccess) return e;
    uint64_t keep = UINT64_MAX;
    e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e != cudaSuccess) return e;
    g_pool_ready[dev] = true;
    return cudaSuccess;
}

cudaError_t dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = prepare_pool();
    if (e != cudaSuccess) return e;
    e = cudaMallocAsync(p, bytes ? bytes : 1, 0);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    return e;
}

void dev_free(void* p) {
    if (p) cudaFreeAsync(p, 0);
}

}  // namespace tcmis
