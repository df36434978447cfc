// mem.cu -- device memory for the library: the stream-ordered pool allocator.
//
// Graph handles, workspaces and create-time temporaries come from the
// device's default memory pool with its release threshold raised, so memory
// freed by one create or destroy is reused by the next without returning to
// the driver.  Allocations are stream-ordered on the legacy default stream and
// made visible to every stream before the call returns.
#include <cstdint>
#include <mutex>
#include <vector>

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
    cudaError_t e = dev_alloc_deferred(p, bytes);
    if (e == cudaSuccess) e = cudaStreamSynchronize(0);
    return e;
}

cudaError_t dev_alloc_deferred(void** p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = prepare_pool();
    if (e != cudaSuccess) return e;
    return cudaMallocAsync(p, bytes ? bytes : 1, 0);
}

cudaError_t dev_alloc_fence() { return cudaStreamSynchronize(0); }

// ---------------------------------------------------------------- pinned host
//
// Small pinned host blocks (control-block and statistics staging, seeds) come
// from slabs that are allocated once and never returned: cudaMallocHost and
// cudaFreeHost cost tens of microseconds each, and cudaFreeHost can wait for
// the whole device.  A block carries a 64-byte header with its size class;
// class k holds blocks of 512 << k bytes, header included.  Larger requests
// go to cudaMallocHost directly.

namespace {
constexpr size_t kHostHdr = 64;
constexpr int kHostClasses = 8;  // 512 B .. 64 KB
constexpr size_t kHostSlab = 1 << 20;
std::mutex g_host_mu;
std::vector<unsigned char*> g_host_free[kHostClasses];
}  // namespace

void* host_small_alloc(size_t bytes) {
    int k = 0;
    while (k < kHostClasses && (size_t(512) << k) < bytes + kHostHdr) ++k;
    unsigned char* b = nullptr;
    if (k == kHostClasses) {
        if (cudaMallocHost((void**)&b, bytes + kHostHdr) != cudaSuccess) return nullptr;
    } else {
        std::lock_guard<std::mutex> lk(g_host_mu);
        std::vector<unsigned char*>& fl = g_host_free[k];
        if (fl.empty()) {
            const size_t bs = size_t(512) << k;
            unsigned char* slab = nullptr;
            if (cudaMallocHost((void**)&slab, kHostSlab) != cudaSuccess) return nullptr;
            for (size_t off = 0; off + bs <= kHostSlab; off += bs) fl.push_back(slab + off);
        }
        b = fl.back();
        fl.pop_back();
    }
    *reinterpret_cast<int*>(b) = k;
    return b + kHostHdr;
}

void host_small_free(void* p) {
    if (!p) return;
    unsigned char* b = static_cast<unsigned char*>(p) - kHostHdr;
    const int k = *reinterpret_cast<int*>(b);
    if (k >= kHostClasses) {
        cudaFreeHost(b);
        return;
    }
    std::lock_guard<std::mutex> lk(g_host_mu);
    g_host_free[k].push_back(b);
}

void dev_free(void* p) {
    if (p) cudaFreeAsync(p, 0);
}

}  // namespace tcmis
