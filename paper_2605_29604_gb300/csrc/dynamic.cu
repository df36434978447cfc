// dynamic.cu -- edge updates of a resident graph, and incremental repair of
// an MIS after them: the dynamic setting (edge insertions and deletions) that
// the paper's conclusion names as future work.
//
// mis_update_edges rebuilds the graph on the device: the arcs become 64-bit
// keys (row << 32 | column), already sorted; the deleted ones are dropped,
// the sorted insertions (both directions) merged in, and a unique pass gives
// the new sorted, duplicate-free, symmetric CSR, from which every create-time
// structure is rebuilt exactly as mis_create_ex builds it.
//
// mis_repair turns the MIS of the graph before a set of edge changes into
// the MIS of the graph after them, equal to a full solve of the new graph.
// It relies on a fact of Algorithm 2 with fixed priorities: its result is the
// greedy MIS in priority order, where a vertex is in exactly when no
// neighbour that outranks it is in.  So a changed edge {a, b} can only change
// the state of its lower endpoint directly, and a vertex whose state flips
// only that of the neighbours it outranks.  The repair runs in passes: the
// first re-decides the lower endpoints, every other vertex fixed; each next
// pass re-decides the lower-priority neighbours of the vertices that flipped,
// until nothing flips.  Within a pass the rounds apply the greedy rule to the
// listed vertices.  This needs priorities that do not depend on the graph:
// the H1 hash keys (Sec. 3.3).  Eq. 1's key divides by the average degree
// d-bar, so any edge change moves every key and a repair would be a full
// solve.
#include <algorithm>
#include <vector>

#include <cub/cub.cuh>

#include "common.cuh"
#include "graph.h"
#include "internal.h"

namespace tcmis {

namespace {

constexpr unsigned long long kGone = ~0ull;  // key of a deleted arc

struct NotGone {
    __host__ __device__ bool operator()(const unsigned long long& k) const { return k != kGone; }
};

// One warp per row: the 64-bit key of every arc, kGone for the arcs listed
// (sorted) in del.
__global__ void arc_keys_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                int32_t n, const unsigned long long* __restrict__ del,
                                int64_t ndel, unsigned long long* __restrict__ keys) {
    const long long v = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (v >= n) return;
    const int b = rp[v], e = rp[v + 1];
    for (int p = b + (int)lane_id(); p < e; p += 32) {
        const unsigned long long k = ((unsigned long long)v << 32) | (unsigned)col[p];
        long long lo = 0, hi = ndel;  // first del entry >= k
        while (lo < hi) {
            const long long mid = (lo + hi) / 2;
            if (del[mid] < k) lo = mid + 1;
            else hi = mid;
        }
        keys[p] = (lo < ndel && del[lo] == k) ? kGone : k;
    }
}

// rp[v] = the first arc of row v among the sorted keys; col = their low words.
__global__ void csr_of_keys_kernel(const unsigned long long* __restrict__ keys, int64_t arcs,
                                   int32_t n, int32_t* __restrict__ rp,
                                   int32_t* __restrict__ col) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < arcs) col[i] = (int32_t)(keys[i] & 0xFFFFFFFFull);
    if (i <= n) {
        const unsigned long long k = (unsigned long long)i << 32;
        long long lo = 0, hi = arcs;
        while (lo < hi) {
            const long long mid = (lo + hi) / 2;
            if (keys[mid] < k) lo = mid + 1;
            else hi = mid;
        }
        rp[i] = (int32_t)lo;
    }
}

// ---- repair

// H1 key of v for the seed (seed_mix = mix64(seed), as in every solve).
__device__ __forceinline__ uint32_t hash_key(uint64_t seed, int v) {
    return priority_key(kPrioHash, 0.f, 1, mix64(seed), (uint32_t)v);
}

// Does u outrank v (fixed keys; ties to the larger id, as in the rounds)?
__device__ __forceinline__ bool above(uint32_t ku, int u, uint32_t kv, int v) {
    return ku > kv || (ku == kv && u > v);
}

// Every vertex keeps its state for now: word = in or out from out[].
__global__ void fixed_words_kernel(const uint8_t* __restrict__ out, int32_t n,
                                   uint32_t* __restrict__ word) {
    const long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) word[v] = out[v] ? kWordInMin : kWordOut;
}

// Puts v on a pass's list, once: mark[v] holds the stamp of the last pass
// that listed it.
__device__ __forceinline__ void enlist(int v, int stamp, int* __restrict__ mark,
                                       int32_t* __restrict__ list, int* __restrict__ len) {
    if (atomicExch(mark + v, stamp) != stamp) list[atomicAdd(len, 1)] = v;
}

// The first pass: the lower endpoint of each changed edge.
__global__ void seed_dirty_kernel(const int32_t* __restrict__ pairs, int64_t m, uint64_t seed,
                                  int stamp, int* __restrict__ mark, int32_t* __restrict__ list,
                                  int* __restrict__ len) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int a = pairs[2 * i], b = pairs[2 * i + 1];
    enlist(above(hash_key(seed, a), a, hash_key(seed, b), b) ? b : a, stamp, mark, list, len);
}

// The pass's vertices are undecided again: their keys, 0 in the result, and
// their previous state kept in old[i].
__global__ void open_dirty_kernel(const int32_t* __restrict__ list, int len, uint64_t seed,
                                  uint32_t* __restrict__ word, uint8_t* __restrict__ out,
                                  uint8_t* __restrict__ old) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= len) return;
    const int v = list[i];
    old[i] = out[v];
    word[v] = undecided_word(kPrioHash, hash_key(seed, v));
    out[v] = 0;
}

// One warp per vertex of the pass: if its state flipped, every neighbour it
// outranks goes on the next pass's list.
__global__ void propagate_kernel(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const int32_t* __restrict__ list, int len, uint64_t seed,
                                 const uint8_t* __restrict__ out, const uint8_t* __restrict__ old,
                                 int stamp, int* __restrict__ mark, int32_t* __restrict__ next,
                                 int* __restrict__ next_len) {
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (i >= len) return;
    const int v = list[i];
    if (out[v] == old[i]) return;
    const uint32_t kv = hash_key(seed, v);
    for (int p = rp[v] + (int)lane_id(); p < rp[v + 1]; p += 32) {
        const int u = col[p];
        if (above(kv, v, hash_key(seed, u), u)) enlist(u, stamp, mark, next, next_len);
    }
}

// One round over W (one warp per vertex), by the greedy rule the rounds of
// Algorithm 2 compute: v goes out when a neighbour that outranks it is in,
// goes in when every neighbour that outranks it is out, and stays otherwise.
// Neighbours below v do not matter (those of the vertices that flip are
// re-decided in the next pass).  A state, once decided, is final, so reading
// one decided in the same round by another warp is safe.
__global__ void repair_round_kernel(const int32_t* __restrict__ rp,
                                    const int32_t* __restrict__ col,
                                    const int32_t* __restrict__ wl, int len, uint64_t seed,
                                    uint32_t* __restrict__ word, uint8_t* __restrict__ out,
                                    int32_t* __restrict__ next, int* __restrict__ next_len) {
    const long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) / 32;
    if (i >= len) return;
    const int v = wl[i];
    const uint32_t kv = hash_key(seed, v);
    bool in_above = false, open_above = false;
    for (int p0 = rp[v]; p0 < rp[v + 1] && !in_above; p0 += 32) {
        const int p = p0 + (int)lane_id();
        bool in_u = false, open_u = false;
        if (p < rp[v + 1]) {
            const int u = col[p];
            if (above(hash_key(seed, u), u, kv, v)) {
                const uint32_t wu = __ldcg(word + u);
                in_u = wu >= kWordInMin;
                open_u = (wu >> 29) == 1u;
            }
        }
        in_above = __any_sync(0xFFFFFFFFu, in_u);
        open_above = open_above || __any_sync(0xFFFFFFFFu, open_u);
    }
    if (lane_id() != 0) return;
    if (in_above) {
        word[v] = kWordOut;
    } else if (!open_above) {
        word[v] = kWordInMin | kv;
        out[v] = 1;
    } else {
        next[atomicAdd(next_len, 1)] = v;
    }
}

__global__ void count_in_kernel(const uint8_t* __restrict__ out, int32_t n,
                                unsigned long long* __restrict__ total) {
    const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nthreads = (long long)gridDim.x * blockDim.x;
    unsigned c = 0;
    for (long long v = tid; v < n; v += nthreads) c += out[v] != 0;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
    if (lane_id() == 0 && c) atomicAdd(total, (unsigned long long)c);
}

unsigned warp_blocks(long long items) { return (unsigned)((32LL * items + 255) / 256); }
unsigned thread_blocks(long long items) { return (unsigned)((items + 255) / 256); }

__global__ void fill_kernel(int32_t* __restrict__ p, int32_t count, int32_t value) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) p[i] = value;
}

// The handle takes the graph (n, rp, col: device CSR, valid and symmetric),
// built by the same create path as mis_create_ex with its options; its old
// data is freed.  On error the handle keeps its old graph.
int adopt_csr(mis_graph* g, int32_t n, const int32_t* rp, const int32_t* col, void* stream) {
    mis_options o = g->opt;
    o.check_symmetry = 0;  // symmetric by construction
    mis_graph* g2 = mis_create_ex(n, rp, col, 1, &o, stream);
    if (!g2) return MIS_EDEVICE;  // the error is already recorded
    std::swap(g->d, g2->d);
    g->path = g2->path;
    g->tpr = g2->tpr;
    g->grid = g2->grid;
    g->tile_grid = g2->tile_grid;
    g->tile_slots = g2->tile_slots;
    g->csr_pending = g2->csr_pending;
    g->csr_range0 = g2->csr_range0;
    g->tile_payload = g2->tile_payload;
    g->cluster = g2->cluster;
    mis_destroy(g2);  // frees the old graph's data
    return MIS_OK;
}

// Checks pairs of vertex ids: 0 <= u, v < n, u != v.
bool pairs_ok(const int32_t* pairs, int64_t m, int32_t n) {
    for (int64_t i = 0; i < m; ++i) {
        const int32_t u = pairs[2 * i], v = pairs[2 * i + 1];
        if (u < 0 || v < 0 || u >= n || v >= n || u == v) return false;
    }
    return true;
}

}  // namespace

}  // namespace tcmis

using namespace tcmis;

extern "C" {

int mis_update_edges(mis_graph* g, int64_t n_ins, const int32_t* ins, int64_t n_del,
                     const int32_t* del, void* stream) {
    clear_error();
    if (!g || n_ins < 0 || n_del < 0 || (n_ins > 0 && !ins) || (n_del > 0 && !del))
        return set_error(MIS_EINVAL, "mis_update_edges: null graph, negative count or null pairs");
    if (g->d.count != 0) return set_error(MIS_EINVAL, "mis_update_edges: a batch cannot be updated");
    if (g->inflight.load() != 0)
        return set_error(MIS_EBUSY, "mis_update_edges: served requests of this graph in flight");
    if (g->replays.load() != 0)
        return set_error(MIS_EBUSY, "mis_update_edges: captured solves of this graph exist "
                                    "(they hold its device memory; destroy them first)");
    const int32_t n = g->d.n;
    if (!pairs_ok(ins, n_ins, n) || !pairs_ok(del, n_del, n))
        return set_error(MIS_EINVAL, "mis_update_edges: a pair is out of range or a self-loop");
    const int64_t arcs = g->d.arcs;
    const int64_t total = arcs + 2 * n_ins;
    if (total > (int64_t)INT32_MAX - 16)
        return set_error(MIS_EINVAL, "mis_update_edges: more than 2^31 arcs");
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;

    // deletions (both directions, sorted) and insertions as arc keys
    std::vector<unsigned long long> hdel, hins;
    hdel.reserve(2 * n_del);
    for (int64_t i = 0; i < n_del; ++i) {
        const unsigned long long u = (unsigned)del[2 * i], v = (unsigned)del[2 * i + 1];
        hdel.push_back(u << 32 | v);
        hdel.push_back(v << 32 | u);
    }
    std::sort(hdel.begin(), hdel.end());
    hins.reserve(2 * n_ins);
    for (int64_t i = 0; i < n_ins; ++i) {
        const unsigned long long u = (unsigned)ins[2 * i], v = (unsigned)ins[2 * i + 1];
        hins.push_back(u << 32 | v);
        hins.push_back(v << 32 | u);
    }
    std::sort(hins.begin(), hins.end());
    hins.erase(std::unique(hins.begin(), hins.end()), hins.end());
    const int64_t nins = (int64_t)hins.size();

    // The old arcs are sorted keys already (rows ascending, columns ascending
    // within a row): drop the deleted ones, merge in the sorted insertions,
    // and drop the insertions of edges that exist -- three linear passes.
    unsigned long long *keys = nullptr, *work = nullptr, *dd = nullptr, *ik = nullptr;
    int32_t *rp = nullptr, *col = nullptr;
    int* nsel = nullptr;
    void* temp = nullptr;
    size_t tb_sel = 0, tb_merge = 0, tb_uniq = 0;
    const size_t tot = (size_t)std::max<int64_t>(total, 1);
    e = dev_alloc((void**)&keys, sizeof(unsigned long long) * tot);
    if (e == cudaSuccess) e = dev_alloc((void**)&work, sizeof(unsigned long long) * tot);
    if (e == cudaSuccess) e = dev_alloc((void**)&dd, sizeof(unsigned long long) * (hdel.size() + 1));
    if (e == cudaSuccess) e = dev_alloc((void**)&ik, sizeof(unsigned long long) * (size_t)(nins + 1));
    if (e == cudaSuccess) e = dev_alloc((void**)&nsel, 2 * sizeof(int));
    if (e == cudaSuccess && !hdel.empty())
        e = cudaMemcpyAsync(dd, hdel.data(), sizeof(unsigned long long) * hdel.size(),
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && nins > 0)
        e = cudaMemcpyAsync(ik, hins.data(), sizeof(unsigned long long) * (size_t)nins,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && n > 0 && arcs > 0) {
        arc_keys_kernel<<<warp_blocks(n), 256, 0, s>>>(g->d.rp, g->d.col, n, dd,
                                                       (int64_t)hdel.size(), keys);
        e = cudaGetLastError();
    }
    const NotGone kept_op;
    if (e == cudaSuccess)
        e = cub::DeviceSelect::If(nullptr, tb_sel, keys, work, nsel, (int)std::max<int64_t>(arcs, 1),
                                  kept_op, s);
    if (e == cudaSuccess)
        e = cub::DeviceMerge::MergeKeys(nullptr, tb_merge, work, (int64_t)arcs, ik, nins, keys,
                                        ::cuda::std::less<unsigned long long>{}, s);
    if (e == cudaSuccess)
        e = cub::DeviceSelect::Unique(nullptr, tb_uniq, keys, work, nsel + 1, (int)tot, s);
    if (e == cudaSuccess)
        e = dev_alloc(&temp, std::max<size_t>(std::max(tb_sel, std::max(tb_merge, tb_uniq)), 1));
    int nkept = 0;
    if (e == cudaSuccess && arcs > 0)
        e = cub::DeviceSelect::If(temp, tb_sel, keys, work, nsel, (int)arcs, kept_op, s);
    if (e == cudaSuccess && arcs > 0)
        e = cudaMemcpyAsync(&nkept, nsel, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const int64_t merged = nkept + nins;
    if (e == cudaSuccess && merged > 0)
        e = cub::DeviceMerge::MergeKeys(temp, tb_merge, work, (int64_t)nkept, ik, nins, keys,
                                        ::cuda::std::less<unsigned long long>{}, s);
    int hn = 0;
    if (e == cudaSuccess && merged > 0)
        e = cub::DeviceSelect::Unique(temp, tb_uniq, keys, work, nsel + 1, (int)merged, s);
    if (e == cudaSuccess && merged > 0)
        e = cudaMemcpyAsync(&hn, nsel + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const int64_t new_arcs = hn;
    if (e == cudaSuccess) e = dev_alloc((void**)&rp, sizeof(int32_t) * ((size_t)n + 1));
    if (e == cudaSuccess) e = dev_alloc((void**)&col, sizeof(int32_t) * ((size_t)new_arcs + 1));
    if (e == cudaSuccess) {
        csr_of_keys_kernel<<<thread_blocks(std::max<int64_t>(new_arcs, (int64_t)n + 1)), 256, 0,
                             s>>>(work, new_arcs, n, rp, col);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    dev_free(keys);
    dev_free(work);
    dev_free(dd);
    dev_free(ik);
    dev_free(nsel);
    dev_free(temp);
    if (e != cudaSuccess) {
        dev_free(rp);
        dev_free(col);
        return set_cuda_error(e, "mis_update_edges");
    }
    const int rc = adopt_csr(g, n, rp, col, stream);
    dev_free(rp);
    dev_free(col);
    return rc;
}

int mis_add_vertices(mis_graph* g, int32_t k, void* stream) {
    clear_error();
    if (!g || k < 0) return set_error(MIS_EINVAL, "mis_add_vertices: null graph or k < 0");
    if (g->d.count != 0) return set_error(MIS_EINVAL, "mis_add_vertices: not for a batch");
    if (g->inflight.load() != 0)
        return set_error(MIS_EBUSY, "mis_add_vertices: served requests of this graph in flight");
    if (g->replays.load() != 0)
        return set_error(MIS_EBUSY, "mis_add_vertices: captured solves of this graph exist "
                                    "(they hold its device memory; destroy them first)");
    const int32_t n = g->d.n;
    if ((int64_t)n + k > (int64_t)INT32_MAX - 16)
        return set_error(MIS_EINVAL, "mis_add_vertices: more than 2^31 vertices");
    if (k == 0) return MIS_OK;
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    // the same arcs; the new rows are empty: row_ptr[n + 1 ..] = arcs
    const int32_t n2 = n + k;
    int32_t *rp = nullptr, *col = nullptr;
    e = dev_alloc((void**)&rp, sizeof(int32_t) * ((size_t)n2 + 1));
    if (e == cudaSuccess) e = dev_alloc((void**)&col, sizeof(int32_t) * ((size_t)g->d.arcs + 1));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rp, g->d.rp, sizeof(int32_t) * ((size_t)n + 1), cudaMemcpyDeviceToDevice,
                            s);
    if (e == cudaSuccess) {
        fill_kernel<<<thread_blocks(k), 256, 0, s>>>(rp + n + 1, k, (int32_t)g->d.arcs);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && g->d.arcs > 0)
        e = cudaMemcpyAsync(col, g->d.col, sizeof(int32_t) * (size_t)g->d.arcs,
                            cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    int rc = e == cudaSuccess ? adopt_csr(g, n2, rp, col, stream)
                              : set_cuda_error(e, "mis_add_vertices");
    dev_free(rp);
    dev_free(col);
    return rc;
}

int mis_repair(mis_graph* g, uint64_t seed, int64_t n_changed, const int32_t* changed,
               uint8_t* out_status, int64_t* mis_size, int32_t* rounds, void* stream) {
    clear_error();
    if (!g || n_changed < 0 || (n_changed > 0 && !changed) || (!out_status && g && g->d.n > 0))
        return set_error(MIS_EINVAL, "mis_repair: null graph, pairs or result");
    if (g->d.count != 0) return set_error(MIS_EINVAL, "mis_repair: not for a batch");
    if (g->opt.priority != MIS_PRIORITY_HASH)
        return set_error(MIS_EINVAL,
                         "mis_repair needs MIS_PRIORITY_HASH: Eq. 1 keys depend on the average "
                         "degree, so an edge change moves every key (solve again instead)");
    const int32_t n = g->d.n;
    if (!pairs_ok(changed, n_changed, n))
        return set_error(MIS_EINVAL, "mis_repair: a pair is out of range or a self-loop");
    cudaError_t e = cudaSetDevice(g->d.device);
    if (e != cudaSuccess) return set_cuda_error(e, "cudaSetDevice");
    cudaStream_t s = (cudaStream_t)stream;
    if (rounds) *rounds = 0;
    if (mis_size) *mis_size = 0;
    if (n == 0) return MIS_OK;
    GraphData& d = g->d;
    // per-graph scratch: the pass stamps of every vertex, and four counters
    if (!d.dyn_mark) {
        if ((e = dev_alloc((void**)&d.dyn_mark, sizeof(int) * (size_t)n)) != cudaSuccess ||
            (e = dev_alloc((void**)&d.dyn_cnt, 4 * sizeof(int))) != cudaSuccess ||
            (e = cudaMemsetAsync(d.dyn_mark, 0, sizeof(int) * (size_t)n, s)) != cudaSuccess)
            return set_cuda_error(e, "mis_repair: scratch");
        d.dyn_stamp = 0;
        d.footprint += 4 * (int64_t)n + 16;
    }
    if (d.dyn_stamp > INT32_MAX - 2 * (n + 2)) {  // stamps would wrap: start over
        if ((e = cudaMemsetAsync(d.dyn_mark, 0, sizeof(int) * (size_t)n, s)) != cudaSuccess)
            return set_cuda_error(e, "mis_repair: scratch");
        d.dyn_stamp = 0;
    }
    Workspace& w = d.ws;
    uint32_t* word = w.word;
    // lists in the workspace (each int4 array holds 4 ints per vertex)
    int32_t* wa = reinterpret_cast<int32_t*>(w.wl0);
    int32_t* wb = reinterpret_cast<int32_t*>(w.wl1);
    int32_t* list = reinterpret_cast<int32_t*>(w.wlp);
    int32_t* next = list + w.cap;
    uint8_t* old = reinterpret_cast<uint8_t*>(list + 2 * w.cap);
    int* cnt = d.dyn_cnt;  // [0] list length, [1] next round's length
    int32_t* dpairs = nullptr;
    unsigned long long* dsum = nullptr;
    e = dev_alloc((void**)&dpairs, sizeof(int32_t) * (2 * (size_t)n_changed + 2));
    if (e == cudaSuccess) e = dev_alloc((void**)&dsum, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(dsum, 0, sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, 4 * sizeof(int), s);
    if (e == cudaSuccess && n_changed > 0)
        e = cudaMemcpyAsync(dpairs, changed, sizeof(int32_t) * 2 * (size_t)n_changed,
                            cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        fixed_words_kernel<<<thread_blocks(n), 256, 0, s>>>(out_status, n, word);
        e = cudaGetLastError();
    }
    int stamp = ++d.dyn_stamp;
    if (e == cudaSuccess && n_changed > 0) {
        seed_dirty_kernel<<<thread_blocks(n_changed), 256, 0, s>>>(dpairs, n_changed, seed, stamp,
                                                                    d.dyn_mark, list, cnt);
        e = cudaGetLastError();
    }
    // passes: re-decide the listed vertices with every other vertex fixed;
    // the lower-priority neighbours of those that flipped form the next pass
    int len = 0, r = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&len, cnt, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    while (e == cudaSuccess && len > 0) {
        open_dirty_kernel<<<thread_blocks(len), 256, 0, s>>>(list, len, seed, word, out_status, old);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(wa, list, sizeof(int32_t) * (size_t)len, cudaMemcpyDeviceToDevice, s);
        // Algorithm 2's rounds on the listed vertices
        int wl = len;
        int32_t *x = wa, *y = wb;
        while (e == cudaSuccess && wl > 0) {
            if (r > 2 * n + 2) {
                e = cudaErrorUnknown;
                break;
            }
            e = cudaMemsetAsync(cnt + 1, 0, sizeof(int), s);
            if (e == cudaSuccess) {
                repair_round_kernel<<<warp_blocks(wl), 256, 0, s>>>(d.rp, d.col, x, wl, seed, word,
                                                                    out_status, y, cnt + 1);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(&wl, cnt + 1, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            std::swap(x, y);
            ++r;
        }
        // the flips, and the next pass
        stamp = ++d.dyn_stamp;
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt + 2, 0, sizeof(int), s);
        if (e == cudaSuccess) {
            propagate_kernel<<<warp_blocks(len), 256, 0, s>>>(d.rp, d.col, list, len, seed,
                                                              out_status, old, stamp, d.dyn_mark,
                                                              next, cnt + 2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&len, cnt + 2, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        std::swap(list, next);
    }
    unsigned long long hsum = 0;
    if (e == cudaSuccess && mis_size) {
        count_in_kernel<<<std::min<unsigned>(thread_blocks(n), 1024), 256, 0, s>>>(out_status, n,
                                                                                    dsum);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&hsum, dsum, sizeof(hsum), cudaMemcpyDeviceToHost, s);
    }
    const cudaError_t se = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = se;
    dev_free(dsum);
    dev_free(dpairs);
    if (e != cudaSuccess) return set_cuda_error(e, "mis_repair");
    if (rounds) *rounds = r;
    if (mis_size) *mis_size = (int64_t)hsum;
    return MIS_OK;
}

}  // extern "C"
