// serve.cu -- continuous-batching request loop (mis_submit / mis_poll / mis_wait).
//
// A few scheduler threads per process (kWorkers) share max_slots solve
// slots: worker w owns slots w, w + kWorkers, ...  A slot holds a CUDA
// stream, an event, a solve workspace (grown on demand) and pinned staging
// for the result.  Each worker loops over its own slots:
//
//   retire   every slot whose event has fired: copy its result bytes to the
//            caller's host buffer (outside the library lock), record the
//            status, release the slot;
//   admit    queued requests, oldest first, while a slot is free and the
//            workspace bytes of all admitted requests stay within the HBM
//            budget (a request is always admitted when nothing runs);
//   group    queued requests on the same single graph (CSR path) ride one
//            slot together, up to 8: one multi-seed launch solves them all
//            (kernels_multi.cu), every neighbour gather serving each of them;
//            only requests already queued are grouped, nothing waits for a
//            group to fill;
//   launch   each admitted request (or group) on its slot's stream: on a graph
//            of up to kSingleBlockMax vertices as one block (a lone request
//            through an ordinary launch), else as a cooperative grid of at
//            most serve_blocks blocks (default: half the SMs), so that
//            requests admitted while others run share the device with them.
//
// Graphs stay resident: a request names a graph created earlier with
// mis_create*.  A graph destroyed while requests on it are in flight is freed
// when the last of them retires.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "graph.h"
#include "tcmis.h"

namespace tcmis {

namespace {

constexpr int32_t kSingleBlockMax = 16384;  // vertices solved by one block
constexpr int kDefaultSlots = 64;
constexpr int kWorkers = 4;  // scheduler threads; worker w owns slots w, w + kWorkers, ...
constexpr int64_t kStagingBytes = 2 << 20;  // pinned result staging per slot at start
constexpr int kGroupScan = 1024;  // queue entries searched for a request's group

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Request {
    int64_t t_submit = 0;
    int64_t t_done = 0;
    mis_ticket id = 0;
    mis_graph* g = nullptr;
    uint64_t seed = 0;
    uint8_t* host_out = nullptr;
    int status = MIS_ENOTREADY;
    bool done = false;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    Workspace ws;
    uint8_t* pinned_out = nullptr;
    int64_t pinned_cap = 0;
    uint64_t* seeds_pinned = nullptr;
    int32_t seeds_cap = 0;
    Ctl* ctl_pinned = nullptr;
    uint32_t* word8 = nullptr;     // multi-seed state, kMaxMulti words per vertex
    int64_t word8_cap = 0;         // vertices
    uint8_t* out_multi = nullptr;  // multi-seed results, kMaxMulti * n bytes
    int64_t out_multi_cap = 0;     // bytes
    Request* reqs[kMaxMulti] = {};
    int nreq = 0;                  // requests riding this slot (0 = free)
    int64_t charge = 0;
};

class Server {
  public:
    static Server& get() {
        static Server s;
        return s;
    }

    ~Server() { shutdown(); }

    int configure(const mis_options* o) {
        std::lock_guard<std::mutex> lk(mu_);
        if (running_) return set_error(MIS_EBUSY, "serving already started");
        mis_options d;
        mis_options_init(&d);
        if (o) d = *o;
        device_ = d.device;
        max_slots_ = d.max_slots > 0 ? d.max_slots : kDefaultSlots;
        budget_ = d.hbm_budget;
        serve_blocks_ = d.serve_blocks;
        return MIS_OK;
    }

    int submit(mis_graph* g, uint64_t seed, uint8_t* out, mis_ticket* t) {
        if (!g || !t || (g->d.result_bytes > 0 && !out))
            return set_error(MIS_EINVAL, "null graph, output or ticket");
        if (g->destroy_pending.load()) return set_error(MIS_EINVAL, "graph is being destroyed");
        std::lock_guard<std::mutex> lk(mu_);
        if (!running_) {
            const int rc = start_locked();
            if (rc != MIS_OK) return rc;
        }
        Request* r = new Request();
        r->t_submit = now_ns();
        r->id = next_id_++;
        r->g = g;
        r->seed = seed;
        r->host_out = out;
        g->inflight.fetch_add(1);
        reqs_[r->id] = r;
        queue_.push_back(r);
        *t = r->id;
        cv_work_.notify_all();
        return MIS_OK;
    }

    int poll(mis_ticket t, int64_t* latency_ns = nullptr) {
        std::lock_guard<std::mutex> lk(mu_);
        return finish_locked(t, latency_ns);
    }

    int wait(mis_ticket t, int64_t us) {
        std::unique_lock<std::mutex> lk(mu_);
        auto it = reqs_.find(t);
        if (it == reqs_.end()) return set_error(MIS_EINVAL, "unknown ticket");
        Request* r = it->second;
        auto ready = [r] { return r->done; };
        if (us < 0) {
            cv_done_.wait(lk, ready);
        } else if (!cv_done_.wait_for(lk, std::chrono::microseconds(us), ready)) {
            return set_error(MIS_ETIMEDOUT, "request still in flight");
        }
        return finish_locked(t);
    }

    // Frees g now if no served request uses it, else when the last one retires.
    void release(mis_graph* g) {
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (g->inflight.load() > 0) {
                g->destroy_pending.store(true);
                return;
            }
        }
        free_graph(g);
    }

    void shutdown() {
        std::vector<std::thread> ths;
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (!running_) return;
            stop_ = true;
            cv_work_.notify_all();
            ths = std::move(threads_);
            threads_.clear();
        }
        for (std::thread& th : ths)
            if (th.joinable()) th.join();
        std::lock_guard<std::mutex> lk(mu_);
        cudaSetDevice(device_);
        free_slots();
        running_ = false;
        stop_ = false;
    }

    // Releases every slot's stream, event, workspace and buffers.
    void free_slots() {
        for (Slot& s : slots_) {
            if (s.stream) cudaStreamSynchronize(s.stream);
            ws_free(s.ws);
            dev_free(s.word8);
            dev_free(s.out_multi);
            if (s.pinned_out) cudaFreeHost(s.pinned_out);
            if (s.seeds_pinned) cudaFreeHost(s.seeds_pinned);
            if (s.ctl_pinned) cudaFreeHost(s.ctl_pinned);
            if (s.ev) cudaEventDestroy(s.ev);
            if (s.stream) cudaStreamDestroy(s.stream);
        }
        slots_.clear();
    }

  private:
    int start_locked() {
        cudaError_t e = cudaSetDevice(device_);
        if (e != cudaSuccess) return set_cuda_error(e, "serving: cudaSetDevice");
        if (cudaDeviceGetAttribute(&sms_, cudaDevAttrMultiProcessorCount, device_) != cudaSuccess)
            sms_ = 1;
        if (budget_ <= 0) {
            size_t free_b = 0, total_b = 0;
            e = cudaMemGetInfo(&free_b, &total_b);
            if (e != cudaSuccess) return set_cuda_error(e, "serving: cudaMemGetInfo");
            budget_ = (int64_t)(free_b / 2);
        }
        stop_ = false;
        running_ = true;
        // every slot exists from the start, so that its owner never changes,
        // with its stream, event and 2 MB of pinned result staging made here
        // rather than while solves run
        slots_.clear();
        slots_.resize((size_t)max_slots_);
        for (Slot& sl : slots_) {
            if ((e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaMallocHost((void**)&sl.ctl_pinned, sizeof(Ctl))) != cudaSuccess ||
                (e = cudaMallocHost((void**)&sl.pinned_out, kStagingBytes)) != cudaSuccess) {
                running_ = false;
                const int rc = set_cuda_error(e, "serving: slot setup");
                free_slots();
                return rc;
            }
            sl.pinned_cap = kStagingBytes;
        }
        const int nw = std::max(1, std::min(kWorkers, max_slots_));
        for (int w = 0; w < nw; ++w) threads_.emplace_back([this, w, nw] { loop(w, nw); });
        return MIS_OK;
    }

    // Caller holds mu_.  Releases a finished request's ticket.
    int finish_locked(mis_ticket t, int64_t* latency_ns = nullptr) {
        auto it = reqs_.find(t);
        if (it == reqs_.end()) return set_error(MIS_EINVAL, "unknown ticket");
        Request* r = it->second;
        if (!r->done) return MIS_ENOTREADY;
        const int st = r->status;
        if (latency_ns) *latency_ns = r->t_done - r->t_submit;
        reqs_.erase(it);
        delete r;
        if (st != MIS_OK) set_error(st, "served request failed");
        return st;
    }

    // Bytes a slot holds for k requests on graph d.
    static int64_t charge_for(const GraphData& d, int k) {
        int64_t b = ws_bytes_for(d.n, d.count) + d.result_bytes;
        if (k > 1) b += 4 * (int64_t)kMaxMulti * ((d.n + 15) / 16 * 16) + k * d.result_bytes;
        return b;
    }

    // Starts the k requests rs (all on the same graph, taken off the queue
    // and assigned to slot s) on slot s; MIS_OK or an error (the requests are
    // then finished with that error by the caller).  Called by the scheduler
    // thread without mu_: only that thread touches the slots.
    int launch_unlocked(Slot& s, Request* const* rs, int k) {
        mis_graph* g = rs[0]->g;
        GraphData& d = g->d;
        cudaError_t e = cudaSuccess;
        if (!s.stream) {
            if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess ||
                (e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming)) != cudaSuccess ||
                (e = cudaMallocHost((void**)&s.ctl_pinned, sizeof(Ctl))) != cudaSuccess)
                return set_cuda_error(e, "serving: slot setup");
        }
        if ((e = ws_reserve(s.ws, d.n, d.count)) != cudaSuccess)
            return set_cuda_error(e, "serving: workspace");
        const int64_t out_bytes = (int64_t)k * d.result_bytes;
        // buffers grow geometrically: freeing pinned or cudaMalloc'd memory
        // synchronises the whole device, so regrowth must stay rare
        if (s.pinned_cap < out_bytes) {
            const int64_t cap = std::max(out_bytes, 2 * s.pinned_cap);
            if (s.pinned_out) cudaFreeHost(s.pinned_out);
            s.pinned_out = nullptr;
            s.pinned_cap = 0;
            if ((e = cudaMallocHost((void**)&s.pinned_out, (size_t)cap)) != cudaSuccess)
                return set_cuda_error(e, "serving: pinned result");
            s.pinned_cap = cap;
        }
        const int32_t count = std::max(1, d.count);
        if (s.seeds_cap < count) {
            if (s.seeds_pinned) cudaFreeHost(s.seeds_pinned);
            s.seeds_pinned = nullptr;
            s.seeds_cap = 0;
            if ((e = cudaMallocHost((void**)&s.seeds_pinned, 8 * (size_t)count)) != cudaSuccess)
                return set_cuda_error(e, "serving: pinned seeds");
            s.seeds_cap = count;
        }
        uint8_t* dev_out = s.ws.out;
        if (k > 1) {
            // from the stream-ordered pool (no device-wide synchronisation);
            // the slot's previous solve has finished, so its buffers are free
            const int64_t cap = std::max<int64_t>((d.n + 15) / 16 * 16, 2 * s.word8_cap);
            if (s.word8_cap < (int64_t)(d.n + 15) / 16 * 16) {
                dev_free(s.word8);
                s.word8 = nullptr;
                s.word8_cap = 0;
                if ((e = dev_alloc((void**)&s.word8, 4 * (size_t)kMaxMulti * cap)) != cudaSuccess)
                    return set_cuda_error(e, "serving: multi-seed state");
                s.word8_cap = cap;
            }
            if (s.out_multi_cap < out_bytes) {
                const int64_t ocap = std::max(out_bytes, 2 * s.out_multi_cap);
                dev_free(s.out_multi);
                s.out_multi = nullptr;
                s.out_multi_cap = 0;
                if ((e = dev_alloc((void**)&s.out_multi, (size_t)ocap)) != cudaSuccess)
                    return set_cuda_error(e, "serving: multi-seed results");
                s.out_multi_cap = ocap;
            }
            dev_out = s.out_multi;
        }
        int rc;
        {
            std::lock_guard<std::mutex> glk(g->mu);
            int blocks = serve_blocks_ > 0 ? serve_blocks_ : std::max(1, sms_ / 2);
            if (d.n <= kSingleBlockMax) blocks = 1;
            if (k > 1) {
                uint64_t seeds[kMaxMulti];
                for (int i = 0; i < k; ++i) seeds[i] = rs[i]->seed;
                rc = solve_multi_in(g, s.ws, s.word8, k, seeds, dev_out, s.stream, blocks);
            } else {
                std::vector<uint64_t> seeds((size_t)count);
                for (int32_t i = 0; i < count; ++i) seeds[(size_t)i] = rs[0]->seed + (uint64_t)i;
                rc = solve_in(g, s.ws, seeds.data(), s.seeds_pinned, dev_out, s.stream, blocks);
            }
        }
        if (rc != MIS_OK) return rc;
        if (out_bytes > 0)
            e = cudaMemcpyAsync(s.pinned_out, dev_out, (size_t)out_bytes, cudaMemcpyDeviceToHost,
                                s.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.ctl_pinned, s.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                                s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.stream);
        if (e != cudaSuccess) return set_cuda_error(e, "serving: enqueue");
        return MIS_OK;
    }

    // Caller holds mu_.  Takes the oldest queued request and, when its graph
    // can be solved by the multi-seed kernel, up to kmax - 1 more queued
    // requests on the same graph (searching kGroupScan entries).
    int take_group_locked(Request** rs, int kmax) {
        Request* r = queue_.front();
        queue_.pop_front();
        rs[0] = r;
        int k = 1;
        const GraphData& d = r->g->d;
        const bool groupable = d.count == 0 && d.n > 0 && r->g->path == MIS_PATH_CSR;
        if (!groupable) return k;
        int scanned = 0;
        for (auto it = queue_.begin(); it != queue_.end() && k < kmax && scanned < kGroupScan;
             ++scanned) {
            if ((*it)->g == r->g) {
                rs[k++] = *it;
                it = queue_.erase(it);
            } else {
                ++it;
            }
        }
        return k;
    }

    // Caller holds mu_ (released around the free of a destroyed graph).
    void complete_locked(std::unique_lock<std::mutex>& lk, Request* r, int status) {
        r->t_done = now_ns();
        r->status = status;
        r->done = true;
        mis_graph* g = r->g;
        const int left = g->inflight.fetch_sub(1) - 1;
        if (left == 0 && g->destroy_pending.load()) {
            lk.unlock();
            free_graph(g);
            lk.lock();
        }
        cv_done_.notify_all();
    }

    struct Job {
        Slot* slot = nullptr;
        Request* rs[kMaxMulti] = {};
        int k = 0;
        int64_t need = 0;
        int rc = MIS_OK;
    };

    // Worker w of nw: retires, admits and launches on its own slots (w, w +
    // nw, ...); the queue, the budget and the requests are shared under mu_.
    // A finished slot's results are copied to the callers' buffers without
    // the lock, then its requests are completed under it.
    void loop(int w, int nw) {
        cudaSetDevice(device_);
        std::vector<Job> jobs;
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            bool progressed = false;
            int busy = 0;
            // retire
            for (size_t si = (size_t)w; si < slots_.size(); si += (size_t)nw) {
                Slot& s = slots_[si];
                if (s.nreq == 0) continue;
                const cudaError_t q = cudaEventQuery(s.ev);
                if (q == cudaErrorNotReady) {
                    ++busy;
                    continue;
                }
                const int k = s.nreq;
                Request* rs[kMaxMulti];
                for (int i = 0; i < k; ++i) rs[i] = s.reqs[i];
                int st = MIS_OK;
                if (q != cudaSuccess) {
                    cudaGetLastError();
                    st = MIS_EDEVICE;
                } else {
                    if (s.ctl_pinned->err == kErrTimedOut) st = MIS_ETIMEDOUT;
                    else if (s.ctl_pinned->err != 0) st = MIS_EINTERNAL;
                }
                // the slot and its requests belong to this worker until they
                // are completed: copy the results without holding the lock
                const int64_t nb = rs[0]->g->d.result_bytes;
                lk.unlock();
                if (st == MIS_OK && nb > 0)
                    for (int i = 0; i < k; ++i)
                        std::memcpy(rs[i]->host_out, s.pinned_out + i * nb, (size_t)nb);
                lk.lock();
                s.nreq = 0;
                used_ -= s.charge;
                s.charge = 0;
                for (int i = 0; i < k; ++i) complete_locked(lk, rs[i], st);
                progressed = true;
            }
            // admit: choose slots and groups under the lock ...
            jobs.clear();
            while (!queue_.empty()) {
                Slot* free_slot = nullptr;
                for (size_t si = (size_t)w; si < slots_.size(); si += (size_t)nw)
                    if (slots_[si].nreq == 0) {
                        free_slot = &slots_[si];
                        break;
                    }
                if (!free_slot) break;
                const GraphData& d = queue_.front()->g->d;
                // admission by HBM footprint (a lone request always fits)
                if (used_ > 0 && used_ + charge_for(d, 1) > budget_) break;
                // the largest group that fits the budget and the slot's pinned
                // staging (regrowing that would synchronise the device)
                int kmax = kMaxMulti;
                while (kmax > 1 && used_ > 0 && used_ + charge_for(d, kmax) > budget_) --kmax;
                if (d.result_bytes > 0)
                    kmax = (int)std::max<int64_t>(
                        1, std::min<int64_t>(kmax, free_slot->pinned_cap / d.result_bytes));
                Job j;
                j.slot = free_slot;
                j.k = take_group_locked(j.rs, kmax);
                j.need = charge_for(d, j.k);
                free_slot->nreq = j.k;
                for (int i = 0; i < j.k; ++i) free_slot->reqs[i] = j.rs[i];
                free_slot->charge = j.need;
                used_ += j.need;
                jobs.push_back(j);
            }
            // ... and launch without it, so that submitters and pollers are not
            // held up by the CUDA calls (the requests taken are off the queue)
            if (!jobs.empty()) {
                lk.unlock();
                for (Job& j : jobs) j.rc = launch_unlocked(*j.slot, j.rs, j.k);
                lk.lock();
                for (Job& j : jobs) {
                    if (j.rc != MIS_OK) {
                        j.slot->nreq = 0;
                        used_ -= j.need;
                        j.slot->charge = 0;
                        for (int i = 0; i < j.k; ++i) complete_locked(lk, j.rs[i], j.rc);
                    } else {
                        ++busy;
                    }
                }
                progressed = true;
            }
            if (stop_ && queue_.empty() && busy == 0) break;
            if (!progressed) {
                if (busy == 0 && queue_.empty()) {
                    cv_work_.wait(lk);
                } else {
                    // solves in flight: poll again at once (a timed sleep rounds
                    // up to the host's timer slack, tens of microseconds, which
                    // delays every retirement and admission behind it)
                    lk.unlock();
                    std::this_thread::yield();
                    lk.lock();
                }
            }
        }
    }

    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::list<Request*> queue_;  // list: grouping erases from the middle
    std::unordered_map<mis_ticket, Request*> reqs_;
    std::deque<Slot> slots_;  // all max_slots_ made at start; slots never move
    std::vector<std::thread> threads_;
    bool running_ = false;
    bool stop_ = false;
    int device_ = 0;
    int max_slots_ = kDefaultSlots;
    int64_t budget_ = 0;
    int64_t used_ = 0;
    int serve_blocks_ = 0;
    int sms_ = 1;
    mis_ticket next_id_ = 1;
};

}  // namespace

void serve_release_graph(mis_graph* g) { Server::get().release(g); }

}  // namespace tcmis

using namespace tcmis;

extern "C" {

int mis_submit(mis_graph* g, uint64_t seed, uint8_t* out_status, mis_ticket* ticket) {
    clear_error();
    return Server::get().submit(g, seed, out_status, ticket);
}

int mis_poll(mis_ticket t) {
    clear_error();
    return Server::get().poll(t);
}

int mis_poll_ex(mis_ticket t, int64_t* latency_ns) {
    clear_error();
    return Server::get().poll(t, latency_ns);
}

int mis_wait(mis_ticket t, int64_t timeout_us) {
    clear_error();
    return Server::get().wait(t, timeout_us);
}

int mis_serve_configure(const mis_options* opt) {
    clear_error();
    return Server::get().configure(opt);
}

void mis_serve_shutdown(void) { Server::get().shutdown(); }

}  // extern "C"
