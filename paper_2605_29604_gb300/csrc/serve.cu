// serve.cu -- continuous-batching request loop (mis_submit / mis_poll / mis_wait).
//
// One scheduler thread per process owns up to max_slots solve slots.  A slot
// holds a CUDA stream, an event, a solve workspace (grown on demand) and
// pinned staging for the result.  The scheduler loops:
//
//   retire   every slot whose event has fired: copy its result bytes to the
//            caller's host buffer, record the status, release the slot;
//   admit    queued requests, oldest first, while a slot is free and the
//            workspace bytes of all admitted requests stay within the HBM
//            budget (a request is always admitted when nothing runs);
//   launch   each admitted request on its slot's stream: graphs of up to
//            kSingleBlockMax vertices run the round kernel as one block
//            through an ordinary launch, larger ones a cooperative grid of at
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
    Request* req = nullptr;
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
        cv_work_.notify_one();
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
        std::thread th;
        {
            std::lock_guard<std::mutex> lk(mu_);
            if (!running_) return;
            stop_ = true;
            cv_work_.notify_all();
            th = std::move(thread_);
        }
        if (th.joinable()) th.join();
        std::lock_guard<std::mutex> lk(mu_);
        cudaSetDevice(device_);
        for (Slot& s : slots_) {
            if (s.stream) cudaStreamSynchronize(s.stream);
            ws_free(s.ws);
            if (s.pinned_out) cudaFreeHost(s.pinned_out);
            if (s.seeds_pinned) cudaFreeHost(s.seeds_pinned);
            if (s.ctl_pinned) cudaFreeHost(s.ctl_pinned);
            if (s.ev) cudaEventDestroy(s.ev);
            if (s.stream) cudaStreamDestroy(s.stream);
        }
        slots_.clear();
        running_ = false;
        stop_ = false;
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
        thread_ = std::thread([this] { loop(); });
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

    // Caller holds mu_.  Starts request r on slot s; MIS_OK or an error (the
    // request is then finished with that error by the caller).
    int launch_locked(Slot& s, Request* r) {
        mis_graph* g = r->g;
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
        if (s.pinned_cap < d.result_bytes) {
            if (s.pinned_out) cudaFreeHost(s.pinned_out);
            s.pinned_out = nullptr;
            if ((e = cudaMallocHost((void**)&s.pinned_out, (size_t)d.result_bytes)) != cudaSuccess)
                return set_cuda_error(e, "serving: pinned result");
            s.pinned_cap = d.result_bytes;
        }
        const int32_t count = std::max(1, d.count);
        if (s.seeds_cap < count) {
            if (s.seeds_pinned) cudaFreeHost(s.seeds_pinned);
            s.seeds_pinned = nullptr;
            if ((e = cudaMallocHost((void**)&s.seeds_pinned, 8 * (size_t)count)) != cudaSuccess)
                return set_cuda_error(e, "serving: pinned seeds");
            s.seeds_cap = count;
        }
        std::vector<uint64_t> seeds((size_t)count);
        for (int32_t i = 0; i < count; ++i) seeds[(size_t)i] = r->seed + (uint64_t)i;
        int rc;
        {
            std::lock_guard<std::mutex> glk(g->mu);
            int blocks = serve_blocks_ > 0 ? serve_blocks_ : std::max(1, sms_ / 2);
            if (d.n <= kSingleBlockMax) blocks = 1;
            rc = solve_in(g, s.ws, seeds.data(), s.seeds_pinned, s.ws.out, s.stream, blocks);
        }
        if (rc != MIS_OK) return rc;
        if (d.result_bytes > 0)
            e = cudaMemcpyAsync(s.pinned_out, s.ws.out, (size_t)d.result_bytes,
                                cudaMemcpyDeviceToHost, s.stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(s.ctl_pinned, s.ws.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost,
                                s.stream);
        if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.stream);
        if (e != cudaSuccess) return set_cuda_error(e, "serving: enqueue");
        s.req = r;
        return MIS_OK;
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

    void loop() {
        cudaSetDevice(device_);
        std::unique_lock<std::mutex> lk(mu_);
        for (;;) {
            bool progressed = false;
            int busy = 0;
            // retire
            for (Slot& s : slots_) {
                if (!s.req) continue;
                const cudaError_t q = cudaEventQuery(s.ev);
                if (q == cudaErrorNotReady) {
                    ++busy;
                    continue;
                }
                Request* r = s.req;
                s.req = nullptr;
                used_ -= s.charge;
                s.charge = 0;
                int st = MIS_OK;
                if (q != cudaSuccess) {
                    cudaGetLastError();
                    st = MIS_EDEVICE;
                } else {
                    if (r->g->d.result_bytes > 0)
                        std::memcpy(r->host_out, s.pinned_out, (size_t)r->g->d.result_bytes);
                    if (s.ctl_pinned->err == kErrTimedOut) st = MIS_ETIMEDOUT;
                    else if (s.ctl_pinned->err != 0) st = MIS_EINTERNAL;
                }
                complete_locked(lk, r, st);
                progressed = true;
            }
            // admit and launch
            while (!queue_.empty()) {
                Slot* free_slot = nullptr;
                for (Slot& s : slots_)
                    if (!s.req) {
                        free_slot = &s;
                        break;
                    }
                if (!free_slot && (int)slots_.size() < max_slots_) {
                    slots_.emplace_back();
                    free_slot = &slots_.back();
                }
                if (!free_slot) break;
                Request* r = queue_.front();
                const GraphData& d = r->g->d;
                const int64_t need = ws_bytes_for(d.n, d.count) + d.result_bytes;
                if (used_ > 0 && used_ + need > budget_) break;  // admission by HBM footprint
                queue_.pop_front();
                const int rc = launch_locked(*free_slot, r);
                if (rc != MIS_OK) {
                    complete_locked(lk, r, rc);
                } else {
                    free_slot->charge = need;
                    used_ += need;
                    ++busy;
                }
                progressed = true;
            }
            if (stop_ && queue_.empty() && busy == 0) break;
            if (!progressed) {
                if (busy == 0 && queue_.empty()) {
                    cv_work_.wait(lk);
                } else {
                    lk.unlock();
                    std::this_thread::sleep_for(std::chrono::microseconds(5));
                    lk.lock();
                }
            }
        }
    }

    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::deque<Request*> queue_;
    std::unordered_map<mis_ticket, Request*> reqs_;
    std::deque<Slot> slots_;  // deque: slots never move once created
    std::thread thread_;
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
