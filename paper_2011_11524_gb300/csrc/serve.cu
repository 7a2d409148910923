// serve.cu -- the serving loop behind dmul_submit / dmul_poll / dmul_wait (see serve.h).
#include "serve.h"

#include <algorithm>
#include <chrono>

namespace dml {

Server::Server(dmul_ctx *c) : ctx_(c) {
    set_device(c);
    // admission budget for in-flight scratch: what the context's HBM budget leaves free now
    budget_ = c->budget > c->used ? (c->budget - c->used) : 0;
    init_ok_ = true;
    // A stream-ordered pool of its own that keeps up to the admission budget mapped between
    // batches.  The default pool returns freed memory to the CUDA driver at every synchronization, so
    // each large batch would map its scratch afresh (hundreds of microseconds for tens of MB).
    int dev = 0;
    cudaGetDevice(&dev);
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if (cudaMemPoolCreate(&pool_, &props) != cudaSuccess) {
        pool_ = nullptr;
        init_ok_ = false;
    } else {
        uint64_t keep = budget_;
        if (cudaMemPoolSetAttribute(pool_, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess)
            init_ok_ = false;
    }
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    for (int i = 0; i < kSlots + kShortSlots; ++i) {
        auto s = std::make_unique<Slot>();
        s->owner = this;
        s->short_only = i >= kSlots;
        if (cudaStreamCreateWithPriority(&s->stream, cudaStreamNonBlocking, s->short_only ? greatest : least) !=
            cudaSuccess)
            init_ok_ = false;
        if (cudaEventCreateWithFlags(&s->done_ev, cudaEventDisableTiming) != cudaSuccess) init_ok_ = false;
        if (cudaMalloc(&s->status, 64) != cudaSuccess || cudaMemset(s->status, 0, 64) != cudaSuccess)
            init_ok_ = false;
        if (init_batch_state(&s->bs, s->short_only ? greatest : least) != DMUL_OK) init_ok_ = false;
        slots_.push_back(std::move(s));
    }
    worker_ = std::thread([this] { loop(); });
}

Server::~Server() {
    {
        std::lock_guard<std::mutex> g(mu_);
        stop_ = true;
        gen_.fetch_add(1, std::memory_order_release);
    }
    cv_.notify_all();
    if (worker_.joinable()) worker_.join();
    set_device(ctx_);
    for (auto &s : slots_) {
        if (s->stream) cudaStreamSynchronize(s->stream);
        free_batch_state(ctx_, &s->bs);
        if (s->status) cudaFree(s->status);
        if (s->done_ev) cudaEventDestroy(s->done_ev);
        if (s->stream) cudaStreamDestroy(s->stream);
    }
    if (pool_) cudaMemPoolDestroy(pool_);
}

int Server::submit(const dmul_job &job, uint64_t *ticket) {
    if (!init_ok_) return DMUL_ERR_CUDA;
    if (!job.x || !job.y || !job.z || job.nx == 0 || job.ny == 0) return DMUL_ERR_INVALID;
    const uint64_t L = job.nx + job.ny;
    if (job.z_cap < L) return DMUL_ERR_CAPACITY;
    if (!choose_N_small(L) && !choose_N(L)) return DMUL_ERR_TOO_LARGE;
    bool four = false;
    const size_t bytes = job_scratch_bytes(ctx_, job, &four);
    if (bytes > budget_) return DMUL_ERR_NOMEM;
    const bool short_job = choose_N_small(L) && !(ctx_->cfg.flags & (DMUL_FLAG_SIXSTEP | DMUL_FLAG_NO_SMALL));
    std::lock_guard<std::mutex> g(mu_);
    uint64_t t = next_++;
    Ticket &tk = tickets_[t];
    tk.job = job;
    tk.bytes = bytes;
    tk.four = four;
    tk.short_job = short_job;
    queue_[short_job ? 0 : 1].push_back(t);
    gen_.fetch_add(1, std::memory_order_release);
    *ticket = t;
    cv_.notify_all();
    return DMUL_OK;
}

// A ticket's result is handed out once: the dmul_poll that sees it done, or dmul_wait, releases
// it, so the table holds only tickets that are queued, running or completed and unclaimed.
int Server::poll(uint64_t ticket, int *done) {
    std::lock_guard<std::mutex> g(mu_);
    auto it = tickets_.find(ticket);
    if (it == tickets_.end()) return DMUL_ERR_UNKNOWN_TICKET;
    if (!it->second.done) {
        *done = 0;
        return DMUL_OK;
    }
    *done = 1;
    const int rc = it->second.status;
    tickets_.erase(it);
    return rc;
}

int Server::wait(uint64_t ticket) {
    std::unique_lock<std::mutex> g(mu_);
    if (tickets_.find(ticket) == tickets_.end()) return DMUL_ERR_UNKNOWN_TICKET;
    // looked up on every wake-up: another thread may release the ticket meanwhile
    done_cv_.wait(g, [&] {
        auto it = tickets_.find(ticket);
        return it == tickets_.end() || it->second.done;
    });
    auto it = tickets_.find(ticket);
    if (it == tickets_.end()) return DMUL_ERR_UNKNOWN_TICKET;
    const int rc = it->second.status;
    tickets_.erase(it);
    return rc;
}

void Server::stats(dmul_serve_info *out) {
    std::lock_guard<std::mutex> g(mu_);
    out->queued = queue_[0].size() + queue_[1].size();
    out->running = running_;
    out->held = tickets_.size();
    out->peak_running = peak_running_;
    out->admit_budget_bytes = budget_;
    out->inflight_bytes = inflight_;
}

// The worker saw the slot's completion event (the batch, and the copy of its jobs' status words,
// are done): complete each launched ticket with its own job's status; rc != DMUL_OK (the event
// reported a failure) completes them all with rc.  Called with the lock held.
void Server::complete(Slot &s, int rc) {
    const BatchState &b = s.bs;
    for (size_t i = 0; i < b.launched; ++i) {
        auto it = tickets_.find(s.tickets[b.order[i]]);
        if (it == tickets_.end()) continue;
        it->second.status = rc ? rc : device_code(((volatile uint32_t *)b.hstat)[i]);
        it->second.done = true;
    }
    running_ -= b.launched;
    s.tickets.clear();
    s.finished = true;
    done_cv_.notify_all();
}

// A finished slot (its tickets already completed by complete()): release its budget.
void Server::retire(Slot &s, std::unique_lock<std::mutex> &g) {
    (void)g;
    s.busy = false;
    s.finished = false;
    inflight_ -= s.bytes;
    s.bytes = 0;
}

// Admit pending requests of queue q into a free slot and launch them as one batch.
bool Server::launch(Slot &s, int q, std::unique_lock<std::mutex> &g) {
    std::vector<dmul_job> jobs;
    std::vector<uint8_t> four;
    size_t bytes = 0;
    std::deque<uint64_t> &queue = queue_[q];
    while (!queue.empty() && jobs.size() < kMaxBatch) {
        Ticket &tk = tickets_[queue.front()];
        if (inflight_ + bytes + tk.bytes > budget_) break;  // wait for memory to free up
        bytes += tk.bytes;
        jobs.push_back(tk.job);
        four.push_back(tk.four ? 1 : 0);
        s.tickets.push_back(queue.front());
        queue.pop_front();
    }
    if (jobs.empty()) return false;
    std::vector<int> hs(jobs.size(), DMUL_OK);
    const std::vector<uint64_t> tick = s.tickets;
    s.busy = true;
    s.bytes = bytes;
    inflight_ += bytes;
    running_ += jobs.size();
    peak_running_ = std::max(peak_running_, running_);
    g.unlock();
    int rc = DMUL_OK;
    void *arena = nullptr;
    if (bytes) {
        if (cudaMallocFromPoolAsync(&arena, bytes, pool_, s.stream) != cudaSuccess) rc = DMUL_ERR_NOMEM;
    }
    if (rc == DMUL_OK) {
        // the scratch of this batch is the pool allocation; the state never reallocates it
        s.bs.arena = (uint8_t *)arena;
        s.bs.arena_cap = bytes;
        // the batch spreads its groups (transform lengths, short classes) over the state's
        // streams, which have the slot's priority
        rc = run_batch_on(ctx_, &s.bs, jobs.data(), jobs.size(), s.stream, s.status, false, hs.data(), four.data(),
                          true);
        s.bs.arena = nullptr;
        s.bs.arena_cap = 0;
    }
    if (arena) cudaFreeAsync(arena, s.stream);
    if (rc == DMUL_OK && cudaEventRecord(s.done_ev, s.stream) != cudaSuccess) rc = DMUL_ERR_CUDA;
    g.lock();
    if (rc != DMUL_OK) {
        // nothing of this batch will complete on the stream (no completion event was recorded)
        for (uint64_t t : tick) {
            tickets_[t].status = rc;
            tickets_[t].done = true;
        }
        running_ -= tick.size();
        s.tickets.clear();
        s.busy = false;
        inflight_ -= s.bytes;
        s.bytes = 0;
        done_cv_.notify_all();
    } else {
        // requests the host checks rejected were left out of the launch: they complete now, with
        // their own code; the launched ones complete when the slot's event does
        bool any = false;
        for (size_t k = 0; k < hs.size(); ++k)
            if (hs[k]) {
                tickets_[tick[k]].status = hs[k];
                tickets_[tick[k]].done = true;
                --running_;
                any = true;
            }
        if (any) done_cv_.notify_all();
    }
    return true;
}

// The worker: launches admitted requests into free slots and completes slots whose event has
// passed.  While a batch is in flight, or for a short while after the last activity, it polls
// instead of sleeping, so that a completion or a new request is seen within microseconds rather
// than after a host callback and a thread wake-up; otherwise it sleeps until a request arrives.
// The polling itself takes no lock: the slots' busy / finished flags are written by this thread
// only, the events are queried without the lock, and new requests (or shutdown) show as a change
// of gen_; the lock is taken only when there is something to do, so submitting and polling
// threads never queue behind the worker.
void Server::loop() {
    set_device(ctx_);
    auto last = std::chrono::steady_clock::now();
    uint64_t seen = gen_.load(std::memory_order_acquire) - 1;  // the first pass looks at everything
    std::vector<int> done(slots_.size());
    for (;;) {
        bool any_done = false, any_busy = false;
        for (size_t i = 0; i < slots_.size(); ++i) {
            done[i] = -1;
            Slot &s = *slots_[i];
            if (!s.busy || s.finished) continue;
            any_busy = true;
            const cudaError_t q = cudaEventQuery(s.done_ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) cudaGetLastError();
            done[i] = q == cudaSuccess ? DMUL_OK : DMUL_ERR_CUDA;
            any_done = true;
        }
        const uint64_t gen = gen_.load(std::memory_order_acquire);
        auto now = std::chrono::steady_clock::now();
        if (!any_done && gen == seen) {
            if (any_busy || now - last < std::chrono::microseconds(kIdlePollUs)) {
                std::this_thread::yield();
                continue;
            }
            std::unique_lock<std::mutex> g(mu_);
            cv_.wait(g, [&] { return gen_.load(std::memory_order_acquire) != seen; });
            last = std::chrono::steady_clock::now();
            continue;
        }
        seen = gen;
        last = now;
        std::unique_lock<std::mutex> g(mu_);
        for (size_t i = 0; i < slots_.size(); ++i)
            if (done[i] >= 0) complete(*slots_[i], done[i]);
        for (auto &s : slots_)
            if (s->busy && s->finished) {
                retire(*s, g);
                mem_blocked_[0] = mem_blocked_[1] = false;  // memory came back: retry the heads
            }
        any_busy = false;
        for (auto &s : slots_) any_busy |= s->busy;
        if (stop_) {
            if (any_busy) continue;  // the batches in flight complete first
            for (auto &queue : queue_) {
                for (uint64_t t : queue) {  // never started: the context is going away
                    tickets_[t].status = DMUL_ERR_INVALID;
                    tickets_[t].done = true;
                }
                queue.clear();
            }
            done_cv_.notify_all();
            return;
        }
        for (auto &s : slots_) {
            if (s->busy) continue;
            // a short-only slot takes short requests; a general one long requests first
            const int order[2] = {s->short_only ? 0 : 1, s->short_only ? -1 : 0};
            for (int q : order) {
                if (q < 0 || queue_[q].empty() || mem_blocked_[q]) continue;
                if (launch(*s, q, g)) {
                    any_busy = true;
                    break;
                }
                // the head request does not fit the admission budget next to the batches in
                // flight: wait for one of them to retire
                mem_blocked_[q] = any_busy;
                if (!any_busy) {  // cannot happen (submit rejects such requests); fail it
                    Ticket &tk = tickets_[queue_[q].front()];
                    tk.status = DMUL_ERR_NOMEM;
                    tk.done = true;
                    queue_[q].pop_front();
                    done_cv_.notify_all();
                }
            }
        }
        // requests that arrived while this pass held (or dropped, in launch) the lock are seen
        // by the next pass through gen_; a queue left non-empty because every slot is busy waits
        // for a completion
    }
}

}  // namespace dml
