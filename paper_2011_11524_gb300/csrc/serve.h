// serve.h -- batched and served forms of libdmul (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dmul.h"
#include "ctx.h"

namespace dml {

// One multiplication enqueued on stream s through the plain pipeline (api.cu).
int ctx_enqueue_mul(dmul_ctx *c, const dmul_job &j, cudaStream_t s);

// dmul_batch implementation (batch.cu).
int run_batch(dmul_ctx *c, dmul_job *jobs, size_t count, cudaStream_t s);

// The serving loop behind dmul_submit / dmul_poll / dmul_wait (serve.cu).
//
// Continuous batching: a worker thread keeps up to kSlots batches in flight, each on its own
// stream with its own scratch.  Whenever a slot is free it takes every pending request (FIFO) whose
// scratch still fits the admission budget, launches them as one batch (grouped by transform
// length, see batch.cu) and returns to the queue; requests that arrive while batches run join the
// next one.  Scratch comes from the server's stream-ordered memory pool (allocated and freed on
// the slot's stream), so admitting and retiring batches never synchronizes the device.  A slot's
// completion is an event recorded after its batch, which the worker polls while anything is in
// flight (and for kIdlePollUs after its last activity) instead of sleeping: a completion or a new
// request is seen within microseconds, at the price of one host core kept busy meanwhile.
//
// Short requests (transform length <= 24576, the one-cluster class) queue apart from long ones.
// kShortSlots extra slots take short requests only, on streams of the highest priority, so that a
// short request waits neither for a long request batched with it nor for a free general slot, and
// the GPU's block scheduler runs its CTAs ahead of a long batch's as SMs free up; the kSlots
// general slots take long requests first and short ones when no long one is queued.
class Server {
  public:
    explicit Server(dmul_ctx *c);
    ~Server();
    int submit(const dmul_job &job, uint64_t *ticket);
    int poll(uint64_t ticket, int *done);
    int wait(uint64_t ticket);
    void stats(dmul_serve_info *out);

    static constexpr int kSlots = 4;       // general slots
    static constexpr int kShortSlots = 2;  // short requests only, highest stream priority
    static constexpr size_t kMaxBatch = 1024;
    static constexpr int kIdlePollUs = 300;  // the worker keeps polling this long after its last activity

  private:
    struct Ticket {
        dmul_job job;
        size_t bytes = 0;
        bool four = false;  // its scratch covers the four-step path (a short job; see run_batch_on)
        bool short_job = false;  // the one-cluster length class: queue_[0]
        int status = DMUL_OK;
        bool done = false;
    };
    struct Slot {
        Server *owner = nullptr;
        BatchState bs;
        cudaStream_t stream = nullptr;
        cudaEvent_t done_ev = nullptr;  // recorded after each batch (the worker polls it)
        uint32_t *status = nullptr;  // launch status word of this slot's batches (every job also
                                     // has its own, in the batch state: bs.hstat / bs.order)
        std::vector<uint64_t> tickets;  // the batch's requests, in the order they were passed
        size_t bytes = 0;
        void *arena = nullptr;
        bool busy = false;
        bool finished = false;
        bool short_only = false;
    };
    void complete(Slot &s, int rc);
    void loop();
    void retire(Slot &s, std::unique_lock<std::mutex> &g);
    bool launch(Slot &s, int q, std::unique_lock<std::mutex> &g);

    dmul_ctx *ctx_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::deque<uint64_t> queue_[2];  // [0] short requests, [1] long ones (FIFO each)
    std::unordered_map<uint64_t, Ticket> tickets_;  // issued and not yet released
    uint64_t next_ = 1;
    uint64_t running_ = 0;  // requests in launched batches
    std::atomic<uint64_t> gen_{0};  // bumped by every submission and by shutdown (the worker's wake-up)
    uint64_t peak_running_ = 0;
    bool stop_ = false;
    bool init_ok_ = false;
    bool mem_blocked_[2] = {false, false};  // a queue's head waits for in-flight scratch to be released
    std::vector<std::unique_ptr<Slot>> slots_;
    size_t budget_ = 0, inflight_ = 0;
    cudaMemPool_t pool_ = nullptr;  // in-flight scratch (stream-ordered, kept mapped up to budget_)
    std::thread worker_;
};

}  // namespace dml
