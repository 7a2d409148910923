// serve.h -- batched and served forms of libdmul (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "../../include/dmul.h"

namespace dml {

// One multiplication enqueued on stream s through the plain pipeline (api.cu).
int ctx_enqueue_mul(dmul_ctx *c, const dmul_job &j, cudaStream_t s);

// dmul_batch implementation (batch.cu).
int run_batch(dmul_ctx *c, const dmul_job *jobs, size_t count, cudaStream_t s);

// The serving loop behind dmul_submit / dmul_poll / dmul_wait (serve.cu).
class Server {
  public:
    explicit Server(dmul_ctx *c);
    ~Server();
    int submit(const dmul_job &job, uint64_t *ticket);
    int poll(uint64_t ticket, int *done);
    int wait(uint64_t ticket);

  private:
    struct Ticket {
        dmul_job job;
        int status = DMUL_OK;
        bool done = false;
    };
    void loop();
    dmul_ctx *ctx_;
    std::mutex mu_;
    std::condition_variable cv_, done_cv_;
    std::deque<uint64_t> queue_;
    std::map<uint64_t, Ticket> tickets_;
    uint64_t next_ = 1;
    bool stop_ = false;
    cudaStream_t stream_ = nullptr;
    std::thread worker_;
};

}  // namespace dml
