// serve.cu -- the serving loop behind dmul_submit / dmul_poll / dmul_wait.
#include "serve.h"

namespace dml {

Server::Server(dmul_ctx *c) : ctx_(c) {
    cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking);
    worker_ = std::thread([this] { loop(); });
}

Server::~Server() {
    {
        std::lock_guard<std::mutex> g(mu_);
        stop_ = true;
    }
    cv_.notify_all();
    if (worker_.joinable()) worker_.join();
    if (stream_) cudaStreamDestroy(stream_);
}

int Server::submit(const dmul_job &job, uint64_t *ticket) {
    std::lock_guard<std::mutex> g(mu_);
    uint64_t t = next_++;
    tickets_[t].job = job;
    queue_.push_back(t);
    *ticket = t;
    cv_.notify_one();
    return DMUL_OK;
}

int Server::poll(uint64_t ticket, int *done) {
    std::lock_guard<std::mutex> g(mu_);
    auto it = tickets_.find(ticket);
    if (it == tickets_.end()) return DMUL_ERR_UNKNOWN_TICKET;
    *done = it->second.done ? 1 : 0;
    return DMUL_OK;
}

int Server::wait(uint64_t ticket) {
    std::unique_lock<std::mutex> g(mu_);
    auto it = tickets_.find(ticket);
    if (it == tickets_.end()) return DMUL_ERR_UNKNOWN_TICKET;
    done_cv_.wait(g, [&] { return tickets_[ticket].done; });
    return tickets_[ticket].status;
}

void Server::loop() {
    for (;;) {
        uint64_t t;
        dmul_job job;
        {
            std::unique_lock<std::mutex> g(mu_);
            cv_.wait(g, [&] { return stop_ || !queue_.empty(); });
            if (stop_ && queue_.empty()) return;
            t = queue_.front();
            queue_.pop_front();
            job = tickets_[t].job;
        }
        int rc = ctx_enqueue_mul(ctx_, job, stream_);
        if (rc == DMUL_OK) rc = dmul_sync(ctx_, stream_);
        {
            std::lock_guard<std::mutex> g(mu_);
            tickets_[t].status = rc;
            tickets_[t].done = true;
        }
        done_cv_.notify_all();
    }
}

}  // namespace dml
