// ctx.h -- the library context and the helpers the plain, batched and served forms share.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <tuple>
#include <memory>
#include <mutex>
#include <vector>

#include "../../include/dmul.h"
#include "kernels.cuh"
#include "plan.h"

namespace dml {

struct PlanEntry {
    HostPlan hp;
    PlanDev pd;
    void *dtables = nullptr;  // one allocation holding the three per-prime tables
    size_t bytes = 0;
};

struct SmallPlanEntry {
    SmallPlanDev sp;
    void *dtables = nullptr;
    size_t bytes = 0;
};

struct StageTimer {
    const char *name;
    double ms = 0;
    uint64_t launches = 0;
};

class Server;

constexpr int kBatchStreams = 4;
constexpr int kMaxSmallPlans = 32;  // distinct short transform lengths (there are 17)

struct GroupLaunch {
    bool small;
    uint64_t N;
    size_t first, count;   // range in the descriptor array
    uint32_t maxtiles;
    bool aligned = false;  // every operand of the group 16-byte aligned (specialized kernels allowed)
};

struct BatchState {
    uint8_t *arena = nullptr;
    size_t arena_cap = 0;
    JobDev *djobs = nullptr;
    JobDev *hjobs = nullptr;  // pinned
    size_t jobs_cap = 0;
    cudaStream_t streams[kBatchStreams] = {};
    cudaEvent_t fork = nullptr, join[kBatchStreams] = {};
    cudaEvent_t done = nullptr;  // recorded after each batch launched on this state
    SmallPlanDev *dplans = nullptr, *hplans = nullptr;  // plans of the short products (device, pinned)
    uint32_t *dcounter = nullptr;                       // job counter of the persistent launch
    bool done_recorded = false;
    // per-job status: one device word per descriptor (zeroed with the descriptor upload), copied
    // to the pinned hstat at the end of the batch; order[i] = the caller's index of descriptor i
    uint32_t *dstat = nullptr, *hstat = nullptr;
    std::vector<size_t> order;
    size_t launched = 0;  // descriptors of the last batch launched on this state
    // dmul_batch: the caller's job array whose status fields the next flush fills
    dmul_job *pend_jobs = nullptr;
    bool pending = false;
    // graph cache keyed by the batch shape
    std::map<std::vector<std::tuple<int, uint64_t, size_t>>, cudaGraphExec_t> graphs;
};

// First-use times (ms, cold L2) of a lone short product on each path; a path not timed keeps
// the 1e30 of "not a candidate" (its *_timed flag tells it apart from one that failed to run).
struct ShortTimes {
    float small = 1e30f, four = 1e30f, fused = 1e30f;
    bool small_timed = false, fused_timed = false;
};



}  // namespace dml

struct dmul_ctx {
    int device = 0;
    dmul_config cfg{};
    uint64_t budget = 0;
    uint64_t used = 0;  // library-owned device bytes
    std::map<uint64_t, std::unique_ptr<dml::PlanEntry>> plans;
    std::map<uint64_t, std::unique_ptr<dml::SmallPlanEntry>> small_plans;
    std::map<uint64_t, bool> small_single;  // per short length: small kernel faster than four-step
    std::map<uint64_t, dml::ShortTimes> short_times;  // per lone short product's lengths (Ns, N)
    std::map<uint64_t, std::unique_ptr<dml::PlanEntry>> fused_plans;  // N1 x 256 plans of the fused kernel
    mutable std::mutex small_mu;            // guards small_single, short_times (read by dmul_submit callers)
    // scratch of the plain form (one set, used by one call at a time)
    uint32_t *X = nullptr, *Y = nullptr;
    size_t res_words = 0;  // capacity of X and of Y, in words
    uint2 *spill = nullptr;
    size_t spill_cap = 0;
    void *ctl = nullptr;
    size_t ctl_cap = 0;
    uint32_t *status = nullptr;  // device status word
    // per-prime hand-off counters from the forward column pass to the row pass (device, never
    // reset) and the host's running total of the columns the plain path has sent through them
    uint32_t *fwd_sync = nullptr;
    uint32_t fwd_cols = 0;
    // the fused short-product kernel's grid barrier word (in fwd_sync's allocation; never reset)
    uint32_t *grid_sync = nullptr;
    // bound of every device-side wait of this context's kernels, in polls (0: the defaults;
    // DMUL_FLAG_SHORT_WAITS makes it short, so that tests can make a wait run out quickly)
    uint32_t spin_limit = 0;
    // host-buffer path staging
    uint32_t *hx = nullptr, *hy = nullptr;  // operand staging (pageable operands), h_in_cap words each
    uint32_t *hz = nullptr;                 // digit sums (and, staged, the limbs), h_cap words
    uint64_t *hnz = nullptr;
    size_t h_cap = 0, h_in_cap = 0;
    uint64_t *h_tail_dev = nullptr;         // device address of h_tail
    uint64_t *h_tail = nullptr;            // pinned: [0] normalized length, [1] status word
    cudaStream_t copy_stream = nullptr;    // uploads of the second operand
    cudaEvent_t ev_start = nullptr, ev_y = nullptr;
    cudaStream_t own_stream = nullptr;
    cudaStream_t last_stream = nullptr;
    // stage timing
    bool timing = false;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pool;
    size_t ev_used = 0;
    std::vector<std::pair<int, size_t>> ev_log;  // (stage id, event pair index)
    std::vector<dml::StageTimer> timers;
    // batched form
    std::unique_ptr<dml::BatchState> batch;
    int batch_err = DMUL_OK;  // a batch job's device error found before the next dmul_sync
    // serving (created on the first dmul_submit, under server_mu)
    std::mutex server_mu;
    std::unique_ptr<dml::Server> server;
};

namespace dml {

enum StageId { kStColFwd = 0, kStRowMul, kStColInv, kStCarry, kStTranspose, kStRowDft, kStCrt,
               kStPack, kStSmall, kStBatch, kStFused, kNumStages };

int set_device(dmul_ctx *c);
int dev_alloc(dmul_ctx *c, void **p, size_t bytes);
void dev_free(dmul_ctx *c, void *p, size_t bytes);
int get_plan(dmul_ctx *c, uint64_t N, PlanEntry **out);
int get_small_plan(dmul_ctx *c, uint64_t N, SmallPlanEntry **out);
// The plain form's residue buffers (3 N words each), spills and carry control block for L limbs.
int ensure_scratch(dmul_ctx *c, uint64_t N, uint64_t L, bool need_y);
bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes);
uint64_t max_min_limbs();

// RAII CUDA-event pair around a stage when the context records stage timings.
struct Timed {
    dmul_ctx *c;
    int id;
    cudaStream_t s;
    size_t idx = 0;
    Timed(dmul_ctx *c_, int id_, cudaStream_t s_);
    ~Timed();
};

void destroy_batch_state(dmul_ctx *c);
// priority: of the state's fork/join streams (0, the default, or a value of
// cudaDeviceGetStreamPriorityRange)
int init_batch_state(BatchState *b, int priority = 0);
void free_batch_state(dmul_ctx *c, BatchState *b);
// One batch on a given state (arena, descriptors); device errors go to *status.  use_graph:
// capture/replay per batch shape with groups forked over the state's streams; otherwise plain
// launches on s (fork_plain: forked over the state's streams, joined back to s).
//
// A size class of short products with fewer jobs than it would take to fill the GPU with clusters
// runs as four-step groups instead when a lone product of that length is faster there (the
// plain form's measured choice, prefer_small_single).  four_ok (null: every job) marks the jobs
// whose scratch allows that: the serving loop admits a short job's four-step scratch only when the
// choice was already known at submission.
//
// Per job: host_status[i] (every entry written) receives the job's host-side verdict -- DMUL_OK
// for a job that was launched, else the code that rejected it (bad pointers or sizes, capacity,
// aliasing, too large); rejected jobs are left out of the launch.  The device-side status of each
// launched job lands in b->hstat[i] for descriptor i (job b->order[i]) once the stream has
// passed the batch (b->done).
int run_batch_on(dmul_ctx *c, BatchState *b, const dmul_job *jobs, size_t count, cudaStream_t s,
                 uint32_t *status, bool use_graph, int *host_status, const uint8_t *four_ok = nullptr,
                 bool fork_plain = false);
// DMUL_OK, DMUL_ERR_TIMEOUT or DMUL_ERR_INVALID for a device status word.
inline int device_code(uint32_t st) {
    return !st ? DMUL_OK : ((st & kStatusTimeout) ? DMUL_ERR_TIMEOUT : DMUL_ERR_INVALID);
}
// Waits for the last dmul_batch on b, writes each launched job's final status into the caller's
// array and returns the first device-side error among them (DMUL_OK if none, or nothing pending).
int flush_batch_status(BatchState *b);
// Library scratch a job needs on the four-step path: 0 for a short product, unless the measured
// choice for its length is the four-step pipeline (then *four = true, when four is non-null).
size_t job_scratch_bytes(const dmul_ctx *c, const dmul_job &j, bool *four = nullptr);
// The measured choice for short products of transform length Ns: 1 the small kernel (one cluster),
// 0 the four-step pipeline, -1 not measured yet.
int small_single_cached(const dmul_ctx *c, uint64_t Ns);
int prefer_small_single(dmul_ctx *c, uint64_t Ns, uint64_t N, bool *use_small);

}  // namespace dml
