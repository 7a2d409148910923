// api.cu -- the C ABI of libdmul (include/dmul.h): contexts, plan cache, scratch, the pipeline.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/dmul.h"
#include "kernels.cuh"
#include "plan.h"
#include "ctx.h"
#include "serve.h"

using namespace dml;

namespace dml {

// Bound of every device-side wait under DMUL_FLAG_SHORT_WAITS: a few milliseconds of polling,
// long enough for any legitimate wait of a product.
constexpr uint32_t kShortWaitPolls = 1u << 13;

static int cuda_fail(cudaError_t e) {
    (void)e;
    return DMUL_ERR_CUDA;
}

#define CK(call)                                         \
    do {                                                 \
        cudaError_t _e = (call);                         \
        if (_e != cudaSuccess) return cuda_fail(_e);     \
    } while (0)

static const char *kStageNames[kNumStages] = {"col_fwd", "row_mul", "col_inv_crt", "carry_scan",
                                              "transpose", "row_dft", "crt", "pack_transpose",
                                              "small_mul", "batch", "short_fused"};

Timed::Timed(dmul_ctx *c_, int id_, cudaStream_t s_) : c(c_), id(id_), s(s_) {
        if (!c->timing) return;
        if (c->ev_used == c->ev_pool.size()) {
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            c->ev_pool.push_back({a, b});
        }
        idx = c->ev_used++;
        cudaEventRecord(c->ev_pool[idx].first, s);
}

Timed::~Timed() {
        if (!c->timing) return;
        cudaEventRecord(c->ev_pool[idx].second, s);
        c->ev_log.push_back({id, idx});
}

int set_device(dmul_ctx *c) {
    CK(cudaSetDevice(c->device));
    return DMUL_OK;
}

int dev_alloc(dmul_ctx *c, void **p, size_t bytes) {
    if (c->used + bytes > c->budget) return DMUL_ERR_NOMEM;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return DMUL_ERR_NOMEM;
    }
    c->used += bytes;
    return DMUL_OK;
}

void dev_free(dmul_ctx *c, void *p, size_t bytes) {
    if (!p) return;
    cudaFree(p);
    c->used -= bytes;
}

static int build_plan_entry(dmul_ctx *c, const HostPlan &hp, std::unique_ptr<PlanEntry> *out) {
    auto pe = std::make_unique<PlanEntry>();
    pe->hp = hp;
    std::vector<uint32_t> tab[kPrimes];
    build_tables(pe->hp, &pe->pd, tab);
    size_t words = tab[0].size();
    pe->bytes = words * sizeof(uint32_t) * kPrimes;
    int rc = dev_alloc(c, &pe->dtables, pe->bytes);
    if (rc) return rc;
    for (int i = 0; i < kPrimes; ++i) {
        uint32_t *dst = (uint32_t *)pe->dtables + i * words;
        CK(cudaMemcpy(dst, tab[i].data(), words * sizeof(uint32_t), cudaMemcpyHostToDevice));
        pe->pd.tw[i] = (const uint2 *)dst;
    }
    // tables of up to 4 MB (transforms up to about 2^20) are prefetched by the forward column pass
    pe->pd.tw_bytes = pe->bytes <= (4u << 20) ? pe->bytes & ~(size_t)15 : 0;
    *out = std::move(pe);
    return DMUL_OK;
}

int ensure_scratch(dmul_ctx *c, uint64_t N, uint64_t L, bool need_y);

// Autotuner: the first time a transform length is planned (never inside a capture: plans are
// built before any capture begins), time the forward column pass, the fused row pass and the
// inverse column pass of a full-length product for every candidate split N1 x N2 and CTA size,
// and keep the fastest.  Results are identical for every candidate (the arithmetic is exact);
// only the time differs.
static int autotune_plan(dmul_ctx *c, uint64_t N, std::unique_ptr<PlanEntry> *best) {
    std::vector<uint32_t> n1s;
    for (uint32_t n1 : candidate_n1(N))
        if (n1 >= 64 && N / n1 >= 256) n1s.push_back(n1);
    HostPlan def;
    if (!make_host_plan(N, &def)) return DMUL_ERR_TOO_LARGE;
    if (n1s.empty()) n1s.push_back(def.N1);
    // the timing runs reuse the plain form's scratch: earlier work on any stream must be done.
    // The status word is kept as earlier calls left it (an error they set is still reported by
    // the next dmul_sync); whatever the timing runs set is discarded.
    CK(cudaDeviceSynchronize());
    uint32_t saved_status = 0;
    CK(cudaMemcpy(&saved_status, c->status, 4, cudaMemcpyDeviceToHost));
    int rc = ensure_scratch(c, N, N, true);
    if (rc) return rc;
    uint32_t *in = nullptr, *zt = nullptr;
    uint2 *sp = nullptr;
    const size_t nsp = N / 32 + 1;
    rc = dev_alloc(c, (void **)&in, N * 4);
    if (!rc) rc = dev_alloc(c, (void **)&zt, N * 4);
    if (!rc) rc = dev_alloc(c, (void **)&sp, nsp * sizeof(uint2));
    if (rc) {
        dev_free(c, in, N * 4);
        dev_free(c, zt, N * 4);
        return rc;
    }
    cudaStream_t s = c->own_stream;
    int sms_i = 152;
    cudaDeviceGetAttribute(&sms_i, cudaDevAttrMultiProcessorCount, c->device);
    const uint32_t sms = (uint32_t)sms_i;
    cudaMemsetAsync(in, 0x11, N * 4, s);  // valid nonzero limbs (0x11111111 < 10^9)
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best_ms = 1e30f;
    for (uint32_t n1 : n1s) {
        HostPlan hp;
        if (!make_host_plan(N, &hp, n1)) continue;
        std::unique_ptr<PlanEntry> cand;
        rc = build_plan_entry(c, hp, &cand);
        if (rc) break;
        float cand_ms = 1e30f;
        uint32_t cand_ct = 0, cand_rt = 0, cand_tma = 0, cand_grid = 0, cand_half = 0;
        // column-pass variants: full-width tiles (256 or 512 threads; 128 for short columns) or
        // half tiles (128 or 256; 64 for short columns)
        std::vector<std::pair<uint32_t, uint32_t>> colv = {{0u, 256u}, {0u, 512u}};
        if (n1 <= 384) colv.push_back({0u, 128u});
        if (col_half_supported(hp)) {
            colv.push_back({1u, 128u});
            colv.push_back({1u, 256u});
            if (n1 <= 192) colv.push_back({1u, 64u});
        }
        // row-pass variants: plain (one CTA per row) or persistent TMA-fed with G CTAs per prime
        std::vector<std::pair<uint32_t, uint32_t>> rowv = {{0u, 0u}};
        if (6ull * (N / n1) * 4 + 16 <= 227ull * 1024)
            for (uint32_t G : {sms / 3, 2 * sms / 3, sms})
                if (G >= 1 && G <= n1) rowv.push_back({1u, G});
        for (auto cv : colv) {
            const uint32_t ct = cv.second;
            for (uint32_t rt : {128u, 256u}) {
                for (auto rv : rowv) {
                    cand->pd.col_half = cv.first;
                    cand->pd.col_threads = ct;
                    cand->pd.row_threads = rt;
                    cand->pd.row_tma = rv.first;
                    cand->pd.row_grid = rv.second;
                    float t = 1e30f;
                    for (int it = 0; it < 3; ++it) {
                        cudaEventRecord(e0, s);
                        launch_col_fwd(cand->pd, in, N / 2, in + N / 2, N / 2, c->X, c->Y, c->status, s);
                        launch_row_any(cand->pd, c->X, c->Y, false, c->status, s);
                        launch_col_inv(cand->pd, c->X, N, kInvDigits, zt, sp, s);
                        cudaEventRecord(e1, s);
                        cudaEventSynchronize(e1);
                        float ms = 0;
                        cudaEventElapsedTime(&ms, e0, e1);
                        if (it > 0) t = std::min(t, ms);  // the first run warms up
                    }
                    if (cudaGetLastError() != cudaSuccess) t = 1e30f;
                    if (t < cand_ms) {
                        cand_ms = t;
                        cand_ct = ct;
                        cand_rt = rt;
                        cand_tma = rv.first;
                        cand_grid = rv.second;
                        cand_half = cv.first;
                    }
                }
            }
        }
        if (cand_ms < best_ms) {
            best_ms = cand_ms;
            cand->hp.col_threads = cand_ct;
            cand->hp.row_threads = cand_rt;
            cand->hp.row_tma = cand_tma;
            cand->hp.row_grid = cand_grid;
            cand->hp.col_half = cand_half;
            if (*best) dev_free(c, (*best)->dtables, (*best)->bytes);
            *best = std::move(cand);
        } else {
            dev_free(c, cand->dtables, cand->bytes);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaMemcpy(c->status, &saved_status, 4, cudaMemcpyHostToDevice);
    dev_free(c, in, N * 4);
    dev_free(c, zt, N * 4);
    dev_free(c, sp, nsp * sizeof(uint2));
    if (!*best) return rc ? rc : DMUL_ERR_CUDA;
    (*best)->pd.col_threads = (*best)->hp.col_threads;
    (*best)->pd.row_threads = (*best)->hp.row_threads;
    (*best)->pd.row_tma = (*best)->hp.row_tma;
    (*best)->pd.row_grid = (*best)->hp.row_grid;
    (*best)->pd.col_half = (*best)->hp.col_half;
    return DMUL_OK;
}

// The plan a context uses without autotuning: the default split, with the row / column pass
// variants its flags force (DMUL_FLAG_ROW_TMA, DMUL_FLAG_COL_HALF).
static bool fixed_host_plan(const dmul_ctx *c, uint64_t N, HostPlan *hp) {
    const bool six = (c->cfg.flags & DMUL_FLAG_SIXSTEP) != 0;
    if (!(six ? make_host_plan_sixstep(N, hp) : make_host_plan(N, hp))) return false;
    if (six) return true;
    if ((c->cfg.flags & DMUL_FLAG_ROW_TMA) && 6ull * hp->N2 * 4 + 16 <= 227ull * 1024) {
        int sms = 152;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device);
        hp->row_tma = 1;
        hp->row_grid = std::max<uint32_t>(1, std::min<uint32_t>(hp->N1, (uint32_t)sms / 3));
    }
    if ((c->cfg.flags & DMUL_FLAG_COL_HALF) && col_half_supported(*hp)) {
        hp->col_half = 1;
        hp->col_threads = 256;
    }
    return true;
}

int get_plan(dmul_ctx *c, uint64_t N, PlanEntry **out) {
    auto it = c->plans.find(N);
    if (it != c->plans.end()) {
        *out = it->second.get();
        return DMUL_OK;
    }
    std::unique_ptr<PlanEntry> pe;
    const bool six = (c->cfg.flags & DMUL_FLAG_SIXSTEP) != 0;
    int rc;
    if (six || (c->cfg.flags & DMUL_FLAG_NO_AUTOTUNE)) {
        HostPlan hp;
        if (!fixed_host_plan(c, N, &hp)) return DMUL_ERR_TOO_LARGE;
        rc = build_plan_entry(c, hp, &pe);
    } else {
        rc = autotune_plan(c, N, &pe);
    }
    if (rc) return rc;
    *out = pe.get();
    c->plans[N] = std::move(pe);
    return DMUL_OK;
}

int get_small_plan(dmul_ctx *c, uint64_t N, SmallPlanEntry **out) {
    auto it = c->small_plans.find(N);
    if (it != c->small_plans.end()) {
        *out = it->second.get();
        return DMUL_OK;
    }
    auto se = std::make_unique<SmallPlanEntry>();
    std::vector<uint32_t> tab[kPrimes];
    build_small_tables(N, &se->sp, tab);
    size_t words = tab[0].size();
    se->bytes = std::max<size_t>(words, 2) * sizeof(uint32_t) * kPrimes;
    int rc = dev_alloc(c, &se->dtables, se->bytes);
    if (rc) return rc;
    for (int i = 0; i < kPrimes; ++i) {
        uint32_t *dst = (uint32_t *)se->dtables + i * std::max<size_t>(words, 2);
        if (words) CK(cudaMemcpy(dst, tab[i].data(), words * sizeof(uint32_t), cudaMemcpyHostToDevice));
        se->sp.tw[i] = (const uint2 *)dst;
    }
    *out = se.get();
    c->small_plans[N] = std::move(se);
    return DMUL_OK;
}

int ensure_scratch(dmul_ctx *c, uint64_t N, uint64_t L, bool need_y) {
    (void)need_y;
    const size_t words = (size_t)kPrimes * N;
    if (words > c->res_words) {
        dev_free(c, c->X, c->res_words * 4);
        dev_free(c, c->Y, c->res_words * 4);
        c->X = c->Y = nullptr;
        c->res_words = 0;
        int rc = dev_alloc(c, (void **)&c->X, words * 4);
        if (rc) return rc;
        rc = dev_alloc(c, (void **)&c->Y, words * 4);
        if (rc) { dev_free(c, c->X, words * 4); c->X = nullptr; return rc; }
        c->res_words = words;
    }
    const size_t nsp = (L + kChunk - 1) / kChunk + 1;
    if (nsp > c->spill_cap) {
        dev_free(c, c->spill, c->spill_cap * sizeof(uint2));
        c->spill = nullptr;
        c->spill_cap = 0;
        int rc = dev_alloc(c, (void **)&c->spill, nsp * sizeof(uint2));
        if (rc) return rc;
        c->spill_cap = nsp;
    }
    const size_t cb = carry_ctl_bytes(L);
    if (cb > c->ctl_cap) {
        dev_free(c, c->ctl, c->ctl_cap);
        c->ctl = nullptr;
        c->ctl_cap = 0;
        int rc = dev_alloc(c, &c->ctl, cb);
        if (rc) return rc;
        c->ctl_cap = cb;
    }
    return DMUL_OK;
}

bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes) {
    uintptr_t a0 = (uintptr_t)a, a1 = a0 + abytes, b0 = (uintptr_t)b, b1 = b0 + bbytes;
    return a0 < b1 && b0 < a1;
}

uint64_t max_min_limbs() {
    typedef unsigned __int128 u128;
    u128 P = (u128)kPrimeSet[0] * kPrimeSet[1] * kPrimeSet[2];
    u128 b1 = (u128)(kBase - 1) * (kBase - 1);
    return (uint64_t)((P - 1) / b1);
}

int check_sizes(dmul_ctx *c, size_t nx, size_t ny, uint64_t *N) {
    if (nx == 0 || ny == 0) return DMUL_ERR_INVALID;
    uint64_t L = (uint64_t)nx + ny;
    if (std::min(nx, ny) > max_min_limbs()) return DMUL_ERR_TOO_LARGE;  // eq. product_inequality
    if (c->cfg.max_limbs && L > c->cfg.max_limbs) return DMUL_ERR_TOO_LARGE;
    *N = (c->cfg.flags & DMUL_FLAG_SIXSTEP) ? choose_N_pow2(L) : choose_N(L, !(c->cfg.flags & DMUL_FLAG_NO_RADIX5));
    if (*N == 0) return DMUL_ERR_TOO_LARGE;
    return DMUL_OK;
}

// The forward transforms of x (and y), the pointwise product and the inverse transforms; the
// residues of the convolution are then in c->X (four-step order: inverse column pass pending).
// y_ready (optional): an event after which y may be read -- the forward pass of x is enqueued
// before the wait, so that y's upload overlaps it.
int enqueue_transforms(dmul_ctx *c, PlanEntry *pe, const uint32_t *x, size_t nx,
                       const uint32_t *y, size_t ny, bool square, cudaStream_t s,
                       cudaEvent_t y_ready = nullptr);

// A lone short product can run three ways: as one cluster (the small kernel: one launch, three
// SMs), as the four-step pipeline (four launches, many CTAs), or -- at N = N1 x 256 with N1 in
// {64, 80, 96} -- as the four-step steps in one cooperative launch over every SM (shortfused.cu).
// Which is fastest depends on the length: the first product of each length times the candidates
// on operands of nonzero limbs (the work of a real product) and keeps the fastest.  small_single
// holds the small kernel against the four-step pipeline alone (the batched form's choice for its
// short groups), short_path the lone product's choice among every candidate.
int small_single_cached(const dmul_ctx *c, uint64_t Ns) {
    std::lock_guard<std::mutex> g(c->small_mu);
    auto it = c->small_single.find(Ns);
    return it == c->small_single.end() ? -1 : (it->second ? 1 : 0);
}

// The fused kernel's plan for N: the split N1 x 256 whatever the autotuner picked for the pipeline.
static int get_fused_plan(dmul_ctx *c, uint64_t N, PlanEntry **out) {
    auto it = c->fused_plans.find(N);
    if (it != c->fused_plans.end()) {
        *out = it->second.get();
        return DMUL_OK;
    }
    HostPlan hp;
    if (N % 256 || !make_host_plan(N, &hp, (uint32_t)(N / 256))) return DMUL_ERR_INVALID;
    std::unique_ptr<PlanEntry> pe;
    int rc = build_plan_entry(c, hp, &pe);
    if (rc) return rc;
    if (!short_fused_supported(pe->pd)) {
        dev_free(c, pe->dtables, pe->bytes);
        return DMUL_ERR_INVALID;
    }
    *out = pe.get();
    c->fused_plans[N] = std::move(pe);
    return DMUL_OK;
}

// Whether a lone product of transform length N may take the fused kernel: the length and the
// operands' alignment suit it.  (A product inside a stream capture never does: the caller leaves
// the cooperative launch out of a capture.)
static bool fused_candidate(const dmul_ctx *c, uint64_t N, const void *x, const void *y) {
    if (c->cfg.flags & (DMUL_FLAG_SIXSTEP | DMUL_FLAG_NO_FUSED)) return false;
    const uint64_t n1 = N / 256;
    if (N % 256 || (n1 != 64 && n1 != 80 && n1 != 96)) return false;
    if ((((uintptr_t)x) | ((uintptr_t)y)) & 15) return false;
    return current_device_sms() >= 48;  // a CTA per column task of both operands
}

static cudaError_t launch_fused_product(dmul_ctx *c, const PlanEntry *fe, const JobDev &jd, cudaStream_t s) {
    return launch_short_fused(fe->pd, fe->bytes, jd.x, jd.nx, jd.y, jd.ny, c->X, c->Y, jd.z, jd.nz, c->spill,
                              (CarryCtl *)c->ctl, c->status, c->grid_sync, c->spin_limit,
                              (uint32_t)current_device_sms(), s);
}

// Times a product of length min(Ns, N) (or N without a small plan) on each candidate path: the
// small kernel (Ns > 0), the pipeline, the fused kernel (fused).  The best of three cold-cache runs
// after a warm-up; the context's status word is kept for the next dmul_sync.
static int time_short_paths(dmul_ctx *c, uint64_t Ns, uint64_t N, bool fused, ShortTimes *t) {
    SmallPlanEntry *se = nullptr;
    PlanEntry *pe = nullptr, *fe = nullptr;
    int rc = Ns ? get_small_plan(c, Ns, &se) : DMUL_OK;
    if (!rc) rc = get_plan(c, N, &pe);
    if (!rc && fused) rc = get_fused_plan(c, N, &fe);
    if (rc) return rc;
    CK(cudaDeviceSynchronize());
    uint32_t saved_status = 0;
    CK(cudaMemcpy(&saved_status, c->status, 4, cudaMemcpyDeviceToHost));
    const uint64_t Lt = Ns ? std::min(Ns, N) : N;
    rc = ensure_scratch(c, N, Lt, true);
    if (rc) return rc;
    uint32_t *buf = nullptr;
    uint64_t *nzb = nullptr;
    if ((rc = dev_alloc(c, (void **)&buf, 2 * Lt * 4))) return rc;
    if ((rc = dev_alloc(c, (void **)&nzb, 64))) { dev_free(c, buf, 2 * Lt * 4); return rc; }
    cudaStream_t s = c->own_stream;
    // operands of valid nonzero limbs (0x11111111 < 10^9): every path does the work of a real product
    cudaMemsetAsync(buf, 0x11, 2 * Lt * 4, s);
    JobDev jd;
    memset(&jd, 0, sizeof(jd));
    jd.x = buf; jd.y = buf + Lt / 2; jd.z = buf + Lt; jd.nz = nzb; jd.nx = Lt / 2; jd.ny = Lt - Lt / 2; jd.L = Lt;
    // Each timed run starts with L2 cold, as a lone product after other work meets it (and as the
    // benchmark times it): a write over twice the L2 size first, which also keeps the GPU busy
    // while the host enqueues the run.  Without room in the budget for that buffer, runs are warm.
    int l2 = 0;
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device);
    size_t flush_bytes = 2 * (size_t)std::max(l2, 0);
    void *flush = nullptr;
    if (flush_bytes && dev_alloc(c, &flush, flush_bytes)) {
        flush = nullptr;
        flush_bytes = 0;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    auto timed = [&](float &best, int it, auto &&body) {
        float ms = 0;
        if (flush) cudaMemsetAsync(flush, it & 0xff, flush_bytes, s);
        cudaEventRecord(e0, s);
        body();
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        cudaEventElapsedTime(&ms, e0, e1);
        if (it) best = std::min(best, ms);  // the first run warms up
    };
    for (int it = 0; it < 4; ++it) {
        if (se) timed(t->small, it, [&] { launch_small_mul_one(se->sp, jd, c->status, s); });
        timed(t->four, it, [&] {
            launch_col_fwd(pe->pd, jd.x, jd.nx, jd.y, jd.ny, c->X, c->Y, c->status, s);
            launch_row_any(pe->pd, c->X, c->Y, false, c->status, s);
            launch_col_inv(pe->pd, c->X, Lt, kInvDigits, jd.z, c->spill, s, c->ctl, carry_ctl_bytes(Lt));
            launch_carry(jd.z, c->spill, Lt, (CarryCtl *)c->ctl, nzb, c->status, s);
        });
        if (fe) {
            // a cooperative launch the device refuses (too few SMs free for its grid) leaves the
            // fused kernel out of the choice; the refusal is not a sticky error
            bool ok = true;
            timed(t->fused, it, [&] { ok = launch_fused_product(c, fe, jd, s) == cudaSuccess; });
            if (!ok) {
                cudaGetLastError();
                t->fused = 1e30f;
                fe = nullptr;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaMemcpy(c->status, &saved_status, 4, cudaMemcpyHostToDevice);
    dev_free(c, buf, 2 * Lt * 4);
    dev_free(c, nzb, 64);
    if (flush) dev_free(c, flush, flush_bytes);
    if (cudaGetLastError() != cudaSuccess) return DMUL_ERR_CUDA;
    return DMUL_OK;
}

int prefer_small_single(dmul_ctx *c, uint64_t Ns, uint64_t N, bool *use_small) {
    const int known = small_single_cached(c, Ns);
    if (known >= 0) {
        *use_small = known == 1;
        return DMUL_OK;
    }
    ShortTimes t;
    int rc = time_short_paths(c, Ns, N, false, &t);
    if (rc) return rc;
    *use_small = t.small <= t.four;
    std::lock_guard<std::mutex> g(c->small_mu);
    c->small_single[Ns] = *use_small;
    return DMUL_OK;
}

enum ShortPath { kPathFour = 0, kPathSmall = 1, kPathFused = 2 };

static bool stream_capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cap != cudaStreamCaptureStatusNone;
}

// The lone product's path among the allowed candidates (small_ok: the small kernel of length Ns;
// fused_ok: the fused kernel; the pipeline always), by the first-use times of the lengths (Ns, N).
// An allowed candidate without a time yet is timed now -- except inside a stream capture, where
// nothing may synchronize: there only the candidates already timed compete, and with none the
// pipeline runs.
static int prefer_short_path(dmul_ctx *c, uint64_t Ns, uint64_t N, bool small_ok, bool fused_ok, bool capturing,
                             int *path) {
    const uint64_t key = (Ns << 40) | N;
    ShortTimes t;
    bool have = false;
    {
        std::lock_guard<std::mutex> g(c->small_mu);
        auto it = c->short_times.find(key);
        if (it != c->short_times.end()) {
            t = it->second;
            have = true;
        }
    }
    const bool need = !have || (small_ok && !t.small_timed) || (fused_ok && !t.fused_timed);
    if (need && !capturing) {
        ShortTimes nt;
        int rc = time_short_paths(c, small_ok ? Ns : 0, N, fused_ok, &nt);
        if (rc) return rc;
        // the candidates timed before and not now keep their times
        if (!small_ok && t.small_timed) { nt.small = t.small; nt.small_timed = true; }
        if (small_ok) nt.small_timed = true;
        if (!fused_ok && t.fused_timed) { nt.fused = t.fused; nt.fused_timed = true; }
        if (fused_ok) nt.fused_timed = true;
        t = nt;
        have = true;
        std::lock_guard<std::mutex> g(c->small_mu);
        if (small_ok && !c->small_single.count(Ns)) c->small_single[Ns] = t.small <= t.four;
        c->short_times[key] = t;
    }
    *path = kPathFour;
    if (!have) return DMUL_OK;
    float best = t.four;
    if (small_ok && t.small_timed && t.small <= best) { *path = kPathSmall; best = t.small; }
    if (fused_ok && t.fused_timed && t.fused < best) *path = kPathFused;
    return DMUL_OK;
}

// Whether a product of L limbs on transform length N (small: the small kernel's length) needs no
// allocation and no planning: its plan cached, the scratch large enough.
static bool planned_for_capture(const dmul_ctx *c, uint64_t N, bool small, uint64_t L) {
    if (small) return c->small_plans.count(N) != 0;
    return c->plans.count(N) != 0 && (size_t)kPrimes * N <= c->res_words &&
           (L + kChunk - 1) / kChunk + 1 <= c->spill_cap && carry_ctl_bytes(L) <= c->ctl_cap;
}

// z_out (optional, digits mode, four-step or six-step path): where the carry writes the limbs --
// pinned host memory for the host-buffer entry point; z then only holds the digit sums.
int enqueue_mul(dmul_ctx *c, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny,
                uint32_t *z, size_t z_cap, uint64_t *nz, cudaStream_t s, InvMode mode,
                uint32_t *mode_out, cudaEvent_t y_ready = nullptr, uint32_t *z_out = nullptr) {
    uint64_t N;
    int rc = check_sizes(c, nx, ny, &N);
    if (rc) return rc;
    const uint64_t L = (uint64_t)nx + ny;
    if (mode == kInvDigits) {
        if (!z || z_cap < L) return DMUL_ERR_CAPACITY;
        if (overlaps(z, L * 4, x, nx * 4) || overlaps(z, L * 4, y, ny * 4)) return DMUL_ERR_INVALID;
    }
    rc = set_device(c);
    if (rc) return rc;
    const uint64_t Ns = choose_N_small(L);
    // Inside a stream capture nothing may allocate or synchronize: the lengths must have been
    // planned (by a product of the same lengths outside the capture), and the scratch be in place.
    const bool capturing = stream_capturing(s);
    const bool small_ok = mode == kInvDigits && Ns && !(c->cfg.flags & (DMUL_FLAG_SIXSTEP | DMUL_FLAG_NO_SMALL));
    const bool fused_ok = mode == kInvDigits && !capturing && fused_candidate(c, N, x, y);
    int path = kPathFour;
    if (small_ok || fused_ok) {
        if (c->cfg.flags & DMUL_FLAG_NO_AUTOTUNE) path = small_ok ? kPathSmall : kPathFused;
        else if ((rc = prefer_short_path(c, Ns, N, small_ok, fused_ok, capturing, &path))) return rc;
    }
    if (capturing && !planned_for_capture(c, path == kPathSmall ? Ns : N, path == kPathSmall, L))
        return DMUL_ERR_INVALID;
    if (path != kPathFour) {
        JobDev jd;
        memset(&jd, 0, sizeof(jd));
        jd.x = x; jd.y = y; jd.z = z; jd.nz = nz; jd.nx = nx; jd.ny = ny; jd.L = L;
        jd.square = (x == y && nx == ny) ? 1u : 0u;
        if (path == kPathSmall) {
            // the whole product in one cluster launch (batch.cu): transforms, CRT and carry in SMEM
            SmallPlanEntry *se;
            rc = get_small_plan(c, Ns, &se);
            if (rc) return rc;
            c->last_stream = s;
            if (y_ready) CK(cudaStreamWaitEvent(s, y_ready, 0));
            Timed t(c, kStSmall, s);
            CK(launch_small_mul_one(se->sp, jd, c->status, s));
        } else {
            // the four-step steps in one cooperative launch (shortfused.cu)
            PlanEntry *fe;
            rc = get_fused_plan(c, N, &fe);
            if (!rc) rc = ensure_scratch(c, N, L, true);
            if (rc) return rc;
            c->last_stream = s;
            if (y_ready) CK(cudaStreamWaitEvent(s, y_ready, 0));
            Timed t(c, kStFused, s);
            CK(launch_fused_product(c, fe, jd, s));
        }
        // both kernels leave the limbs in z: they are copied out afterwards
        if (z_out) CK(cudaMemcpyAsync(z_out, z, L * 4, cudaMemcpyDefault, s));
        return DMUL_OK;
    }
    PlanEntry *pe;
    rc = get_plan(c, N, &pe);
    if (rc) return rc;
    rc = ensure_scratch(c, N, L, true);
    if (rc) return rc;
    c->last_stream = s;
    const bool square = (x == y && nx == ny);
    rc = enqueue_transforms(c, pe, x, nx, y, ny, square, s, y_ready);
    if (rc) return rc;
    const bool six = (c->cfg.flags & DMUL_FLAG_SIXSTEP) != 0;
    if (six) {
        Timed t(c, kStCrt, s);
        CK(launch_crt_transposed(c->X, pe->pd.N1, pe->pd.N2, L, mode, mode == kInvDigits ? z : mode_out, c->spill, s));
        if (mode == kInvDigits) CK(cudaMemsetAsync(c->ctl, 0, carry_ctl_bytes(L), s));
    } else {
        // the inverse pass also clears the carry scan's control block (no memset in between)
        Timed t(c, kStColInv, s);
        CK(launch_col_inv(pe->pd, c->X, L, mode, mode == kInvDigits ? z : mode_out, c->spill, s,
                          mode == kInvDigits ? c->ctl : nullptr, mode == kInvDigits ? carry_ctl_bytes(L) : 0));
    }
    if (mode == kInvDigits) {
        Timed t(c, kStCarry, s);
        CK(launch_carry(z, c->spill, L, (CarryCtl *)c->ctl, nz, c->status, s, z_out, c->spin_limit));
    }
    return DMUL_OK;
}

int enqueue_transforms(dmul_ctx *c, PlanEntry *pe, const uint32_t *x, size_t nx,
                       const uint32_t *y, size_t ny, bool square, cudaStream_t s, cudaEvent_t y_ready) {
    if (!(c->cfg.flags & DMUL_FLAG_SIXSTEP)) {
        // The row pass of a prime starts once that prime's forward columns are done (per-prime
        // counters, running totals: this call adds operands x N2 columns to every prime's count).
        // The counters are never reset: a row CTA may start, through the chain of early
        // (programmatic) launches, while the previous call's kernels still run, and a total that
        // only grows can never be met by that call's columns.  The host's total therefore counts
        // only launches that were accepted.  Inside a stream capture the hand-off is off (the row
        // pass waits for the whole column grid): a replayed graph would move the device counters
        // without the host's total.
        PlanDev pd = pe->pd;
        pd.spin = c->spin_limit;
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        CK(cudaStreamIsCapturing(s, &cap));
        const bool handoff = cap == cudaStreamCaptureStatusNone;
        const uint32_t before = c->fwd_cols;
        if (handoff) {
            pd.fsync = c->fwd_sync;
            pd.ftarget = before + (square ? 1u : 2u) * pd.N2;
        } else {
            pd.fsync = nullptr;
        }
        cudaError_t e;
        if (y_ready && !square) {
            // x's forward pass first, then (once y is uploaded) y's
            Timed t(c, kStColFwd, s);
            e = launch_col_fwd(pd, x, nx, nullptr, 0, c->X, nullptr, c->status, s);
            if (e == cudaSuccess) {
                if (handoff) c->fwd_cols += pd.N2;
                e = cudaStreamWaitEvent(s, y_ready, 0);
                if (e == cudaSuccess) e = launch_col_fwd(pd, y, ny, nullptr, 0, c->Y, nullptr, c->status, s);
                if (e == cudaSuccess && handoff) c->fwd_cols += pd.N2;
            }
        } else {
            e = y_ready ? cudaStreamWaitEvent(s, y_ready, 0) : cudaSuccess;
            Timed t(c, kStColFwd, s);
            if (e == cudaSuccess) e = launch_col_fwd(pd, x, nx, square ? nullptr : y, ny, c->X, c->Y, c->status, s);
            if (e == cudaSuccess && handoff) c->fwd_cols += (square ? 1u : 2u) * pd.N2;
        }
        if (e != cudaSuccess) return DMUL_ERR_CUDA;
        Timed t(c, kStRowMul, s);
        CK(launch_row_any(pd, c->X, c->Y, square, c->status, s));
        return DMUL_OK;
    }
    const PlanDev &pd = pe->pd;
    // Six-step form (Sec. 7.2): [N1 x N2] -> transpose -> row DFTs of length N1 -> transpose
    // back -> (twiddle fused into the row DFT kernel) -> fused row pass -> and the mirror.
    if (y_ready) CK(cudaStreamWaitEvent(s, y_ready, 0));
    const uint64_t N = pd.N;
    for (int op = 0; op < (square ? 1 : 2); ++op) {
        uint32_t *A = op ? c->Y : c->X;
        {
            // packing and step 1 in one out-of-place pass: limbs -> the primes' N2 x N1 transposes
            Timed t(c, kStPack, s);
            CK(launch_pack_transpose(op ? y : x, op ? ny : nx, pd.N1, pd.N2, A, c->status, s));
        }
        {
            Timed t(c, kStRowDft, s);
            CK(rowdft6_specialized(pd) ? launch_rowdft6_ct(pd, A, false, s) : launch_rowdft_fwd_tw(pd, A, s));
        }
        Timed t(c, kStTranspose, s);
        CK(launch_transpose(A, pd.N2, pd.N1, kPrimes, N, s, c->status));
    }
    {
        Timed t(c, kStRowMul, s);
        CK(launch_row_any(pd, c->X, c->Y, square, c->status, s));
    }
    {
        Timed t(c, kStTranspose, s);
        CK(launch_transpose(c->X, pd.N1, pd.N2, kPrimes, N, s, c->status));
    }
    Timed t(c, kStRowDft, s);
    CK(rowdft6_specialized(pd) ? launch_rowdft6_ct(pd, c->X, true, s) : launch_rowdft_inv_tw(pd, c->X, s));
    // the last transpose is fused into the CRT that follows (launch_crt_transposed)
    return DMUL_OK;
}

static void collect_timers(dmul_ctx *c) {
    if (!c->timing || c->ev_log.empty()) return;
    for (auto &pr : c->ev_log) {
        auto &ev = c->ev_pool[pr.second];
        cudaEventSynchronize(ev.second);
        float ms = 0;
        cudaEventElapsedTime(&ms, ev.first, ev.second);
        c->timers[pr.first].ms += ms;
        c->timers[pr.first].launches += 1;
    }
    c->ev_log.clear();
    c->ev_used = 0;
}

}  // namespace dml

// ================================================================================================
// C ABI
// ================================================================================================
extern "C" {

const char *dmul_strerror(int st) {
    switch (st) {
        case DMUL_OK: return "ok";
        case DMUL_ERR_INVALID: return "invalid argument or input limb";
        case DMUL_ERR_TOO_LARGE: return "operands too large for the prime set / transform lengths";
        case DMUL_ERR_NOMEM: return "out of device memory (HBM budget)";
        case DMUL_ERR_TIMEOUT: return "a bounded device wait expired";
        case DMUL_ERR_CUDA: return "CUDA runtime error";
        case DMUL_ERR_CAPACITY: return "output capacity too small";
        case DMUL_ERR_UNKNOWN_TICKET: return "unknown ticket";
        case DMUL_PENDING: return "pending";
        default: return "unknown status";
    }
}

int dmul_primes(uint32_t out[3]) {
    std::vector<uint64_t> p = find_primes(31, 23, 3);
    if (p.size() != 3) return DMUL_ERR_INVALID;
    // ascending
    out[0] = (uint32_t)p[2];
    out[1] = (uint32_t)p[1];
    out[2] = (uint32_t)p[0];
    return DMUL_OK;
}

int dmul_lambda(int w, int l, int log2M) { return lambda_max_digits(w, l, log2M); }

uint64_t dmul_max_min_limbs(void) { return max_min_limbs(); }

int dmul_get_plan(const dmul_ctx *ctx, uint64_t L, dmul_plan_info *out) {
    if (!out || L < 2) return DMUL_ERR_INVALID;
    const bool six = ctx && (ctx->cfg.flags & DMUL_FLAG_SIXSTEP);
    uint64_t N = six ? choose_N_pow2(L) : choose_N(L, !(ctx && (ctx->cfg.flags & DMUL_FLAG_NO_RADIX5)));
    if (!N) return DMUL_ERR_TOO_LARGE;
    HostPlan hp;
    if (!(six ? make_host_plan_sixstep(N, &hp) : make_host_plan(N, &hp))) return DMUL_ERR_TOO_LARGE;
    if (ctx) {
        auto it = ctx->plans.find(N);
        if (it != ctx->plans.end()) hp = it->second->hp;  // the split the autotuner chose
        else if (six || (ctx->cfg.flags & DMUL_FLAG_NO_AUTOTUNE)) fixed_host_plan(ctx, N, &hp);
    }
    memset(out, 0, sizeof(*out));
    for (int i = 0; i < kPrimes; ++i) out->primes[i] = kPrimeSet[i];
    out->N = hp.N;
    out->N1 = hp.N1;
    out->N2 = hp.N2;
    for (size_t i = 0; i < hp.col_radix.size() && i < 8; ++i) out->col_radix[i] = hp.col_radix[i];
    for (size_t i = 0; i < hp.row_radix.size() && i < 8; ++i) out->row_radix[i] = hp.row_radix[i];
    out->sixstep = (ctx && (ctx->cfg.flags & DMUL_FLAG_SIXSTEP)) ? 1u : 0u;
    out->col_threads = hp.col_threads ? hp.col_threads : (hp.N1 >= 512 ? 512 : 256);
    out->row_threads = hp.row_threads ? hp.row_threads : 256;
    out->row_tma = hp.row_tma;
    out->row_grid = hp.row_grid;
    out->col_half = hp.col_half;
    return DMUL_OK;
}

int dmul_init(dmul_ctx **out, const dmul_config *cfg) {
    if (!out) return DMUL_ERR_INVALID;
    *out = nullptr;
    uint32_t pr[3];
    if (dmul_primes(pr) != DMUL_OK) return DMUL_ERR_INVALID;
    for (int i = 0; i < 3; ++i)
        if (pr[i] != kPrimeSet[i]) return DMUL_ERR_INVALID;  // FindPrimes must give the compiled set
    auto c = std::make_unique<dmul_ctx>();
    if (cfg) c->cfg = *cfg;
    c->device = c->cfg.device;
    c->budget = c->cfg.hbm_budget_bytes ? c->cfg.hbm_budget_bytes : (16ull << 30);
    c->timing = (c->cfg.flags & DMUL_FLAG_STAGE_TIMING) != 0;
    if (c->cfg.flags & DMUL_FLAG_SHORT_WAITS) c->spin_limit = kShortWaitPolls;
    for (int i = 0; i < kNumStages; ++i) c->timers.push_back(StageTimer{kStageNames[i]});
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c->device < 0 || c->device >= ndev) {
        cudaGetLastError();
        return DMUL_ERR_CUDA;
    }
    CK(cudaSetDevice(c->device));
    PrimeConst pc[kPrimes];
    CrtConst crt;
    make_prime_consts(pc);
    make_crt_consts(&crt);
    CK(upload_constants_main(pc, crt));
    CK(upload_constants_sixstep(pc, crt));
    CK(upload_constants_batch(pc, crt));
    CK(upload_constants_rowpass(pc, crt));
    CK(upload_constants_colpass(pc, crt));
    CK(upload_constants_shortfused(pc, crt));
    CK(init_kernel_attributes_main());
    CK(init_kernel_attributes_sixstep());
    CK(init_kernel_attributes_batch());
    CK(init_kernel_attributes_rowpass());
    CK(init_kernel_attributes_colpass());
    int rc = dev_alloc(c.get(), (void **)&c->status, 256);
    if (rc) return rc;
    CK(cudaMemset(c->status, 0, 256));
    rc = dev_alloc(c.get(), (void **)&c->fwd_sync, 256);
    if (rc) return rc;
    CK(cudaMemset(c->fwd_sync, 0, 256));
    c->grid_sync = c->fwd_sync + 32;
    CK(cudaStreamCreateWithFlags(&c->own_stream, cudaStreamNonBlocking));
    *out = c.release();
    return DMUL_OK;
}

void dmul_destroy(dmul_ctx *c) {
    if (!c) return;
    cudaSetDevice(c->device);
    c->server.reset();
    cudaDeviceSynchronize();
    for (auto &kv : c->plans) dev_free(c, kv.second->dtables, kv.second->bytes);
    for (auto &kv : c->fused_plans) dev_free(c, kv.second->dtables, kv.second->bytes);
    dev_free(c, c->X, c->res_words * 4);
    dev_free(c, c->Y, c->res_words * 4);
    dev_free(c, c->spill, c->spill_cap * sizeof(uint2));
    dev_free(c, c->ctl, c->ctl_cap);
    dev_free(c, c->status, 256);
    dev_free(c, c->fwd_sync, 256);
    destroy_batch_state(c);

    if (c->hx) { cudaFree(c->hx); cudaFree(c->hy); }
    if (c->hz) { cudaFree(c->hz); cudaFree(c->hnz); }
    if (c->h_tail) {
        cudaFreeHost(c->h_tail);
        cudaStreamDestroy(c->copy_stream);
        cudaEventDestroy(c->ev_start);
        cudaEventDestroy(c->ev_y);
    }
    for (auto &e : c->ev_pool) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    if (c->own_stream) cudaStreamDestroy(c->own_stream);
    delete c;
}

int dmul_sync(dmul_ctx *c, void *stream) {
    if (!c) return DMUL_ERR_INVALID;
    int rc = set_device(c);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    CK(cudaStreamSynchronize(s));
    uint32_t st = 0;
    CK(cudaMemcpy(&st, c->status, 4, cudaMemcpyDeviceToHost));
    if (st) CK(cudaMemset(c->status, 0, 4));
    // the last dmul_batch's jobs get their own statuses; a failed one is reported here too
    int jb = c->batch ? flush_batch_status(c->batch.get()) : DMUL_OK;
    if (c->batch_err && jb != DMUL_ERR_TIMEOUT) jb = jb ? jb : c->batch_err;
    if (c->batch_err == DMUL_ERR_TIMEOUT) jb = DMUL_ERR_TIMEOUT;
    c->batch_err = DMUL_OK;
    if ((st & kStatusTimeout) || jb == DMUL_ERR_TIMEOUT) return DMUL_ERR_TIMEOUT;
    if (st & kStatusInvalid) return DMUL_ERR_INVALID;
    return jb;
}

int dmul_mul(dmul_ctx *c, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny, uint32_t *z,
             size_t z_cap, uint64_t *nz, void *stream) {
    if (!c || !x || !y) return DMUL_ERR_INVALID;
    return enqueue_mul(c, x, nx, y, ny, z, z_cap, nz, (cudaStream_t)stream, kInvDigits, nullptr);
}

int dmul_sqr(dmul_ctx *c, const uint32_t *x, size_t nx, uint32_t *z, size_t z_cap, uint64_t *nz,
             void *stream) {
    if (!c || !x) return DMUL_ERR_INVALID;
    return enqueue_mul(c, x, nx, x, nx, z, z_cap, nz, (cudaStream_t)stream, kInvDigits, nullptr);
}

int dmul_conv_residues(dmul_ctx *c, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny,
                       uint32_t *r, void *stream) {
    if (!c || !x || !y || !r) return DMUL_ERR_INVALID;
    return enqueue_mul(c, x, nx, y, ny, nullptr, 0, nullptr, (cudaStream_t)stream, kInvResidues, r);
}

int dmul_conv_coeffs(dmul_ctx *c, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny,
                     uint32_t *d, void *stream) {
    if (!c || !x || !y || !d) return DMUL_ERR_INVALID;
    return enqueue_mul(c, x, nx, y, ny, nullptr, 0, nullptr, (cudaStream_t)stream, kInvTriples, d);
}

int dmul_carry(dmul_ctx *c, const uint32_t *d, size_t L, uint32_t *z, size_t z_cap, uint64_t *nz,
               void *stream) {
    if (!c || !d || !z || L == 0) return DMUL_ERR_INVALID;
    if (z_cap < L) return DMUL_ERR_CAPACITY;
    if (overlaps(z, L * 4, d, L * 12)) return DMUL_ERR_INVALID;
    int rc = set_device(c);
    if (rc) return rc;
    rc = ensure_scratch(c, 0, L, false);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    CK(launch_triples_to_digits(d, L, z, c->spill, c->status, s));
    CK(cudaMemsetAsync(c->ctl, 0, carry_ctl_bytes(L), s));
    if (c->cfg.flags & DMUL_FLAG_TEST_STALL_CARRY) {
        // fault injection on the host side: the scan's tile ticket starts at 1, so no CTA becomes
        // tile 0 and tile 1 waits for a publication that never comes (bounded by spin_limit)
        static const uint32_t one = 1;
        CK(cudaMemcpyAsync(c->ctl, &one, 4, cudaMemcpyHostToDevice, s));
    }
    Timed t(c, kStCarry, s);
    CK(launch_carry(z, c->spill, L, (CarryCtl *)c->ctl, nz, c->status, s, nullptr, c->spin_limit));
    return DMUL_OK;
}

int dmul_transpose(dmul_ctx *c, uint32_t *a, size_t rows, size_t cols, void *stream) {
    if (!c || !a) return DMUL_ERR_INVALID;
    if (rows % 32 || cols % 32 || rows == 0 || cols == 0) return DMUL_ERR_INVALID;
    // square, or n x Cn / Cn x n with C n <= 16384 (the permuted row lives in shared memory)
    const size_t lo = rows < cols ? rows : cols, hi = rows < cols ? cols : rows;
    if (hi % lo || (hi != lo && hi > 16384)) return DMUL_ERR_INVALID;
    int rc = set_device(c);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    c->last_stream = s;
    Timed t(c, kStTranspose, s);
    CK(launch_transpose(a, rows, cols, 1, rows * cols, s, c->status));
    return DMUL_OK;
}

// The device address of the host buffer [p, p + bytes) when it is page-locked (cudaHostAlloc,
// cudaMallocHost, cudaHostRegister: both ends inside registered memory), else nullptr.
static void *pinned_view(const void *p, size_t bytes) {
    cudaPointerAttributes a, b;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    const char *last = (const char *)p + bytes - 1;
    if (cudaPointerGetAttributes(&b, last) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type != cudaMemoryTypeHost || b.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
    if ((const char *)b.devicePointer != (const char *)a.devicePointer + (bytes - 1)) return nullptr;
    return a.devicePointer;
}

int dmul_host_direct(dmul_ctx *c, const void *p, size_t bytes) {
    if (!c || !p || !bytes) return 0;
    if (set_device(c)) return 0;
    return pinned_view(p, bytes) ? 1 : 0;
}

int dmul_mul_host(dmul_ctx *c, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny,
                  uint32_t *z, size_t z_cap, size_t *nz) {
    if (!c || !x || !y || !z) return DMUL_ERR_INVALID;
    const bool square = (x == y && nx == ny);
    uint64_t N;
    int rc = check_sizes(c, nx, ny, &N);
    if (rc) return rc;
    const size_t L = nx + ny;
    if (z_cap < L) return DMUL_ERR_CAPACITY;
    if (overlaps(z, L * 4, x, nx * 4) || overlaps(z, L * 4, y, ny * 4)) return DMUL_ERR_INVALID;
    rc = set_device(c);
    if (rc) return rc;
    if (!c->h_tail) {
        CK(cudaMallocHost(&c->h_tail, 64));
        CK(cudaHostGetDevicePointer((void **)&c->h_tail_dev, c->h_tail, 0));
        CK(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&c->ev_start, cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&c->ev_y, cudaEventDisableTiming));
    }
    // Page-locked buffers of short products are read and written in place by the kernels (the
    // operands by the forward pass, the limbs and their count by the carry scan): the bytes cross
    // the host link while the kernels run, not in copies before and after them.  Pageable buffers
    // (or the DMUL_FLAG_HOST_STAGED_* flags) go through device staging buffers with
    // cudaMemcpyAsync.  Longer products (unless the DMUL_FLAG_HOST_DIRECT_* flags ask otherwise)
    // copy too: each prime's column pass reads the operand tile again, which over the host link
    // costs more than one copy up front; and the carry scan's stores of a long product into host
    // memory ran at 0.350 ms per 2^24-digit product on some runs and 0.472 ms on another, where
    // the copy after the scan took 0.356-0.360 ms on every run.
    const uint32_t fl = c->cfg.flags;
    const bool in_place_in = !(fl & DMUL_FLAG_HOST_STAGED_IN) &&
                             ((fl & DMUL_FLAG_HOST_DIRECT_IN) || L <= DMUL_HOST_IN_PLACE_LIMBS);
    const bool in_place_out = !(fl & DMUL_FLAG_HOST_STAGED_OUT) &&
                              ((fl & DMUL_FLAG_HOST_DIRECT_OUT) || L <= DMUL_HOST_IN_PLACE_LIMBS);
    const uint32_t *xd = in_place_in ? (const uint32_t *)pinned_view(x, nx * 4) : nullptr;
    const uint32_t *yd = square ? xd : in_place_in ? (const uint32_t *)pinned_view(y, ny * 4) : nullptr;
    if (!xd || !yd) xd = yd = nullptr;  // both operands one way
    uint32_t *zd = in_place_out ? (uint32_t *)pinned_view(z, L * 4) : nullptr;
    if (c->h_cap < L) {
        if (c->hz) { cudaFree(c->hz); cudaFree(c->hnz); c->used -= c->h_cap * 4 + 64; }
        c->hz = nullptr;
        c->hnz = nullptr;
        c->h_cap = 0;
        if (c->used + L * 4 + 64 > c->budget) return DMUL_ERR_NOMEM;
        CK(cudaMalloc(&c->hz, L * 4));
        CK(cudaMalloc(&c->hnz, 64));
        c->used += L * 4 + 64;
        c->h_cap = L;
    }
    if (!xd && c->h_in_cap < L) {
        if (c->hx) { cudaFree(c->hx); cudaFree(c->hy); c->used -= c->h_in_cap * 8; }
        c->hx = c->hy = nullptr;
        c->h_in_cap = 0;
        if (c->used + L * 8 > c->budget) return DMUL_ERR_NOMEM;
        CK(cudaMalloc(&c->hx, L * 4));
        CK(cudaMalloc(&c->hy, L * 4));
        c->used += L * 8;
        c->h_in_cap = L;
    }
    cudaStream_t s = c->own_stream;
    cudaEvent_t y_ready = nullptr;
    const uint32_t *xa = xd, *ya = yd;
    if (!xd) {
        // x is uploaded on the compute stream; y on the copy stream, overlapping x's forward pass
        CK(cudaMemcpyAsync(c->hx, x, nx * 4, cudaMemcpyHostToDevice, s));
        xa = c->hx;
        ya = square ? c->hx : c->hy;
        if (!square) {
            CK(cudaEventRecord(c->ev_start, s));  // earlier work on s (readers of hy) is done first
            CK(cudaStreamWaitEvent(c->copy_stream, c->ev_start, 0));
            CK(cudaMemcpyAsync(c->hy, y, ny * 4, cudaMemcpyHostToDevice, c->copy_stream));
            CK(cudaEventRecord(c->ev_y, c->copy_stream));
            y_ready = c->ev_y;
        }
    }
    rc = enqueue_mul(c, xa, nx, ya, ny, c->hz, L, zd ? &c->h_tail_dev[0] : c->hnz, s, kInvDigits, nullptr,
                     y_ready, zd);
    if (rc) {
        cudaStreamSynchronize(c->copy_stream);
        return rc;
    }
    // the status word (and, staged, the normalized length) into pinned memory ahead of the
    // product, so that the product's copy ends the stream: one synchronization
    if (!zd) CK(cudaMemcpyAsync(&c->h_tail[0], c->hnz, 8, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&c->h_tail[1], c->status, 4, cudaMemcpyDeviceToHost, s));
    if (!zd) CK(cudaMemcpyAsync(z, c->hz, L * 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (nz) *nz = (size_t)c->h_tail[0];
    const uint32_t st = (uint32_t)c->h_tail[1];
    if (st) {
        CK(cudaMemsetAsync(c->status, 0, 4, s));
        CK(cudaStreamSynchronize(s));
    }
    if (st & kStatusTimeout) return DMUL_ERR_TIMEOUT;
    if (st & kStatusInvalid) return DMUL_ERR_INVALID;
    return DMUL_OK;
}

int dmul_batch(dmul_ctx *c, dmul_job *jobs, size_t count, void *stream) {
    if (!c) {
        for (size_t i = 0; jobs && i < count; ++i) jobs[i].status = DMUL_ERR_INVALID;
        return DMUL_ERR_INVALID;
    }
    if (!jobs && count) return DMUL_ERR_INVALID;
    return dml::run_batch(c, jobs, count, (cudaStream_t)stream);
}

static dml::Server *server_of(dmul_ctx *c, bool create) {
    std::lock_guard<std::mutex> g(c->server_mu);
    if (!c->server && create) c->server = std::make_unique<dml::Server>(c);
    return c->server.get();
}

int dmul_submit(dmul_ctx *c, const dmul_job *job, uint64_t *ticket) {
    if (!c || !job || !ticket) return DMUL_ERR_INVALID;
    return server_of(c, true)->submit(*job, ticket);
}

int dmul_poll(dmul_ctx *c, uint64_t ticket, int *done) {
    if (!c || !done) return DMUL_ERR_INVALID;
    dml::Server *s = server_of(c, false);
    if (!s) return DMUL_ERR_UNKNOWN_TICKET;
    return s->poll(ticket, done);
}

int dmul_wait(dmul_ctx *c, uint64_t ticket) {
    if (!c) return DMUL_ERR_INVALID;
    dml::Server *s = server_of(c, false);
    if (!s) return DMUL_ERR_UNKNOWN_TICKET;
    return s->wait(ticket);
}

int dmul_serve_stats(dmul_ctx *c, dmul_serve_info *out) {
    if (!c || !out) return DMUL_ERR_INVALID;
    memset(out, 0, sizeof(*out));
    dml::Server *s = server_of(c, false);
    if (s) s->stats(out);
    return DMUL_OK;
}

int dmul_stage_times(dmul_ctx *c, const char **names, double *ms, uint64_t *launches, int *n) {
    if (!c || !n) return DMUL_ERR_INVALID;
    if (c->last_stream || c->ev_used) {
        set_device(c);
        collect_timers(c);
    }
    int k = 0;
    for (int i = 0; i < kNumStages; ++i) {
        if (c->timers[i].launches == 0) continue;
        if (k < *n) {
            if (names) names[k] = c->timers[i].name;
            if (ms) ms[k] = c->timers[i].ms;
            if (launches) launches[k] = c->timers[i].launches;
        }
        ++k;
        c->timers[i].ms = 0;
        c->timers[i].launches = 0;
    }
    *n = k;
    return DMUL_OK;
}

int dmul_stage_timing(dmul_ctx *c, int on) {
    if (!c) return DMUL_ERR_INVALID;
    if (c->timing && !on && c->ev_used) {
        int rc = set_device(c);
        if (rc) return rc;
        collect_timers(c);  // keep what was recorded so far for dmul_stage_times
    }
    c->timing = on != 0;
    return DMUL_OK;
}

int dmul_probe_imad(dmul_ctx *c, double *imad_per_s) {
    if (!c || !imad_per_s) return DMUL_ERR_INVALID;
    int rc = set_device(c);
    if (rc) return rc;
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device));
    uint32_t *sink;
    CK(cudaMalloc(&sink, 4096 * 4));
    cudaStream_t s = c->own_stream;
    const int blocks = sms * 8, iters = 4096;
    CK(launch_imad_probe(sink, blocks, iters, s));  // warm-up
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    CK(launch_imad_probe(sink, blocks, iters, s));
    cudaEventRecord(b, s);
    CK(cudaEventSynchronize(b));
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    cudaFree(sink);
    const double ops = (double)blocks * 256 * iters * 16 * 8;
    *imad_per_s = ops / (ms * 1e-3);
    return DMUL_OK;
}

}  // extern "C"

// ---- internal entry points used by the batch and serve layers ------------------------------------
namespace dml {

int ctx_enqueue_mul(dmul_ctx *c, const dmul_job &j, cudaStream_t s) {
    return enqueue_mul(c, j.x, j.nx, j.y, j.ny, j.z, j.z_cap, j.nz, s, kInvDigits, nullptr);
}

}  // namespace dml
