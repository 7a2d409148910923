// batch.cu -- the batched form (dmul_batch) and the fused small-product kernel.
//
// Small products (transform length N <= 24576) run whole in one cluster of three CTAs, one per
// prime: limbs -> residues in shared memory, forward transform of x (and y), pointwise product
// fused with the first inverse stage, inverse transform with the 2^32 N^-1 scale (Sec. 6), then
// the cluster's CRT through distributed shared memory (Sec. 8.2.2) and the carry recurrence as
// a block-wide scan of carry maps (Sec. 3.2) in the rank-0 CTA.  One launch; the residues never
// leave shared memory (only the digit sums pass through z on their way to the carry).  A size
// class with too few short jobs to fill the GPU runs them as four-step groups instead, where that
// measured faster for a lone product of their length (run_batch_on).
//
// Larger products run the four-step pipeline (column pass, fused row pass, inverse column pass
// with CRT, lookahead carry) with a job index in the grid: one launch per stage serves every job of
// the same transform length.  Groups of different lengths are independent and run on several
// streams at once.  A batch whose shape (lengths and job counts) repeats replays a captured CUDA
// graph; only the job descriptors change between replays.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "ctx.h"
#include "kernels.cuh"
#include "modarith.cuh"
#include "serve.h"
#include "stages.cuh"

namespace cg = cooperative_groups;

namespace dml {

DMUL_DEFINE_UPLOAD(upload_constants_batch)

// ---------------------------------------------------------------------------------------------
// fused small product
// ---------------------------------------------------------------------------------------------
// The transform buffers hold one padding word after every 16 (index a + a/16, N + N/16 words): the
// rows base + u*s of a stage (every stride s of these schedules is a multiple of 16) sit at
// spidx(base) + u*(s + s/16), one address per group with constant steps, and the radix-16 center's
// 16 consecutive rows at 17b + u.
__device__ __forceinline__ uint32_t spidx(uint32_t a) { return a + (a >> 4); }
__host__ __device__ constexpr uint32_t small_np(uint32_t N) { return N + N / 16; }
// CTA size of the one-cluster kernels: one CTA per SM holds a product from N = 8192 up (its shared
// memory), so it takes the most warps the register file allows (1024 threads at 64 registers) to
// hide the latency of its twiddle loads and cluster exchanges.
__host__ __device__ constexpr uint32_t small_threads(uint32_t N) { return N >= 8192 ? 1024u : 256u; }

// forward stage t < ns-1 (twiddled: outputs k > 0 go to their twiddle products unreduced)
template <int PI, int R>
__device__ __forceinline__ void sfwd_stage(const Stage &st, const uint2 *tw, uint32_t *sx, uint32_t *sy,
                                           uint32_t n, uint32_t nops) {
    const uint32_t stride = st.m / R, ps = stride + (stride >> 4);
    const uint32_t per_op = n / R;
    for (uint32_t g = threadIdx.x; g < per_op * nops; g += blockDim.x) {
        const bool second = g >= per_op;
        const uint32_t gg = second ? g - per_op : g;
        const uint32_t blk = gg / stride, j = gg - blk * stride;
        uint32_t *pb = (second ? sy : sx) + spidx(blk * st.m + j);
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = pb[u * ps];
        dft<PI, 0, R, 1>(v);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = v[outpos<R>(k)];
            if (k > 0) {
                const uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
                o = shoup<PI>(o, w.x, w.y);
            }
            pb[k * ps] = o;
        }
    }
}

// inverse stage t < ns-1: input 0 reduced (its producer left it unreduced), the others untwiddled;
// outputs unreduced (the next inverse stage, or the final scaling, multiplies them)
template <int PI, int R>
__device__ __forceinline__ void sinv_stage(const Stage &st, const uint2 *tw, uint32_t *sb, uint32_t n) {
    const uint32_t stride = st.m / R, ps = stride + (stride >> 4);
    const uint32_t groups = n / R;
    for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        const uint32_t blk = g / stride, j = g - blk * stride;
        uint32_t *pb = sb + spidx(blk * st.m + j);
        uint32_t v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = pb[k * ps];
        v[0] = red2p<PI>(v[0]);
#pragma unroll
        for (int k = 1; k < R; ++k) {
            const uint2 w = ldtw(tw + st.twi + (k - 1) * stride + j);
            v[k] = shoup<PI>(v[k], w.x, w.y);
        }
        dft<PI, 1, R, 2>(v);
#pragma unroll
        for (int u = 0; u < R; ++u) pb[u * ps] = v[outpos<R>(u)];
    }
}

// last forward stage (radix 16) of every operand, pointwise product (or square), first inverse stage
template <int PI, bool SQR>
__device__ __forceinline__ void scenter(uint32_t *sx, const uint32_t *sy, uint32_t n) {
    constexpr int R = 16;
    for (uint32_t b = threadIdx.x; b < n / R; b += blockDim.x) {
        uint32_t v[2][R];
#pragma unroll
        for (int op = 0; op < (SQR ? 1 : 2); ++op) {
            const uint32_t *sb = (op ? sy : sx) + 17 * b;
#pragma unroll
            for (int u = 0; u < R; ++u) v[op][u] = sb[u];
            dft<PI, 0, R>(v[op]);
        }
        uint32_t z[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t a = v[0][outpos<R>(k)];
            z[k] = pointwise<PI>(a, SQR ? a : v[1][outpos<R>(k)]);
        }
        dft<PI, 1, R, 2>(z);
        uint32_t *sb = sx + 17 * b;
#pragma unroll
        for (int u = 0; u < R; ++u) sb[u] = z[outpos<R>(u)];
    }
}

template <int PI>
__device__ __forceinline__ void small_transform(const SmallPlanDev &sp, const JobDev &J, uint32_t *sx, uint32_t *sy,
                                uint32_t *status) {
    const uint32_t N = sp.N;
    const uint2 *tw = sp.tw[PI];
    const bool sq = J.square != 0;
    uint32_t bad = 0;
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
        uint32_t a = i < J.nx ? J.x[i] : 0u;
        bad |= (a >= kBase);
        if (PI == 0) a = red2p<0>(a);
        sx[spidx(i)] = a;
        if (!sq) {
            uint32_t b = i < J.ny ? J.y[i] : 0u;
            bad |= (b >= kBase);
            if (PI == 0) b = red2p<0>(b);
            sy[spidx(i)] = b;
        }
    }
    const int any_bad = __syncthreads_or((int)bad);
    if (PI == 0 && any_bad && threadIdx.x == 0) atomicOr(status, kStatusInvalid);
    const int ns = sp.ns;
    const uint32_t nops = sq ? 1u : 2u;
    for (int t = 0; t < ns - 1; ++t) {
        DMUL_RADIX_SWITCH(sp.st[t].R, (sfwd_stage<PI, RR>(sp.st[t], tw, sx, sy, N, nops)));
        __syncthreads();
    }
    if (sq) scenter<PI, true>(sx, sy, N);
    else scenter<PI, false>(sx, sy, N);
    __syncthreads();
    for (int t = ns - 2; t >= 0; --t) {
        DMUL_RADIX_SWITCH(sp.st[t].R, (sinv_stage<PI, RR>(sp.st[t], tw, sx, N)));
        __syncthreads();
    }
    for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
        const uint32_t a = spidx(i);
        sx[a] = red1p<PI>(shoup<PI>(sx[a], sp.scale[PI], sp.scales[PI]));
    }
    __syncthreads();
}

// Carry recurrence over the whole (short) product in one CTA: every thread maps a contiguous
// segment, a block scan of the carry maps gives each segment its incoming carry.
__device__ __forceinline__ void small_carry(const JobDev &J, const uint2 *spb, uint32_t *status) {
    __shared__ uint32_t s_w[32];
    __shared__ uint64_t s_top[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
    const uint64_t L = J.L;
    const uint64_t per = (L + blockDim.x - 1) / blockDim.x;
    const uint64_t b0 = (uint64_t)tid * per;
    const uint64_t b1 = b0 + per < L ? b0 + per : L;
    auto digit = [&](uint64_t k) -> uint32_t {
        uint32_t v = J.z[k];
        if (k >= 32 && (k & 31) == 0) v += spb[(k >> 5) - 1].x;
        if (k >= 33 && (k & 31) == 1) v += spb[(k >> 5) - 1].y;
        return v;
    };
    // the segment's map: constant when its last position's carry-out ignores its carry-in (the
    // usual case), else the three carry chains
    uint32_t c0 = 0, c1 = 0, c2 = 0;
    const uint32_t vl = b1 > b0 ? digit(b1 - 1) : 0u;
    const uint32_t ql = qdig(vl);
    if (b1 > b0 && qdig(vl + 2u) == ql) {
        c0 = c1 = c2 = ql;
    } else {
        c1 = 1;
        c2 = 2;
        for (uint64_t k = b0; k < b1; ++k) {
            uint32_t v = digit(k);
            c0 = qdig(v + c0);
            c1 = qdig(v + c1);
            c2 = qdig(v + c2);
        }
    }
    uint32_t f = c0 | (c1 << 2) | (c2 << 4);
    uint32_t inc = f;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, inc, dd);
        if (lane >= dd) inc = map_compose(inc, o);
    }
    uint32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc = kIdentityMap;
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    if (tid == 0) {
        uint32_t agg = kIdentityMap;
        for (int w = 0; w < nw; ++w) {
            uint32_t wf = s_w[w];
            s_w[w] = agg;
            agg = map_compose(wf, agg);
        }
    }
    __syncthreads();
    uint32_t c = map_apply(map_compose(exc, s_w[warp]), 0);
    uint64_t top = 0;
    for (uint64_t k = b0; k < b1; ++k) {
        uint32_t t = digit(k) + c;
        uint32_t q = qdig(t);
        uint32_t o = t - q * kBase;
        c = q;
        if (o) top = k + 1;
        if (k == L - 1 && c) atomicOr(status, kStatusInvalid);
        // the digit() of later positions reads z[k + 1...] and spills only, never z[k]: safe
        J.z[k] = o;
    }
#pragma unroll
    for (int dd = 16; dd >= 1; dd >>= 1) {
        uint64_t o = __shfl_down_sync(0xffffffffu, top, dd);
        top = o > top ? o : top;
    }
    if (lane == 0) s_top[warp] = top;
    __syncthreads();
    if (tid == 0) {
        uint64_t t = 0;
        for (int w = 0; w < nw; ++w) t = s_top[w] > t ? s_top[w] : t;
        if (J.nz) *J.nz = t ? t : 1;
    }
}

// jobs == null: the single job `one` (passed by value, so a lone product needs no descriptor copy)
__global__ void __launch_bounds__(1024) k_small_mul(const SmallPlanDev sp, const JobDev *__restrict__ jobs,
                                                   const JobDev one, uint32_t *status) {
    extern __shared__ uint32_t sm[];
    cg::cluster_group cluster = cg::this_cluster();
    const int pi = (int)cluster.block_rank();
    const JobDev J = jobs ? jobs[blockIdx.y] : one;
    status = job_status(J, status);
    uint32_t *sx = sm, *sy = sm + small_np(sp.N);
    uint2 *spb = (uint2 *)(sm + 2 * small_np(sp.N));
    DMUL_PRIME_SWITCH(pi, (small_transform<PI>(sp, J, sx, sy, status)));
    cluster.sync();
    const uint32_t *s0 = cluster.map_shared_rank(sx, 0);
    const uint32_t *s1 = cluster.map_shared_rank(sx, 1);
    const uint32_t *s2 = cluster.map_shared_rank(sx, 2);
    uint2 *sp0 = cluster.map_shared_rank(spb, 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t nch = (uint32_t)((J.L + 31) >> 5);
    for (uint32_t c = pi + kPrimes * warp; c < nch; c += kPrimes * nw) {
        const uint32_t k = c * 32 + lane;  // < N: L <= N and 32 | N
        uint32_t d0, d1, d2;
        crt_digits(s0[spidx(k)], s1[spidx(k)], s2[spidx(k)], d0, d1, d2);
        uint32_t sv;
        uint2 spv;
        chunk_digits(d0, d1, d2, sv, spv);
        if (k < J.L) J.z[k] = sv;
        if (lane == 31) sp0[c] = spv;
    }
    __threadfence();
    cluster.sync();
    if (pi != 0) return;
    small_carry(J, spb, status);
}

// Persistent form: the cluster's rank-0 CTA draws the next job from the counter and hands it to
// the other two through distributed shared memory; all three then run the job as k_small_mul
// does.  The loop ends when the counter passes the job count.
__global__ void __launch_bounds__(1024) k_small_persist(const SmallPlanDev *__restrict__ plans,
                                                       const JobDev *__restrict__ jobs, uint32_t njobs,
                                                       uint32_t maxN, uint32_t *counter,
                                                       uint32_t *status) {
    extern __shared__ uint32_t sm[];
    __shared__ uint32_t s_job;
    cg::cluster_group cluster = cg::this_cluster();
    const int pi = (int)cluster.block_rank();
    uint32_t *sx = sm, *sy = sm + small_np(maxN);
    uint2 *spb = (uint2 *)(sm + 2 * small_np(maxN));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (;;) {
        if (pi == 0 && threadIdx.x == 0) {
            const uint32_t j = atomicAdd(counter, 1u);
            for (int r = 0; r < kPrimes; ++r) *cluster.map_shared_rank(&s_job, r) = j;
        }
        cluster.sync();
        const uint32_t j = s_job;
        if (j >= njobs) break;
        const JobDev J = jobs[j];
        const SmallPlanDev &sp = plans[J.plan];
        uint32_t *jst = job_status(J, status);
        DMUL_PRIME_SWITCH(pi, (small_transform<PI>(sp, J, sx, sy, jst)));
        cluster.sync();
        const uint32_t *s0 = cluster.map_shared_rank(sx, 0);
        const uint32_t *s1 = cluster.map_shared_rank(sx, 1);
        const uint32_t *s2 = cluster.map_shared_rank(sx, 2);
        uint2 *sp0 = cluster.map_shared_rank(spb, 0);
        const uint32_t nch = (uint32_t)((J.L + 31) >> 5);
        for (uint32_t c = pi + kPrimes * warp; c < nch; c += kPrimes * nw) {
            const uint32_t k = c * 32 + lane;
            uint32_t d0, d1, d2;
            crt_digits(s0[spidx(k)], s1[spidx(k)], s2[spidx(k)], d0, d1, d2);
            uint32_t sv;
            uint2 spv;
            chunk_digits(d0, d1, d2, sv, spv);
            if (k < J.L) J.z[k] = sv;
            if (lane == 31) sp0[c] = spv;
        }
        __threadfence();
        cluster.sync();
        if (pi == 0) small_carry(J, spb, jst);
        cluster.sync();  // shared memory is reused by the next job
    }
}

cudaError_t launch_small_persistent(const SmallPlanDev *plans, uint32_t maxN, const JobDev *jobs,
                                    uint32_t njobs, uint32_t *counter, uint32_t *status, cudaStream_t s) {
    const int sms = current_device_sms();
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(small_threads(maxN), 1, 1);
    cfg.dynamicSmemBytes = (size_t)2 * small_np(maxN) * 4 + (size_t)(maxN / 32) * sizeof(uint2);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kPrimes;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    // resident clusters for this shared-memory size: queried once per size (the query costs tens
    // of microseconds, a short product's whole run)
    static std::mutex occ_mu;
    static std::map<std::pair<int, size_t>, int> occ;  // (device, shared-memory bytes)
    int clusters = 0, dev = 0;
    cudaGetDevice(&dev);
    const std::pair<int, size_t> key(dev, cfg.dynamicSmemBytes);
    {
        std::lock_guard<std::mutex> g(occ_mu);
        auto it = occ.find(key);
        if (it != occ.end()) {
            clusters = it->second;
        } else {
            cfg.gridDim = dim3(kPrimes, 1, 1);
            if (cudaOccupancyMaxActiveClusters(&clusters, k_small_persist, &cfg) != cudaSuccess || clusters < 1) {
                cudaGetLastError();
                clusters = sms / kPrimes;
            }
            occ[key] = clusters;
        }
    }
    uint32_t n = std::min<uint32_t>(njobs, (uint32_t)std::max(1, clusters));
    cfg.gridDim = dim3(kPrimes * n, 1, 1);
    return cudaLaunchKernelEx(&cfg, k_small_persist, plans, jobs, njobs, maxN, counter, status);
}

static size_t small_smem(uint32_t N) { return (size_t)2 * small_np(N) * 4 + (size_t)(N / 32) * sizeof(uint2); }

static cudaError_t small_launch(const SmallPlanDev &sp, const JobDev *jobs, int njobs, const JobDev &one,
                                uint32_t *status, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kPrimes, (unsigned)njobs, 1);
    cfg.blockDim = dim3(small_threads(sp.N), 1, 1);
    cfg.dynamicSmemBytes = small_smem(sp.N);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kPrimes;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_small_mul, sp, jobs, one, status);
}

cudaError_t launch_small_mul(const SmallPlanDev &sp, const JobDev *jobs, int njobs, uint32_t *status,
                             cudaStream_t s) {
    JobDev none;
    memset(&none, 0, sizeof(none));
    return small_launch(sp, jobs, njobs, none, status, s);
}

cudaError_t launch_small_mul_one(const SmallPlanDev &sp, const JobDev &job, uint32_t *status,
                                 cudaStream_t s) {
    return small_launch(sp, nullptr, 1, job, status, s);
}

// ---------------------------------------------------------------------------------------------
// batched four-step pipeline (job = blockIdx.z, or blockIdx.y for the carry)
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_col_fwd_b(const PlanDev pd, const JobDev *__restrict__ jobs,
                                                   uint32_t *status) {
    extern __shared__ uint32_t sm[];
    const JobDev &J = jobs[blockIdx.z];
    const bool second = blockIdx.y != 0;
    if (second && J.square) return;
    const int pi = blockIdx.x % kPrimes;
    const uint32_t tile = blockIdx.x / kPrimes;
    const uint32_t *src = second ? J.y : J.x;
    const uint64_t n = second ? J.ny : J.nx;
    uint32_t *dst = (second ? J.Y : J.X) + (uint64_t)pi * pd.N;
    DMUL_PRIME_SWITCH(pi, (col_fwd_body<PI>(pd, sm, src, n, dst, tile, job_status(J, status))));
}

__global__ void __launch_bounds__(256) k_row_mul_b(const PlanDev pd, const JobDev *__restrict__ jobs) {
    extern __shared__ uint32_t sm[];
    const JobDev &J = jobs[blockIdx.z];
    const uint32_t row = blockIdx.x;
    const int pi = blockIdx.y;
    uint32_t *xr = J.X + (uint64_t)pi * pd.N + (uint64_t)row * pd.N2;
    if (J.square) {
        DMUL_PRIME_SWITCH(pi, (row_mul_body<PI, true>(pd, sm, xr, nullptr)));
    } else {
        const uint32_t *yr = J.Y + (uint64_t)pi * pd.N + (uint64_t)row * pd.N2;
        DMUL_PRIME_SWITCH(pi, (row_mul_body<PI, false>(pd, sm, xr, yr)));
    }
}

__global__ void __launch_bounds__(512) k_col_inv_b(const PlanDev pd, const JobDev *__restrict__ jobs) {
    extern __shared__ uint32_t sm[];
    const JobDev &J = jobs[blockIdx.z];
    col_inv_crt(pd, J.X, J.L, kInvDigits, J.z, J.spill, sm);
}

__global__ void __launch_bounds__(256) k_carry_b(const JobDev *__restrict__ jobs, uint32_t *status) {
    const JobDev &J = jobs[blockIdx.y];
    if (blockIdx.x >= J.ntiles) return;
    carry_tile<256, 8>(J.z, J.z, J.spill, J.L, J.ctl, J.nz, job_status(J, status), J.ntiles);
}

cudaError_t init_kernel_attributes_batch() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_small_mul, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)small_smem(kSmallMaxN))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_small_persist, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)small_smem(kSmallMaxN))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_col_fwd_b, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMaxN1 * 32 * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row_mul_b, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  2 * kMaxN2 * 4)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_col_inv_b, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxN1 * 32 * 4);
}

cudaError_t launch_col_fwd_b(const PlanDev &pd, const JobDev *jobs, int njobs, uint32_t *status,
                             cudaStream_t s) {
    dim3 grid(kPrimes * (pd.N2 / 32), 2, (unsigned)njobs);
    k_col_fwd_b<<<grid, pd.col_threads, (size_t)pd.N1 * 32 * 4, s>>>(pd, jobs, status);
    return cudaGetLastError();
}

cudaError_t launch_row_mul_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s) {
    dim3 grid(pd.N1, kPrimes, (unsigned)njobs);
    k_row_mul_b<<<grid, pd.row_threads, (size_t)2 * pd.N2 * 4, s>>>(pd, jobs);
    return cudaGetLastError();
}

cudaError_t launch_col_inv_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(kPrimes * (pd.N2 / 32), 1, (unsigned)njobs);
    cfg.blockDim = dim3(pd.col_threads, 1, 1);
    cfg.dynamicSmemBytes = (size_t)pd.N1 * 32 * 4;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = kPrimes;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_col_inv_b, pd, jobs);
}

cudaError_t launch_carry_b(const JobDev *jobs, int njobs, uint32_t maxtiles, uint32_t *status,
                           cudaStream_t s) {
    k_carry_b<<<dim3(maxtiles, (unsigned)njobs), 256, 0, s>>>(jobs, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------
static size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

void destroy_batch_state(dmul_ctx *c) {
    if (!c->batch) return;
    free_batch_state(c, c->batch.get());
    c->batch.reset();
}

int init_batch_state(BatchState *b, int priority) {
    for (int i = 0; i < kBatchStreams; ++i) {
        if (cudaStreamCreateWithPriority(&b->streams[i], cudaStreamNonBlocking, priority) != cudaSuccess)
            return DMUL_ERR_CUDA;
        if (cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess) return DMUL_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) return DMUL_ERR_CUDA;
    if (cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) return DMUL_ERR_CUDA;
    return DMUL_OK;
}

void free_batch_state(dmul_ctx *c, BatchState *b) {
    if (b->done_recorded) cudaEventSynchronize(b->done);
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
    if (b->arena) dev_free(c, b->arena, b->arena_cap);
    if (b->djobs) dev_free(c, b->djobs, b->jobs_cap * sizeof(JobDev));
    if (b->dstat) dev_free(c, b->dstat, b->jobs_cap * sizeof(uint32_t));
    if (b->hjobs) cudaFreeHost(b->hjobs);
    if (b->hstat) cudaFreeHost(b->hstat);
    b->arena = nullptr;
    b->djobs = nullptr;
    b->dstat = nullptr;
    b->hjobs = nullptr;
    b->hstat = nullptr;
    b->pending = false;
    b->pend_jobs = nullptr;
    for (int i = 0; i < kBatchStreams; ++i) {
        if (b->streams[i]) cudaStreamDestroy(b->streams[i]);
        if (b->join[i]) cudaEventDestroy(b->join[i]);
        b->streams[i] = nullptr;
        b->join[i] = nullptr;
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->done) cudaEventDestroy(b->done);
    if (b->dcounter) dev_free(c, b->dcounter, 256);
    if (b->dplans) dev_free(c, b->dplans, kMaxSmallPlans * sizeof(SmallPlanDev));
    if (b->hplans) cudaFreeHost(b->hplans);
    b->dcounter = nullptr;
    b->dplans = nullptr;
    b->hplans = nullptr;
    b->fork = b->done = nullptr;
}

static int batch_state(dmul_ctx *c, BatchState **out) {
    if (!c->batch) {
        c->batch = std::make_unique<BatchState>();
        int rc = init_batch_state(c->batch.get());
        if (rc) return rc;
    }
    *out = c->batch.get();
    return DMUL_OK;
}

// Enqueue the launches of every group (on the fork/join streams).  The short products run in up
// to three persistent launches by size class (transform length up to 1536, 6144, 24576): each
// launch sizes its shared memory for its class, so that clusters of short jobs pack several to an
// SM instead of each holding the room of the largest job in the batch.  Each group of longer
// products of one transform length runs as the four batched pipeline launches.  Work items are
// spread over the given streams.
constexpr int kSmallClasses = 3;
inline int small_class(uint64_t N) { return N <= 1536 ? 0 : (N <= 6144 ? 1 : 2); }
struct SmallClass {
    size_t first = 0, count = 0;
    uint32_t maxN = 0;
};
struct SmallLaunch {
    size_t count = 0;  // all short products
    SmallClass cls[kSmallClasses];
    size_t nplans = 0;
};

static int launch_work(dmul_ctx *c, BatchState *b, const std::vector<GroupLaunch> &groups,
                       const SmallLaunch &sl, cudaStream_t *streams, int nstreams, uint32_t *status,
                       bool rows) {
    int si = 0;
    for (int k = 0; k < kSmallClasses; ++k) {
        const SmallClass &sc = sl.cls[k];
        if (!sc.count) continue;
        if (launch_small_persistent(b->dplans, sc.maxN, b->djobs + sc.first, (uint32_t)sc.count, b->dcounter + k,
                                    status, streams[si++ % nstreams]) != cudaSuccess)
            return DMUL_ERR_CUDA;
    }
    for (const GroupLaunch &G : groups) {
        if (G.small) continue;
        cudaStream_t st = streams[si++ % nstreams];
        const JobDev *jd = b->djobs + G.first;
        PlanEntry *pe;
        int rc = get_plan(c, G.N, &pe);
        if (rc) return rc;
        const PlanDev &pd = pe->pd;
        // the specialized passes where the plan has their schedule (the column passes also need
        // 16-byte aligned operands), else the generic ones
        const bool cs = G.aligned && col_pass_specialized(pd), rs = row_pass_specialized(pd);
        if ((cs ? launch_col_fwd_bs(pd, jd, (int)G.count, status, st)
                : launch_col_fwd_b(pd, jd, (int)G.count, status, st)) != cudaSuccess)
            return DMUL_ERR_CUDA;
        if ((rs ? launch_row_pass_ct_b(pd, jd, (int)G.count, st, rows) : launch_row_mul_b(pd, jd, (int)G.count, st)) !=
            cudaSuccess)
            return DMUL_ERR_CUDA;
        if ((col_pass_specialized(pd) ? launch_col_inv_bs(pd, jd, (int)G.count, st)
                                      : launch_col_inv_b(pd, jd, (int)G.count, st)) != cudaSuccess)
            return DMUL_ERR_CUDA;
        if (launch_carry_b(jd, (int)G.count, G.maxtiles, status, st) != cudaSuccess) return DMUL_ERR_CUDA;
    }
    return DMUL_OK;
}

// Descriptor uploads and zeroing of the control words, then the work.
static int upload_and_launch(dmul_ctx *c, BatchState *b, const std::vector<GroupLaunch> &groups,
                             const SmallLaunch &sl, cudaStream_t s, size_t njobs, size_t ctl_off,
                             size_t ctl_bytes, uint32_t *status, bool fork, bool rows) {
    if (cudaMemcpyAsync(b->djobs, b->hjobs, njobs * sizeof(JobDev), cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(b->dstat, 0, njobs * sizeof(uint32_t), s) != cudaSuccess)
        return DMUL_ERR_CUDA;
    if (sl.count) {
        if (cudaMemcpyAsync(b->dplans, b->hplans, sl.nplans * sizeof(SmallPlanDev), cudaMemcpyHostToDevice, s) !=
                cudaSuccess ||
            cudaMemsetAsync(b->dcounter, 0, kSmallClasses * sizeof(uint32_t), s) != cudaSuccess)
            return DMUL_ERR_CUDA;
    }
    if (ctl_bytes && cudaMemsetAsync(b->arena + ctl_off, 0, ctl_bytes, s) != cudaSuccess) return DMUL_ERR_CUDA;
    // the serving loop keeps one row per CTA (rows = false); a whole batch takes several
    // (rowpass.cuh).  fork: the groups spread over the state's streams, joined back to s.
    if (!fork) {
        int rc = launch_work(c, b, groups, sl, &s, 1, status, rows);
        if (rc) return rc;
    } else {
        if (cudaEventRecord(b->fork, s) != cudaSuccess) return DMUL_ERR_CUDA;
        for (int i = 0; i < kBatchStreams; ++i)
            if (cudaStreamWaitEvent(b->streams[i], b->fork, 0) != cudaSuccess) return DMUL_ERR_CUDA;
        int rc = launch_work(c, b, groups, sl, b->streams, kBatchStreams, status, rows);
        if (rc) return rc;
        for (int i = 0; i < kBatchStreams; ++i) {
            if (cudaEventRecord(b->join[i], b->streams[i]) != cudaSuccess) return DMUL_ERR_CUDA;
            if (cudaStreamWaitEvent(s, b->join[i], 0) != cudaSuccess) return DMUL_ERR_CUDA;
        }
    }
    // every job's own status word, for the caller (dmul_batch) or the serving loop's tickets
    if (cudaMemcpyAsync(b->hstat, b->dstat, njobs * sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return DMUL_ERR_CUDA;
    return DMUL_OK;
}

int flush_batch_status(BatchState *b) {
    if (!b->pending) return DMUL_OK;
    b->pending = false;
    if (b->done_recorded && cudaEventSynchronize(b->done) != cudaSuccess) return DMUL_ERR_CUDA;
    int agg = DMUL_OK;
    for (size_t i = 0; i < b->launched; ++i) {
        const int rc = device_code(b->hstat[i]);
        b->pend_jobs[b->order[i]].status = rc;
        if (rc == DMUL_ERR_TIMEOUT || (rc && !agg)) agg = rc;
    }
    b->pend_jobs = nullptr;
    return agg;
}

int run_batch(dmul_ctx *c, dmul_job *jobs, size_t count, cudaStream_t s) {
    BatchState *b;
    auto fail_all = [&](int rc) {
        for (size_t i = 0; i < count; ++i) jobs[i].status = rc;
        return rc;
    };
    int rc = set_device(c);
    if (rc) return fail_all(rc);
    rc = batch_state(c, &b);
    if (rc) return fail_all(rc);
    // the previous batch's jobs get their statuses before this batch reuses the state; an error
    // among them is kept for the next dmul_sync
    const int prev = flush_batch_status(b);
    if (prev && c->batch_err != DMUL_ERR_TIMEOUT) c->batch_err = prev;
    c->last_stream = s;
    std::vector<int> hs(count, DMUL_OK);
    {
        Timed t(c, kStBatch, s);
        rc = run_batch_on(c, b, jobs, count, s, c->status, true, hs.data());
    }
    if (rc) return fail_all(rc);
    for (size_t i = 0; i < count; ++i) jobs[i].status = hs[i] ? hs[i] : DMUL_PENDING;
    b->pend_jobs = jobs;
    b->pending = true;
    return DMUL_OK;
}

size_t job_scratch_bytes(const dmul_ctx *c, const dmul_job &j, bool *four) {
    const uint64_t L = j.nx + j.ny;
    if (four) *four = false;
    const uint64_t Ns = choose_N_small(L);
    if (Ns && !(c->cfg.flags & (DMUL_FLAG_SIXSTEP | DMUL_FLAG_NO_SMALL))) {
        if (small_single_cached(c, Ns) != 0) return 0;
        if (four) *four = true;  // may run as a four-step group (see run_batch_on)
    }
    const uint64_t N = choose_N(L, !(c->cfg.flags & DMUL_FLAG_NO_RADIX5));
    const bool sq = j.x == j.y && j.nx == j.ny;
    return align256((size_t)kPrimes * N * 4) * (sq ? 1 : 2) + align256(((L + 31) / 32 + 1) * sizeof(uint2)) +
           align256(carry_ctl_bytes(L));
}

// The host-side verdict on one job: DMUL_OK, or the code that keeps it out of the launch.
static int check_job(const dmul_ctx *c, const dmul_job &j) {
    if (!j.x || !j.y || !j.z || j.nx == 0 || j.ny == 0) return DMUL_ERR_INVALID;
    const uint64_t L = j.nx + j.ny;
    if (j.z_cap < L) return DMUL_ERR_CAPACITY;
    if (overlaps(j.z, L * 4, j.x, j.nx * 4) || overlaps(j.z, L * 4, j.y, j.ny * 4)) return DMUL_ERR_INVALID;
    if (std::min(j.nx, j.ny) > max_min_limbs()) return DMUL_ERR_TOO_LARGE;
    if (c->cfg.max_limbs && L > c->cfg.max_limbs) return DMUL_ERR_TOO_LARGE;
    if (c->cfg.flags & DMUL_FLAG_SIXSTEP) return DMUL_ERR_INVALID;  // the batched form is four-step only
    if (!choose_N_small(L) && !choose_N(L, !(c->cfg.flags & DMUL_FLAG_NO_RADIX5))) {
        return DMUL_ERR_TOO_LARGE;
    }
    return DMUL_OK;
}

int run_batch_on(dmul_ctx *c, BatchState *b, const dmul_job *jobs, size_t count_in, cudaStream_t s,
                 uint32_t *status, bool use_graph, int *host_status, const uint8_t *four_ok, bool fork_plain) {
    int rc = DMUL_OK;
    b->launched = 0;
    // validate (per job: a rejected job is left out, the others run) and classify
    struct Item { size_t idx; bool small; uint64_t N; bool square; };
    std::vector<Item> items;
    items.reserve(count_in);
    for (size_t i = 0; i < count_in; ++i) {
        const dmul_job &j = jobs[i];
        host_status[i] = check_job(c, j);
        if (host_status[i]) continue;
        const uint64_t L = j.nx + j.ny;
        Item it{i, false, 0, j.x == j.y && j.nx == j.ny};
        uint64_t Ns = choose_N_small(L);
        if (Ns && !(c->cfg.flags & (DMUL_FLAG_SIXSTEP | DMUL_FLAG_NO_SMALL))) {
            it.small = true;
            it.N = Ns;
        } else {
            it.N = choose_N(L, !(c->cfg.flags & DMUL_FLAG_NO_RADIX5));
        }
        items.push_back(it);
    }
    const size_t count = items.size();
    if (count == 0) return DMUL_OK;
    // Size classes with too few short jobs to fill the GPU with clusters: where the plain form
    // measured the four-step pipeline faster for a lone product of that length, those jobs run as
    // four-step groups (a lone short job waits on one cluster's three SMs otherwise).
    {
        const int sms = current_device_sms();
        size_t per_class[kSmallClasses] = {0, 0, 0};
        for (const Item &it : items)
            if (it.small) per_class[small_class(it.N)]++;
        for (Item &it : items) {
            if (!it.small || per_class[small_class(it.N)] * kPrimes >= (size_t)std::max(sms, 1)) continue;
            bool use_small = true;
            if (four_ok) {
                // the serving loop: its scratch was admitted at submission
                if (!four_ok[it.idx]) {
                    if (small_single_cached(c, it.N) < 0) {
                        const dmul_job &j = jobs[it.idx];
                        const uint64_t N4 = choose_N(j.nx + j.ny, !(c->cfg.flags & DMUL_FLAG_NO_RADIX5));
                        if ((rc = prefer_small_single(c, it.N, N4, &use_small))) return rc;  // for later
                    }
                    continue;
                }
                use_small = false;
            } else {
                const dmul_job &j = jobs[it.idx];
                const uint64_t N4 = choose_N(j.nx + j.ny, !(c->cfg.flags & DMUL_FLAG_NO_RADIX5));
                if ((rc = prefer_small_single(c, it.N, N4, &use_small))) return rc;
            }
            if (!use_small) {
                const dmul_job &j = jobs[it.idx];
                it.small = false;
                it.N = choose_N(j.nx + j.ny, !(c->cfg.flags & DMUL_FLAG_NO_RADIX5));
                if (!it.N) return DMUL_ERR_TOO_LARGE;
            }
        }
    }
    // group by (kind, N): the largest transforms first
    std::sort(items.begin(), items.end(), [](const Item &a, const Item &b) {
        if (a.small != b.small) return !a.small;
        if (a.N != b.N) return a.N > b.N;
        return a.idx < b.idx;
    });
    std::vector<GroupLaunch> groups;
    for (size_t i = 0; i < count; ++i) {
        if (groups.empty() || groups.back().small != items[i].small || groups.back().N != items[i].N)
            groups.push_back(GroupLaunch{items[i].small, items[i].N, i, 0, 0});
        groups.back().count++;
    }
    // arena: per medium job X, Y, spill; then all carry control blocks contiguously
    size_t off = 0;
    std::vector<size_t> offX(count), offY(count), offS(count), offC(count);
    for (size_t i = 0; i < count; ++i) {
        const Item &it = items[i];
        if (it.small) continue;
        const dmul_job &j = jobs[it.idx];
        offX[i] = off;
        off = align256(off + (size_t)kPrimes * it.N * 4);
        offY[i] = off;
        if (!it.square) off = align256(off + (size_t)kPrimes * it.N * 4);
        offS[i] = off;
        off = align256(off + ((j.nx + j.ny + 31) / 32 + 1) * sizeof(uint2));
    }
    const size_t ctl_off = off;
    for (size_t i = 0; i < count; ++i) {
        const Item &it = items[i];
        if (it.small) continue;
        const dmul_job &j = jobs[it.idx];
        offC[i] = off;
        off = align256(off + carry_ctl_bytes(j.nx + j.ny));
    }
    const size_t ctl_bytes = off - ctl_off;
    const size_t need = off;  // 0 when every job takes the fused short path
    if (need > b->arena_cap) {
        for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
        b->graphs.clear();
        if (b->done_recorded && cudaEventSynchronize(b->done) != cudaSuccess) return DMUL_ERR_CUDA;
        if (b->arena) dev_free(c, b->arena, b->arena_cap);
        b->arena = nullptr;
        b->arena_cap = 0;
        rc = dev_alloc(c, (void **)&b->arena, need);
        if (rc) return rc;
        b->arena_cap = need;
    }
    if (count > b->jobs_cap) {
        for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
        b->graphs.clear();
        if (b->done_recorded && cudaEventSynchronize(b->done) != cudaSuccess) return DMUL_ERR_CUDA;
        if (b->djobs) dev_free(c, b->djobs, b->jobs_cap * sizeof(JobDev));
        if (b->dstat) dev_free(c, b->dstat, b->jobs_cap * sizeof(uint32_t));
        if (b->hjobs) cudaFreeHost(b->hjobs);
        if (b->hstat) cudaFreeHost(b->hstat);
        b->djobs = nullptr;
        b->dstat = nullptr;
        b->hjobs = nullptr;
        b->hstat = nullptr;
        b->jobs_cap = 0;
        rc = dev_alloc(c, (void **)&b->djobs, count * sizeof(JobDev));
        if (rc) return rc;
        rc = dev_alloc(c, (void **)&b->dstat, count * sizeof(uint32_t));
        if (rc) return rc;
        if (cudaMallocHost(&b->hjobs, count * sizeof(JobDev)) != cudaSuccess) return DMUL_ERR_NOMEM;
        if (cudaMallocHost(&b->hstat, count * sizeof(uint32_t)) != cudaSuccess) return DMUL_ERR_NOMEM;
        b->jobs_cap = count;
    }
    // the previous batch on this state may still read its descriptors (hjobs) and arena
    if (b->done_recorded && cudaEventSynchronize(b->done) != cudaSuccess) return DMUL_ERR_CUDA;
    for (size_t i = 0; i < count; ++i) {
        const Item &it = items[i];
        const dmul_job &j = jobs[it.idx];
        JobDev &d = b->hjobs[i];
        memset(&d, 0, sizeof(d));
        d.x = j.x;
        d.y = j.y;
        d.z = j.z;
        d.nz = j.nz;
        d.nx = j.nx;
        d.ny = j.ny;
        d.L = j.nx + j.ny;
        d.square = it.square ? 1u : 0u;
        d.stat = b->dstat + i;
        if (!it.small) {
            d.X = (uint32_t *)(b->arena + offX[i]);
            d.Y = it.square ? nullptr : (uint32_t *)(b->arena + offY[i]);
            d.spill = (uint2 *)(b->arena + offS[i]);
            d.ctl = (CarryCtl *)(b->arena + offC[i]);
            d.ntiles = (uint32_t)((d.L + kCarryLimbs - 1) / kCarryLimbs);
        }
    }
    for (auto &G : groups) {
        uint32_t mt = 0;
        bool al = true;
        for (size_t i = G.first; i < G.first + G.count; ++i) {
            mt = std::max(mt, b->hjobs[i].ntiles);
            al = al && ((uintptr_t)b->hjobs[i].x & 15) == 0 && ((uintptr_t)b->hjobs[i].y & 15) == 0;
        }
        G.maxtiles = mt;
        G.aligned = al;
    }
    // plans are built outside any capture
    for (auto &G : groups) {
        if (G.small) { SmallPlanEntry *se; rc = get_small_plan(c, G.N, &se); }
        else { PlanEntry *pe; rc = get_plan(c, G.N, &pe); }
        if (rc) return rc;
    }
    // the persistent launch for the short products: their plan table and counter
    SmallLaunch sl;
    size_t small_first = 0;
    for (size_t i = 0; i < count; ++i) {
        if (!items[i].small) continue;
        if (!sl.count) small_first = i;
        ++sl.count;
        // the short items are sorted by decreasing N: each class is one contiguous range
        SmallClass &sc = sl.cls[small_class(items[i].N)];
        if (!sc.count) sc.first = i;
        ++sc.count;
        sc.maxN = std::max<uint32_t>(sc.maxN, (uint32_t)items[i].N);
    }
    if (sl.count) {
        if (!b->dcounter) {
            if ((rc = dev_alloc(c, (void **)&b->dcounter, 256))) return rc;
            if ((rc = dev_alloc(c, (void **)&b->dplans, kMaxSmallPlans * sizeof(SmallPlanDev)))) return rc;
            if (cudaMallocHost(&b->hplans, kMaxSmallPlans * sizeof(SmallPlanDev)) != cudaSuccess) return DMUL_ERR_NOMEM;
        }
        std::vector<uint64_t> ns;
        for (size_t i = small_first; i < small_first + sl.count; ++i) {
            auto f = std::find(ns.begin(), ns.end(), items[i].N);
            uint32_t id = (uint32_t)(f - ns.begin());
            if (f == ns.end()) {
                if (ns.size() == (size_t)kMaxSmallPlans) return DMUL_ERR_INVALID;
                ns.push_back(items[i].N);
                SmallPlanEntry *se;
                if ((rc = get_small_plan(c, items[i].N, &se))) return rc;
                b->hplans[id] = se->sp;
            }
            b->hjobs[i].plan = id;
        }
        sl.nplans = ns.size();
    }
    b->order.resize(count);
    for (size_t i = 0; i < count; ++i) b->order[i] = items[i].idx;
    b->launched = count;
    if (!use_graph) {
        // plain launches (the serving loop's slots: shapes vary, slots overlap), on s or, with
        // fork_plain, spread over the state's streams
        rc = upload_and_launch(c, b, groups, sl, s, count, ctl_off, ctl_bytes, status, fork_plain, false);
        if (rc) return rc;
        if (cudaEventRecord(b->done, s) != cudaSuccess) return DMUL_ERR_CUDA;
        b->done_recorded = true;
        return DMUL_OK;
    }
    std::vector<std::tuple<int, uint64_t, size_t>> key;
    for (auto &G : groups) key.emplace_back((G.small ? 1 : 0) | (G.aligned ? 2 : 0), G.N, G.count);
    for (size_t i = 0; i < count; ++i) key.emplace_back(2, (uint64_t)b->hjobs[i].square, b->hjobs[i].ntiles);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaGraph_t graph;
        cudaStream_t cap = b->streams[0];
        // capture on a private stream, joined to s through events
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return DMUL_ERR_CUDA;
        rc = upload_and_launch(c, b, groups, sl, cap, count, ctl_off, ctl_bytes, status, true, true);
        cudaError_t ce = cudaStreamEndCapture(cap, &graph);
        if (rc) return rc;
        if (ce != cudaSuccess) return DMUL_ERR_CUDA;
        cudaGraphExec_t exec;
        ce = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) return DMUL_ERR_CUDA;
        it = b->graphs.emplace(key, exec).first;
    }
    if (cudaGraphLaunch(it->second, s) != cudaSuccess) return DMUL_ERR_CUDA;
    if (cudaEventRecord(b->done, s) != cudaSuccess) return DMUL_ERR_CUDA;
    b->done_recorded = true;
    return DMUL_OK;
}

}  // namespace dml
