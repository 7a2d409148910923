// rowpass.cuh -- the fused row pass specialized at compile time on the row length N2, as templates;
// rowpass_big.cu (N2 = 1024 .. 8192) and rowpass_small.cu (N2 = 256, 512) instantiate them and
// rowpass.cu dispatches on the plan.
//
// Same arithmetic and data layout as the generic row pass (stages.cuh: forward row DFTs of X and
// Y, pointwise Montgomery product, inverse row DFTs, Sec. 5.4 / 6 / 7.1), but the row length is
// a template parameter, so every stage's radix, span and stride are compile-time constants: group
// indices become shifts and masks, and most swizzled shared-memory addresses fold into immediate
// offsets.  The radix schedule is the planner's (a small radix first, then radix 16); the
// dispatcher checks that the plan has exactly that schedule and otherwise uses the generic pass.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "modarith.cuh"
#include "stages.cuh"

namespace dml {

// Compile-time radix schedule of a power-of-two length N (the planner's pow2_schedule).
template <uint32_t N>
struct Pow2Sched {
    static constexpr int A = ilog2c((int)N);
    static constexpr int NS = (A % 4 ? 1 : 0) + A / 4;
    static constexpr uint32_t radix(int t) { return (A % 4 && t == 0) ? (1u << (A % 4)) : 16u; }
    static constexpr uint32_t span(int t) {  // m of stage t
        uint32_t m = N;
        for (int i = 0; i < t; ++i) m /= radix(i);
        return m;
    }
};

// Working buffers of the specialized pass: one padding word after every 16 (index a + a/16, N + N/16
// words per row).  Every stage's rows base + u*s (s a multiple of 16, or the 16 consecutive rows
// of the center) then sit at pidx(base) + u*(s + s/16): one address per group, immediate offsets
// per row.  Banks: conflict-free for s = 16 and the center; one lane pair of a warp shares a bank
// in the stages with s >= 256 (a CPU check over every access of the four schedules).
template <uint32_t N>
struct RowPad {
    static constexpr uint32_t NP = N + N / 16;
};
__device__ __forceinline__ uint32_t pidx(uint32_t a) { return a + (a >> 4); }

// Rows per CTA of the batched one-CTA-per-rows pass: short rows leave most of a CTA idle (a row of
// N = 256 has 16 radix-16 groups per stage), so for a batch a CTA takes up to 4096 / N consecutive
// rows of one prime: as many as divide the row count N1 and still leave at least two CTAs per SM
// in the grid.  The launcher stores the choice in the plan copy it launches with
// (PlanDev::row_rows).  Lone products and the serving loop's batches keep one row per CTA: with
// the GPU shared between several batches in flight, the finer CTAs gave lower latency (served at
// 70 % load: p50 0.80 against 1.01 ms), while a whole batch gained 11 % throughput from the rows.  Consecutive rows r
// form one padded buffer: pidx(r N + a) = r NP + pidx(a), so the stages run over the rows as one
// longer row whose blocks never straddle two rows.
template <uint32_t N>
static uint32_t row_rows(uint32_t n1, uint64_t rows_total) {
    const int sms = current_device_sms();
    uint32_t r = N >= 4096 ? 1u : 4096u / N;
    while (r > 1 && ((n1 % r) || rows_total / r < 2 * (uint64_t)sms)) r >>= 1;
    return r;
}

template <int PI, uint32_t R, uint32_t M, uint32_t N>
__device__ __forceinline__ void fwd_stage_ct(const Stage &st, const uint2 *tw, uint32_t *sx,
                                             uint32_t *sy, const uint32_t *gx, const uint32_t *gy,
                                             bool from_plain, uint32_t nops, uint32_t rows) {
    constexpr uint32_t stride = M / R;
    constexpr uint32_t pstride = stride + stride / 16;
    static_assert(stride % 16 == 0, "padded rows need strides that are multiples of 16");
    const uint32_t per_op = rows * (N / R);
    constexpr bool has_tw = M > R;
    for (uint32_t g = threadIdx.x; g < per_op * nops; g += blockDim.x) {
        const bool second = g >= per_op;
        const uint32_t gg = second ? g - per_op : g;
        uint32_t *sb = second ? sy : sx;
        const uint32_t blk = gg / stride, j = gg % stride;
        const uint32_t base = blk * M + j;
        uint32_t *pb = sb + pidx(base);
        uint32_t v[R];
        if (from_plain) {
            const uint32_t *src = second ? gy : gx;
#pragma unroll
            for (uint32_t u = 0; u < R; ++u) v[u] = src[base + u * stride];
        } else {
#pragma unroll
            for (uint32_t u = 0; u < R; ++u) v[u] = pb[u * pstride];
        }
        dft<PI, 0, (int)R, has_tw ? 1 : 0>(v);  // outputs k > 0 go straight into the twiddle product
#pragma unroll
        for (uint32_t k = 0; k < R; ++k) {
            uint32_t o = v[outpos<(int)R>((int)k)];
            if (k > 0 && has_tw) {
                const uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
                o = shoup<PI>(o, w.x, w.y);
            }
            pb[k * pstride] = o;
        }
    }
}

// The same stage on X and Y at once (a product, not a square): the groups of X and Y with the
// same index share their twiddle index j, so each thread loads the R - 1 twiddles once for both,
// and the two independent DFTs give the scheduler twice the instruction-level parallelism.
template <int PI, uint32_t R, uint32_t M, uint32_t N>
__device__ __forceinline__ void fwd_stage_pair(const Stage &st, const uint2 *tw, uint32_t *sx, uint32_t *sy,
                                               const uint32_t *gx, const uint32_t *gy, bool from_plain,
                                               uint32_t rows) {
    constexpr uint32_t stride = M / R;
    constexpr uint32_t pstride = stride + stride / 16;
    static_assert(stride % 16 == 0, "padded rows need strides that are multiples of 16");
    const uint32_t per_op = rows * (N / R);
    constexpr bool has_tw = M > R;
    for (uint32_t g = threadIdx.x; g < per_op; g += blockDim.x) {
        const uint32_t blk = g / stride, j = g % stride;
        const uint32_t base = blk * M + j;
        uint32_t *px = sx + pidx(base), *py = sy + pidx(base);
        uint32_t v[R], u[R];
        if (from_plain) {
#pragma unroll
            for (uint32_t k = 0; k < R; ++k) {
                v[k] = gx[base + k * stride];
                u[k] = gy[base + k * stride];
            }
        } else {
#pragma unroll
            for (uint32_t k = 0; k < R; ++k) {
                v[k] = px[k * pstride];
                u[k] = py[k * pstride];
            }
        }
        dft<PI, 0, (int)R, has_tw ? 1 : 0>(v);
        dft<PI, 0, (int)R, has_tw ? 1 : 0>(u);
#pragma unroll
        for (uint32_t k = 0; k < R; ++k) {
            uint32_t o = v[outpos<(int)R>((int)k)], o2 = u[outpos<(int)R>((int)k)];
            if (k > 0 && has_tw) {
                const uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
                o = shoup<PI>(o, w.x, w.y);
                o2 = shoup<PI>(o2, w.x, w.y);
            }
            px[k * pstride] = o;
            py[k * pstride] = o2;
        }
    }
}

template <int PI, uint32_t R, uint32_t M, uint32_t N>
__device__ __forceinline__ void inv_stage_ct(const Stage &st, const uint2 *tw, uint32_t *sb,
                                             uint32_t *gout, uint32_t rows) {
    constexpr uint32_t stride = M / R;
    constexpr uint32_t pstride = stride + stride / 16;
    static_assert(stride % 16 == 0, "padded rows need strides that are multiples of 16");
    const uint32_t groups = rows * (N / R);
    constexpr bool has_tw = M > R;
    for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        const uint32_t blk = g / stride, j = g % stride;
        const uint32_t base = blk * M + j;
        uint32_t *pb = sb + pidx(base);
        uint32_t v[R];
#pragma unroll
        for (uint32_t k = 0; k < R; ++k) v[k] = pb[k * pstride];
        // The previous inverse stage left its outputs unreduced: input 0 is reduced here, the
        // others go through their twiddle product.  This stage's outputs stay unreduced too: the
        // next inverse stage does the same, and after the last one the inverse column pass
        // multiplies every input by a four-step twiddle.
        static_assert(has_tw, "every inverse row stage after the center has twiddles");
        v[0] = red2p<PI>(v[0]);
#pragma unroll
        for (uint32_t k = 1; k < R; ++k) {
            const uint2 w = ldtw(tw + st.twi + (k - 1) * stride + j);
            v[k] = shoup<PI>(v[k], w.x, w.y);
        }
        dft<PI, 1, (int)R, 2>(v);
        if (gout) {
#pragma unroll
            for (uint32_t u = 0; u < R; ++u) gout[base + u * stride] = v[outpos<(int)R>((int)u)];
        } else {
#pragma unroll
            for (uint32_t u = 0; u < R; ++u) pb[u * pstride] = v[outpos<(int)R>((int)u)];
        }
    }
}

// Between the last forward stage (span 256), the center and the first inverse stage (span 256)
// each thread reads only words that its own warp wrote: a group of those stages covers the 16
// words j + 16u of one 256-word block, a center group 16 consecutive words, so the center group
// b and the stage groups of its block, 16 b .. 16 b + 15, have indices in one 32-aligned range,
// which the loops' common stride (the CTA size, a multiple of 32) hands to one warp.  A warp
// barrier then orders these two hand-offs; a CPU check over every row length, rows per CTA and
// CTA size found no word read across warps.  The unpaired forward form gives Y's groups to other
// threads than X's (its operand loop runs past per_op), so products there keep the CTA barrier.
#ifdef DMUL_ROW_UNPAIRED
template <bool SQR>
constexpr bool kCenterWarpLocal = SQR;
#else
template <bool SQR>
constexpr bool kCenterWarpLocal = true;
#endif
template <bool SQR>
__device__ __forceinline__ void center_barrier() {
    if constexpr (kCenterWarpLocal<SQR>) __syncwarp();
    else __syncthreads();
}

// forward stages 0 .. NS-2, then the center, then inverse stages NS-2 .. 0
template <int PI, uint32_t N, int T, bool SQR>
__device__ __forceinline__ void fwd_stages_ct(const PlanDev &pd, const uint2 *tw, uint32_t *sx,
                                              uint32_t *sy, const uint32_t *gx, const uint32_t *gy,
                                              uint32_t rows) {
    using S = Pow2Sched<N>;
    if constexpr (T < S::NS - 1) {
#ifndef DMUL_ROW_UNPAIRED
        if constexpr (!SQR)
            fwd_stage_pair<PI, S::radix(T), S::span(T), N>(pd.rs[T], tw, sx, sy, gx, gy, T == 0, rows);
        else
#endif
            fwd_stage_ct<PI, S::radix(T), S::span(T), N>(pd.rs[T], tw, sx, sy, gx, gy, T == 0, SQR ? 1u : 2u,
                                                          rows);
        if constexpr (T == S::NS - 2) center_barrier<SQR>();  // the center reads this warp's words
        else __syncthreads();
        fwd_stages_ct<PI, N, T + 1, SQR>(pd, tw, sx, sy, gx, gy, rows);
    }
}

template <int PI, uint32_t N, int T>
__device__ __forceinline__ void inv_stages_ct(const PlanDev &pd, const uint2 *tw, uint32_t *sx,
                                              uint32_t *xout, uint32_t rows) {
    using S = Pow2Sched<N>;
    if constexpr (T >= 0) {
        inv_stage_ct<PI, S::radix(T), S::span(T), N>(pd.rs[T], tw, sx, T == 0 ? xout : nullptr, rows);
        if (T > 0) __syncthreads();
        inv_stages_ct<PI, N, T - 1>(pd, tw, sx, xout, rows);
    }
}

// Last forward stage of x (and y), pointwise Montgomery product, first inverse stage, on the 16
// consecutive rows 16b .. 16b+15 (padded index 17b + u); the inverse outputs stay unreduced.
template <int PI, bool SQR>
__device__ __forceinline__ void row_center_ct(uint32_t *sx, const uint32_t *sy, uint32_t groups) {
    constexpr int R = 16;
    for (uint32_t b = threadIdx.x; b < groups; b += blockDim.x) {
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

template <int PI, uint32_t N, bool SQR>
__device__ __forceinline__ void row_core_ct(const PlanDev &pd, uint32_t *sx, uint32_t *sy,
                                            const uint32_t *xin, const uint32_t *yin,
                                            uint32_t *__restrict__ xout, uint32_t rows = 1) {
    using S = Pow2Sched<N>;
    const uint2 *tw = pd.tw[PI];
    fwd_stages_ct<PI, N, 0, SQR>(pd, tw, sx, sy, xin, yin, rows);
    static_assert(S::radix(S::NS - 1) == 16, "the center stage is radix 16");
    row_center_ct<PI, SQR>(sx, sy, rows * (N / 16));
    center_barrier<SQR>();  // the first inverse stage reads this warp's words
    inv_stages_ct<PI, N, S::NS - 2>(pd, tw, sx, xout, rows);
}

template <uint32_t N, bool SQR>
__global__ void __launch_bounds__(256) k_row_ct(const PlanDev pd, uint32_t *X, const uint32_t *Y,
                                                uint32_t *status) {
    extern __shared__ uint32_t sm[];
    pdl_trigger();
    row_wait_prime(pd, blockIdx.y, status);
    const uint32_t rows = pd.row_rows ? pd.row_rows : 1u;
    const uint32_t row = blockIdx.x * rows;
    const int pi = blockIdx.y;
    uint32_t *xr = X + (uint64_t)pi * pd.N + (uint64_t)row * N;
    const uint32_t *yr = SQR ? nullptr : Y + (uint64_t)pi * pd.N + (uint64_t)row * N;
    DMUL_PRIME_SWITCH(pi, (row_core_ct<PI, N, SQR>(pd, sm, sm + rows * RowPad<N>::NP, xr, yr, xr, rows)));
}

// the plain form for a batch of jobs of one transform length (job = blockIdx.z)
template <uint32_t N>
__global__ void __launch_bounds__(256) k_row_ct_b(const PlanDev pd, const JobDev *__restrict__ jobs) {
    extern __shared__ uint32_t sm[];
    const JobDev &J = jobs[blockIdx.z];
    const uint32_t rows = pd.row_rows ? pd.row_rows : 1u;
    const uint32_t row = blockIdx.x * rows;
    const int pi = blockIdx.y;
    uint32_t *xr = J.X + (uint64_t)pi * pd.N + (uint64_t)row * N;
    uint32_t *sy = sm + rows * RowPad<N>::NP;
    if (J.square) {
        DMUL_PRIME_SWITCH(pi, (row_core_ct<PI, N, true>(pd, sm, sy, xr, nullptr, xr, rows)));
    } else {
        const uint32_t *yr = J.Y + (uint64_t)pi * pd.N + (uint64_t)row * N;
        DMUL_PRIME_SWITCH(pi, (row_core_ct<PI, N, false>(pd, sm, sy, xr, yr, xr, rows)));
    }
}

// persistent TMA-fed form (see row_mul_tma_body in stages.cuh for the protocol)
template <int PI, uint32_t N, bool SQR>
__device__ __forceinline__ void row_tma_ct_body(const PlanDev &pd, uint32_t *sm, uint32_t *X,
                                                const uint32_t *Y, uint32_t *status) {
    constexpr uint32_t NP = RowPad<N>::NP;
    uint32_t *land = sm;
    uint32_t *sx = sm + 4 * N, *sy = sm + 4 * N + NP;
    uint64_t *bar = (uint64_t *)(sm + 4 * N + 2 * NP);  // an even word offset: 8-byte aligned
    const uint32_t G = gridDim.x;
    const uint64_t base = (uint64_t)PI * pd.N;
    constexpr uint32_t bytes = N * 4;
    constexpr uint32_t per_row = (SQR ? 1u : 2u) * bytes;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t r = blockIdx.x;
    if (threadIdx.x == 0 && r < pd.N1) {
        mbar_expect_tx(&bar[0], per_row);
        tma_load_1d(land, X + base + (uint64_t)r * N, bytes, &bar[0]);
        if (!SQR) tma_load_1d(land + N, Y + base + (uint64_t)r * N, bytes, &bar[0]);
    }
    for (uint32_t it = 0; r < pd.N1; ++it, r += G) {
        const uint32_t b = it & 1u;
        const uint32_t rn = r + G;
        if (threadIdx.x == 0 && rn < pd.N1) {
            uint32_t *dst = land + (b ^ 1u) * 2 * N;
            fence_proxy_async();
            mbar_expect_tx(&bar[b ^ 1u], per_row);
            tma_load_1d(dst, X + base + (uint64_t)rn * N, bytes, &bar[b ^ 1u]);
            if (!SQR) tma_load_1d(dst + N, Y + base + (uint64_t)rn * N, bytes, &bar[b ^ 1u]);
        }
        const int ok = __syncthreads_and(mbar_wait(&bar[b], (it >> 1) & 1u, pd.spin) ? 1 : 0);
        if (!ok) {
            if (threadIdx.x == 0) {
                atomicOr(status, kStatusTimeout);
                if (rn < pd.N1) mbar_wait(&bar[b ^ 1u], ((it + 1) >> 1) & 1u);
            }
            return;
        }
        const uint32_t *lx = land + b * 2 * N;
        row_core_ct<PI, N, SQR>(pd, sx, sy, lx, lx + N, X + base + (uint64_t)r * N);
        __syncthreads();
    }
}

template <uint32_t N, bool SQR>
__global__ void __launch_bounds__(256) k_row_tma_ct(const PlanDev pd, uint32_t *X, const uint32_t *Y,
                                                    uint32_t *status) {
    extern __shared__ __align__(16) uint32_t sm[];
    pdl_trigger();
    row_wait_prime(pd, blockIdx.y, status);
    const int pi = blockIdx.y;
    DMUL_PRIME_SWITCH(pi, (row_tma_ct_body<PI, N, SQR>(pd, sm, X, Y, status)));
}

// landing area (two rows of x and y, plain) + padded working buffers + two mbarriers
template <uint32_t N>
static constexpr size_t row_tma_ct_smem() { return ((size_t)4 * N + 2 * RowPad<N>::NP) * 4 + 16; }

template <uint32_t N>
static bool schedule_matches(const PlanDev &pd) {
    using S = Pow2Sched<N>;
    if (pd.N2 != N || pd.nrs != S::NS) return false;
    for (int t = 0; t < S::NS; ++t)
        if (pd.rs[t].R != S::radix(t) || pd.rs[t].m != S::span(t)) return false;
    return true;
}

template <uint32_t N>
static cudaError_t launch_ct(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,
                             uint32_t *status, cudaStream_t s) {
    if (pd.row_tma) {
        dim3 grid(pd.row_grid ? pd.row_grid : 256, kPrimes);
        const size_t smem = row_tma_ct_smem<N>();
        if (square) return launch_pdl(k_row_tma_ct<N, true>, grid, dim3(pd.row_threads), smem, s, 1, pd, X, Y, status);
        return launch_pdl(k_row_tma_ct<N, false>, grid, dim3(pd.row_threads), smem, s, 1, pd, X, Y, status);
    } else {
        PlanDev p = pd;
        p.row_rows = 1;
        dim3 grid(pd.N1, kPrimes);
        const size_t smem = (size_t)(square ? 1 : 2) * RowPad<N>::NP * 4;
        if (square) return launch_pdl(k_row_ct<N, true>, grid, dim3(pd.row_threads), smem, s, 1, p, X, Y, status);
        return launch_pdl(k_row_ct<N, false>, grid, dim3(pd.row_threads), smem, s, 1, p, X, Y, status);
    }
    return cudaGetLastError();
}



template <uint32_t N>
static cudaError_t attrs_ct() {
    cudaError_t e;
    // the rows form holds up to 4096 / N rows (N < 4096)
    const int plain = 2 * (N >= 4096 ? 1 : 4096 / N) * RowPad<N>::NP * 4, tma = (int)row_tma_ct_smem<N>();
    if ((e = cudaFuncSetAttribute(k_row_ct<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, plain)))
        return e;
    if ((e = cudaFuncSetAttribute(k_row_ct<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, plain)))
        return e;
    if ((e = cudaFuncSetAttribute(k_row_ct_b<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, plain)))
        return e;
    if ((e = cudaFuncSetAttribute(k_row_tma_ct<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, tma)))
        return e;
    return cudaFuncSetAttribute(k_row_tma_ct<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, tma);
}


template <uint32_t N>
static cudaError_t launch_ct_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s, bool rows) {
    PlanDev p = pd;
    p.row_rows = rows ? row_rows<N>(pd.N1, (uint64_t)pd.N1 * kPrimes * (uint64_t)njobs) : 1u;
    dim3 grid(pd.N1 / p.row_rows, kPrimes, (unsigned)njobs);
    k_row_ct_b<N><<<grid, pd.row_threads, (size_t)2 * p.row_rows * RowPad<N>::NP * 4, s>>>(p, jobs);
    return cudaGetLastError();
}


// ---- step 2 of the six-step form (Sec. 7.2) and its inverse, specialized the same way --------------
// The length-N DFTs (the column schedule, pd.cs) along the contiguous rows of the N2 x N matrix,
// with the four-step twiddle xi_N^(k1 n2) = Q[k][n2] A[b][n2] on the last forward stage's outputs
// (the inverse: the scaled inverse tables on the first stage's inputs).  n2 is the CTA's row, so
// the R - 1 factors Q[k][n2] are shared by the CTA.  Same tables, stage order and output order as
// the generic k_rowdft6 (sixstep.cu); the inverse ends reduced to [0, p) for the natural CRT.
template <int PI, uint32_t N, int T>
__device__ __forceinline__ void fwd6_stages(const Stage *cs, const uint2 *tw, uint32_t *sb, const uint32_t *g) {
    using S = Pow2Sched<N>;
    if constexpr (T < S::NS - 1) {
        fwd_stage_ct<PI, S::radix(T), S::span(T), N>(cs[T], tw, sb, nullptr, g, nullptr, T == 0, 1u, 1u);
        __syncthreads();
        fwd6_stages<PI, N, T + 1>(cs, tw, sb, g);
    }
}

template <int PI, uint32_t N, int T>
__device__ __forceinline__ void inv6_stages(const Stage *cs, const uint2 *tw, uint32_t *sb) {
    if constexpr (T >= 0) {
        using S = Pow2Sched<N>;
        inv_stage_ct<PI, S::radix(T), S::span(T), N>(cs[T], tw, sb, nullptr, 1u);
        __syncthreads();
        inv6_stages<PI, N, T - 1>(cs, tw, sb);
    }
}

template <int PI, uint32_t N, bool INV>
__device__ __forceinline__ void rowdft6_body(const PlanDev &pd, uint32_t *sb, uint2 *qs, uint32_t *row, uint32_t n2) {
    using S = Pow2Sched<N>;
    static_assert(S::radix(S::NS - 1) == 16, "the last stage is radix 16");
    constexpr uint32_t nb = N / 16;
    const uint2 *tw = pd.tw[PI];
    const uint2 *A = tw + (INV ? pd.offAi : pd.offA);
    if (threadIdx.x >= 1 && threadIdx.x < 16)
        qs[threadIdx.x] = ldtw(tw + (INV ? pd.offQi : pd.offQ) + (uint64_t)threadIdx.x * pd.N2 + n2);
    if (!INV) {
        fwd6_stages<PI, N, 0>(pd.cs, tw, sb, row);  // ends with a barrier (qs visible too)
        for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
            uint32_t v[16];
            const uint32_t *s = sb + 17 * b;
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = s[u];
            dft<PI, 0, 16, 2>(v);  // every output goes straight into the twiddle products
            const uint2 a = ldtw(A + (uint64_t)b * pd.N2 + n2);
            uint32_t o[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                uint32_t x = v[outpos<16>(k)];
                if (k > 0) x = shoup<PI>(x, qs[k].x, qs[k].y);
                o[k] = shoup<PI>(x, a.x, a.y);
            }
            uint4 *dst = (uint4 *)(row + 16 * b);
#pragma unroll
            for (int i = 0; i < 4; ++i) dst[i] = make_uint4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
        }
    } else {
        __syncthreads();  // qs
        for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
            const uint2 a = ldtw(A + (uint64_t)b * pd.N2 + n2);
            const uint4 *src = (const uint4 *)(row + 16 * b);
            uint32_t v[16];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint4 t = src[i];
                v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                uint32_t x = v[k];
                if (k > 0) x = shoup<PI>(x, qs[k].x, qs[k].y);
                v[k] = shoup<PI>(x, a.x, a.y);
            }
            dft<PI, 1, 16, 2>(v);  // the next inverse stage reduces / untwiddles its inputs
            uint32_t *s = sb + 17 * b;
#pragma unroll
            for (int u = 0; u < 16; ++u) s[u] = v[outpos<16>(u)];
        }
        __syncthreads();
        inv6_stages<PI, N, S::NS - 2>(pd.cs, tw, sb);
        for (uint32_t i = threadIdx.x; i < N / 4; i += blockDim.x) {
            uint32_t o[4];
#pragma unroll
            for (int t = 0; t < 4; ++t) o[t] = red1p<PI>(red2p<PI>(sb[pidx(4 * i + t)]));
            ((uint4 *)row)[i] = make_uint4(o[0], o[1], o[2], o[3]);
        }
    }
}

template <uint32_t N, bool INV>
__global__ void __launch_bounds__(256) k_rowdft6_ct(const PlanDev pd, uint32_t *A) {
    extern __shared__ uint32_t sm[];
    __shared__ uint2 qs[16];
    const uint32_t n2 = blockIdx.x;
    const int pi = blockIdx.y;
    uint32_t *row = A + (uint64_t)pi * pd.N + (uint64_t)n2 * N;
    DMUL_PRIME_SWITCH(pi, (rowdft6_body<PI, N, INV>(pd, sm, qs, row, n2)));
}

template <uint32_t N>
static bool cols_schedule_matches(const PlanDev &pd) {
    using S = Pow2Sched<N>;
    if (pd.N1 != N || pd.ncs != S::NS) return false;
    for (int t = 0; t < S::NS; ++t)
        if (pd.cs[t].R != S::radix(t) || pd.cs[t].m != S::span(t)) return false;
    return true;
}

template <uint32_t N>
static cudaError_t launch_dft6(const PlanDev &pd, uint32_t *A, bool inv, cudaStream_t s) {
    const unsigned threads = N / 16 < 64 ? 64u : (N / 16 > 256 ? 256u : N / 16);
    const size_t smem = (size_t)RowPad<N>::NP * 4;
    dim3 grid(pd.N2, kPrimes);
    if (inv) k_rowdft6_ct<N, true><<<grid, threads, smem, s>>>(pd, A);
    else k_rowdft6_ct<N, false><<<grid, threads, smem, s>>>(pd, A);
    return cudaGetLastError();
}

template <uint32_t... Ns>
struct RowSet {
    static bool dft6_matches(const PlanDev &pd) {
        bool r = false;
        (void)((pd.N1 == Ns && (r = cols_schedule_matches<Ns>(pd), true)) || ...);
        return r;
    }
    static cudaError_t dft6(const PlanDev &pd, uint32_t *A, bool inv, cudaStream_t s) {
        cudaError_t r = cudaErrorInvalidValue;
        (void)((pd.N1 == Ns && (r = launch_dft6<Ns>(pd, A, inv, s), true)) || ...);
        return r;
    }
    static bool matches(const PlanDev &pd) {
        bool r = false;
        (void)((pd.N2 == Ns && (r = schedule_matches<Ns>(pd), true)) || ...);
        return r;
    }
    static cudaError_t run(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square, uint32_t *status,
                           cudaStream_t s) {
        cudaError_t r = cudaErrorInvalidValue;
        (void)((pd.N2 == Ns && (r = launch_ct<Ns>(pd, X, Y, square, status, s), true)) || ...);
        return r;
    }
    static cudaError_t run_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s, bool rows) {
        cudaError_t r = cudaErrorInvalidValue;
        (void)((pd.N2 == Ns && (r = launch_ct_b<Ns>(pd, jobs, njobs, s, rows), true)) || ...);
        return r;
    }
    static cudaError_t attrs() {
        cudaError_t r = cudaSuccess;
        (void)(((r = attrs_ct<Ns>()) != cudaSuccess) || ...);
        return r;
    }
};

// The entry points each instantiating translation unit defines for its set (TAG: big, small).
#define DMUL_ROWPASS_SET(TAG, ...)                                                                    \
    DMUL_DEFINE_UPLOAD(upload_constants_rowpass_##TAG)                                                 \
    using RowSet_##TAG = RowSet<__VA_ARGS__>;                                                          \
    bool rowpass_##TAG##_matches(const PlanDev &pd) { return RowSet_##TAG::matches(pd); }             \
    cudaError_t rowpass_##TAG##_run(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,   \
                                   uint32_t *status, cudaStream_t s) {                                 \
        return RowSet_##TAG::run(pd, X, Y, square, status, s);                                         \
    }                                                                                                  \
    cudaError_t rowpass_##TAG##_run_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s, \
                                     bool rows) {                                                      \
        return RowSet_##TAG::run_b(pd, jobs, njobs, s, rows);                                          \
    }                                                                                                  \
    cudaError_t rowpass_##TAG##_attrs() { return RowSet_##TAG::attrs(); }                            \
    bool rowpass_##TAG##_dft6_matches(const PlanDev &pd) { return RowSet_##TAG::dft6_matches(pd); }   \
    cudaError_t rowpass_##TAG##_dft6(const PlanDev &pd, uint32_t *A, bool inv, cudaStream_t s) {      \
        return RowSet_##TAG::dft6(pd, A, inv, s);                                                      \
    }

}  // namespace dml
