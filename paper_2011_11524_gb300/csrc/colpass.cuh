// colpass.cuh -- the column passes specialized at compile time on the column length N1, as
// templates; colpass_big.cu and colpass_small.cu instantiate them for their sets of N1 (separate
// translation units that compile in parallel) and colpass.cu dispatches on the plan.
//
// Same arithmetic, layout and order as the generic column passes (stages.cuh: column DFTs of
// length N1 with the four-step twiddle, Sec. 7.1 / 7.8; the inverse with the 2^32 N^-1 scale of
// Sec. 6 and the cluster CRT of Sec. 8.2.2), with N1 a template parameter so that each stage's
// radix, span and stride are compile-time constants (group indices become shifts, shared-memory
// addresses immediate offsets).  The dispatcher uses them only when the plan's column schedule is
// the planner's (radix 3 or 5 first for 3*2^a or 5*2^a, then a small power of two, then radix 16).
#pragma once
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "modarith.cuh"
#include "stages.cuh"

namespace cg = cooperative_groups;

namespace dml {

template <uint32_t N1>
struct ColSched {
    static constexpr uint32_t F = (N1 % 3) == 0 ? 3u : (N1 % 5) == 0 ? 5u : 1u;  // odd factor
    static constexpr uint32_t P = N1 / F;
    static constexpr int A = ilog2c((int)P);
    static constexpr int NS = (F > 1 ? 1 : 0) + (A % 4 ? 1 : 0) + A / 4;
    static constexpr uint32_t radix(int t) {
        if (F > 1) {
            if (t == 0) return F;
            t -= 1;
        }
        return (A % 4 && t == 0) ? (1u << (A % 4)) : 16u;
    }
    static constexpr uint32_t span(int t) {
        uint32_t m = N1;
        for (int i = 0; i < t; ++i) m /= radix(i);
        return m;
    }
};

// stage 0 of the forward pass on the staged limb tile (in place)
template <int PI, uint32_t R, uint32_t N1>
__device__ __forceinline__ void colf0_ct(const Stage &st, const uint2 *tw, uint32_t *sm, uint32_t &bad) {
    constexpr uint32_t stride = N1 / R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t j = warp; j < stride; j += nw) {
        uint32_t v[R];
#pragma unroll
        for (uint32_t u = 0; u < R; ++u) {
            uint32_t a = sm[(j + u * stride) * 32 + lane];
            if (PI == 0) bad |= (a >= kBase);  // prime 0's CTAs report invalid limbs
            if (PI == 0) a = red2p<PI>(a);  // 10^9 < 4 p0: [0, 10^9) -> [0, 2 p0)
            v[u] = a;
        }
        dft<PI, 0, (int)R, 1>(v);
#pragma unroll
        for (uint32_t k = 0; k < R; ++k) {
            uint32_t o = v[outpos<(int)R>((int)k)];
            if (k > 0) {
                const uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
                o = shoup<PI>(o, w.x, w.y);
            }
            sm[(j + k * stride) * 32 + lane] = o;
        }
    }
}

// a middle stage (forward: DFT then twiddle; inverse: untwiddle then DFT), in place
template <int PI, uint32_t R, uint32_t M, uint32_t N1, bool INV>
__device__ __forceinline__ void colmid_ct(const Stage &st, const uint2 *tw, uint32_t *sm,
                                          bool final_reduce) {
    constexpr uint32_t stride = M / R;
    constexpr uint32_t groups = N1 / R;
    constexpr bool has_tw = M > R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t g = warp; g < groups; g += nw) {
        const uint32_t blk = g / stride, j = g % stride;
        const uint32_t base = blk * M + j;
        uint32_t v[R];
#pragma unroll
        for (uint32_t u = 0; u < R; ++u) v[u] = sm[(base + u * stride) * 32 + lane];
        if (!INV) {
            dft<PI, 0, (int)R, has_tw ? 1 : 0>(v);
#pragma unroll
            for (uint32_t k = 0; k < R; ++k) {
                uint32_t o = v[outpos<(int)R>((int)k)];
                if (k > 0 && has_tw) {
                    const uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
                    o = shoup<PI>(o, w.x, w.y);
                }
                sm[(base + k * stride) * 32 + lane] = o;
            }
        } else {
            // inputs left unreduced by the previous inverse stage: 0 reduced, the others
            // multiplied by their twiddles; outputs unreduced unless this is the last stage
            static_assert(has_tw, "every inverse column stage after the first has twiddles");
            v[0] = red2p<PI>(v[0]);
#pragma unroll
            for (uint32_t k = 1; k < R; ++k) {
                const uint2 w = ldtw(tw + st.twi + (k - 1) * stride + j);
                v[k] = shoup<PI>(v[k], w.x, w.y);
            }
            if (final_reduce) {
                dft<PI, 1, (int)R>(v);
#pragma unroll
                for (uint32_t u = 0; u < R; ++u) sm[(base + u * stride) * 32 + lane] = red1p<PI>(v[outpos<(int)R>((int)u)]);
            } else {
                dft<PI, 1, (int)R, 2>(v);
#pragma unroll
                for (uint32_t u = 0; u < R; ++u) sm[(base + u * stride) * 32 + lane] = v[outpos<(int)R>((int)u)];
            }
        }
    }
}

// Q[k][n2] for k = 1..R-1: the lane's column n2 is fixed for the whole tile, so the R-1 factors
// are loaded once and kept in registers across the N1/R groups.
template <int PI, uint32_t R>
__device__ __forceinline__ void load_q(const uint2 *Q, uint32_t N2, uint32_t n2, uint2 (&q)[R]) {
#pragma unroll
    for (uint32_t k = 1; k < R; ++k) q[k] = ldtw(Q + (uint64_t)k * N2 + n2);
}

// last forward stage (m == R) + four-step twiddle Q[k][n2] * A[b][n2] + store of the residues
template <int PI, uint32_t R, uint32_t N1>
__device__ __forceinline__ void colf_last_ct(const PlanDev &pd, const uint32_t *sm,
                                             uint32_t *__restrict__ dst, uint32_t n2) {
    constexpr uint32_t nb = N1 / R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint2 *A = pd.tw[PI] + pd.offA;
    uint2 q[R];
    load_q<PI, R>(pd.tw[PI] + pd.offQ, pd.N2, n2, q);
    for (uint32_t b = warp; b < nb; b += nw) {
        uint32_t v[R];
#pragma unroll
        for (uint32_t u = 0; u < R; ++u) v[u] = sm[(b * R + u) * 32 + lane];
        const uint2 a = ldtw(A + (uint64_t)b * pd.N2 + n2);
        dft<PI, 0, (int)R, 2>(v);
#pragma unroll
        for (uint32_t k = 0; k < R; ++k) {
            uint32_t o = v[outpos<(int)R>((int)k)];
            if (k > 0) o = shoup<PI>(o, q[k].x, q[k].y);
            o = shoup<PI>(o, a.x, a.y);
            dst[(uint64_t)(b * R + k) * pd.N2 + n2] = o;
        }
    }
}

// first inverse stage on the staged residue tile: inverse four-step twiddle, inverse DFT
template <int PI, uint32_t R, uint32_t N1>
__device__ __forceinline__ void coli_first_ct(const PlanDev &pd, uint32_t *sm, uint32_t n2) {
    constexpr uint32_t nb = N1 / R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint2 *A = pd.tw[PI] + pd.offAi;
    uint2 q[R];
    load_q<PI, R>(pd.tw[PI] + pd.offQi, pd.N2, n2, q);
    for (uint32_t b = warp; b < nb; b += nw) {
        uint32_t v[R];
        const uint2 a = ldtw(A + (uint64_t)b * pd.N2 + n2);
#pragma unroll
        for (uint32_t k = 0; k < R; ++k) {
            uint32_t o = sm[(b * R + k) * 32 + lane];
            if (k > 0) o = shoup<PI>(o, q[k].x, q[k].y);
            v[k] = shoup<PI>(o, a.x, a.y);
        }
        dft<PI, 1, (int)R, 2>(v);  // the next inverse stage reduces / untwiddles its inputs
#pragma unroll
        for (uint32_t u = 0; u < R; ++u) sm[(b * R + u) * 32 + lane] = v[outpos<(int)R>((int)u)];
    }
}

// forward middle stages t = T .. NS-2
template <int PI, uint32_t N1, int T>
__device__ __forceinline__ void colf_mids_ct(const PlanDev &pd, uint32_t *sm) {
    using S = ColSched<N1>;
    if constexpr (T < S::NS - 1) {
        colmid_ct<PI, S::radix(T), S::span(T), N1, false>(pd.cs[T], pd.tw[PI], sm, false);
        __syncthreads();
        colf_mids_ct<PI, N1, T + 1>(pd, sm);
    }
}

// inverse middle stages t = T .. 0 (the last one reduces to [0, p))
template <int PI, uint32_t N1, int T>
__device__ __forceinline__ void coli_mids_ct(const PlanDev &pd, uint32_t *sm) {
    using S = ColSched<N1>;
    if constexpr (T >= 0) {
        colmid_ct<PI, S::radix(T), S::span(T), N1, true>(pd.cs[T], pd.tw[PI], sm, T == 0);
        __syncthreads();
        coli_mids_ct<PI, N1, T - 1>(pd, sm);
    }
}

template <int PI, uint32_t N1>
__device__ __forceinline__ void col_fwd_ct_body(const PlanDev &pd, uint32_t *sm,
                                                const uint32_t *__restrict__ src, uint64_t n,
                                                uint32_t *__restrict__ dst, uint32_t tile,
                                                uint32_t *status) {
    using S = ColSched<N1>;
    const uint32_t n2 = tile * 32 + (threadIdx.x & 31);
    uint32_t bad = 0;
    tile_load_async(sm, src, n, N1, pd.N2, tile * 32);
    colf0_ct<PI, S::radix(0), N1>(pd.cs[0], pd.tw[PI], sm, bad);
    if (PI == 0 && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusInvalid);
    __syncthreads();
    colf_mids_ct<PI, N1, 1>(pd, sm);
    colf_last_ct<PI, S::radix(S::NS - 1), N1>(pd, sm, dst, n2);
}

template <int PI, uint32_t N1>
__device__ __forceinline__ void col_inv_ct_body(const PlanDev &pd, const uint32_t *__restrict__ src,
                                                uint32_t *sm, uint32_t n2) {
    using S = ColSched<N1>;
    tile_load_async(sm, src, pd.N, N1, pd.N2, n2 & ~31u);
    coli_first_ct<PI, S::radix(S::NS - 1), N1>(pd, sm, n2);
    __syncthreads();
    coli_mids_ct<PI, N1, S::NS - 2>(pd, sm);
}

// grid (3 * N2/32, operands): blockIdx.x = 3 * tile + prime; x and y 16-byte aligned
template <uint32_t N1>
__global__ void __launch_bounds__(512) k_col_fwd_ct(const PlanDev pd, const uint32_t *__restrict__ x,
                                                    uint64_t nx, const uint32_t *__restrict__ y,
                                                    uint64_t ny, uint32_t *X, uint32_t *Y,
                                                    uint32_t *status) {
    extern __shared__ __align__(16) uint32_t sm[];
    pdl_trigger();
    prefetch_tables(pd);
    pdl_wait();
    uint32_t pi, tile;
    bool second;
    fwd_order(pi, tile, second);
    const uint32_t *src = second ? y : x;
    const uint64_t n = second ? ny : nx;
    uint32_t *dst = (second ? Y : X) + (uint64_t)pi * pd.N;
    DMUL_PRIME_SWITCH((int)pi, (col_fwd_ct_body<PI, N1>(pd, sm, src, n, dst, tile, status)));
    fwd_done(pd, pi, 32);
}

// the same for a batch of jobs of one transform length (job = blockIdx.z)
template <uint32_t N1>
__global__ void __launch_bounds__(512) k_col_fwd_ct_b(const PlanDev pd, const JobDev *__restrict__ jobs,
                                                      uint32_t *status) {
    extern __shared__ __align__(16) uint32_t sm[];
    const JobDev &J = jobs[blockIdx.z];
    const bool second = blockIdx.y != 0;
    if (second && J.square) return;
    const int pi = blockIdx.x % kPrimes;
    const uint32_t tile = blockIdx.x / kPrimes;
    uint32_t *dst = (second ? J.Y : J.X) + (uint64_t)pi * pd.N;
    DMUL_PRIME_SWITCH(pi, (col_fwd_ct_body<PI, N1>(pd, sm, second ? J.y : J.x, second ? J.ny : J.nx, dst,
                                                   tile, job_status(J, status))));
}

// cluster of three CTAs (rank = prime) per 32-column tile, then the CRT epilogue
template <uint32_t N1, int MODE>
__global__ void __launch_bounds__(512) k_col_inv_ct(const PlanDev pd, const uint32_t *__restrict__ X,
                                                    uint64_t L, uint32_t *__restrict__ out,
                                                    uint2 *__restrict__ spill, uint64_t *zero,
                                                    uint32_t nzero) {
    extern __shared__ __align__(16) uint32_t sm[];
    pdl_trigger();
    pdl_wait();
    zero_words(zero, nzero);
    const int pi = (int)cg::this_cluster().block_rank();
    const uint32_t n2 = (blockIdx.x / kPrimes) * 32 + (threadIdx.x & 31);
    const uint32_t *src = X + (uint64_t)pi * pd.N;
    DMUL_PRIME_SWITCH(pi, (col_inv_ct_body<PI, N1>(pd, src, sm, n2)));
    col_crt_epilogue(pd, L, MODE, out, spill, sm);
}

// the same (digit sums) for a batch of jobs of one transform length (job = blockIdx.z)
template <uint32_t N1>
__global__ void __launch_bounds__(512) k_col_inv_ct_b(const PlanDev pd, const JobDev *__restrict__ jobs) {
    extern __shared__ __align__(16) uint32_t sm[];
    const JobDev &J = jobs[blockIdx.z];
    const int pi = (int)cg::this_cluster().block_rank();
    const uint32_t n2 = (blockIdx.x / kPrimes) * 32 + (threadIdx.x & 31);
    DMUL_PRIME_SWITCH(pi, (col_inv_ct_body<PI, N1>(pd, J.X + (uint64_t)pi * pd.N, sm, n2)));
    col_crt_epilogue(pd, J.L, kInvDigits, J.z, J.spill, sm);
}

template <uint32_t N1>
static bool col_schedule_matches(const PlanDev &pd) {
    using S = ColSched<N1>;
    if (pd.N1 != N1 || pd.ncs != S::NS) return false;
    for (int t = 0; t < S::NS; ++t)
        if (pd.cs[t].R != S::radix(t) || pd.cs[t].m != S::span(t)) return false;
    return true;
}


template <uint32_t N1>
static cudaError_t launch_fwd_ct(const PlanDev &pd, const uint32_t *x, uint64_t nx, const uint32_t *y,
                                 uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *status,
                                 cudaStream_t s) {
    const size_t smem = (size_t)N1 * 32 * sizeof(uint32_t);
    dim3 grid(kPrimes * (pd.N2 / 32), y ? 2 : 1);
    return launch_pdl(k_col_fwd_ct<N1>, grid, dim3(pd.col_threads), smem, s, 1, pd, x, nx, y, ny, X, Y, status);
}


template <uint32_t N1, int MODE>
static cudaError_t launch_inv_ct_mode(const PlanDev &pd, const uint32_t *X, uint64_t L,
                                      uint32_t *out, uint2 *spill, cudaStream_t s, uint64_t *zero,
                                      uint32_t nzero) {
    return launch_pdl(k_col_inv_ct<N1, MODE>, dim3(kPrimes * (pd.N2 / 32)), dim3(pd.col_threads),
                      (size_t)N1 * 32 * sizeof(uint32_t), s, kPrimes, pd, X, L, out, spill, zero, nzero);
}





}  // namespace dml

// =============================================================================================
// Half-width tiles: N1 rows x 16 columns (64 KB at N1 = 1024), so that two or three CTAs share an
// SM and one CTA's tile load overlaps another's arithmetic.  A warp works on two groups at once,
// one per half-warp (lane = 16 h + c, c = column).  Row r of the tile sits at slot
// phys(r) = r ^ ((r >> 4) & 1) (16 words per slot): the two half-warps then always touch slots of
// different parity -- rows j, j + 1 (j even) in the strided stages, rows 16 b + u, 16 (b + 1) + u
// in the last forward / first inverse stage -- i.e. different 16-bank halves.
// =============================================================================================
namespace dml {

__device__ __forceinline__ uint32_t hphys(uint32_t r) { return r ^ ((r >> 4) & 1u); }

// Issue (without waiting) the copies of the half tile's rows r with HALF * K/2 <= r mod K <
// (HALF + 1) * K/2 as one cp.async group (words >= n read as 0; src 16-byte aligned).  With
// K = N1 these are rows [0, N1/2) or [N1/2, N1): the groups of 16 consecutive rows of the inverse
// first stage's first or second half.
template <uint32_t N1, uint32_t K, uint32_t HALF>
__device__ __forceinline__ void htile_issue(uint32_t *sm, const uint32_t *__restrict__ src, uint64_t n,
                                            uint32_t N2, uint32_t j0) {
    constexpr uint32_t per = K / 2;
    constexpr uint32_t chunks = (N1 / K) * per * 4;  // 16-byte chunks: 4 per 16-word row
    for (uint32_t idx = threadIdx.x; idx < chunks; idx += blockDim.x) {
        const uint32_t rr = idx >> 2, q = idx & 3;
        const uint32_t row = (rr / per) * K + HALF * per + rr % per;
        const uint64_t g = (uint64_t)row * N2 + j0 + 4 * q;
        const uint32_t valid = g >= n ? 0u : (n - g >= 4 ? 4u : (uint32_t)(n - g));
        const uint32_t *s = valid ? src + g : src;
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(sm + hphys(row) * 16 + 4 * q);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(s), "r"(valid * 4)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int PENDING>
__device__ __forceinline__ void cp_async_wait_sync() {
    asm volatile("cp.async.wait_group %0;" ::"n"(PENDING) : "memory");
    __syncthreads();
}

// Word offset of row (base + u * S) for a group whose first row is `base`, for the row strides
// the schedules produce: S a multiple of 32 (phys is linear in u), S = 16 (base has bit 4 clear:
// odd u flips bit 0 of the row), S = 1 with base = 16 b (odd b flips bit 0 of u).  odd_off is the
// per-thread correction added for odd u (S = 16) or to every u (S = 1: see hoff1).
template <uint32_t S>
__device__ __forceinline__ uint32_t hbase(uint32_t base, uint32_t c) {
    if constexpr (S % 32 == 0) return hphys(base) * 16 + c;
    else return base * 16 + c;
}
template <uint32_t S>
__device__ __forceinline__ int hodd(uint32_t base) {
    if constexpr (S == 16) return (base & 1u) ? -16 : 16;  // row ^ 1
    else if constexpr (S == 1) return ((base >> 4) & 1u) ? 16 : 0;  // u -> u ^ 1 when b is odd
    else return 0;
}
template <uint32_t S, uint32_t U>
__device__ __forceinline__ uint32_t hoff(uint32_t b0, int odd) {
    static_assert(S % 32 == 0 || S == 16 || S == 1, "row stride without a half-tile layout");
    if constexpr (S % 32 == 0) return b0 + U * S * 16;
    else if constexpr (S == 16) return b0 + U * 256 + ((U & 1) ? odd : 0);
    else return (U & 1) ? b0 + U * 16 - odd : b0 + U * 16 + odd;  // (u ^ (b & 1)) * 16, odd = 16 (b & 1)
}

template <int PI, uint32_t R, uint32_t S, uint32_t U = 0>
__device__ __forceinline__ void hload(const uint32_t *sm, uint32_t b0, int odd, uint32_t (&v)[R]) {
    if constexpr (U < R) {
        v[U] = sm[hoff<S, U>(b0, odd)];
        hload<PI, R, S, U + 1>(sm, b0, odd, v);
    }
}
// store v[outpos(k)] to row k of the group
template <int PI, uint32_t R, uint32_t S, uint32_t K = 0>
__device__ __forceinline__ void hstore_out(uint32_t *sm, uint32_t b0, int odd, const uint32_t (&v)[R]) {
    if constexpr (K < R) {
        sm[hoff<S, K>(b0, odd)] = v[outpos<(int)R>((int)K)];
        hstore_out<PI, R, S, K + 1>(sm, b0, odd, v);
    }
}

// stage 0 of the forward pass (limbs in, in place)
template <int PI, uint32_t R, uint32_t N1>
__device__ __forceinline__ void hcolf0(const Stage &st, const uint2 *tw, uint32_t *sm, uint32_t &bad) {
    constexpr uint32_t stride = N1 / R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t c = lane & 15, h = lane >> 4;
    for (uint32_t j = 2 * warp + h; j < stride; j += 2 * nw) {
        const uint32_t b0 = hbase<stride>(j, c);
        const int odd = hodd<stride>(j);
        uint32_t v[R];
        hload<PI, R, stride>(sm, b0, odd, v);
#pragma unroll
        for (uint32_t u = 0; u < R; ++u) {
            if (PI == 0) bad |= (v[u] >= kBase);  // prime 0's CTAs report invalid limbs
            if (PI == 0) v[u] = red2p<PI>(v[u]);  // 10^9 < 4 p0: [0, 10^9) -> [0, 2 p0)
        }
        dft<PI, 0, (int)R, 1>(v);
#pragma unroll
        for (uint32_t k = 1; k < R; ++k) {
            const uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
            v[outpos<(int)R>((int)k)] = shoup<PI>(v[outpos<(int)R>((int)k)], w.x, w.y);
        }
        hstore_out<PI, R, stride>(sm, b0, odd, v);
    }
}

// a middle stage (forward: DFT then twiddle; inverse: untwiddle then DFT), in place
template <int PI, uint32_t R, uint32_t M, uint32_t N1, bool INV>
__device__ __forceinline__ void hcolmid(const Stage &st, const uint2 *tw, uint32_t *sm, bool final_reduce) {
    constexpr uint32_t stride = M / R;
    constexpr uint32_t groups = N1 / R;
    constexpr bool has_tw = M > R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t c = lane & 15, h = lane >> 4;
    for (uint32_t g = 2 * warp + h; g < groups; g += 2 * nw) {
        const uint32_t blk = g / stride, j = g % stride;
        const uint32_t base = blk * M + j;
        const uint32_t b0 = hbase<stride>(base, c);
        const int odd = hodd<stride>(base);
        uint32_t v[R];
        hload<PI, R, stride>(sm, b0, odd, v);
        if (!INV) {
            dft<PI, 0, (int)R, has_tw ? 1 : 0>(v);
            if (has_tw) {
#pragma unroll
                for (uint32_t k = 1; k < R; ++k) {
                    const uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
                    v[outpos<(int)R>((int)k)] = shoup<PI>(v[outpos<(int)R>((int)k)], w.x, w.y);
                }
            }
        } else {
            // as colmid_ct: input 0 reduced, the others untwiddled; outputs unreduced unless last
            static_assert(has_tw, "every inverse column stage after the first has twiddles");
            v[0] = red2p<PI>(v[0]);
#pragma unroll
            for (uint32_t k = 1; k < R; ++k) {
                const uint2 w = ldtw(tw + st.twi + (k - 1) * stride + j);
                v[k] = shoup<PI>(v[k], w.x, w.y);
            }
            if (final_reduce) {
                dft<PI, 1, (int)R>(v);
#pragma unroll
                for (uint32_t u = 0; u < R; ++u) v[u] = red1p<PI>(v[u]);
            } else {
                dft<PI, 1, (int)R, 2>(v);
            }
        }
        hstore_out<PI, R, stride>(sm, b0, odd, v);
    }
}

// last forward stage (rows 16 b + u, R = 16) + four-step twiddle + store of the residues
template <int PI, uint32_t R, uint32_t N1>
__device__ __forceinline__ void hcolf_last(const PlanDev &pd, const uint32_t *sm,
                                           uint32_t *__restrict__ dst, uint32_t n2) {
    static_assert(R == 16, "half tiles need a last stage of radix 16");
    constexpr uint32_t nb = N1 / R;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t c = lane & 15, h = lane >> 4;
    const uint2 *A = pd.tw[PI] + pd.offA;
    uint2 q[R];
    load_q<PI, R>(pd.tw[PI] + pd.offQ, pd.N2, n2, q);
    for (uint32_t b = 2 * warp + h; b < nb; b += 2 * nw) {
        uint32_t v[R];
        hload<PI, R, 1>(sm, hbase<1>(b * R, c), hodd<1>(b * R), v);
        const uint2 a = ldtw(A + (uint64_t)b * pd.N2 + n2);
        dft<PI, 0, (int)R, 2>(v);
#pragma unroll
        for (uint32_t k = 0; k < R; ++k) {
            uint32_t o = v[outpos<(int)R>((int)k)];
            if (k > 0) o = shoup<PI>(o, q[k].x, q[k].y);
            o = shoup<PI>(o, a.x, a.y);
            dst[(uint64_t)(b * R + k) * pd.N2 + n2] = o;
        }
    }
}

// first inverse stage on the staged half tile: inverse four-step twiddle, inverse DFT
template <int PI, uint32_t R, uint32_t N1>
__device__ __forceinline__ void hcoli_first(const PlanDev &pd, uint32_t *sm, uint32_t n2, const uint2 (&q)[R],
                                            uint32_t b_lo, uint32_t b_hi) {
    static_assert(R == 16, "half tiles need a last stage of radix 16");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t c = lane & 15, h = lane >> 4;
    const uint2 *A = pd.tw[PI] + pd.offAi;
    for (uint32_t b = b_lo + 2 * warp + h; b < b_hi; b += 2 * nw) {
        const uint32_t b0 = hbase<1>(b * R, c);
        const int odd = hodd<1>(b * R);
        uint32_t v[R];
        hload<PI, R, 1>(sm, b0, odd, v);
        const uint2 a = ldtw(A + (uint64_t)b * pd.N2 + n2);
#pragma unroll
        for (uint32_t k = 0; k < R; ++k) {
            uint32_t o = v[k];
            if (k > 0) o = shoup<PI>(o, q[k].x, q[k].y);
            v[k] = shoup<PI>(o, a.x, a.y);
        }
        dft<PI, 1, (int)R, 2>(v);  // the next inverse stage reduces / untwiddles its inputs
        hstore_out<PI, R, 1>(sm, b0, odd, v);
    }
}

template <int PI, uint32_t N1, int T>
__device__ __forceinline__ void hcolf_mids(const PlanDev &pd, uint32_t *sm) {
    using S = ColSched<N1>;
    if constexpr (T < S::NS - 1) {
        hcolmid<PI, S::radix(T), S::span(T), N1, false>(pd.cs[T], pd.tw[PI], sm, false);
        __syncthreads();
        hcolf_mids<PI, N1, T + 1>(pd, sm);
    }
}

template <int PI, uint32_t N1, int T>
__device__ __forceinline__ void hcoli_mids(const PlanDev &pd, uint32_t *sm) {
    using S = ColSched<N1>;
    if constexpr (T >= 0) {
        hcolmid<PI, S::radix(T), S::span(T), N1, true>(pd.cs[T], pd.tw[PI], sm, T == 0);
        __syncthreads();
        hcoli_mids<PI, N1, T - 1>(pd, sm);
    }
}

// grid (3 * N2/16, operands): blockIdx.x = 3 * half_tile + prime; x and y 16-byte aligned
template <uint32_t N1>
__device__ __forceinline__ void col_fwd_h_run(const PlanDev &pd, uint32_t *sm, const uint32_t *__restrict__ src,
                                              uint64_t n, uint32_t *__restrict__ dst, uint32_t j0, int pi,
                                              uint32_t *status) {
    using S = ColSched<N1>;
    const uint32_t n2 = j0 + (threadIdx.x & 15);
    uint32_t bad = 0;
    // the whole tile, then the first stage (starting the first stage on half the tile measured
    // slower here than waiting for all of it: three CTAs per SM already overlap loads)
    htile_issue<N1, N1, 0>(sm, src, n, pd.N2, j0);
    htile_issue<N1, N1, 1>(sm, src, n, pd.N2, j0);
    cp_async_wait_sync<0>();
    DMUL_PRIME_SWITCH(pi, (hcolf0<PI, S::radix(0), N1>(pd.cs[0], pd.tw[PI], sm, bad)));
    if (pi == 0 && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusInvalid);
    __syncthreads();
    DMUL_PRIME_SWITCH(pi, (hcolf_mids<PI, N1, 1>(pd, sm)));
    DMUL_PRIME_SWITCH(pi, (hcolf_last<PI, S::radix(S::NS - 1), N1>(pd, sm, dst, n2)));
}

template <uint32_t N1>
__global__ void __launch_bounds__(256, 3) k_col_fwd_h(const PlanDev pd, const uint32_t *__restrict__ x,
                                                      uint64_t nx, const uint32_t *__restrict__ y,
                                                      uint64_t ny, uint32_t *X, uint32_t *Y,
                                                      uint32_t *status) {
    extern __shared__ __align__(16) uint32_t sm[];
    pdl_trigger();
    prefetch_tables(pd);
    pdl_wait();
    uint32_t pi, tile;
    bool second;
    fwd_order(pi, tile, second);
    col_fwd_h_run<N1>(pd, sm, second ? y : x, second ? ny : nx, (second ? Y : X) + (uint64_t)pi * pd.N,
                      tile * 16, (int)pi, status);
    fwd_done(pd, pi, 16);
}

// the same for a batch of jobs of one transform length (job = blockIdx.z)
template <uint32_t N1>
__global__ void __launch_bounds__(256, 3) k_col_fwd_h_b(const PlanDev pd, const JobDev *__restrict__ jobs,
                                                        uint32_t *status) {
    extern __shared__ __align__(16) uint32_t sm[];
    const JobDev &J = jobs[blockIdx.z];
    const bool second = blockIdx.y != 0;
    if (second && J.square) return;
    const int pi = blockIdx.x % kPrimes;
    col_fwd_h_run<N1>(pd, sm, second ? J.y : J.x, second ? J.ny : J.nx,
                      (second ? J.Y : J.X) + (uint64_t)pi * pd.N, (blockIdx.x / kPrimes) * 16, pi,
                      job_status(J, status));
}

template <int PI, uint32_t N1>
__device__ __forceinline__ void hcol_inv_body(const PlanDev &pd, const uint32_t *__restrict__ src,
                                              uint32_t *sm, uint32_t j0) {
    using S = ColSched<N1>;
    constexpr uint32_t R = S::radix(S::NS - 1), nb = N1 / R;
    const uint32_t n2 = j0 + (threadIdx.x & 15);
    // the tile in two halves of rows; the four-step Q twiddles load while the copies fly, and the
    // first stage starts on the first half while the second half lands
    htile_issue<N1, N1, 0>(sm, src, pd.N, pd.N2, j0);
    htile_issue<N1, N1, 1>(sm, src, pd.N, pd.N2, j0);
    uint2 q[R];
    load_q<PI, R>(pd.tw[PI] + pd.offQi, pd.N2, n2, q);
    cp_async_wait_sync<1>();
    hcoli_first<PI, R, N1>(pd, sm, n2, q, 0, nb / 2);
    cp_async_wait_sync<0>();
    hcoli_first<PI, R, N1>(pd, sm, n2, q, nb / 2, nb);
    __syncthreads();
    hcoli_mids<PI, N1, S::NS - 2>(pd, sm);
}

// Cluster of six CTAs per 32-column tile: rank = 3 * half + prime, half 0 / 1 holding columns
// [0, 16) / [16, 32) of the tile.  After the inverse column DFTs, each 32-coefficient chunk of a
// row is recovered by CRT from the six CTAs' shared memory (lanes 0-15 read the CTAs of half 0,
// lanes 16-31 those of half 1), so the chunk digit sums and spills are those of the full-width
// pass.
template <uint32_t N1, int MODE>
__device__ __forceinline__ void col_inv_h_run(const PlanDev &pd, uint32_t *sm, const uint32_t *__restrict__ X,
                                              uint64_t L, uint32_t *__restrict__ out,
                                              uint2 *__restrict__ spill) {
    cg::cluster_group cluster = cg::this_cluster();
    const uint32_t rank = cluster.block_rank();
    const uint32_t half = rank / kPrimes, pi = rank % kPrimes;
    const uint32_t t0 = (blockIdx.x / (2 * kPrimes)) * 32;  // first column of the 32-column tile
    const uint32_t j0 = t0 + 16 * half;
    const uint32_t *src = X + (uint64_t)pi * pd.N;
    DMUL_PRIME_SWITCH((int)pi, (hcol_inv_body<PI, N1>(pd, src, sm, j0)));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t c = lane & 15, hl = lane >> 4;
    if (MODE == kInvResidues) {
        for (uint32_t r = 2 * warp + hl; r < N1; r += 2 * nw) {
            const uint64_t k = (uint64_t)r * pd.N2 + j0 + c;
            if (k < L) out[(uint64_t)pi * L + k] = sm[hphys(r) * 16 + c];
        }
        return;
    }
    cluster.sync();
    const uint32_t *s0 = cluster.map_shared_rank(sm, kPrimes * hl + 0);
    const uint32_t *s1 = cluster.map_shared_rank(sm, kPrimes * hl + 1);
    const uint32_t *s2 = cluster.map_shared_rank(sm, kPrimes * hl + 2);
#pragma unroll 2
    for (uint32_t r = rank + 2 * kPrimes * warp; r < N1; r += 2 * kPrimes * nw) {
        const uint64_t k0 = (uint64_t)r * pd.N2 + t0;  // first coefficient of this chunk
        if (k0 >= L) continue;                          // warp-uniform
        const uint32_t off = hphys(r) * 16 + c;
        uint32_t d0, d1, d2;
        crt_digits(s0[off], s1[off], s2[off], d0, d1, d2);
        const uint64_t k = k0 + lane;
        if (MODE == kInvTriples) {
            if (k < L) { out[3 * k] = d0; out[3 * k + 1] = d1; out[3 * k + 2] = d2; }
        } else {
            uint32_t sv;
            uint2 sp;
            chunk_digits(d0, d1, d2, sv, sp);
            if (k < L) out[k] = sv;
            if (lane == 31) spill[k0 >> 5] = sp;
        }
    }
    cluster.sync();
}

template <uint32_t N1, int MODE>
__global__ void __launch_bounds__(256, 3) k_col_inv_h(const PlanDev pd, const uint32_t *__restrict__ X,
                                                      uint64_t L, uint32_t *__restrict__ out,
                                                      uint2 *__restrict__ spill, uint64_t *zero,
                                                      uint32_t nzero) {
    extern __shared__ __align__(16) uint32_t sm[];
    pdl_trigger();
    pdl_wait();
    zero_words(zero, nzero);
    col_inv_h_run<N1, MODE>(pd, sm, X, L, out, spill);
}

// the same (digit sums) for a batch of jobs of one transform length (job = blockIdx.z)
template <uint32_t N1>
__global__ void __launch_bounds__(256, 3) k_col_inv_h_b(const PlanDev pd, const JobDev *__restrict__ jobs) {
    extern __shared__ __align__(16) uint32_t sm[];
    const JobDev &J = jobs[blockIdx.z];
    col_inv_h_run<N1, kInvDigits>(pd, sm, J.X, J.L, J.z, J.spill);
}

template <uint32_t N1>
static cudaError_t launch_fwd_h(const PlanDev &pd, const uint32_t *x, uint64_t nx, const uint32_t *y,
                                uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *status, cudaStream_t s) {
    const size_t smem = (size_t)N1 * 16 * sizeof(uint32_t);
    dim3 grid(kPrimes * (pd.N2 / 16), y ? 2 : 1);
    return launch_pdl(k_col_fwd_h<N1>, grid, dim3(pd.col_threads), smem, s, 1, pd, x, nx, y, ny, X, Y, status);
}

template <uint32_t N1, int MODE>
static cudaError_t launch_inv_h_mode(const PlanDev &pd, const uint32_t *X, uint64_t L, uint32_t *out,
                                     uint2 *spill, cudaStream_t s, uint64_t *zero, uint32_t nzero) {
    return launch_pdl(k_col_inv_h<N1, MODE>, dim3(2 * kPrimes * (pd.N2 / 32)), dim3(pd.col_threads),
                      (size_t)N1 * 16 * sizeof(uint32_t), s, 2 * kPrimes, pd, X, L, out, spill, zero, nzero);
}






// ---- batched launches (the medium products of dmul_batch, one transform length per launch) ----
template <uint32_t N1>
static cudaError_t launch_fwd_b(const PlanDev &pd, const JobDev *jobs, int njobs, uint32_t *status,
                                cudaStream_t s) {
    if (pd.col_half) {
        dim3 grid(kPrimes * (pd.N2 / 16), 2, (unsigned)njobs);
        k_col_fwd_h_b<N1><<<grid, pd.col_threads, (size_t)N1 * 16 * 4, s>>>(pd, jobs, status);
    } else {
        dim3 grid(kPrimes * (pd.N2 / 32), 2, (unsigned)njobs);
        k_col_fwd_ct_b<N1><<<grid, pd.col_threads, (size_t)N1 * 32 * 4, s>>>(pd, jobs, status);
    }
    return cudaGetLastError();
}

template <uint32_t N1>
static cudaError_t launch_inv_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(pd.col_threads, 1, 1);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (pd.col_half) {
        cfg.gridDim = dim3(2 * kPrimes * (pd.N2 / 32), 1, (unsigned)njobs);
        cfg.dynamicSmemBytes = (size_t)N1 * 16 * 4;
        at[0].val.clusterDim.x = 2 * kPrimes;
        return cudaLaunchKernelEx(&cfg, k_col_inv_h_b<N1>, pd, jobs);
    }
    cfg.gridDim = dim3(kPrimes * (pd.N2 / 32), 1, (unsigned)njobs);
    cfg.dynamicSmemBytes = (size_t)N1 * 32 * 4;
    at[0].val.clusterDim.x = kPrimes;
    return cudaLaunchKernelEx(&cfg, k_col_inv_ct_b<N1>, pd, jobs);
}





// ---- one set of column lengths: dispatch on pd.N1 over the set (C++17 folds) ---------------
template <uint32_t N1>
static cudaError_t attrs_col_all() {
    cudaError_t e;
    const int full = (int)(N1 * 32 * 4), half = (int)(N1 * 16 * 4);
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if ((e = cudaFuncSetAttribute(k_col_fwd_ct<N1>, a, full))) return e;
    if ((e = cudaFuncSetAttribute(k_col_inv_ct<N1, kInvDigits>, a, full))) return e;
    if ((e = cudaFuncSetAttribute(k_col_fwd_h<N1>, a, half))) return e;
    if ((e = cudaFuncSetAttribute(k_col_inv_h<N1, kInvDigits>, a, half))) return e;
    if ((e = cudaFuncSetAttribute(k_col_fwd_ct_b<N1>, a, full))) return e;
    if ((e = cudaFuncSetAttribute(k_col_inv_ct_b<N1>, a, full))) return e;
    if ((e = cudaFuncSetAttribute(k_col_fwd_h_b<N1>, a, half))) return e;
    return cudaFuncSetAttribute(k_col_inv_h_b<N1>, a, half);
}

template <uint32_t... Ns>
struct ColSet {
    static bool matches(const PlanDev &pd) {
        bool r = false;
        (void)((pd.N1 == Ns && (r = col_schedule_matches<Ns>(pd), true)) || ...);
        return r;
    }
    static cudaError_t fwd(const PlanDev &pd, const uint32_t *x, uint64_t nx, const uint32_t *y, uint64_t ny,
                           uint32_t *X, uint32_t *Y, uint32_t *status, cudaStream_t s) {
        cudaError_t r = cudaErrorInvalidValue;
        (void)((pd.N1 == Ns && (r = pd.col_half ? launch_fwd_h<Ns>(pd, x, nx, y, ny, X, Y, status, s)
                                               : launch_fwd_ct<Ns>(pd, x, nx, y, ny, X, Y, status, s),
                                true)) || ...);
        return r;
    }
    static cudaError_t inv(const PlanDev &pd, const uint32_t *X, uint64_t L, uint32_t *out, uint2 *spill,
                           cudaStream_t s, uint64_t *zero, uint32_t nzero) {
        cudaError_t r = cudaErrorInvalidValue;
        (void)((pd.N1 == Ns &&
                (r = pd.col_half ? launch_inv_h_mode<Ns, kInvDigits>(pd, X, L, out, spill, s, zero, nzero)
                                 : launch_inv_ct_mode<Ns, kInvDigits>(pd, X, L, out, spill, s, zero, nzero),
                 true)) || ...);
        return r;
    }
    static cudaError_t fwd_b(const PlanDev &pd, const JobDev *jobs, int njobs, uint32_t *status, cudaStream_t s) {
        cudaError_t r = cudaErrorInvalidValue;
        (void)((pd.N1 == Ns && (r = launch_fwd_b<Ns>(pd, jobs, njobs, status, s), true)) || ...);
        return r;
    }
    static cudaError_t inv_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s) {
        cudaError_t r = cudaErrorInvalidValue;
        (void)((pd.N1 == Ns && (r = launch_inv_b<Ns>(pd, jobs, njobs, s), true)) || ...);
        return r;
    }
    static cudaError_t attrs() {
        cudaError_t r = cudaSuccess;
        (void)(((r = attrs_col_all<Ns>()) != cudaSuccess) || ...);
        return r;
    }
};

// The entry points each instantiating translation unit defines for its set (TAG: big, small).
#define DMUL_COLPASS_SET(TAG, ...)                                                                    \
    DMUL_DEFINE_UPLOAD(upload_constants_colpass_##TAG)                                                 \
    using ColSet_##TAG = ColSet<__VA_ARGS__>;                                                          \
    bool colpass_##TAG##_matches(const PlanDev &pd) { return ColSet_##TAG::matches(pd); }             \
    cudaError_t colpass_##TAG##_fwd(const PlanDev &pd, const uint32_t *x, uint64_t nx, const uint32_t *y, \
                                   uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *status,            \
                                   cudaStream_t s) {                                                   \
        return ColSet_##TAG::fwd(pd, x, nx, y, ny, X, Y, status, s);                                   \
    }                                                                                                  \
    cudaError_t colpass_##TAG##_inv(const PlanDev &pd, const uint32_t *X, uint64_t L, uint32_t *out,   \
                                   uint2 *spill, cudaStream_t s, uint64_t *zero, uint32_t nzero) {     \
        return ColSet_##TAG::inv(pd, X, L, out, spill, s, zero, nzero);                                \
    }                                                                                                  \
    cudaError_t colpass_##TAG##_fwd_b(const PlanDev &pd, const JobDev *jobs, int njobs, uint32_t *status, \
                                     cudaStream_t s) {                                                 \
        return ColSet_##TAG::fwd_b(pd, jobs, njobs, status, s);                                        \
    }                                                                                                  \
    cudaError_t colpass_##TAG##_inv_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s) { \
        return ColSet_##TAG::inv_b(pd, jobs, njobs, s);                                                \
    }                                                                                                  \
    cudaError_t colpass_##TAG##_attrs() { return ColSet_##TAG::attrs(); }

}  // namespace dml
