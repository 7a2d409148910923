// stages.cuh -- device-side building blocks of the pipeline, shared by the kernel translation
// units (each instantiates its own copies; there is no relocatable device code).
//
// Transform structure (Sec. 7.1, four-step form): a length-N vector is an N1 x N2 row-major matrix
// (Sec. 7, row-major convention).  The forward transform runs length-N1 DFTs down the columns,
// multiplies element <k1, n2> by xi_N^(k1 n2), then runs length-N2 DFTs along the rows; nothing is
// transposed and no bit reversal is performed: the forward output order is a fixed permutation,
// and the inverse walks the exact mirror of the forward stages, so the pointwise product (which is
// order-blind, Sec. 5.4 eq. cdot_permutation_invariance and Sec. 7.4) sees matching orders.
//
// Each length-n DFT is a sequence of radix-R stages (R in {2,3,4,8,16}).  Stage t splits
// sub-transforms of length m into R interleaved pieces: for j < m/R it takes the R elements
// j + u m/R of a sub-transform, computes their R-point DFT in registers (modarith.cuh), multiplies
// output k by xi_m^(j k) (inter-stage twiddles, precomputed per stage in coalesced tables) and stores
// it back to position j + k m/R.  The inverse stage undoes this exactly (twiddle xi_m^(-jk) first,
// then the inverse R-point DFT).
#pragma once
#include <cooperative_groups.h>
#include <stdint.h>

#include "kernels.cuh"
#include "modarith.cuh"
#include "tma.cuh"

namespace dml {

// ---------------------------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------------------------
#define DMUL_RADIX_SWITCH(R, CALL)                \
    switch (R) {                                  \
        case 2: { constexpr int RR = 2; CALL; } break;   \
        case 3: { constexpr int RR = 3; CALL; } break;   \
        case 4: { constexpr int RR = 4; CALL; } break;   \
        case 5: { constexpr int RR = 5; CALL; } break;   \
        case 8: { constexpr int RR = 8; CALL; } break;   \
        default: { constexpr int RR = 16; CALL; } break; \
    }

#define DMUL_PRIME_SWITCH(pi, CALL)                 \
    switch (pi) {                                   \
        case 0: { constexpr int PI = 0; CALL; } break; \
        case 1: { constexpr int PI = 1; CALL; } break; \
        default: { constexpr int PI = 2; CALL; } break; \
    }

__device__ __forceinline__ uint2 ldtw(const uint2 *p) { return __ldg(p); }

// The forward column pass brings the whole plan's twiddle tables (every prime, contiguous at
// pd.tw[0], pd.tw_bytes bytes; 0 for long transforms, whose tables stay cached across their many
// CTAs anyway) into L2 for the passes after it: one bulk prefetch of up to 4 KB per thread of the
// grid's first row of CTAs.  Short products otherwise meet every table cold, one dependent miss
// per stage.  The tables are never written, so this runs before waiting on the predecessor.
__device__ __forceinline__ void prefetch_tables(const PlanDev &pd) {
    if (!pd.tw_bytes || blockIdx.y != 0) return;
    const uint64_t nblk = (pd.tw_bytes + 4095) / 4096;
    const uint8_t *base = (const uint8_t *)pd.tw[0];
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nblk;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t off = i * 4096, left = pd.tw_bytes - off;
        const uint32_t bytes = (uint32_t)(left < 4096 ? left : 4096);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(base + off), "r"(bytes) : "memory");
    }
}

// ---- hand-off from the forward column pass to the row pass, per prime ------------------------
// The forward column CTAs run prime by prime (CTA order lin = blockIdx.y * gridDim.x + blockIdx.x,
// prime-major), so that the rows of a prime can start while later primes' columns still run.
__device__ __forceinline__ void fwd_order(uint32_t &pi, uint32_t &tile, bool &second) {
    const uint32_t nt = gridDim.x / kPrimes;  // tiles per prime and operand
    const uint32_t per_prime = nt * gridDim.y;
    const uint32_t lin = blockIdx.y * gridDim.x + blockIdx.x;
    pi = lin / per_prime;
    const uint32_t r = lin - pi * per_prime;
    second = r >= nt;
    tile = second ? r - nt : r;
}
__device__ __forceinline__ void fwd_sync_add(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t fwd_sync_ld(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// end of a forward column CTA: its columns of prime pi are in memory.  Each warp posts its share
// (cols / warps) once its own stores are ordered before the release (a warp barrier, then lane 0),
// so no warp waits for the others' stores.
__device__ __forceinline__ void fwd_done(const PlanDev &pd, uint32_t pi, uint32_t cols) {
    if (!pd.fsync) return;
    __syncwarp();
    if ((threadIdx.x & 31) == 0) fwd_sync_add(pd.fsync + pi, cols / (blockDim.x >> 5));
}
// start of a row CTA of prime pi: wait for the columns of its prime (bounded), or for the whole
// previous grid when there is no per-prime hand-off
__device__ __forceinline__ void row_wait_prime(const PlanDev &pd, uint32_t pi, uint32_t *status) {
    if (!pd.fsync) {
        pdl_wait();
        return;
    }
    if (threadIdx.x == 0) {
        uint32_t spins = 0;
        const uint32_t limit = pd.spin ? pd.spin : (1u << 24);
        while ((int32_t)(fwd_sync_ld(pd.fsync + pi) - pd.ftarget) < 0) {
            if (++spins > limit) {
                if (status) atomicOr(status, kStatusTimeout);
                break;
            }
            __nanosleep(64);
        }
    }
    __syncthreads();
}

// Grid-strided zeroing of n words (the next pipeline stage's control block; p may be null).
__device__ __forceinline__ void zero_words(uint64_t *p, uint32_t n) {
    if (!p) return;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) p[i] = 0;
}

// Row-buffer index with an XOR swizzle of the 32-word bank rows: bank = (a mod 32) ^ f(a div 32),
// f(r) = (r mod 16) | ((r >> 3) & 1) << 4.  Every stage pattern of every row schedule the planner
// emits (a small radix first, then radix 16) then hits 32 distinct banks per warp access.
__device__ __forceinline__ uint32_t swz(uint32_t a) {
    uint32_t r = a >> 5;
    uint32_t f = (r & 15u) | (((r >> 3) & 1u) << 4);
    return a ^ f;
}

// ---------------------------------------------------------------------------------------------
// Forward column pass: limbs -> column DFTs (length N1) -> four-step twiddle -> residues.
// CTA = one tile of 32 adjacent columns for one prime and one operand; the tile lives in shared
// memory as N1 rows x 32 words, warp lane = column.
// ---------------------------------------------------------------------------------------------
template <int PI, int R>
__device__ __forceinline__ void colf_first(const PlanDev &pd, const Stage &st, uint32_t *sm,
                                           const uint32_t *__restrict__ src, uint64_t n,
                                           uint32_t n2, uint32_t &bad) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t stride = st.m / R;
    const uint2 *tw = pd.tw[PI] + st.tw;
    for (uint32_t j = warp; j < stride; j += nw) {
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            uint64_t idx = (uint64_t)(j + u * stride) * pd.N2 + n2;
            uint32_t a = idx < n ? __ldg(src + idx) : 0u;
            bad |= (a >= kBase);
            if (PI == 0) a = red2p<PI>(a);  // 10^9 < 4 p0: [0, 10^9) -> [0, 2 p0)
            v[u] = a;
        }
        dft<PI, 0, R>(v);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = v[outpos<R>(k)];
            if (k > 0 && st.m > (uint32_t)R) {
                uint2 w = ldtw(tw + (k - 1) * stride + j);
                o = shoup<PI>(o, w.x, w.y);
            }
            sm[(j + k * stride) * 32 + lane] = o;
        }
    }
}

// Stage the N1 x 32 tile at word offset j0 of a row-major matrix with row length N2 into shared
// memory with asynchronous 16-byte copies (all in flight at once); words at or beyond n read as 0
// (the zero padding of Sec. 3.2).  src must be 16-byte aligned.
__device__ __forceinline__ void tile_load_async(uint32_t *sm, const uint32_t *__restrict__ src,
                                                uint64_t n, uint32_t N1, uint32_t N2, uint32_t j0) {
    const uint32_t chunks = N1 * 8;  // 16-byte chunks: 8 per 32-word row
    for (uint32_t idx = threadIdx.x; idx < chunks; idx += blockDim.x) {
        const uint32_t row = idx >> 3, q = idx & 7;
        const uint64_t g = (uint64_t)row * N2 + j0 + 4 * q;
        const uint32_t valid = g >= n ? 0u : (n - g >= 4 ? 4u : (uint32_t)(n - g));
        const uint32_t *s = valid ? src + g : src;  // a readable address even when nothing is read
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(sm + row * 32 + 4 * q);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(s), "r"(valid * 4)
                     : "memory");
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
}

// First forward column stage from a tile already in shared memory (limbs), in place.
template <int PI, int R>
__device__ __forceinline__ void colf_first_sm(const PlanDev &pd, const Stage &st, uint32_t *sm,
                                              uint32_t &bad) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t stride = st.m / R;
    const uint2 *tw = pd.tw[PI] + st.tw;
    for (uint32_t j = warp; j < stride; j += nw) {
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) {
            uint32_t a = sm[(j + u * stride) * 32 + lane];
            bad |= (a >= kBase);
            if (PI == 0) a = red2p<PI>(a);  // 10^9 < 4 p0: [0, 10^9) -> [0, 2 p0)
            v[u] = a;
        }
        dft<PI, 0, R>(v);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = v[outpos<R>(k)];
            if (k > 0 && st.m > (uint32_t)R) {
                uint2 w = ldtw(tw + (k - 1) * stride + j);
                o = shoup<PI>(o, w.x, w.y);
            }
            sm[(j + k * stride) * 32 + lane] = o;
        }
    }
}

template <int PI, int R, bool INV>
__device__ __forceinline__ void col_mid(const PlanDev &pd, const Stage &st, uint32_t *sm,
                                        bool final_reduce) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t stride = st.m / R;
    const uint32_t groups = pd.N1 / R;
    const uint2 *tw = pd.tw[PI] + (INV ? st.twi : st.tw);
    const bool has_tw = st.m > (uint32_t)R;
    for (uint32_t g = warp; g < groups; g += nw) {
        uint32_t blk = g / stride, j = g - blk * stride;
        uint32_t base = blk * st.m + j;
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = sm[(base + u * stride) * 32 + lane];
        if (!INV) {
            dft<PI, 0, R>(v);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                uint32_t o = v[outpos<R>(k)];
                if (k > 0 && has_tw) {
                    uint2 w = ldtw(tw + (k - 1) * stride + j);
                    o = shoup<PI>(o, w.x, w.y);
                }
                sm[(base + k * stride) * 32 + lane] = o;
            }
        } else {
            if (has_tw) {
#pragma unroll
                for (int k = 1; k < R; ++k) {
                    uint2 w = ldtw(tw + (k - 1) * stride + j);
                    v[k] = shoup<PI>(v[k], w.x, w.y);
                }
            }
            dft<PI, 1, R>(v);
#pragma unroll
            for (int u = 0; u < R; ++u) {
                uint32_t o = v[outpos<R>(u)];
                if (final_reduce) o = red1p<PI>(o);
                sm[(base + u * stride) * 32 + lane] = o;
            }
        }
    }
}

// Last forward column stage (m == R): DFT, then the four-step twiddle xi_N^(k1 n2) with
// k1 = F(b) + (N1/R) k, applied as Q[k][n2] * A[b][n2], then the store to the residue array.
template <int PI, int R>
__device__ __forceinline__ void colf_last(const PlanDev &pd, const Stage &st, const uint32_t *sm,
                                          uint32_t *__restrict__ dst, uint32_t n2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t nb = pd.N1 / R;
    const uint2 *A = pd.tw[PI] + pd.offA;
    const uint2 *Q = pd.tw[PI] + pd.offQ;
    for (uint32_t b = warp; b < nb; b += nw) {
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = sm[(b * R + u) * 32 + lane];
        dft<PI, 0, R>(v);
        uint2 a = ldtw(A + (uint64_t)b * pd.N2 + n2);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = v[outpos<R>(k)];
            if (k > 0) {
                uint2 q = ldtw(Q + (uint64_t)k * pd.N2 + n2);
                o = shoup<PI>(o, q.x, q.y);
            }
            o = shoup<PI>(o, a.x, a.y);
            dst[(uint64_t)(b * R + k) * pd.N2 + n2] = o;
        }
    }
}

template <int PI>
__device__ __forceinline__ void col_fwd_body(const PlanDev &pd, uint32_t *sm, const uint32_t *__restrict__ src,
                             uint64_t n, uint32_t *__restrict__ dst, uint32_t tile,
                             uint32_t *status) {
    const uint32_t n2 = tile * 32 + (threadIdx.x & 31);
    uint32_t bad = 0;
    if ((((uintptr_t)src) & 15) == 0) {
        tile_load_async(sm, src, n, pd.N1, pd.N2, tile * 32);
        DMUL_RADIX_SWITCH(pd.cs[0].R, (colf_first_sm<PI, RR>(pd, pd.cs[0], sm, bad)));
    } else {
        DMUL_RADIX_SWITCH(pd.cs[0].R, (colf_first<PI, RR>(pd, pd.cs[0], sm, src, n, n2, bad)));
    }
    if (PI == 0 && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(status, kStatusInvalid);
    __syncthreads();
    for (int t = 1; t < pd.ncs - 1; ++t) {
        DMUL_RADIX_SWITCH(pd.cs[t].R, (col_mid<PI, RR, false>(pd, pd.cs[t], sm, false)));
        __syncthreads();
    }
    const Stage &last = pd.cs[pd.ncs - 1];
    DMUL_RADIX_SWITCH(last.R, (colf_last<PI, RR>(pd, last, sm, dst, n2)));
}

// ---------------------------------------------------------------------------------------------
// Row pass (fused): forward row DFTs of X (and Y), pointwise Montgomery product (or square),
// inverse row DFTs; the last forward stage, the product and the first inverse stage run on the
// same registers.  CTA = one row of one prime.
// ---------------------------------------------------------------------------------------------
template <int PI, int R>
__device__ __forceinline__ void rowf_first(const Stage &st, const uint2 *tw,
                                           const uint32_t *__restrict__ g, uint32_t *sbuf) {
    const uint32_t stride = st.m / R;
    for (uint32_t j = threadIdx.x; j < stride; j += blockDim.x) {
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = g[j + u * stride];
        dft<PI, 0, R>(v);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = v[outpos<R>(k)];
            if (k > 0) {
                uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
                o = shoup<PI>(o, w.x, w.y);
            }
            sbuf[swz(j + k * stride)] = o;
        }
    }
}

template <int PI, int R, bool INV>
__device__ __forceinline__ void row_mid(const Stage &st, const uint2 *tw, uint32_t *sbuf,
                                        uint32_t n) {
    const uint32_t stride = st.m / R;
    const uint32_t groups = n / R;
    const bool has_tw = st.m > (uint32_t)R;
    for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        uint32_t blk = g / stride, j = g - blk * stride;
        uint32_t base = blk * st.m + j;
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = sbuf[swz(base + u * stride)];
        if (!INV) {
            dft<PI, 0, R>(v);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                uint32_t o = v[outpos<R>(k)];
                if (k > 0 && has_tw) {
                    uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
                    o = shoup<PI>(o, w.x, w.y);
                }
                sbuf[swz(base + k * stride)] = o;
            }
        } else {
            if (has_tw) {
#pragma unroll
                for (int k = 1; k < R; ++k) {
                    uint2 w = ldtw(tw + st.twi + (k - 1) * stride + j);
                    v[k] = shoup<PI>(v[k], w.x, w.y);
                }
            }
            dft<PI, 1, R>(v);
#pragma unroll
            for (int u = 0; u < R; ++u) sbuf[swz(base + u * stride)] = v[outpos<R>(u)];
        }
    }
}

// last forward stage of X and Y + pointwise product + first inverse stage (m == R)
template <int PI, int R, bool SQR>
__device__ __forceinline__ void row_fused_center(uint32_t *sx, const uint32_t *sy, uint32_t n) {
    const uint32_t groups = n / R;
    for (uint32_t b = threadIdx.x; b < groups; b += blockDim.x) {
        uint32_t vx[R], vy[R], z[R];
#pragma unroll
        for (int u = 0; u < R; ++u) vx[u] = sx[swz(b * R + u)];
        dft<PI, 0, R>(vx);
        if (!SQR) {
#pragma unroll
            for (int u = 0; u < R; ++u) vy[u] = sy[swz(b * R + u)];
            dft<PI, 0, R>(vy);
        }
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t a = vx[outpos<R>(k)];
            z[k] = pointwise<PI>(a, SQR ? a : vy[outpos<R>(k)]);
        }
        dft<PI, 1, R>(z);
#pragma unroll
        for (int u = 0; u < R; ++u) sx[swz(b * R + u)] = z[outpos<R>(u)];
    }
}

template <int PI, int R>
__device__ __forceinline__ void rowi_last(const Stage &st, const uint2 *tw, const uint32_t *sbuf,
                                          uint32_t *__restrict__ g) {
    const uint32_t stride = st.m / R;
    for (uint32_t j = threadIdx.x; j < stride; j += blockDim.x) {
        uint32_t v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = sbuf[swz(j + k * stride)];
#pragma unroll
        for (int k = 1; k < R; ++k) {
            uint2 w = ldtw(tw + st.twi + (k - 1) * stride + j);
            v[k] = shoup<PI>(v[k], w.x, w.y);
        }
        dft<PI, 1, R>(v);
#pragma unroll
        for (int u = 0; u < R; ++u) g[j + u * stride] = v[outpos<R>(u)];
    }
}

// Forward row stage on every operand at once (groups of operand 0 first).  Stage 0 reads its
// inputs from `gin` (plain layout, global or shared), the others from the swizzled buffers.
// Looping over operands and stages keeps one copy of the DFT code per radix, which the
// instruction cache holds.
template <int PI, int R>
__device__ __forceinline__ void row_fwd_stage(const Stage &st, const uint2 *tw, uint32_t *sx,
                                              uint32_t *sy, const uint32_t *gx, const uint32_t *gy,
                                              bool from_plain, uint32_t n, uint32_t nops) {
    const uint32_t stride = st.m / R;
    const uint32_t per_op = n / R;
    const bool has_tw = st.m > (uint32_t)R;
    for (uint32_t g = threadIdx.x; g < per_op * nops; g += blockDim.x) {
        const bool second = g >= per_op;
        const uint32_t gg = second ? g - per_op : g;
        uint32_t *sb = second ? sy : sx;
        const uint32_t blk = gg / stride, j = gg - blk * stride;
        const uint32_t base = blk * st.m + j;
        uint32_t v[R];
        if (from_plain) {
            const uint32_t *src = second ? gy : gx;
#pragma unroll
            for (int u = 0; u < R; ++u) v[u] = src[base + u * stride];
        } else {
#pragma unroll
            for (int u = 0; u < R; ++u) v[u] = sb[swz(base + u * stride)];
        }
        dft<PI, 0, R>(v);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = v[outpos<R>(k)];
            if (k > 0 && has_tw) {
                uint2 w = ldtw(tw + st.tw + (k - 1) * stride + j);
                o = shoup<PI>(o, w.x, w.y);
            }
            sb[swz(base + k * stride)] = o;
        }
    }
}

// Inverse row stage on the product buffer; the last one (stage 0) writes to `gout` (plain).
template <int PI, int R>
__device__ __forceinline__ void row_inv_stage(const Stage &st, const uint2 *tw, uint32_t *sb,
                                              uint32_t *gout, uint32_t n) {
    const uint32_t stride = st.m / R;
    const uint32_t groups = n / R;
    const bool has_tw = st.m > (uint32_t)R;
    for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        const uint32_t blk = g / stride, j = g - blk * stride;
        const uint32_t base = blk * st.m + j;
        uint32_t v[R];
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = sb[swz(base + k * stride)];
        if (has_tw) {
#pragma unroll
            for (int k = 1; k < R; ++k) {
                uint2 w = ldtw(tw + st.twi + (k - 1) * stride + j);
                v[k] = shoup<PI>(v[k], w.x, w.y);
            }
        }
        dft<PI, 1, R>(v);
        if (gout) {
#pragma unroll
            for (int u = 0; u < R; ++u) gout[base + u * stride] = v[outpos<R>(u)];
        } else {
#pragma unroll
            for (int u = 0; u < R; ++u) sb[swz(base + u * stride)] = v[outpos<R>(u)];
        }
    }
}

// Last forward stage (m == R) of every operand, pointwise product (or square), first inverse stage.
// LAZY_OUT: the inverse DFT's outputs stay in [0, 4p) (the next inverse stage reduces its
// untwiddled input k = 0 and multiplies the others by their twiddles first).
template <int PI, int R, bool SQR, bool LAZY_OUT>
__device__ __forceinline__ void row_center_lazy(uint32_t *sx, const uint32_t *sy, uint32_t n) {
    const uint32_t groups = n / R;
    for (uint32_t b = threadIdx.x; b < groups; b += blockDim.x) {
        uint32_t v[2][R];
#pragma unroll
        for (int op = 0; op < (SQR ? 1 : 2); ++op) {
            const uint32_t *sb = op ? sy : sx;
#pragma unroll
            for (int u = 0; u < R; ++u) v[op][u] = sb[swz(b * R + u)];
            dft<PI, 0, R>(v[op]);
        }
        uint32_t z[R];
#pragma unroll
        for (int k = 0; k < R; ++k) {
            const uint32_t a = v[0][outpos<R>(k)];
            z[k] = pointwise<PI>(a, SQR ? a : v[1][outpos<R>(k)]);
        }
        dft<PI, 1, R, LAZY_OUT ? 2 : 0>(z);
#pragma unroll
        for (int u = 0; u < R; ++u) sx[swz(b * R + u)] = z[outpos<R>(u)];
    }
}

template <int PI, int R, bool SQR>
__device__ __forceinline__ void row_center(uint32_t *sx, const uint32_t *sy, uint32_t n) {
    row_center_lazy<PI, R, SQR, false>(sx, sy, n);
}

// The fused row pass on one row: inputs read from xin / yin (plain layout: global memory, or a
// landing buffer in shared memory), working buffers sx / sy (swizzled), result written to xout.
template <int PI, bool SQR>
__device__ __forceinline__ void row_mul_core(const PlanDev &pd, uint32_t *sx, uint32_t *sy,
                                             const uint32_t *xin, const uint32_t *yin,
                                             uint32_t *__restrict__ xout) {
    const uint32_t n = pd.N2;
    const uint2 *tw = pd.tw[PI];
    const int ns = pd.nrs;
    const uint32_t nops = SQR ? 1u : 2u;
    for (int t = 0; t < ns - 1; ++t) {
        DMUL_RADIX_SWITCH(pd.rs[t].R, (row_fwd_stage<PI, RR>(pd.rs[t], tw, sx, sy, xin, yin, t == 0, n, nops)));
        __syncthreads();
    }
    DMUL_RADIX_SWITCH(pd.rs[ns - 1].R, (row_center<PI, RR, SQR>(sx, sy, n)));
    __syncthreads();
    for (int t = ns - 2; t >= 0; --t) {
        DMUL_RADIX_SWITCH(pd.rs[t].R, (row_inv_stage<PI, RR>(pd.rs[t], tw, sx, t == 0 ? xout : nullptr, n)));
        if (t > 0) __syncthreads();
    }
}

template <int PI, bool SQR>
__device__ __forceinline__ void row_mul_body(const PlanDev &pd, uint32_t *sm, uint32_t *__restrict__ xr,
                             const uint32_t *__restrict__ yr) {
    row_mul_core<PI, SQR>(pd, sm, sm + pd.N2, xr, yr, xr);
}

// ---- TMA (bulk async copy) helpers -----------------------------------------------------------
// Persistent, TMA-fed row pass: CTA (g, prime) handles rows g, g + G, ...; while it computes one
// row, the bulk-copy engine brings the next row's X and Y into the other landing buffer.
// Shared memory: landing buffers [2][X, Y] (plain layout) + working buffers [X, Y] (swizzled)
// + 2 mbarriers.  On an expired wait the CTA records a timeout, waits (bounded) for its own copy
// in flight and returns.
template <int PI, bool SQR>
__device__ __forceinline__ void row_mul_tma_body(const PlanDev &pd, uint32_t *sm, uint32_t *X, const uint32_t *Y,
                                 uint32_t *status) {
    const uint32_t n = pd.N2;
    uint32_t *land = sm;                      // [2][2][n]
    uint32_t *sx = sm + 4 * n, *sy = sm + 5 * n;
    uint64_t *bar = (uint64_t *)(sm + 6 * n);  // 8-byte aligned: 6n words, n % 32 == 0
    const uint32_t G = gridDim.x;
    const uint64_t base = (uint64_t)PI * pd.N;
    const uint32_t bytes = n * 4;
    const uint32_t per_row = (SQR ? 1u : 2u) * bytes;
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    uint32_t r = blockIdx.x;
    if (threadIdx.x == 0 && r < pd.N1) {
        mbar_expect_tx(&bar[0], per_row);
        tma_load_1d(land, X + base + (uint64_t)r * n, bytes, &bar[0]);
        if (!SQR) tma_load_1d(land + n, Y + base + (uint64_t)r * n, bytes, &bar[0]);
    }
    for (uint32_t it = 0; r < pd.N1; ++it, r += G) {
        const uint32_t b = it & 1u;
        const uint32_t rn = r + G;
        if (threadIdx.x == 0 && rn < pd.N1) {
            uint32_t *dst = land + (b ^ 1u) * 2 * n;
            fence_proxy_async();
            mbar_expect_tx(&bar[b ^ 1u], per_row);
            tma_load_1d(dst, X + base + (uint64_t)rn * n, bytes, &bar[b ^ 1u]);
            if (!SQR) tma_load_1d(dst + n, Y + base + (uint64_t)rn * n, bytes, &bar[b ^ 1u]);
        }
        // every thread polls; the outcome is agreed on so that the CTA leaves (or not) as a whole
        const int ok = __syncthreads_and(mbar_wait(&bar[b], (it >> 1) & 1u, pd.spin) ? 1 : 0);
        if (!ok) {
            if (threadIdx.x == 0) {
                atomicOr(status, kStatusTimeout);
                if (rn < pd.N1) mbar_wait(&bar[b ^ 1u], ((it + 1) >> 1) & 1u);  // our copy in flight
            }
            return;
        }
        const uint32_t *lx = land + b * 2 * n;
        row_mul_core<PI, SQR>(pd, sx, sy, lx, lx + n, X + base + (uint64_t)r * n);
        __syncthreads();  // the landing buffer b and the working buffers are free again
    }
}

// ---------------------------------------------------------------------------------------------
// Inverse column pass.  A cluster of three CTAs (one per prime) shares a tile of 32 columns:
// each runs the inverse four-step twiddle (scaled by 2^32 N^-1, the linearity trick of Sec. 6)
// and the inverse column DFTs, then the three CTAs read each other's shared memory to recover
// every coefficient by CRT (Sec. 8.2.2 generalized to three primes by Garner's method).
// ---------------------------------------------------------------------------------------------
template <int PI, int R>
__device__ __forceinline__ void coli_first(const PlanDev &pd, const uint32_t *__restrict__ src,
                                           uint32_t *sm, uint32_t n2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t nb = pd.N1 / R;
    const uint2 *A = pd.tw[PI] + pd.offAi;
    const uint2 *Q = pd.tw[PI] + pd.offQi;
    for (uint32_t b = warp; b < nb; b += nw) {
        uint32_t v[R];
        uint2 a = ldtw(A + (uint64_t)b * pd.N2 + n2);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = src[(uint64_t)(b * R + k) * pd.N2 + n2];
            if (k > 0) {
                uint2 q = ldtw(Q + (uint64_t)k * pd.N2 + n2);
                o = shoup<PI>(o, q.x, q.y);
            }
            v[k] = shoup<PI>(o, a.x, a.y);
        }
        dft<PI, 1, R>(v);
#pragma unroll
        for (int u = 0; u < R; ++u) sm[(b * R + u) * 32 + lane] = v[outpos<R>(u)];
    }
}

// First inverse column stage (inverse four-step twiddle, inverse DFT) on a staged tile, in place.
template <int PI, int R>
__device__ __forceinline__ void coli_first_sm(const PlanDev &pd, uint32_t *sm, uint32_t n2) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t nb = pd.N1 / R;
    const uint2 *A = pd.tw[PI] + pd.offAi;
    const uint2 *Q = pd.tw[PI] + pd.offQi;
    for (uint32_t b = warp; b < nb; b += nw) {
        uint32_t v[R];
        uint2 a = ldtw(A + (uint64_t)b * pd.N2 + n2);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = sm[(b * R + k) * 32 + lane];
            if (k > 0) {
                uint2 q = ldtw(Q + (uint64_t)k * pd.N2 + n2);
                o = shoup<PI>(o, q.x, q.y);
            }
            v[k] = shoup<PI>(o, a.x, a.y);
        }
        dft<PI, 1, R>(v);
#pragma unroll
        for (int u = 0; u < R; ++u) sm[(b * R + u) * 32 + lane] = v[outpos<R>(u)];
    }
}

template <int PI>
__device__ __forceinline__ void col_inv_body(const PlanDev &pd, const uint32_t *__restrict__ src, uint32_t *sm,
                             uint32_t n2) {
    const int ns = pd.ncs;
    if ((((uintptr_t)src) & 15) == 0) {
        tile_load_async(sm, src, pd.N, pd.N1, pd.N2, n2 & ~31u);
        DMUL_RADIX_SWITCH(pd.cs[ns - 1].R, (coli_first_sm<PI, RR>(pd, sm, n2)));
    } else {
        DMUL_RADIX_SWITCH(pd.cs[ns - 1].R, (coli_first<PI, RR>(pd, src, sm, n2)));
    }
    __syncthreads();
    for (int t = ns - 2; t >= 0; --t) {
        DMUL_RADIX_SWITCH(pd.cs[t].R, (col_mid<PI, RR, true>(pd, pd.cs[t], sm, t == 0)));
        __syncthreads();
    }
    if (ns == 1) {  // a single stage: reduce in place
        for (uint32_t i = threadIdx.x; i < pd.N1 * 32; i += blockDim.x) sm[i] = red1p<PI>(sm[i]);
        __syncthreads();
    }
}

// Garner CRT of (a0, a1, a2), a_i in [0, p_i), p0 < p1 < p2, then the base-10^9 digits of
// c = v0 + p0 v1 + p0 p1 v2 < p0 p1 p2 < 10^27.
__device__ __forceinline__ void crt_digits(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t &d0,
                                           uint32_t &d1, uint32_t &d2) {
    const uint32_t p1 = c_prime[1].p, p2 = c_prime[2].p;
    // v1 = (a1 - a0) p0^-1 mod p1   (a0 < p0 < p1)
    uint32_t v1 = red1p<1>(shoup<1>(a1 - a0 + p1, c_crt.inv01, c_crt.inv01s));
    // v2 = (a2 - a0 - p0 v1) (p0 p1)^-1 mod p2   (a0 < p0 < p2)
    uint32_t t = red1p<2>(shoup<2>(v1, c_crt.p0m2, c_crt.p0m2s));
    uint32_t s = red1p<2>(a2 - a0 + p2);
    s = red1p<2>(s - t + p2);
    uint32_t v2 = red1p<2>(shoup<2>(s, c_crt.inv012, c_crt.inv012s));
    // c = a0 + p0 v1 + (A0 + A1 10^9) v2
    uint64_t S0 = (uint64_t)a0 + (uint64_t)c_prime[0].p * v1 + (uint64_t)c_crt.A0 * v2;
    uint64_t q0 = S0 / kBase;
    d0 = (uint32_t)(S0 - q0 * kBase);
    uint64_t S1 = q0 + (uint64_t)c_crt.A1 * v2;
    uint64_t q1 = S1 / kBase;
    d1 = (uint32_t)(S1 - q1 * kBase);
    d2 = (uint32_t)q1;
}

// Within a warp holding 32 consecutive coefficients (lane = position in the chunk): the chunk's
// digit sums s_c = d0_c + d1_(c-1) + d2_(c-2) (< 3*10^9) and the spill (d1_31 + d2_30, d2_31) that
// belongs to the first two positions of the next chunk.
__device__ __forceinline__ void chunk_digits(uint32_t d0, uint32_t d1, uint32_t d2, uint32_t &sv,
                                             uint2 &spill) {
    const int lane = threadIdx.x & 31;
    uint32_t d1p = __shfl_up_sync(0xffffffffu, d1, 1);
    uint32_t d2p = __shfl_up_sync(0xffffffffu, d2, 2);
    if (lane < 1) d1p = 0;
    if (lane < 2) d2p = 0;
    sv = d0 + d1p + d2p;
    uint32_t d2_30 = __shfl_sync(0xffffffffu, d2, 30);
    spill = make_uint2(d1 + d2_30, d2);
}

// ---------------------------------------------------------------------------------------------
// Carry: the recurrence of Sec. 3.2 (eq. sigmai_and_zi) as a decoupled-lookahead scan.
// After the CRT stage every position holds a digit sum s < 3*10^9 (the spill of the previous
// chunk added in), so the carry into any position is 0, 1 or 2 and each position acts on the
// carry by a map {0,1,2} -> {0,1,2}, c -> floor((s + c) / 10^9).  Maps compose associatively;
// a map is stored as three 2-bit outputs (6 bits).
// ---------------------------------------------------------------------------------------------
constexpr uint32_t kIdentityMap = 0u | (1u << 2) | (2u << 4);

__device__ __forceinline__ uint32_t map_apply(uint32_t f, uint32_t c) { return (f >> (2 * c)) & 3u; }
// g after f
__device__ __forceinline__ uint32_t map_compose(uint32_t g, uint32_t f) {
    return map_apply(g, map_apply(f, 0)) | (map_apply(g, map_apply(f, 1)) << 2) |
           (map_apply(g, map_apply(f, 2)) << 4);
}
__device__ __forceinline__ uint32_t qdig(uint32_t t) { return (t >= kBase) + (t >= 2u * kBase); }

__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_add_release(uint32_t *p, uint32_t v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// Maximum over the CTA (NT threads), returned to every thread; s: NT/32 words of shared memory
// (reused after the final barrier).
template <int NT>
__device__ __forceinline__ uint64_t block_max_u64(uint64_t v, uint64_t *s) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) {
        const uint64_t o = __shfl_down_sync(0xffffffffu, v, d);
        v = o > v ? o : v;
    }
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    uint64_t m = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) m = s[w] > m ? s[w] : m;
    __syncthreads();
    return m;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

constexpr uint32_t kSpinLimit = 1u << 22;  // bounded lookahead wait


// Inverse column pass of one tile (cluster of three CTAs, rank = prime) + CRT epilogue.
// After the inverse column pass of a tile (cluster of three CTAs, rank = prime, residues of the
// tile in [0, p) in each CTA's shared memory): write residues, or CRT each coefficient through
// distributed shared memory and write its digits.
__device__ __forceinline__ void col_crt_epilogue(const PlanDev &pd, uint64_t L, int mode,
                                                 uint32_t *__restrict__ out, uint2 *__restrict__ spill,
                                                 uint32_t *sm) {
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int pi = (int)cluster.block_rank();
    const uint32_t j0 = (blockIdx.x / kPrimes) * 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t n2 = j0 + lane;
    if (mode == kInvResidues) {
        for (uint32_t r = warp; r < pd.N1; r += nw) {
            uint64_t k = (uint64_t)r * pd.N2 + n2;
            if (k < L) out[(uint64_t)pi * L + k] = sm[r * 32 + lane];
        }
        return;
    }
    cluster.sync();
    const uint32_t *s0 = cluster.map_shared_rank(sm, 0);
    const uint32_t *s1 = cluster.map_shared_rank(sm, 1);
    const uint32_t *s2 = cluster.map_shared_rank(sm, 2);
    for (uint32_t r = pi + kPrimes * warp; r < pd.N1; r += kPrimes * nw) {
        const uint64_t k0 = (uint64_t)r * pd.N2 + j0;  // first coefficient of this chunk
        if (k0 >= L) continue;                          // warp-uniform
        uint32_t d0, d1, d2;
        crt_digits(s0[r * 32 + lane], s1[r * 32 + lane], s2[r * 32 + lane], d0, d1, d2);
        const uint64_t k = k0 + lane;
        if (mode == kInvTriples) {
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

// Inverse column pass of one tile (cluster of three CTAs, rank = prime) + CRT epilogue.
__device__ __forceinline__ void col_inv_crt(const PlanDev &pd, const uint32_t *__restrict__ X,
                                            uint64_t L, int mode, uint32_t *__restrict__ out,
                                            uint2 *__restrict__ spill, uint32_t *sm) {
    namespace cg = cooperative_groups;
    const int pi = (int)cg::this_cluster().block_rank();
    const uint32_t n2 = (blockIdx.x / kPrimes) * 32 + (threadIdx.x & 31);
    const uint32_t *src = X + (uint64_t)pi * pd.N;
    DMUL_PRIME_SWITCH(pi, (col_inv_body<PI>(pd, src, sm, n2)));
    col_crt_epilogue(pd, L, mode, out, spill, sm);
}

// One tile (NT threads x PER limbs) of the decoupled-lookahead carry scan.
//
// A tile publishes its aggregate carry map (status 1) and, once it knows its carry-in, its
// carry-out (status 2).  A tile whose map is constant -- its carry-out does not depend on its
// carry-in, the usual case unless its digit sums sit at 10^9 - 1 -- publishes its carry-out at
// once, so successors rarely wait.  The look-back runs on a whole warp: 32 predecessors per round,
// the maps before the nearest finished predecessor composed by a warp reduction.  A flag word holds
// its status and its value together (one 64-bit access), so publishing and polling need no memory
// ordering beyond the word itself.  Every wait is bounded; on expiry the tile records a timeout
// and proceeds with carry 0.
//
// A run of positions maps carries monotonically with out(2) - out(0) <= 1, and its map is constant
// unless every position of the run has a digit sum within 2 of a multiple of 10^9.  The per-thread
// map therefore follows the carry chains from 0 and from 2; only when they end apart (never, for
// random digits) is the chain from 1 followed too.
//
// The digit sums are read from z and the limbs written to zo: the same buffer, or (OOP, the
// host-buffer entry point) pinned host memory, so that the limbs cross the host link as the tiles
// finish instead of in a copy after the kernel.
//
// spin_limit bounds every wait of the tile (polls of a predecessor's flag, of the done count); an
// expired wait sets kStatusTimeout and the tile goes on with carry 0, so the kernel always ends.
template <int NT, int PER, bool OOP = false>
__device__ __forceinline__ void carry_tile(const uint32_t *z, uint32_t *zo, const uint2 *__restrict__ spill,
                                           uint64_t L, CarryCtl *ctl, uint64_t *nz,
                                           uint32_t *status, uint32_t ntiles, uint32_t spin_limit = kSpinLimit) {
    // every 32-limb chunk start (where a spill lands) is the first limb of some thread
    static_assert(NT % 32 == 0 && NT <= 1024 && PER % 4 == 0 && 32 % PER == 0, "tile shape");
    constexpr int NW = NT / 32;
    __shared__ uint32_t s_tile, s_cin, s_early, s_warp[NW];
    __shared__ uint64_t s_top[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) s_tile = atomicAdd(&ctl->ticket, 1u);
    __syncthreads();
    const uint32_t tile = s_tile;
    if (tile >= ntiles) return;  // more CTAs than tiles (a ticket that did not start at 0)
    const uint64_t base = (uint64_t)tile * (NT * PER) + (uint64_t)tid * PER;
    const bool vec = ((((uintptr_t)z) & 15) == 0) && (base + PER <= L);
    uint32_t v[PER];
    if (vec) {
#pragma unroll
        for (int i = 0; i < PER; i += 4) {
            const uint4 a = *(const uint4 *)(z + base + i);
            v[i] = a.x; v[i + 1] = a.y; v[i + 2] = a.z; v[i + 3] = a.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < PER; ++i) v[i] = (base + i < L) ? z[base + i] : 0u;
    }
    if ((base & 31) == 0 && base > 0 && base < L) {
        uint2 sp = spill[(base >> 5) - 1];
        v[0] += sp.x;
        v[1] += sp.y;
    }
    // map of this thread's PER positions.  When the last position's digit sum is not within 2 of
    // a multiple of 10^9 its carry-out ignores its carry-in, so the map is constant: that carry-out
    // (the usual case).  Otherwise follow the chains from carry 0 and 2 (and 1 if they differ).
    const uint32_t ql = qdig(v[PER - 1]);
    uint32_t c0 = ql, c1 = ql, c2 = ql;
    if (qdig(v[PER - 1] + 2u) != ql) {
        c0 = 0;
        c2 = 2;
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            c0 = qdig(v[i] + c0);
            c2 = qdig(v[i] + c2);
        }
        c1 = c0;
        if (c2 != c0) {
            c1 = 1;
#pragma unroll
            for (int i = 0; i < PER; ++i) c1 = qdig(v[i] + c1);
        }
    }
    uint32_t f = c0 | (c1 << 2) | (c2 << 4);
    // The tile's map is the composition of its threads' maps; when the last thread's map is
    // constant, so is the tile's, whatever came before: its carry-out is known now, and that thread
    // publishes it at once (the usual case), ahead of every scan and barrier of the tile.
    const bool early = c0 == c2;
    if (tid == NT - 1 && early) st_relaxed(&ctl->flags[tile], 2ull | ((uint64_t)c0 << 8));
    // inclusive warp scan (earlier lanes first)
    uint32_t inc = f;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= d) inc = map_compose(inc, o);
    }
    uint32_t exc = __shfl_up_sync(0xffffffffu, inc, 1);
    if (lane == 0) exc = kIdentityMap;
    if (lane == 31) s_warp[warp] = inc;
    if (tid == NT - 1) s_early = early ? 1u : 0u;
    __syncthreads();
    // every warp scans the warp maps across its lanes: its own exclusive prefix, and the tile's map
    uint32_t wi = lane < NW ? s_warp[lane] : kIdentityMap;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t o = __shfl_up_sync(0xffffffffu, wi, d);
        if (lane >= d) wi = map_compose(wi, o);
    }
    const uint32_t wpre = warp == 0 ? kIdentityMap : __shfl_sync(0xffffffffu, wi, warp - 1);
    if (warp == 0) {
        const uint32_t agg = __shfl_sync(0xffffffffu, wi, NW - 1);
        const uint32_t a0 = map_apply(agg, 0);
        const bool constant = (a0 == map_apply(agg, 1)) && (a0 == map_apply(agg, 2));
        const bool published = s_early != 0;
        if (lane == 0 && !published) {
            if (tile == 0 || constant) st_relaxed(&ctl->flags[tile], 2ull | ((uint64_t)a0 << 8));
            else st_relaxed(&ctl->flags[tile], 1ull | ((uint64_t)agg << 8));
        }
        uint32_t cin = 0;
        if (tile > 0) {
            uint32_t acc = kIdentityMap;  // maps of the predecessors already passed, newest last-applied
            int64_t top_t = (int64_t)tile - 1;
            for (;;) {
                // poll the window of 32 predecessors until the ones up to the nearest finished
                // one (or all 32, if none has finished) have published: only those are needed
                const int64_t t = top_t - lane;
                uint64_t w;
                unsigned incl;
                int first;
                bool late = false;
                for (uint32_t spins = 0;; ++spins) {
                    w = t >= 0 ? ld_relaxed(&ctl->flags[t]) : 2ull;  // before tile 0: carry-out 0
                    const uint32_t st = (uint32_t)w & 3u;
                    incl = __ballot_sync(0xffffffffu, st == 2u);
                    const unsigned ready = __ballot_sync(0xffffffffu, st != 0u);
                    first = incl ? __ffs(incl) - 1 : 32;
                    const unsigned need = first == 32 ? 0xffffffffu : (2u << first) - 1u;  // lanes 0..first
                    if ((ready & need) == need) break;
                    if (spins >= spin_limit) { late = true; break; }
                }
                if (late) {
                    if (lane == 0) atomicOr(status, kStatusTimeout);
                    cin = 0;
                    break;
                }
                const uint32_t val = (uint32_t)(w >> 8) & 63u;
                if (first == 0) {  // the nearest predecessor is finished: its carry-out
                    cin = map_apply(acc, __shfl_sync(0xffffffffu, val, 0));
                    break;
                }
                // compose the maps of lanes [0, first): newer lanes are applied after older ones
                uint32_t m = (lane < first) ? val : kIdentityMap;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    uint32_t o = __shfl_down_sync(0xffffffffu, m, d);
                    if (lane + d < 32) m = map_compose(m, o);
                }
                const uint32_t G = __shfl_sync(0xffffffffu, m, 0);
                if (incl) {
                    const uint32_t cfirst = __shfl_sync(0xffffffffu, val, first);
                    cin = map_apply(map_compose(acc, G), cfirst);
                    break;
                }
                acc = map_compose(acc, G);
                top_t -= 32;
            }
            if (lane == 0 && !published && !constant)
                st_relaxed(&ctl->flags[tile], 2ull | ((uint64_t)map_apply(agg, cin) << 8));
        }
        if (lane == 0) s_cin = cin;
    }
    __syncthreads();
    uint32_t c = map_apply(map_compose(exc, wpre), s_cin);
    uint32_t o[PER];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const uint32_t t = v[i] + c;
        const uint32_t q = qdig(t);
        o[i] = t - q * kBase;
        c = q;
    }
    if (base < L && base + PER >= L) {  // the thread holding position L-1: a carry out of it means z >= B^L
        uint32_t cc = map_apply(map_compose(exc, wpre), s_cin);
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (base + i < L) cc = qdig(v[i] + cc);
        if (cc != 0) atomicOr(status, kStatusInvalid);
    }
    if constexpr (OOP) {
        // out of place (pinned host memory across the host link, where a store of 16 bytes per
        // lane at a 64-byte stride is as many transactions): the tile goes through shared memory
        // and every warp store covers contiguous bytes.  Slot i of thread T sits at
        // T * G + (i ^ (T mod G)), which halves the bank conflicts of the writes.
        constexpr int G = PER / 4;
        __shared__ uint4 s_out[NT * G];
#pragma unroll
        for (int i = 0; i < G; ++i)
            s_out[tid * G + (i ^ (tid & (G - 1)))] =
                make_uint4(o[4 * i], o[4 * i + 1], o[4 * i + 2], o[4 * i + 3]);
        __syncthreads();
        const uint64_t t0 = (uint64_t)tile * (NT * PER);
        if ((((uintptr_t)zo) & 15) == 0 && t0 + NT * PER <= L) {
            uint4 *dst = (uint4 *)(zo + t0);
#pragma unroll
            for (int j = tid; j < NT * G; j += NT) dst[j] = s_out[(j / G) * G + ((j % G) ^ ((j / G) & (G - 1)))];
        } else {
            const uint32_t *sw = (const uint32_t *)s_out;
            for (int k = tid; k < NT * PER; k += NT) {
                if (t0 + k >= L) break;
                const int T = k / PER, r = k % PER;
                zo[t0 + k] = sw[4 * (T * G + ((r / 4) ^ (T & (G - 1)))) + (r & 3)];
            }
        }
    } else if (vec) {
#pragma unroll
        for (int i = 0; i < PER; i += 4) *(uint4 *)(zo + base + i) = make_uint4(o[i], o[i + 1], o[i + 2], o[i + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < PER; ++i)
            if (base + i < L) zo[base + i] = o[i];
    }
    if (!nz) return;
    // The normalized length: the highest nonzero limb lies in the last tile that has one.  Every
    // tile but the last marks in its flag word whether it has a nonzero limb and counts itself done
    // (release: after its digits); the last tile finds its own highest nonzero limb, and only when
    // it has none waits (bounded) for the others, finds the highest marked tile and scans its digits
    // -- both searches spread over the CTA.
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i) any |= (base + i < L) ? o[i] : 0u;
    if (tile != ntiles - 1) {
        const int tile_any = __syncthreads_or((int)(any != 0));
        if (tid == NT - 1) {
            // c: the carry out of the tile's last limb, the value published before
            st_relaxed(&ctl->flags[tile], 2ull | ((uint64_t)c << 8) | ((uint64_t)(tile_any ? 1 : 0) << 16));
            red_add_release(&ctl->done, 1u);
        }
        return;
    }
    uint64_t top = 0;
#pragma unroll
    for (int i = 0; i < PER; ++i)
        if (base + i < L && o[i]) top = base + i + 1;
    top = block_max_u64<NT>(top, s_top);
    if (top == 0 && tile > 0) {
        if (tid == 0) {
            uint32_t spins = 0;
            while (ld_acquire_u32(&ctl->done) != ntiles - 1) {
                if (++spins > spin_limit) { atomicOr(status, kStatusTimeout); break; }
            }
        }
        __syncthreads();
        // the highest earlier tile with a nonzero limb
        uint64_t hi = 0;  // tile index + 1
        for (uint32_t t = tid; t < tile; t += NT)
            if ((ld_relaxed(&ctl->flags[t]) >> 16) & 1u) hi = t + 1;
        hi = block_max_u64<NT>(hi, s_top);
        if (hi) {
            const uint64_t t0 = (hi - 1) * (uint64_t)(NT * PER);
            for (uint64_t k = t0 + tid; k < t0 + (uint64_t)NT * PER; k += NT)
                if (ld_relaxed_u32(zo + k)) top = top > k + 1 ? top : k + 1;
            top = block_max_u64<NT>(top, s_top);
        }
    }
    if (tid == 0) *nz = top ? top : 1;
}

}  // namespace dml
