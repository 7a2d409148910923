// sixstep.cu -- the six-step form of the transform (Sec. 7.2) with the paper's in-place
// transposes (Sec. 7.5-7.6), and the natural-layout CRT it ends with.
//
// Forward, for N = N1 * N2 = 2^k with N1 = 2^floor(k/2), N2 = 2^ceil(k/2) (Sec. 7.9): pack the limbs
// as an N1 x N2 matrix, transpose it in place (step 1), run length-N1 DFTs on the contiguous rows
// of the N2 x N1 result (step 2) and multiply by the four-step twiddle xi_N^(k1 n2) in the same
// kernel (step 4), transpose back in place (step 3), then the row pass (step 5, fused with the
// pointwise product and the first inverse step).  The final transpose of the forward transform and
// the first one of the inverse are omitted (Sec. 7.4).  The DFTs of step 2 leave their outputs in
// the stage order (no bit reversal): the twiddle is indexed by the true frequency of each position,
// and the inverse mirrors the order, so no reordering pass is needed.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "modarith.cuh"

namespace dml {

DMUL_DEFINE_UPLOAD(upload_constants_sixstep)

#define DMUL_RADIX_SWITCH(R, CALL)                \
    switch (R) {                                  \
        case 2: { constexpr int RR = 2; CALL; } break;   \
        case 4: { constexpr int RR = 4; CALL; } break;   \
        case 8: { constexpr int RR = 8; CALL; } break;   \
        default: { constexpr int RR = 16; CALL; } break; \
    }
#define DMUL_PRIME_SWITCH(pi, CALL)                 \
    switch (pi) {                                   \
        case 0: { constexpr int PI = 0; CALL; } break; \
        case 1: { constexpr int PI = 1; CALL; } break; \
        default: { constexpr int PI = 2; CALL; } break; \
    }

__device__ __forceinline__ uint32_t swz6(uint32_t a) {
    uint32_t r = a >> 5;
    uint32_t f = (r & 15u) | (((r >> 3) & 1u) << 4);
    return a ^ f;
}

// ---- packing: limbs -> residues [3][N], natural order, zero padded (Sec. 3.2) ------------------
__global__ void k_pack(const uint32_t *__restrict__ x, uint64_t nx, uint64_t N, uint32_t *X,
                       uint32_t *status) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    uint32_t a = i < nx ? x[i] : 0u;
    if (a >= kBase) atomicOr(status, kStatusInvalid);
    X[i] = red2p<0>(a);          // [0, 10^9) -> [0, 2 p0)
    X[N + i] = a;                // 10^9 < 2 p1
    X[2 * N + i] = a;            // 10^9 < 2 p2
}

cudaError_t launch_pack(const uint32_t *x, uint64_t nx, uint64_t N, uint32_t *X, uint32_t *status,
                        cudaStream_t s) {
    k_pack<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(x, nx, N, X, status);
    return cudaGetLastError();
}

// ---- in-place transposes -------------------------------------------------------------------------
// TransposeSquareSubMatrix semantics (Sec. 7.5): the n x n submatrix at `a` with row stride `rs`
// is transposed in place.  CTA (I, J), I <= J, swaps the 32 x 32 tiles (I, J) and (J, I) through
// shared memory, each transposed; the diagonal tiles transpose in place.
__global__ void __launch_bounds__(256) k_transpose_square(uint32_t *a, uint64_t n, uint64_t rs,
                                                          uint64_t batch_stride) {
    const uint32_t I = blockIdx.y, J = blockIdx.x;
    if (I > J) return;
    __shared__ uint32_t ta[32][33], tb[32][33];
    uint32_t *m = a + (uint64_t)blockIdx.z * batch_stride;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    for (int r = ty; r < 32; r += 8) {
        ta[r][tx] = m[(uint64_t)(I * 32 + r) * rs + J * 32 + tx];
        if (I != J) tb[r][tx] = m[(uint64_t)(J * 32 + r) * rs + I * 32 + tx];
    }
    __syncthreads();
    for (int r = ty; r < 32; r += 8) {
        if (I != J) m[(uint64_t)(I * 32 + r) * rs + J * 32 + tx] = tb[tx][r];
        m[(uint64_t)(J * 32 + r) * rs + I * 32 + tx] = ta[tx][r];
    }
}

// PermuteRho / UnPermuteRho of Sec. 7.6 on every row of an n x 2n matrix (rows of length 2n):
// rho: p[i] <- z[2i], p[i+n] <- z[2i+1]; inverse: p[2i] <- z[i], p[2i+1] <- z[i+n].  The scratch
// buffer z of 2n words is the CTA's shared memory.
__global__ void __launch_bounds__(256) k_permute_rho(uint32_t *a, uint64_t n, uint64_t batch_stride,
                                                     int inverse) {
    extern __shared__ uint32_t zeta[];
    uint32_t *p = a + (uint64_t)blockIdx.z * batch_stride + (uint64_t)blockIdx.x * 2 * n;
    for (uint64_t i = threadIdx.x; i < 2 * n; i += blockDim.x) zeta[i] = p[i];
    __syncthreads();
    if (!inverse) {
        for (uint64_t i = threadIdx.x; i < 2 * n; i += blockDim.x)
            p[i] = (i < n) ? zeta[2 * i] : zeta[2 * (i - n) + 1];
    } else {
        for (uint64_t i = threadIdx.x; i < 2 * n; i += blockDim.x)
            p[i] = (i & 1) ? zeta[n + (i >> 1)] : zeta[i >> 1];
    }
}

static cudaError_t square_sub(uint32_t *a, uint64_t n, uint64_t rs, uint64_t batch,
                              uint64_t batch_stride, cudaStream_t s) {
    dim3 grid((unsigned)(n / 32), (unsigned)(n / 32), (unsigned)batch);
    k_transpose_square<<<grid, 256, 0, s>>>(a, n, rs, batch_stride);
    return cudaGetLastError();
}

static cudaError_t rho_rows(uint32_t *a, uint64_t n, uint64_t batch, uint64_t batch_stride,
                            int inverse, cudaStream_t s) {
    dim3 grid((unsigned)n, 1, (unsigned)batch);
    k_permute_rho<<<grid, 256, 2 * n * sizeof(uint32_t), s>>>(a, n, batch_stride, inverse);
    return cudaGetLastError();
}

cudaError_t launch_transpose(uint32_t *a, uint64_t rows, uint64_t cols, uint64_t batch,
                             uint64_t batch_stride, cudaStream_t s) {
    cudaError_t e;
    if (rows == cols) return square_sub(a, rows, cols, batch, batch_stride, s);
    if (cols == 2 * rows) {
        // TransposeMatrixNx2N: rho on every row, then the left and right n x n halves (stride 2n)
        const uint64_t n = rows;
        if ((e = rho_rows(a, n, batch, batch_stride, 0, s)) != cudaSuccess) return e;
        if ((e = square_sub(a, n, 2 * n, batch, batch_stride, s)) != cudaSuccess) return e;
        return square_sub(a + n, n, 2 * n, batch, batch_stride, s);
    }
    if (rows == 2 * cols) {
        // TransposeMatrix2NxN: the two halves of the n x 2n view first, then rho^-1 on every row
        const uint64_t n = cols;
        if ((e = square_sub(a, n, 2 * n, batch, batch_stride, s)) != cudaSuccess) return e;
        if ((e = square_sub(a + n, n, 2 * n, batch, batch_stride, s)) != cudaSuccess) return e;
        return rho_rows(a, n, batch, batch_stride, 1, s);
    }
    return cudaErrorInvalidValue;
}

// ---- step 2 (and its inverse): length-N1 DFTs along the contiguous rows of the N2 x N1 matrix,
// with the four-step twiddle fused into the last (forward) / first (inverse) stage. -------------
template <int PI, int R, bool INV>
__device__ __forceinline__ void r6_mid(const Stage &st, const uint2 *tw, uint32_t *sb, uint32_t n) {
    const uint32_t stride = st.m / R;
    const uint32_t groups = n / R;
    const bool has_tw = st.m > (uint32_t)R;
    for (uint32_t g = threadIdx.x; g < groups; g += blockDim.x) {
        uint32_t blk = g / stride, j = g - blk * stride;
        uint32_t base = blk * st.m + j;
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = sb[swz6(base + u * stride)];
        if (!INV) {
            dft<PI, 0, R>(v);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                uint32_t o = v[outpos<R>(k)];
                if (k > 0 && has_tw) {
                    uint2 w = __ldg(tw + st.tw + (k - 1) * stride + j);
                    o = shoup<PI>(o, w.x, w.y);
                }
                sb[swz6(base + k * stride)] = o;
            }
        } else {
            if (has_tw) {
#pragma unroll
                for (int k = 1; k < R; ++k) {
                    uint2 w = __ldg(tw + st.twi + (k - 1) * stride + j);
                    v[k] = shoup<PI>(v[k], w.x, w.y);
                }
            }
            dft<PI, 1, R>(v);
#pragma unroll
            for (int u = 0; u < R; ++u) sb[swz6(base + u * stride)] = v[outpos<R>(u)];
        }
    }
}

// last forward stage with the four-step twiddle, output to global
template <int PI, int R>
__device__ __forceinline__ void r6_last_fwd(const PlanDev &pd, const uint32_t *sb, uint32_t *row,
                                            uint32_t n2) {
    const uint32_t n = pd.N1, nb = n / R;
    const uint2 *A = pd.tw[PI] + pd.offA, *Q = pd.tw[PI] + pd.offQ;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
        uint32_t v[R];
#pragma unroll
        for (int u = 0; u < R; ++u) v[u] = sb[swz6(b * R + u)];
        dft<PI, 0, R>(v);
        uint2 a = __ldg(A + (uint64_t)b * pd.N2 + n2);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = v[outpos<R>(k)];
            if (k > 0) {
                uint2 q = __ldg(Q + (uint64_t)k * pd.N2 + n2);
                o = shoup<PI>(o, q.x, q.y);
            }
            row[b * R + k] = shoup<PI>(o, a.x, a.y);
        }
    }
}

// first inverse stage with the inverse four-step twiddle (scaled), input from global
template <int PI, int R>
__device__ __forceinline__ void r6_first_inv(const PlanDev &pd, const uint32_t *row, uint32_t *sb,
                                             uint32_t n2) {
    const uint32_t n = pd.N1, nb = n / R;
    const uint2 *A = pd.tw[PI] + pd.offAi, *Q = pd.tw[PI] + pd.offQi;
    for (uint32_t b = threadIdx.x; b < nb; b += blockDim.x) {
        uint32_t v[R];
        uint2 a = __ldg(A + (uint64_t)b * pd.N2 + n2);
#pragma unroll
        for (int k = 0; k < R; ++k) {
            uint32_t o = row[b * R + k];
            if (k > 0) {
                uint2 q = __ldg(Q + (uint64_t)k * pd.N2 + n2);
                o = shoup<PI>(o, q.x, q.y);
            }
            v[k] = shoup<PI>(o, a.x, a.y);
        }
        dft<PI, 1, R>(v);
#pragma unroll
        for (int u = 0; u < R; ++u) sb[swz6(b * R + u)] = v[outpos<R>(u)];
    }
}

template <int PI, bool INV>
__device__ void r6_body(const PlanDev &pd, uint32_t *sb, uint32_t *row, uint32_t n2) {
    const uint32_t n = pd.N1;
    const uint2 *tw = pd.tw[PI];
    const int ns = pd.ncs;
    if (!INV) {
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) sb[swz6(i)] = row[i];
        __syncthreads();
        for (int t = 0; t < ns - 1; ++t) {
            DMUL_RADIX_SWITCH(pd.cs[t].R, (r6_mid<PI, RR, false>(pd.cs[t], tw, sb, n)));
            __syncthreads();
        }
        DMUL_RADIX_SWITCH(pd.cs[ns - 1].R, (r6_last_fwd<PI, RR>(pd, sb, row, n2)));
    } else {
        DMUL_RADIX_SWITCH(pd.cs[ns - 1].R, (r6_first_inv<PI, RR>(pd, row, sb, n2)));
        __syncthreads();
        for (int t = ns - 2; t >= 0; --t) {
            DMUL_RADIX_SWITCH(pd.cs[t].R, (r6_mid<PI, RR, true>(pd.cs[t], tw, sb, n)));
            __syncthreads();
        }
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) row[i] = red1p<PI>(sb[swz6(i)]);
    }
}

template <bool INV>
__global__ void __launch_bounds__(256) k_rowdft6(const PlanDev pd, uint32_t *A) {
    extern __shared__ uint32_t sb[];
    const uint32_t n2 = blockIdx.x;  // row of the N2 x N1 matrix = column of the N1 x N2 one
    const int pi = blockIdx.y;
    uint32_t *row = A + (uint64_t)pi * pd.N + (uint64_t)n2 * pd.N1;
    DMUL_PRIME_SWITCH(pi, (r6_body<PI, INV>(pd, sb, row, n2)));
}

cudaError_t launch_rowdft_fwd_tw(const PlanDev &pd, uint32_t *A, cudaStream_t s) {
    k_rowdft6<false><<<dim3(pd.N2, kPrimes), 256, pd.N1 * sizeof(uint32_t), s>>>(pd, A);
    return cudaGetLastError();
}

cudaError_t launch_rowdft_inv_tw(const PlanDev &pd, uint32_t *A, cudaStream_t s) {
    k_rowdft6<true><<<dim3(pd.N2, kPrimes), 256, pd.N1 * sizeof(uint32_t), s>>>(pd, A);
    return cudaGetLastError();
}

// ---- CRT on natural-layout residues (the six-step form ends in natural order) -------------------
__device__ __forceinline__ void crt_digits6(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t &d0,
                                            uint32_t &d1, uint32_t &d2) {
    const uint32_t p1 = c_prime[1].p, p2 = c_prime[2].p;
    uint32_t v1 = red1p<1>(shoup<1>(a1 - a0 + p1, c_crt.inv01, c_crt.inv01s));
    uint32_t t = red1p<2>(shoup<2>(v1, c_crt.p0m2, c_crt.p0m2s));
    uint32_t sdiff = red1p<2>(a2 - a0 + p2);
    sdiff = red1p<2>(sdiff - t + p2);
    uint32_t v2 = red1p<2>(shoup<2>(sdiff, c_crt.inv012, c_crt.inv012s));
    uint64_t S0 = (uint64_t)a0 + (uint64_t)c_prime[0].p * v1 + (uint64_t)c_crt.A0 * v2;
    uint64_t q0 = S0 / kBase;
    d0 = (uint32_t)(S0 - q0 * kBase);
    uint64_t S1 = q0 + (uint64_t)c_crt.A1 * v2;
    uint64_t q1 = S1 / kBase;
    d1 = (uint32_t)(S1 - q1 * kBase);
    d2 = (uint32_t)q1;
}

__global__ void __launch_bounds__(256) k_crt_natural(const uint32_t *__restrict__ X, uint64_t N,
                                                     uint64_t L, int mode, uint32_t *__restrict__ out,
                                                     uint2 *__restrict__ spill) {
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t k0 = k & ~31ull;
    if (k0 >= L) return;  // warp-uniform
    const int lane = threadIdx.x & 31;
    uint32_t a0 = 0, a1 = 0, a2 = 0;
    if (k < L) { a0 = X[k]; a1 = X[N + k]; a2 = X[2 * N + k]; }
    if (mode == kInvResidues) {
        if (k < L) { out[k] = a0; out[L + k] = a1; out[2 * L + k] = a2; }
        return;
    }
    uint32_t d0, d1, d2;
    crt_digits6(a0, a1, a2, d0, d1, d2);
    if (mode == kInvTriples) {
        if (k < L) { out[3 * k] = d0; out[3 * k + 1] = d1; out[3 * k + 2] = d2; }
        return;
    }
    uint32_t d1p = __shfl_up_sync(0xffffffffu, d1, 1);
    uint32_t d2p = __shfl_up_sync(0xffffffffu, d2, 2);
    if (lane < 1) d1p = 0;
    if (lane < 2) d2p = 0;
    uint32_t d2_30 = __shfl_sync(0xffffffffu, d2, 30);
    if (k < L) out[k] = d0 + d1p + d2p;
    if (lane == 31) spill[k0 >> 5] = make_uint2(d1 + d2_30, d2);
}

cudaError_t launch_crt_natural(const uint32_t *X, uint64_t N, uint64_t L, InvMode mode,
                               uint32_t *out, uint2 *spill, cudaStream_t s) {
    k_crt_natural<<<(unsigned)((L + 255) / 256), 256, 0, s>>>(X, N, L, (int)mode, out, spill);
    return cudaGetLastError();
}

cudaError_t init_kernel_attributes_sixstep() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_permute_rho, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  16384 * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_rowdft6<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  8192 * 4)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_rowdft6<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 4);
}

}  // namespace dml
