// sixstep.cu -- the six-step form of the transform (Sec. 7.2) with the paper's in-place
// transposes (Sec. 7.5-7.6), and the CRT it ends with.
//
// Forward, for N = N1 * N2 = 2^k with N1 = 2^floor(k/2), N2 = 2^ceil(k/2) (Sec. 7.9): the limbs seen
// as an N1 x N2 matrix go straight into the primes' N2 x N1 transposes (packing and step 1 in one
// out-of-place pass), length-N1 DFTs run on the contiguous rows of that result (step 2) with the
// four-step twiddle xi_N^(k1 n2) in the same kernel (step 4), an in-place transpose brings it back
// (step 3), then the row pass (step 5, fused with the pointwise product and the first inverse
// step).  The inverse mirrors it; its last transpose is fused into the CRT, which reads the
// transposed tiles.  The final transpose of the forward transform and the first one of the inverse
// are omitted (Sec. 7.4).  The DFTs of step 2 leave their outputs in
// the stage order (no bit reversal): the twiddle is indexed by the true frequency of each position,
// and the inverse mirrors the order, so no reordering pass is needed.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "kernels.cuh"
#include "modarith.cuh"
#include "tma.cuh"

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

// ---- the TMA-fed forms of both (used whenever the matrix is 16-byte aligned) -------------------
constexpr uint64_t kRhoMaxBytes = 16384 * 4 + 16;  // rows of up to 16384 words, and the barrier
constexpr uint64_t kRhoCMaxWords = 16384;          // the longest row rho_C permutes (n x Cn: C n)
// Square tile-pair swap: one CTA per pair of 32 x 32 tiles (I, J), I <= J, of the n x n submatrix
// (pair index p = J (J + 1) / 2 + I, so no CTA is launched for I > J).  Both tiles arrive in shared
// memory through a 3-D tensor map (columns, rows, batch) before anything is written, which makes
// the swap in place.  Each thread then transposes 4 x 4 blocks in registers: 128-bit shared loads
// along a tile row (eight lanes cover one 128-byte row, so no bank conflict) and 128-bit global
// stores.  xoff is the submatrix's first column within the mapped rows (0, or n for the right
// half of an n x 2n matrix).
constexpr uint32_t kTT = 32;

__device__ __forceinline__ void tile_pair(uint32_t p, uint32_t &I, uint32_t &J) {
    uint32_t j = (uint32_t)((sqrtf(8.0f * (float)p + 1.0f) - 1.0f) * 0.5f);
    while ((j + 1) * (j + 2) / 2 <= p) ++j;
    while (j * (j + 1) / 2 > p) --j;
    J = j;
    I = p - j * (j + 1) / 2;
}

__global__ void __launch_bounds__(128) k_transpose_tma(const __grid_constant__ CUtensorMap map, uint32_t *a,
                                                       uint64_t rs, uint64_t batch_stride, uint32_t xoff,
                                                       uint32_t *status) {
    __shared__ __align__(128) uint32_t tile[2][kTT * kTT];
    __shared__ __align__(8) uint64_t bar;
    uint32_t I, J;
    tile_pair(blockIdx.x, I, J);
    const uint32_t z = blockIdx.y;
    const bool diag = I == J;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(&bar, (diag ? 1u : 2u) * kTT * kTT * 4u);
        tma_load_3d(tile[0], &map, (int)(xoff + J * kTT), (int)(I * kTT), (int)z, &bar);
        if (!diag) tma_load_3d(tile[1], &map, (int)(xoff + I * kTT), (int)(J * kTT), (int)z, &bar);
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait(&bar, 0) ? 1 : 0)) {
        if (threadIdx.x == 0) {
            if (status) atomicOr(status, kStatusTimeout);
            mbar_wait(&bar, 0);  // the copies in flight (bounded again)
        }
        return;
    }
    const uint32_t w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const uint32_t sel = w >> 1;  // 0: tile (I, J) goes to (J, I); 1: tile (J, I) goes to (I, J)
    if (sel == 1 && diag) return;
    const uint32_t R = sel ? J : I, C = sel ? I : J;  // the source tile's row and column tile
    const uint32_t c = l & 7, q = (l >> 3) + 4 * (w & 1);
    const uint32_t *S = tile[sel];
    uint4 v[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = *(const uint4 *)&S[(4 * q + i) * kTT + 4 * c];
    uint32_t *m = a + (uint64_t)z * batch_stride;
    const uint64_t col = xoff + R * kTT + 4 * q;
    uint64_t row = (uint64_t)C * kTT + 4 * c;
    *(uint4 *)&m[row * rs + col] = make_uint4(v[0].x, v[1].x, v[2].x, v[3].x);
    *(uint4 *)&m[(row + 1) * rs + col] = make_uint4(v[0].y, v[1].y, v[2].y, v[3].y);
    *(uint4 *)&m[(row + 2) * rs + col] = make_uint4(v[0].z, v[1].z, v[2].z, v[3].z);
    *(uint4 *)&m[(row + 3) * rs + col] = make_uint4(v[0].w, v[1].w, v[2].w, v[3].w);
}

// rho / rho^-1 on every row of an n x 2n matrix, the row brought into shared memory by one bulk
// copy, the permuted row written back with 128-bit stores: rho sends (z[8k], z[8k+2], z[8k+4],
// z[8k+6]) to p[4k..4k+3] and the odd ones to p[n+4k..n+4k+3]; rho^-1 interleaves z[4k..4k+3]
// with z[n+4k..n+4k+3] into p[8k..8k+7].
__global__ void __launch_bounds__(256) k_permute_rho_tma(uint32_t *a, uint64_t n, uint64_t batch_stride,
                                                         int inverse, uint32_t *status) {
    extern __shared__ __align__(128) uint32_t zeta[];
    uint64_t *bar = (uint64_t *)(zeta + 2 * n);
    uint32_t *p = a + (uint64_t)blockIdx.z * batch_stride + (uint64_t)blockIdx.x * 2 * n;
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        mbar_expect_tx(bar, (uint32_t)(8 * n));
        tma_load_1d(zeta, p, (uint32_t)(8 * n), bar);
    }
    __syncthreads();
    if (!__syncthreads_and(mbar_wait(bar, 0) ? 1 : 0)) {
        if (threadIdx.x == 0) {
            if (status) atomicOr(status, kStatusTimeout);
            mbar_wait(bar, 0);
        }
        return;
    }
    for (uint64_t k = threadIdx.x; k < n / 4; k += blockDim.x) {
        if (!inverse) {
            const uint4 lo = *(const uint4 *)&zeta[8 * k], hi = *(const uint4 *)&zeta[8 * k + 4];
            *(uint4 *)&p[4 * k] = make_uint4(lo.x, lo.z, hi.x, hi.z);
            *(uint4 *)&p[n + 4 * k] = make_uint4(lo.y, lo.w, hi.y, hi.w);
        } else {
            const uint4 e = *(const uint4 *)&zeta[4 * k], o = *(const uint4 *)&zeta[n + 4 * k];
            *(uint4 *)&p[8 * k] = make_uint4(e.x, o.x, e.y, o.y);
            *(uint4 *)&p[8 * k + 4] = make_uint4(e.z, o.z, e.w, o.w);
        }
    }
}

// The generalization to n x Cn matrices (the closing remark of Sec. 7.6): with M = [A_0 ... A_{C-1}],
// transposing every n x n block in place gives rows alpha^0_1, alpha^1_1, ..., alpha^{C-1}_1, alpha^0_2
// ... where M^T wants all alpha^0 first, then all alpha^1, and so on: the row permutation
// rho_C(i) = n (i mod C) + (i div C) of the Cn x n view, which equals rho_C on the columns of M
// before the block transposes.  So the forward applies p[k n + i] <- z[C i + k] (k < C, i < n) to
// every row of M, then the C block transposes; the inverse (Cn x n) the block transposes of the
// n x Cn view, then p[C i + k] <- z[k n + i].  The row (Cn words) is the CTA's shared memory; it
// arrives by one bulk copy when the row is 16-byte aligned.
__global__ void __launch_bounds__(256) k_permute_rho_c(uint32_t *a, uint64_t n, uint32_t C, uint64_t batch_stride,
                                                       int inverse, int bulk, uint32_t *status) {
    extern __shared__ __align__(128) uint32_t zeta[];
    const uint64_t len = (uint64_t)C * n;
    uint64_t *bar = (uint64_t *)(zeta + len + (len & 1));
    uint32_t *p = a + (uint64_t)blockIdx.z * batch_stride + (uint64_t)blockIdx.x * len;
    if (bulk) {
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
            mbar_expect_tx(bar, (uint32_t)(4 * len));
            tma_load_1d(zeta, p, (uint32_t)(4 * len), bar);
        }
        __syncthreads();
        if (!__syncthreads_and(mbar_wait(bar, 0) ? 1 : 0)) {
            if (threadIdx.x == 0) {
                if (status) atomicOr(status, kStatusTimeout);
                mbar_wait(bar, 0);
            }
            return;
        }
    } else {
        for (uint64_t i = threadIdx.x; i < len; i += blockDim.x) zeta[i] = p[i];
        __syncthreads();
    }
    for (uint64_t o = threadIdx.x; o < len; o += blockDim.x) {
        if (!inverse) {
            const uint64_t k = o / n, i = o - k * n;  // p[k n + i] <- z[C i + k]
            p[o] = zeta[C * i + k];
        } else {
            const uint64_t i = o / C, k = o - i * C;  // p[C i + k] <- z[k n + i]
            p[o] = zeta[k * n + i];
        }
    }
}

// cuTensorMapEncodeTiled, from the driver through the runtime (no link against libcuda).
using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)f;
        else
            cudaGetLastError();
    });
    return fn;
}

// A tensor map of 32 x 32 uint32 boxes over `batch` matrices of `rows` rows of `cols` words (row
// stride rs words, matrix stride bs words).  False when the base is not 16-byte aligned or the
// driver refuses the map; the caller then takes the plain kernels.
static bool tile_map(CUtensorMap *m, uint32_t *a, uint64_t cols, uint64_t rows, uint64_t batch, uint64_t rs,
                     uint64_t bs) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc || ((uintptr_t)a & 15) || (rs % 4) || (bs % 4)) return false;
    const cuuint64_t dims[3] = {cols, rows, batch};
    const cuuint64_t strides[2] = {rs * 4, bs * 4};
    const cuuint32_t box[3] = {kTT, kTT, 1}, es[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, a, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The n x n submatrix starting at column xoff of the rows of `a` (row stride rs) transposed in place.
static cudaError_t square_sub(uint32_t *a, uint64_t n, uint64_t rs, uint64_t xoff, uint64_t batch,
                              uint64_t batch_stride, cudaStream_t s, uint32_t *status) {
    CUtensorMap map;
    if (tile_map(&map, a, rs, n, batch, rs, batch_stride)) {
        const uint64_t T = n / kTT;
        k_transpose_tma<<<dim3((unsigned)(T * (T + 1) / 2), (unsigned)batch), 128, 0, s>>>(
            map, a, rs, batch_stride, (uint32_t)xoff, status);
        return cudaGetLastError();
    }
    dim3 grid((unsigned)(n / 32), (unsigned)(n / 32), (unsigned)batch);
    k_transpose_square<<<grid, 256, 0, s>>>(a + xoff, n, rs, batch_stride);
    return cudaGetLastError();
}

static cudaError_t rho_rows(uint32_t *a, uint64_t n, uint64_t batch, uint64_t batch_stride,
                            int inverse, cudaStream_t s, uint32_t *status) {
    dim3 grid((unsigned)n, 1, (unsigned)batch);
    if (!((uintptr_t)a & 15) && !(batch_stride % 4) && 8 * n + 16 <= kRhoMaxBytes) {
        k_permute_rho_tma<<<grid, 256, 8 * n + 16, s>>>(a, n, batch_stride, inverse, status);
        return cudaGetLastError();
    }
    k_permute_rho<<<grid, 256, 2 * n * sizeof(uint32_t), s>>>(a, n, batch_stride, inverse);
    return cudaGetLastError();
}

cudaError_t launch_transpose(uint32_t *a, uint64_t rows, uint64_t cols, uint64_t batch,
                             uint64_t batch_stride, cudaStream_t s, uint32_t *status) {
    cudaError_t e;
    if (rows == cols) return square_sub(a, rows, cols, 0, batch, batch_stride, s, status);
    if (cols == 2 * rows) {
        // TransposeMatrixNx2N: rho on every row, then the left and right n x n halves (stride 2n)
        const uint64_t n = rows;
        if ((e = rho_rows(a, n, batch, batch_stride, 0, s, status)) != cudaSuccess) return e;
        if ((e = square_sub(a, n, 2 * n, 0, batch, batch_stride, s, status)) != cudaSuccess) return e;
        return square_sub(a, n, 2 * n, n, batch, batch_stride, s, status);
    }
    if (rows == 2 * cols) {
        // TransposeMatrix2NxN: the two halves of the n x 2n view first, then rho^-1 on every row
        const uint64_t n = cols;
        if ((e = square_sub(a, n, 2 * n, 0, batch, batch_stride, s, status)) != cudaSuccess) return e;
        if ((e = square_sub(a, n, 2 * n, n, batch, batch_stride, s, status)) != cudaSuccess) return e;
        return rho_rows(a, n, batch, batch_stride, 1, s, status);
    }
    // n x Cn and Cn x n for C > 2: rho_C, then the C block transposes (or the mirror)
    const bool wide = cols > rows;
    const uint64_t n = wide ? rows : cols, C = wide ? cols / rows : rows / cols;
    if (C * n != (wide ? cols : rows) || C * n > kRhoCMaxWords) return cudaErrorInvalidValue;
    const int bulk = !((uintptr_t)a & 15) && !(batch_stride % 4);
    const size_t smem = C * n * 4 + 16;
    dim3 grid((unsigned)n, 1, (unsigned)batch);
    if (wide) {
        k_permute_rho_c<<<grid, 256, smem, s>>>(a, n, (uint32_t)C, batch_stride, 0, bulk, status);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    for (uint64_t k = 0; k < C; ++k)
        if ((e = square_sub(a, n, C * n, k * n, batch, batch_stride, s, status)) != cudaSuccess) return e;
    if (!wide) {
        k_permute_rho_c<<<grid, 256, smem, s>>>(a, n, (uint32_t)C, batch_stride, 1, bulk, status);
        return cudaGetLastError();
    }
    return cudaSuccess;
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

// ---- Garner CRT (Sec. 8.2.2 extended to three primes) and the base-10^9 digits of one coefficient --
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

// ---- the first and the last data movement of the six-step form, fused with their neighbours ------
// Packing + step 1: the limbs seen as the N1 x N2 matrix (zero past nx) go straight into the three
// primes' N2 x N1 transposes, out of place (x is the caller's, X the scratch): one read of the limbs
// and one write of the residues instead of a packing pass and an in-place transpose.  Any
// N1 x N2 shape (also n x 2n: out of place no rho is needed).  CTA (J, I) moves the 32 x 32 tile of
// rows 32 I.., columns 32 J.. through shared memory (one padding word per row).
__global__ void __launch_bounds__(256) k_pack_transpose(const uint32_t *__restrict__ x, uint64_t nx, uint32_t N1,
                                                        uint32_t N2, uint64_t N, uint32_t *__restrict__ X,
                                                        uint32_t *status) {
    __shared__ uint32_t t[32][33];
    const uint32_t I = blockIdx.y, J = blockIdx.x;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
    uint32_t bad = 0;
    for (int r = ty; r < 32; r += 8) {
        const uint64_t k = (uint64_t)(I * 32 + r) * N2 + J * 32 + tx;
        const uint32_t a = k < nx ? x[k] : 0u;
        bad |= a >= kBase;
        t[r][tx] = a;
    }
    if (__syncthreads_or((int)bad) && threadIdx.x == 0) atomicOr(status, kStatusInvalid);
    for (int r = ty; r < 32; r += 8) {
        const uint32_t a = t[tx][r];  // element (row 32 I + tx, column 32 J + r)
        const uint64_t o = (uint64_t)(J * 32 + r) * N1 + I * 32 + tx;
        X[o] = red2p<0>(a);  // [0, 10^9) -> [0, 2 p0)
        X[N + o] = a;        // 10^9 < 2 p1
        X[2 * N + o] = a;    // 10^9 < 2 p2
    }
}

cudaError_t launch_pack_transpose(const uint32_t *x, uint64_t nx, uint32_t N1, uint32_t N2, uint32_t *X,
                                  uint32_t *status, cudaStream_t s) {
    if (N1 % 32 || N2 % 32) return cudaErrorInvalidValue;
    k_pack_transpose<<<dim3(N2 / 32, N1 / 32), 256, 0, s>>>(x, nx, N1, N2, (uint64_t)N1 * N2, X, status);
    return cudaGetLastError();
}

// Step 1 of the inverse (the last transpose) + CRT: the residues of the three primes sit in N2 x N1
// matrices, coefficient k = k1 N2 + n2 at [n2][k1].  CTA (I, J) brings the 32 x 32 tile of rows
// 32 J.. (n2), columns 32 I.. (k1) of each prime into shared memory; warp row k1 then covers the 32
// consecutive coefficients k1 N2 + 32 J .. + 31: one chunk of the digit sums.
__global__ void __launch_bounds__(256) k_crt_transposed(const uint32_t *__restrict__ X, uint32_t N1, uint32_t N2,
                                                        uint64_t N, uint64_t L, int mode,
                                                        uint32_t *__restrict__ out, uint2 *__restrict__ spill) {
    __shared__ uint32_t t[3][32][33];
    const uint32_t I = blockIdx.x, J = blockIdx.y;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const uint64_t first = (uint64_t)(I * 32) * N2 + J * 32;  // the tile's smallest coefficient
    if (first >= L) return;  // uniform over the CTA
    for (int r = ty; r < 32; r += 8) {
        const uint64_t o = (uint64_t)(J * 32 + r) * N1 + I * 32 + tx;
        t[0][r][tx] = X[o];
        t[1][r][tx] = X[N + o];
        t[2][r][tx] = X[2 * N + o];
    }
    __syncthreads();
    const int lane = tx;
    for (int r = ty; r < 32; r += 8) {  // k1 = 32 I + r, n2 = 32 J + lane
        const uint64_t k0 = (uint64_t)(I * 32 + r) * N2 + J * 32;
        if (k0 >= L) continue;  // warp-uniform
        const uint64_t k = k0 + lane;
        const bool in = k < L;
        const uint32_t a0 = in ? t[0][lane][r] : 0u, a1 = in ? t[1][lane][r] : 0u, a2 = in ? t[2][lane][r] : 0u;
        if (mode == kInvResidues) {
            if (in) { out[k] = a0; out[L + k] = a1; out[2 * L + k] = a2; }
            continue;
        }
        uint32_t d0, d1, d2;
        crt_digits6(a0, a1, a2, d0, d1, d2);
        if (mode == kInvTriples) {
            if (in) { out[3 * k] = d0; out[3 * k + 1] = d1; out[3 * k + 2] = d2; }
            continue;
        }
        // digit sums within the chunk; the two digits past it go to the chunk's spill
        uint32_t d1p = __shfl_up_sync(0xffffffffu, d1, 1);
        uint32_t d2p = __shfl_up_sync(0xffffffffu, d2, 2);
        if (lane < 1) d1p = 0;
        if (lane < 2) d2p = 0;
        const uint32_t d2_30 = __shfl_sync(0xffffffffu, d2, 30);
        if (in) out[k] = d0 + d1p + d2p;
        if (lane == 31) spill[k0 >> 5] = make_uint2(d1 + d2_30, d2);
    }
}

cudaError_t launch_crt_transposed(const uint32_t *X, uint32_t N1, uint32_t N2, uint64_t L, InvMode mode,
                                  uint32_t *out, uint2 *spill, cudaStream_t s) {
    if (N1 % 32 || N2 % 32) return cudaErrorInvalidValue;
    k_crt_transposed<<<dim3(N1 / 32, N2 / 32), 256, 0, s>>>(X, N1, N2, (uint64_t)N1 * N2, L, (int)mode, out, spill);
    return cudaGetLastError();
}

cudaError_t init_kernel_attributes_sixstep() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_permute_rho, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  16384 * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_permute_rho_tma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kRhoMaxBytes)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_permute_rho_c, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(kRhoCMaxWords * 4 + 16))) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_rowdft6<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  8192 * 4)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_rowdft6<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8192 * 4);
}

}  // namespace dml
