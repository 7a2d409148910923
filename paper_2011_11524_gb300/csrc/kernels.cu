// kernels.cu -- the multiplication pipeline on sm_103a: forward column pass, fused row pass,
// inverse column pass with cluster CRT, decoupled-lookahead carry scan.

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"
#include "modarith.cuh"
#include "stages.cuh"

namespace cg = cooperative_groups;

namespace dml {

DMUL_DEFINE_UPLOAD(upload_constants_main)

__global__ void __launch_bounds__(512) k_col_fwd(const PlanDev pd, const uint32_t *__restrict__ x,
                                                 uint64_t nx, const uint32_t *__restrict__ y,
                                                 uint64_t ny, uint32_t *X, uint32_t *Y,
                                                 uint32_t *status) {
    extern __shared__ uint32_t sm[];
    pdl_trigger();
    prefetch_tables(pd);
    pdl_wait();
    uint32_t pi, tile;
    bool second;
    fwd_order(pi, tile, second);
    const uint32_t *src = second ? y : x;
    const uint64_t n = second ? ny : nx;
    uint32_t *dst = (second ? Y : X) + (uint64_t)pi * pd.N;
    DMUL_PRIME_SWITCH((int)pi, (col_fwd_body<PI>(pd, sm, src, n, dst, tile, status)));
    fwd_done(pd, pi, 32);
}

cudaError_t launch_col_fwd(const PlanDev &pd, const uint32_t *x, uint64_t nx, const uint32_t *y,
                           uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *status, cudaStream_t s) {
    const bool aligned = ((uintptr_t)x & 15) == 0 && ((uintptr_t)y & 15) == 0;
    if (aligned && col_pass_specialized(pd)) return launch_col_fwd_spec(pd, x, nx, y, ny, X, Y, status, s);
    const size_t smem = (size_t)pd.N1 * 32 * sizeof(uint32_t);
    const int threads = (int)pd.col_threads;
    dim3 grid(kPrimes * (pd.N2 / 32), y ? 2 : 1);
    return launch_pdl(k_col_fwd, grid, dim3(threads), smem, s, 1, pd, x, nx, y, ny, X, Y, status);
}

template <bool SQR>
__global__ void __launch_bounds__(256) k_row_mul(const PlanDev pd, uint32_t *X, const uint32_t *Y,
                                                 uint32_t *status) {
    extern __shared__ uint32_t sm[];
    pdl_trigger();
    row_wait_prime(pd, blockIdx.y, status);
    const uint32_t row = blockIdx.x;
    const int pi = blockIdx.y;
    uint32_t *xr = X + (uint64_t)pi * pd.N + (uint64_t)row * pd.N2;
    const uint32_t *yr = SQR ? nullptr : Y + (uint64_t)pi * pd.N + (uint64_t)row * pd.N2;
    DMUL_PRIME_SWITCH(pi, (row_mul_body<PI, SQR>(pd, sm, xr, yr)));
}

template <bool SQR>
__global__ void __launch_bounds__(256) k_row_mul_tma(const PlanDev pd, uint32_t *X, const uint32_t *Y,
                                                     uint32_t *status) {
    extern __shared__ __align__(16) uint32_t sm[];
    pdl_trigger();
    row_wait_prime(pd, blockIdx.y, status);
    const int pi = blockIdx.y;
    DMUL_PRIME_SWITCH(pi, (row_mul_tma_body<PI, SQR>(pd, sm, X, Y, status)));
}

size_t row_tma_smem(const PlanDev &pd) { return (size_t)6 * pd.N2 * 4 + 16; }

cudaError_t launch_row_mul_tma(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,
                               uint32_t *status, cudaStream_t s) {
    dim3 grid(pd.row_grid ? pd.row_grid : 256, kPrimes);
    if (square) return launch_pdl(k_row_mul_tma<true>, grid, dim3(pd.row_threads), row_tma_smem(pd), s, 1, pd, X, Y, status);
    return launch_pdl(k_row_mul_tma<false>, grid, dim3(pd.row_threads), row_tma_smem(pd), s, 1, pd, X, Y, status);
}

cudaError_t launch_row_any(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,
                           uint32_t *status, cudaStream_t s) {
    if (row_pass_specialized(pd)) return launch_row_pass_ct(pd, X, Y, square, status, s);
    if (pd.row_tma) return launch_row_mul_tma(pd, X, Y, square, status, s);
    return launch_row_mul(pd, X, Y, square, s, status);
}

cudaError_t launch_row_mul(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,
                           cudaStream_t s, uint32_t *status) {
    dim3 grid(pd.N1, kPrimes);
    const size_t smem = (size_t)(square ? 1 : 2) * pd.N2 * sizeof(uint32_t);
    if (square) return launch_pdl(k_row_mul<true>, grid, dim3(pd.row_threads), smem, s, 1, pd, X, Y, status);
    return launch_pdl(k_row_mul<false>, grid, dim3(pd.row_threads), smem, s, 1, pd, X, Y, status);
}

template <int MODE>
__global__ void __launch_bounds__(512) k_col_inv(const PlanDev pd, const uint32_t *__restrict__ X,
                                                 uint64_t L, uint32_t *__restrict__ out,
                                                 uint2 *__restrict__ spill, uint64_t *zero, uint32_t nzero) {
    extern __shared__ uint32_t sm[];
    pdl_trigger();
    pdl_wait();
    zero_words(zero, nzero);
    col_inv_crt(pd, X, L, MODE, out, spill, sm);
}

cudaError_t launch_col_inv(const PlanDev &pd, const uint32_t *X, uint64_t L, InvMode mode,
                           uint32_t *out, uint2 *spill, cudaStream_t s, void *zero, size_t zero_bytes) {
    uint64_t *zw = (uint64_t *)zero;
    const uint32_t nzero = (uint32_t)(zero_bytes / 8);
    if (mode == kInvDigits && col_pass_specialized(pd)) return launch_col_inv_spec(pd, X, L, out, spill, s, zw, nzero);
    const dim3 grid(kPrimes * (pd.N2 / 32)), block(pd.col_threads);
    const size_t smem = (size_t)pd.N1 * 32 * sizeof(uint32_t);
    if (mode == kInvTriples)
        return launch_pdl(k_col_inv<kInvTriples>, grid, block, smem, s, kPrimes, pd, X, L, out, spill, zw, nzero);
    if (mode == kInvResidues)
        return launch_pdl(k_col_inv<kInvResidues>, grid, block, smem, s, kPrimes, pd, X, L, out, spill, zw, nzero);
    return launch_pdl(k_col_inv<kInvDigits>, grid, block, smem, s, kPrimes, pd, X, L, out, spill, zw, nzero);
}

// digit triples -> within-chunk digit sums + spills (the CRT stage's epilogue on given triples)
__global__ void k_triples_to_digits(const uint32_t *__restrict__ d, uint64_t L,
                                    uint32_t *__restrict__ out, uint2 *__restrict__ spill,
                                    uint32_t *status) {
    const uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;  // blockDim % 32 == 0
    const uint64_t k0 = k & ~31ull;
    if (k0 >= L) return;  // warp-uniform
    uint32_t d0 = 0, d1 = 0, d2 = 0;
    if (k < L) { d0 = d[3 * k]; d1 = d[3 * k + 1]; d2 = d[3 * k + 2]; }
    uint32_t sv;
    uint2 sp;
    chunk_digits(d0, d1, d2, sv, sp);
    if (k < L) out[k] = sv;
    bool over = (k >= L && sv != 0);  // a digit beyond the L limbs: the sum does not fit
    if ((threadIdx.x & 31) == 31) {
        spill[k0 >> 5] = sp;
        over |= (k0 + 32 >= L) && (sp.x | sp.y);
    }
    if (over) atomicOr(status, kStatusInvalid);
}

cudaError_t launch_triples_to_digits(const uint32_t *d, uint64_t L, uint32_t *out, uint2 *spill,
                                     uint32_t *status, cudaStream_t s) {
    const uint64_t blocks = (L + 255) / 256;
    k_triples_to_digits<<<(unsigned)blocks, 256, 0, s>>>(d, L, out, spill, status);
    return cudaGetLastError();
}

template <int NT, int PER, bool OOP>
__global__ void __launch_bounds__(NT, 1536 / NT) k_carry(const uint32_t *z, uint32_t *zo, const uint2 *__restrict__ spill,
                                              uint64_t L, CarryCtl *ctl, uint64_t *nz, uint32_t *status,
                                              uint32_t ntiles, uint32_t spin) {
    pdl_trigger();
    pdl_wait();
    carry_tile<NT, PER, OOP>(z, zo, spill, L, ctl, nz, status, ntiles, spin);
}

// Long products take 8192-limb tiles (512 threads x 16), so that every tile of a product of a few
// million limbs is resident at once and the look-back chain is short; shorter ones 2048-limb tiles
// (256 x 8) for parallelism.  ctl holds flags for ceil(L / kCarryLimbs) tiles, enough for either;
// it must be zero when the kernel starts.
cudaError_t launch_carry(uint32_t *z, const uint2 *spill, uint64_t L, CarryCtl *ctl, uint64_t *nz,
                         uint32_t *status, cudaStream_t s, uint32_t *zo, uint32_t spin) {
    constexpr uint64_t kBig = 512 * 16;
    if (!spin) spin = kSpinLimit;
    const uint32_t *zi = z;
    const bool oop = zo && zo != z;
    if (!zo) zo = z;
    if (L >= 256 * kBig) {
        const uint64_t ntiles = (L + kBig - 1) / kBig;
        return launch_pdl(oop ? k_carry<512, 16, true> : k_carry<512, 16, false>, dim3((unsigned)ntiles),
                          dim3(512), 0, s, 1, zi, zo, spill, L, ctl, nz, status, (uint32_t)ntiles, spin);
    }
    const uint64_t ntiles = (L + kCarryLimbs - 1) / kCarryLimbs;
    return launch_pdl(oop ? k_carry<256, 8, true> : k_carry<256, 8, false>, dim3((unsigned)ntiles), dim3(256), 0,
                      s, 1, zi, zo, spill, L, ctl, nz, status, (uint32_t)ntiles, spin);
}

// ---------------------------------------------------------------------------------------------
// Integer-pipe probe: independent chains of 32-bit multiply-adds (IMAD) per thread.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_imad_probe(uint32_t *sink, int iters) {
    uint32_t a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 2654435761u + i * 40503u + 1u;
    const uint32_t m = blockIdx.x | 1u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = a[i] * m + (uint32_t)i;  // one IMAD each
        }
    }
    uint32_t acc = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) acc ^= a[i];
    if (acc == 0x9e3779b9u) sink[blockIdx.x] = acc;  // keeps the chains alive
}

cudaError_t launch_imad_probe(uint32_t *sink, int blocks, int iters, cudaStream_t s) {
    k_imad_probe<<<blocks, 256, 0, s>>>(sink, iters);
    return cudaGetLastError();
}

cudaError_t init_kernel_attributes_main() {
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_col_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMaxN1 * 32 * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row_mul<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  2 * kMaxN2 * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row_mul<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMaxN2 * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row_mul_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  6 * kMaxN2 * 4 + 16)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_row_mul_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  6 * kMaxN2 * 4 + 16)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_col_inv<kInvTriples>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMaxN1 * 32 * 4)) != cudaSuccess) return e;
    if ((e = cudaFuncSetAttribute(k_col_inv<kInvResidues>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMaxN1 * 32 * 4)) != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_col_inv<kInvDigits>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kMaxN1 * 32 * 4);
}

}  // namespace dml
