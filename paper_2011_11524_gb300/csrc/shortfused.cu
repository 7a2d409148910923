// shortfused.cu -- the whole four-step product of a short operand pair in one cooperative launch.
//
// A product of up to 24576 limbs runs through the same steps as the four-step pipeline (forward
// column DFTs with the four-step twiddle, Sec. 7.1; fused row pass, Sec. 5.4 / 6; inverse column
// DFTs; three-prime CRT, Sec. 8.2.2; chunk digit sums and the lookahead carry scan, Sec. 3.2), but
// the four kernels become five phases of one grid, separated by grid-wide barriers.  At these
// sizes each kernel of the pipeline does a few microseconds of work; one launch keeps the SMs and
// the data (all of it L2-resident) in place, at the price of a cooperative launch and four grid
// barriers.  Which wins is measured per length on first use (api.cu): at 10^5-digit operands the
// four programmatically chained kernels do (28 against 35 microseconds).  The phases reuse the
// specialized device code of the pipeline kernels (colpass.cuh, rowpass.cuh, stages.cuh) for
// column lengths N1 in {64, 80, 96} and rows of N2 = 256, so the arithmetic, the order of the
// outputs and the results are the pipeline's own.
//
// The launch is cooperative (every CTA resident at once), so a CTA may wait for the others:
// every barrier wait is bounded, and an expired one sets the timeout bit and lets the CTA go on.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "colpass.cuh"
#include "rowpass.cuh"

namespace dml {

DMUL_DEFINE_UPLOAD(upload_constants_shortfused)

namespace {

constexpr uint32_t kFusedN2 = 256;
constexpr uint32_t kFusedThreads = 256;

struct FusedArgs {
    const uint32_t *x, *y;  // operands (y == x for a square), 16-byte aligned
    uint64_t nx, ny, L;
    uint32_t *X, *Y;        // residue scratch [3][N] each
    uint32_t *z;            // product limbs (digit sums between phases 4 and 5)
    uint64_t *nz;
    uint2 *spill;
    CarryCtl *ctl;
    uint32_t *status;
    uint32_t *gbar;         // grid barrier word
    const uint8_t *tables;  // the plan's twiddle tables (all primes, contiguous) and their size
    uint64_t table_bytes;
    uint32_t spin;          // bound of every wait (polls)
    uint32_t rows;          // rows of one prime per row-pass task
    uint32_t ntiles, ctl_words;
};

// Grid-wide barrier on one device word.  Every CTA adds to the word once per barrier: CTA 0 adds
// 2^31 - (G - 1), the others 1, so that once all G have arrived the word has gained exactly 2^31:
// its top bit has flipped and its other bits are back where they were.  A CTA waits (bounded) for
// the top bit to differ from the one its own addition saw.  The word needs no reset between
// barriers or launches (a launch adds 4 * 2^31 = 0 mod 2^32 in all, even when a wait expired).
__device__ __forceinline__ void grid_barrier(const FusedArgs &a) {
    __syncthreads();  // the CTA's writes happen before thread 0's release below
    if (threadIdx.x == 0) {
        const uint32_t add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1) : 1u;
        uint32_t old;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(a.gbar), "r"(add) : "memory");
        for (uint32_t spins = 0; ((ld_acquire_u32(a.gbar) ^ old) & 0x80000000u) == 0;) {
            if (++spins > a.spin) {
                atomicOr(a.status, kStatusTimeout);
                break;
            }
        }
    }
    __syncthreads();  // and every other CTA's writes before this CTA's next reads
}

template <uint32_t N1, bool SQR>
__global__ void __launch_bounds__(kFusedThreads) k_short_fused(const PlanDev pd, const FusedArgs a) {
    extern __shared__ __align__(16) uint32_t sm[];
    const uint32_t G = gridDim.x, b = blockIdx.x;
    constexpr uint32_t tiles = kFusedN2 / 32;
    // phase 1: forward column passes of x (and y), one 32-column tile of one prime per task; the
    // carry scan's control block is cleared on the way, and the CTAs without a column task bring
    // the twiddle tables of the later phases into L2 (bulk prefetches of 4 KB)
    constexpr uint32_t col_tasks = kPrimes * tiles * (SQR ? 1u : 2u);
    if (b == 0)
        for (uint32_t i = threadIdx.x; i < a.ctl_words; i += blockDim.x) ((uint64_t *)a.ctl)[i] = 0;
    if (b >= col_tasks) {
        const uint64_t nblk = (a.table_bytes + 4095) / 4096;
        for (uint64_t i = (uint64_t)(b - col_tasks) * blockDim.x + threadIdx.x; i < nblk;
             i += (uint64_t)(G - col_tasks) * blockDim.x) {
            const uint64_t off = i * 4096, left = a.table_bytes - off;
            const uint32_t bytes = (uint32_t)(left < 4096 ? left : 4096);
            asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a.tables + off), "r"(bytes) : "memory");
        }
    }
    for (uint32_t t = b; t < col_tasks; t += G) {
        const uint32_t pi = t % kPrimes, tile = (t / kPrimes) % tiles, second = t / (kPrimes * tiles);
        DMUL_PRIME_SWITCH((int)pi, (col_fwd_ct_body<PI, N1>(pd, sm, second ? a.y : a.x, second ? a.ny : a.nx,
                                                            (second ? a.Y : a.X) + (uint64_t)pi * pd.N, tile,
                                                            a.status)));
        __syncthreads();
    }
    grid_barrier(a);
    // phase 2: the fused row pass, `rows` consecutive rows of one prime per task (a row of 256 has
    // 16 radix-16 groups per stage: one row would leave all but 16 threads idle)
    for (uint32_t t = b; t < kPrimes * (N1 / a.rows); t += G) {
        const uint32_t pi = t % kPrimes, row = (t / kPrimes) * a.rows;
        uint32_t *xr = a.X + (uint64_t)pi * pd.N + (uint64_t)row * kFusedN2;
        const uint32_t *yr = SQR ? nullptr : a.Y + (uint64_t)pi * pd.N + (uint64_t)row * kFusedN2;
        uint32_t *sy = sm + a.rows * RowPad<kFusedN2>::NP;
        DMUL_PRIME_SWITCH((int)pi, (row_core_ct<PI, kFusedN2, SQR>(pd, sm, sy, xr, yr, xr, a.rows)));
        __syncthreads();
    }
    grid_barrier(a);
    // phase 3: inverse column passes (residues, reduced to [0, p), natural order) into Y
    for (uint32_t t = b; t < kPrimes * tiles; t += G) {
        const uint32_t pi = t % kPrimes, tile = t / kPrimes;
        const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
        DMUL_PRIME_SWITCH((int)pi, (col_inv_ct_body<PI, N1>(pd, a.X + (uint64_t)pi * pd.N, sm, tile * 32 + lane)));
        __syncthreads();
        uint32_t *dst = a.Y + (uint64_t)pi * pd.N;
        for (uint32_t r = warp; r < N1; r += nw) dst[(uint64_t)r * kFusedN2 + tile * 32 + lane] = sm[r * 32 + lane];
        __syncthreads();
    }
    grid_barrier(a);
    // phase 4: CRT of every coefficient and the digit sums of each 32-coefficient chunk (L2 reads:
    // the residues were written by other SMs after this SM may have cached Y in phase 2)
    {
        const uint32_t lane = threadIdx.x & 31, nw = blockDim.x >> 5;
        const uint64_t chunks = (a.L + 31) / 32;
        for (uint64_t c = (uint64_t)b * nw + (threadIdx.x >> 5); c < chunks; c += (uint64_t)G * nw) {
            const uint64_t k = c * 32 + lane;
            uint32_t d0, d1, d2;
            crt_digits(__ldcg(a.Y + k), __ldcg(a.Y + pd.N + k), __ldcg(a.Y + 2 * pd.N + k), d0, d1, d2);
            uint32_t sv;
            uint2 sp;
            chunk_digits(d0, d1, d2, sv, sp);
            if (k < a.L) a.z[k] = sv;
            if (lane == 31) a.spill[c] = sp;
        }
    }
    grid_barrier(a);
    // phase 5: the lookahead carry scan (every tile's CTA is resident, so its waits end)
    carry_tile<kFusedThreads, 8>(a.z, a.z, a.spill, a.L, a.ctl, a.nz, a.status, a.ntiles, a.spin);
}

template <uint32_t N1>
bool fused_schedule_matches(const PlanDev &pd) {
    using S = ColSched<N1>;
    using R = Pow2Sched<kFusedN2>;
    if (pd.N1 != N1 || pd.N2 != kFusedN2 || pd.ncs != S::NS || pd.nrs != R::NS) return false;
    for (int t = 0; t < S::NS; ++t)
        if (pd.cs[t].R != S::radix(t) || pd.cs[t].m != S::span(t)) return false;
    for (int t = 0; t < R::NS; ++t)
        if (pd.rs[t].R != R::radix(t) || pd.rs[t].m != R::span(t)) return false;
    return true;
}

size_t fused_smem(uint32_t N1, uint32_t rows) {
    const size_t col = (size_t)N1 * 32 * 4, row = (size_t)2 * rows * RowPad<kFusedN2>::NP * 4;
    return col > row ? col : row;
}

template <uint32_t N1, bool SQR>
cudaError_t launch_fused(const PlanDev &pd, const FusedArgs &a, uint32_t grid, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kFusedThreads);
    cfg.dynamicSmemBytes = fused_smem(N1, a.rows);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_short_fused<N1, SQR>, pd, a);
}

}  // namespace

bool short_fused_supported(const PlanDev &pd) {
    return fused_schedule_matches<64>(pd) || fused_schedule_matches<80>(pd) || fused_schedule_matches<96>(pd);
}

cudaError_t launch_short_fused(const PlanDev &pd, uint64_t table_bytes, const uint32_t *x, uint64_t nx,
                               const uint32_t *y, uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *z, uint64_t *nz,
                               uint2 *spill, CarryCtl *ctl, uint32_t *status, uint32_t *gbar, uint32_t spin,
                               uint32_t grid, cudaStream_t s) {
    if (grid < 2 * kPrimes * (kFusedN2 / 32) || (((uintptr_t)pd.tw[0]) & 15)) return cudaErrorInvalidValue;
    FusedArgs a;
    a.tables = (const uint8_t *)pd.tw[0];
    a.table_bytes = table_bytes & ~(uint64_t)15;  // a bulk prefetch moves multiples of 16 bytes
    a.x = x;
    a.y = y;
    a.nx = nx;
    a.ny = ny;
    a.L = nx + ny;
    a.X = X;
    a.Y = Y;
    a.z = z;
    a.nz = nz;
    a.spill = spill;
    a.ctl = ctl;
    a.status = status;
    a.gbar = gbar;
    a.spin = spin ? spin : kSpinLimit;
    // the fewest rows per task that still give every row task its own CTA
    a.rows = 1;
    while (kPrimes * (pd.N1 / a.rows) > grid && (pd.N1 % (2 * a.rows)) == 0) a.rows *= 2;
    a.ntiles = (uint32_t)((a.L + kFusedThreads * 8 - 1) / (kFusedThreads * 8));
    a.ctl_words = (uint32_t)(carry_ctl_bytes(a.L) / 8);
    const bool sq = x == y && nx == ny;
    switch (pd.N1) {
        case 64: return sq ? launch_fused<64, true>(pd, a, grid, s) : launch_fused<64, false>(pd, a, grid, s);
        case 80: return sq ? launch_fused<80, true>(pd, a, grid, s) : launch_fused<80, false>(pd, a, grid, s);
        case 96: return sq ? launch_fused<96, true>(pd, a, grid, s) : launch_fused<96, false>(pd, a, grid, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace dml
