// kernels.cuh -- launch interface of the multiplication pipeline kernels (host side).
#pragma once
#include <utility>
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <stdint.h>
#include "common.h"

namespace dml {

// SM count of the current device, cached per device ordinal (thread-safe: launches come from the
// caller's threads and the serving loop's).
inline int current_device_sms() {
    static std::mutex mu;
    static std::map<int, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(dev);
    if (it != cache.end()) return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
        cudaGetLastError();
        sms = 1;
    }
    cache[dev] = sms;
    return sms;
}

// Device-side status bits (accumulated in a context word, read by dmul_sync).
constexpr uint32_t kStatusInvalid = 1u;   // an input limb >= 10^9, or the result overflowed
constexpr uint32_t kStatusTimeout = 2u;   // a bounded wait expired

// Control block of one carry scan (zeroed before each scan).
struct CarryCtl {
    uint32_t ticket;   // dynamic tile counter
    uint32_t done;     // tiles finished
    uint64_t top;      // highest nonzero limb index + 1
    uint64_t flags[1]; // per-tile lookahead words (ntiles entries)
};
inline size_t carry_ctl_bytes(uint64_t L) {
    uint64_t ntiles = (L + kCarryLimbs - 1) / kCarryLimbs;
    return sizeof(CarryCtl) + ntiles * sizeof(uint64_t);
}

// Launch with programmatic stream serialization (the kernel may begin while its predecessor in the
// stream drains; it calls pdl_wait() before touching memory) and, for cluster > 1, a cluster shape.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              unsigned cluster, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[2];
    unsigned n = 0;
    at[n].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[n].val.programmaticStreamSerializationAllowed = 1;
    ++n;
    if (cluster > 1) {
        at[n].id = cudaLaunchAttributeClusterDimension;
        at[n].val.clusterDim.x = cluster;
        at[n].val.clusterDim.y = 1;
        at[n].val.clusterDim.z = 1;
        ++n;
    }
    cfg.attrs = at;
    cfg.numAttrs = n;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// One job of a batched launch (device-resident descriptor).
struct JobDev {
    const uint32_t *x, *y;  // operands (y == x for a squaring)
    uint32_t *z;            // product, L limbs
    uint64_t *nz;           // normalized length or null
    uint64_t nx, ny, L;
    uint32_t *X, *Y;        // residue scratch (medium jobs)
    uint2 *spill;
    CarryCtl *ctl;
    uint32_t square, ntiles;
    uint32_t plan;          // index of the job's small plan (persistent small-job launch)
    uint32_t pad;
    uint32_t *stat;         // the job's own device status word (batched form), or null: the launch's
};

// The status word a job's device-side errors go to: its own (batched form) or the launch's.
__host__ __device__ inline uint32_t *job_status(const JobDev &J, uint32_t *launch_status) {
    return J.stat ? J.stat : launch_status;
}

// Inverse column pass output modes.
enum InvMode { kInvDigits = 0, kInvTriples = 1, kInvResidues = 2 };

cudaError_t upload_constants_main(const PrimeConst pc[kPrimes], const CrtConst &crt);
cudaError_t upload_constants_sixstep(const PrimeConst pc[kPrimes], const CrtConst &crt);
cudaError_t upload_constants_batch(const PrimeConst pc[kPrimes], const CrtConst &crt);

// x (and y) limbs -> forward column transforms + four-step twiddle -> X (and Y) residues [3][N].
cudaError_t launch_col_fwd(const PlanDev &pd, const uint32_t *x, uint64_t nx, const uint32_t *y,
                           uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *status, cudaStream_t s);

// Row pass: forward row transforms, pointwise product (or square), inverse row transforms,
// result in X.
cudaError_t launch_row_mul(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,
                           cudaStream_t s, uint32_t *status = nullptr);

// The same row pass as a persistent kernel fed by bulk asynchronous copies (TMA), pd.row_grid
// CTAs per prime, each prefetching its next row while computing the current one.
cudaError_t launch_row_mul_tma(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,
                               uint32_t *status, cudaStream_t s);

// Specialized row passes for N2 in {256, 512, 1024, 2048, 4096, 8192} with the planner's schedule
// (rowpass.cu), plain or TMA-fed per pd.row_tma.
bool row_pass_specialized(const PlanDev &pd);
cudaError_t launch_row_pass_ct(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,
                               uint32_t *status, cudaStream_t s);
cudaError_t init_kernel_attributes_rowpass();
cudaError_t upload_constants_rowpass(const PrimeConst pc[kPrimes], const CrtConst &crt);

// Specialized column passes (colpass.cuh; N1 in {64, 96, 128, 192, 256, 384, 512, 768, 1024, 1536}
// with the planner's schedule), on full or half tiles per pd.col_half.  launch_col_fwd /
// launch_col_inv dispatch to them when the schedule matches (forward: both operands 16-byte
// aligned; inverse: the digit-sum mode).  The batched forms take a job array (job = blockIdx.z;
// every operand 16-byte aligned).
bool col_pass_specialized(const PlanDev &pd);
cudaError_t launch_col_fwd_spec(const PlanDev &pd, const uint32_t *x, uint64_t nx, const uint32_t *y,
                                uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *status, cudaStream_t s);
cudaError_t launch_col_inv_spec(const PlanDev &pd, const uint32_t *X, uint64_t L, uint32_t *out, uint2 *spill,
                                cudaStream_t s, uint64_t *zero, uint32_t nzero);
cudaError_t launch_col_fwd_bs(const PlanDev &pd, const JobDev *jobs, int njobs, uint32_t *status,
                              cudaStream_t s);
cudaError_t launch_col_inv_bs(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s);
cudaError_t init_kernel_attributes_colpass();
cudaError_t upload_constants_colpass(const PrimeConst pc[kPrimes], const CrtConst &crt);
// The specialized row pass for a batch of medium products of one transform length (plain form;
// squarings per job).
// rows: several short rows per CTA where the batch is large enough (dmul_batch; see rowpass.cuh)
cudaError_t launch_row_pass_ct_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s,
                                 bool rows = false);
cudaError_t upload_constants_colpass(const PrimeConst pc[kPrimes], const CrtConst &crt);

// The row pass the plan asks for: specialized when available, else the generic plain or TMA form.
cudaError_t launch_row_any(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,
                           uint32_t *status, cudaStream_t s);

// Inverse column pass + (mode) CRT and digit split.  kInvDigits writes the within-chunk digit
// sums to out[0..L) and the chunk spills to spill; kInvTriples writes d[3k..3k+2]; kInvResidues
// writes r[pi*L + k].
// zero/zero_bytes (optional, a multiple of 8 bytes): device words the kernel clears after its
// predecessor in the stream has finished -- the carry scan's control block, so that no separate
// memset separates the two kernels.
cudaError_t launch_col_inv(const PlanDev &pd, const uint32_t *X, uint64_t L, InvMode mode,
                           uint32_t *out, uint2 *spill, cudaStream_t s, void *zero = nullptr,
                           size_t zero_bytes = 0);

// Digit triples -> within-chunk digit sums + spills (the tail of the CRT stage, on its own).
cudaError_t launch_triples_to_digits(const uint32_t *d, uint64_t L, uint32_t *out, uint2 *spill,
                                     uint32_t *status, cudaStream_t s);

// Decoupled-lookahead carry scan: z[0..L) (digit sums < 3*10^9) + spills -> base-10^9 limbs in
// zo[0..L) (zo == nullptr: in place in z; else a disjoint buffer, device or pinned host memory),
// *nz (device or pinned host, may be null).  ctl must be zeroed (carry_ctl_bytes(L)) before the
// launch.
// spin (0: the default) bounds each device-side wait of the scan, in polls.
cudaError_t launch_carry(uint32_t *z, const uint2 *spill, uint64_t L, CarryCtl *ctl, uint64_t *nz,
                         uint32_t *status, cudaStream_t s, uint32_t *zo = nullptr, uint32_t spin = 0);

// Six-step pieces (Sec. 7.2, 7.6).
// packing + the first transpose (limbs as N1 x N2 -> the three primes' N2 x N1 residues), out of place
cudaError_t launch_pack_transpose(const uint32_t *x, uint64_t nx, uint32_t N1, uint32_t N2, uint32_t *X,
                                  uint32_t *status, cudaStream_t s);
// In place; 16-byte aligned matrices take the TMA-fed kernels (tensor-map tile loads of the I <= J
// tile pairs, bulk-copied rows for rho).  status (may be null) receives an expired bounded wait.
cudaError_t launch_transpose(uint32_t *a, uint64_t rows, uint64_t cols, uint64_t batch,
                             uint64_t batch_stride, cudaStream_t s, uint32_t *status = nullptr);
cudaError_t launch_rowdft_fwd_tw(const PlanDev &pd, uint32_t *A, cudaStream_t s);
// The same two steps specialized on N1 in {256, ..., 8192} with the planner's schedule (rowpass.cuh).
bool rowdft6_specialized(const PlanDev &pd);
cudaError_t launch_rowdft6_ct(const PlanDev &pd, uint32_t *A, bool inv, cudaStream_t s);
cudaError_t launch_rowdft_inv_tw(const PlanDev &pd, uint32_t *A, cudaStream_t s);
// the last transpose + CRT: residues in N2 x N1 matrices ([n2][k1] = coefficient k1 N2 + n2)
cudaError_t launch_crt_transposed(const uint32_t *X, uint32_t N1, uint32_t N2, uint64_t L, InvMode mode,
                                  uint32_t *out, uint2 *spill, cudaStream_t s);

// Batched forms (batch.cu).  small: one cluster of three CTAs per job does the whole product.
cudaError_t launch_small_mul(const SmallPlanDev &sp, const JobDev *jobs, int njobs, uint32_t *status,
                             cudaStream_t s);
cudaError_t launch_small_mul_one(const SmallPlanDev &sp, const JobDev &job, uint32_t *status,
                                 cudaStream_t s);
// One persistent launch for every short product of a batch: clusters take jobs from *counter
// (zeroed beforehand) until none is left; plans[job.plan] is the job's small plan.
cudaError_t launch_small_persistent(const SmallPlanDev *plans, uint32_t maxN, const JobDev *jobs,
                                    uint32_t njobs, uint32_t *counter, uint32_t *status, cudaStream_t s);
cudaError_t launch_col_fwd_b(const PlanDev &pd, const JobDev *jobs, int njobs, uint32_t *status,
                             cudaStream_t s);
cudaError_t launch_row_mul_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s);
cudaError_t launch_col_inv_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s);
cudaError_t launch_carry_b(const JobDev *jobs, int njobs, uint32_t maxtiles, uint32_t *status,
                           cudaStream_t s);

// A short four-step product in one cooperative launch (shortfused.cu): forward columns, row pass,
// inverse columns, CRT with digit sums, carry scan as five phases separated by grid barriers.
// Supported for the planner's schedules at N1 in {64, 80, 96}, N2 = 256; x and y 16-byte aligned.
// gbar: a device word of the grid barriers (zero-initialized once, never reset; one launch at a
// time per word).  48 <= grid <= the SM count (every CTA resident at once).  pd.tw[0] starts the
// plan's contiguous twiddle tables of table_bytes bytes.
// The carry scan's control block ctl (carry_ctl_bytes(nx + ny)) is cleared by the kernel.
bool short_fused_supported(const PlanDev &pd);
cudaError_t launch_short_fused(const PlanDev &pd, uint64_t table_bytes, const uint32_t *x, uint64_t nx,
                               const uint32_t *y, uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *z, uint64_t *nz,
                               uint2 *spill, CarryCtl *ctl, uint32_t *status, uint32_t *gbar, uint32_t spin,
                               uint32_t grid, cudaStream_t s);
cudaError_t upload_constants_shortfused(const PrimeConst pc[kPrimes], const CrtConst &crt);

// Sets the shared-memory / cluster attributes of every kernel once (outside any graph capture).
cudaError_t init_kernel_attributes_main();
cudaError_t init_kernel_attributes_sixstep();
cudaError_t init_kernel_attributes_batch();

// Integer-pipe probe.
cudaError_t launch_imad_probe(uint32_t *sink, int blocks, int iters, cudaStream_t s);

}  // namespace dml
