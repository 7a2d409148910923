/*
 * dmul.h -- C ABI of libdmul: exact multiplication of large decimal integers on one GB300 GPU.
 *
 * Method (Krapivensky, "Speeding up decimal multiplication", arXiv 2011.11524):
 *   the product of x = <x_0..x_{n-1}> and y = <y_0..y_{m-1}> in base B = 10^9 is recovered from the
 *   cyclic convolution of the zero-padded limb vectors (Sec. 3.2), computed exactly by
 *   number-theoretic transforms modulo three primes p < 2^30 of the form c*3*2^n + 1 (Sec. 3.5,
 *   Sec. 4.5) with the matrix-Fourier four-step / six-step decomposition (Sec. 7), a pointwise
 *   Montgomery product with the linearity trick (Sec. 6), CRT recovery of every coefficient
 *   (Sec. 8.2.2, extended to three primes) and the decimal carry recurrence (Sec. 3.2,
 *   eq. sigmai_and_zi), here as a decoupled-lookahead scan.
 *
 * Number format (all entry points): little-endian base-10^9 limbs, one uint32_t per limb, each
 * limb < 10^9.  Leading zero limbs are allowed (the padding of Sec. 3.2).  Zero is nz = 1,
 * z[0] = 0.
 *
 * Pointers: unless a function says "host", limb pointers are DEVICE pointers owned by the
 * caller, on the context's device.  `stream` is a cudaStream_t passed as void* (NULL = the
 * legacy default stream).  Device-pointer entry points only enqueue work: they return DMUL_OK
 * once the work is queued, and device-side errors (an input limb >= 10^9, an expired bounded
 * wait) are reported by the next dmul_sync() on that context.
 *
 * Threading: a context is not thread-safe.  Its device scratch is shared by the calls made on it,
 * so calls on one context must be issued on one stream (or be otherwise serialized), except the
 * served entry points dmul_submit / dmul_poll / dmul_wait, which may be called from any thread.
 * While the serving loop has work (between the first dmul_submit and the last completion) the
 * context is its own: the loop plans new lengths and times short ones on the context's plans and
 * scratch, so the other entry points must not be called on it meanwhile.
 *
 * Errors: every int-returning function returns one of the DMUL_* codes below.
 */
#ifndef DMUL_H
#define DMUL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------------------------- */
#define DMUL_OK 0
#define DMUL_ERR_INVALID 1   /* bad argument, a limb >= 10^9, aliasing of z with x or y        */
#define DMUL_ERR_TOO_LARGE 2 /* n+m exceeds the longest supported transform or max_limbs, or    */
                             /* (B-1)^2 min(n,m) >= p1 p2 p3 (eq. product_inequality)         */
#define DMUL_ERR_NOMEM 3     /* the context's HBM budget, or a device allocation, is exhausted   */
#define DMUL_ERR_TIMEOUT 4   /* a bounded device-side wait expired (the result is not valid)    */
#define DMUL_ERR_CUDA 5      /* a CUDA runtime call failed                                      */
#define DMUL_ERR_CAPACITY 6  /* z_cap < nx + ny                                                 */
#define DMUL_ERR_UNKNOWN_TICKET 7 /* dmul_poll / dmul_wait on a ticket that was never issued,   */
                                  /* or whose result was already returned (see dmul_wait)        */
#define DMUL_PENDING (-1)         /* dmul_job.status of a job whose batch has not been checked yet */

/* ---- context ------------------------------------------------------------------------------- */
typedef struct dmul_ctx dmul_ctx;

#define DMUL_FLAG_SIXSTEP 1u      /* transforms use the six-step decomposition with the in-place */
                                  /* n x n, n x 2n and 2n x n transposes of Sec. 7.6 instead of   */
                                  /* the four-step form (Sec. 7.1-7.2); results are identical     */
#define DMUL_FLAG_STAGE_TIMING 2u /* record CUDA events around each pipeline stage (see          */
                                  /* dmul_stage_times); adds a little launch overhead             */
#define DMUL_FLAG_NO_SMALL 4u     /* never use the one-cluster kernel for short products          */
                                  /* (transform length <= 24576); they take the four-step path    */
#define DMUL_FLAG_NO_AUTOTUNE 8u  /* plan every length with the default split instead of timing   */
                                  /* the candidate splits and CTA sizes on first use              */
#define DMUL_FLAG_COL_HALF 32u   /* with DMUL_FLAG_NO_AUTOTUNE: run the column passes on N1 x 16 */
                                  /* half tiles (N1 in {512, 768, 1024, 1536}) instead of N1 x 32 */
#define DMUL_FLAG_ROW_TMA 16u     /* with DMUL_FLAG_NO_AUTOTUNE: use the persistent row pass fed  */
                                  /* by bulk asynchronous copies (TMA) instead of one CTA per row */
#define DMUL_FLAG_HOST_STAGED_IN 64u   /* dmul_mul_host: copy page-locked operands into device   */
                                       /* staging buffers instead of reading them in place       */
#define DMUL_FLAG_HOST_DIRECT_IN 256u  /* dmul_mul_host: read page-locked operands in place at   */
                                       /* every length (default: only short products, see below) */
#define DMUL_FLAG_NO_RADIX5 512u       /* transform lengths from {2^k, 3 2^k} only (default: also */
                                       /* 5 2^k, with a radix-5 first column stage)              */
#define DMUL_FLAG_HOST_STAGED_OUT 128u /* dmul_mul_host: write the product to a device buffer    */
                                       /* and copy it out, instead of writing a page-locked z    */
                                       /* in place                                               */
#define DMUL_FLAG_HOST_DIRECT_OUT 8192u /* dmul_mul_host: write a page-locked z in place at     */
                                       /* every length (default: only short products)            */
#define DMUL_FLAG_SHORT_WAITS 1024u    /* bound every device-side wait (carry look-back, column-  */
                                       /* to-row hand-off, bulk-copy barriers) by 2^13 polls, a  */
                                       /* few milliseconds, instead of seconds: an expired wait  */
                                       /* reports DMUL_ERR_TIMEOUT soon (for tests of that path) */
#define DMUL_FLAG_TEST_STALL_CARRY 2048u /* fault injection for tests, on the host side:        */
                                       /* dmul_carry starts its tile ticket at 1, so that tile 0 */
                                       /* never runs and tile 1's bounded look-back wait expires */
                                       /* (DMUL_ERR_TIMEOUT at the next dmul_sync); the kernels  */
                                       /* end normally and the context stays usable              */
#define DMUL_FLAG_NO_FUSED 4096u       /* never run a lone short product (transform length       */
                                       /* 16384, 20480 or 24576, as N1 x 256) as the four-step   */
                                       /* steps in one cooperative launch; it takes the small    */
                                       /* kernel or the four-kernel pipeline                     */

typedef struct {
    int device;                /* CUDA device ordinal                                          */
    uint64_t hbm_budget_bytes; /* cap on library-owned device memory; 0 = 16 GiB               */
    uint64_t max_limbs;        /* longest product (nx + ny) the context must accept; 0 = the   */
                               /* longest transform the primes allow                           */
    uint32_t flags;            /* DMUL_FLAG_*                                                  */
} dmul_config;

/* Create a context on cfg->device: checks the prime set against FindPrimes (Sec. 4.5) and the
 * bound of eq. product_inequality, uploads per-prime constants.  Plans (transform splits,
 * twiddle tables) are built and cached per transform length on first use.  cfg may be NULL
 * (device 0, defaults).  *out receives the context, or NULL on error. */
int dmul_init(dmul_ctx **out, const dmul_config *cfg);

/* Free every device and host resource of the context (synchronizes its device first). */
void dmul_destroy(dmul_ctx *ctx);

/* Human-readable name of a status code (static string). */
const char *dmul_strerror(int status);

/* Synchronize `stream` and return the device-side status accumulated by the work enqueued on
 * this context since the previous dmul_sync (DMUL_OK, DMUL_ERR_INVALID, DMUL_ERR_TIMEOUT), then
 * clear it.  It also fills the status field of every job of the last dmul_batch (see there); a
 * failed batch job makes this return that job's error too.  Returns DMUL_ERR_CUDA if the
 * synchronization itself fails. */
int dmul_sync(dmul_ctx *ctx, void *stream);

/* ---- the plain form -------------------------------------------------------------------------- */
/* z = x * y (Sec. 3.2).  x: nx >= 1 limbs, y: ny >= 1 limbs, z: z_cap >= nx + ny limbs, all
 * device pointers; z must not overlap x or y.  x == y with nx == ny is a squaring (the aliasing
 * case of Sec. 6) and takes the cheaper dmul_sqr path.  All nx + ny limbs of z are written.
 * nz (device pointer to one uint64_t, or NULL) receives the normalized length: the index of the
 * highest nonzero limb + 1, or 1 for a zero product.  Asynchronous on `stream`.
 * A short product (transform length <= 24576) runs, by the first such product's timing, as one
 * cluster kernel, as the four-kernel pipeline or, at lengths 16384, 20480 and 24576 with 16-byte
 * aligned operands and outside a stream capture, as one cooperative launch of the same four-step
 * steps; the limbs are identical on every path (DMUL_FLAG_NO_SMALL / DMUL_FLAG_NO_FUSED rule
 * paths out).
 * Stream capture: a call may be captured into a CUDA graph once a product of the same lengths has
 * run on this context outside the capture (its plan, scratch and path choice then exist); the
 * graph's replays multiply whatever the buffers hold at replay time.  Captured, a product takes
 * the pipeline's plain launches (no cooperative kernel, no per-prime hand-off between the column
 * and row passes).  A call whose lengths are not planned yet returns DMUL_ERR_INVALID inside a
 * capture, having enqueued nothing. */
int dmul_mul(dmul_ctx *ctx, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny,
             uint32_t *z, size_t z_cap, uint64_t *nz, void *stream);

/* z = x^2: one forward transform instead of two (Sec. 6, the x aliasing y case).  z_cap >= 2 nx.
 * Same conventions as dmul_mul. */
int dmul_sqr(dmul_ctx *ctx, const uint32_t *x, size_t nx, uint32_t *z, size_t z_cap,
             uint64_t *nz, void *stream);

/* Host-memory convenience: x, y, z and nz are HOST pointers; the call returns when z and *nz
 * hold the product (it synchronizes).  x == y with nx == ny squares.  z must not overlap x or y.
 * Returns the full status (including device-side errors).
 *  - Page-locked buffers (cudaHostAlloc / cudaMallocHost / cudaHostRegister, both ends of the
 *    buffer inside registered memory; a buffer must not straddle two registrations) of a short
 *    product (nx + ny <= DMUL_HOST_IN_PLACE_LIMBS) are accessed in place: the forward pass reads
 *    the operands and the carry scan writes z, so the bytes cross the host link while the kernels
 *    run.  Longer products copy their page-locked operands (every prime's column pass reads its
 *    operand tile again) and their product (one copy-engine transfer after the carry scan: the
 *    scan's stores across the host link ran at two speeds from one machine state to another,
 *    the copy at one).  DMUL_FLAG_HOST_STAGED_IN / _OUT and DMUL_FLAG_HOST_DIRECT_IN / _OUT
 *    override this.
 *  - Pageable buffers are copied through device staging buffers (cudaMemcpyAsync; y's upload
 *    overlaps x's forward pass).
 * Device memory: nx + ny words for the digit sums, plus 2 (nx + ny) words of operand staging
 * when the operands are copied; DMUL_ERR_NOMEM beyond the context's budget. */
int dmul_mul_host(dmul_ctx *ctx, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny,
                  uint32_t *z, size_t z_cap, size_t *nz);

#define DMUL_HOST_IN_PLACE_LIMBS 524288u

/* 1 when the host buffer [p, p + bytes) is page-locked, so that dmul_mul_host can access it in
 * place, else 0 (pageable memory, or a null / empty range). */
int dmul_host_direct(dmul_ctx *ctx, const void *p, size_t bytes);

/* ---- the batched form -------------------------------------------------------------------------- */
typedef struct {
    const uint32_t *x; /* device pointer                                                 */
    uint64_t nx;
    const uint32_t *y; /* device pointer; y == x with ny == nx makes the job a squaring   */
    uint64_t ny;
    uint32_t *z;       /* device pointer, z_cap >= nx + ny                                */
    uint64_t z_cap;
    uint64_t *nz;      /* device pointer or NULL                                          */
    int status;        /* out (dmul_batch): this job's own status, see dmul_batch          */
} dmul_job;

/* Run `count` independent multiplications (jobs: HOST array of descriptors holding device
 * pointers).  Jobs are grouped by transform length; each group runs as batched launches that
 * process all of its jobs at once, and a repeated batch shape replays a captured CUDA graph.
 * Results are identical to calling dmul_mul on each job.  Asynchronous on `stream`.
 *
 * Every job has its own status, so one bad job does not fail the others:
 *  - a job the host rejects (null pointer, nx or ny = 0, z_cap < nx + ny, z overlapping x or y,
 *    too large) gets that code in jobs[i].status at once and is not run;
 *  - every other job gets DMUL_PENDING, replaced by its final status (DMUL_OK, DMUL_ERR_INVALID
 *    for a limb >= 10^9, DMUL_ERR_TIMEOUT) by the next dmul_sync or dmul_batch on the context,
 *    so `jobs` must stay valid until then.
 * Returns DMUL_OK when the accepted jobs (possibly none) were enqueued; any other code is a
 * failure of the call itself (bad context or array, budget, CUDA), with every job's status set
 * to it and nothing run. */
int dmul_batch(dmul_ctx *ctx, dmul_job *jobs, size_t count, void *stream);

/* ---- the served form ------------------------------------------------------------------------- */
/* Enqueue one job for the context's serving loop (a host thread that continuously batches
 * pending requests by transform length onto several streams, admitting each request only when
 * its device footprint fits the context's HBM budget).  The job's pointers are device pointers
 * that must stay valid until the ticket completes.  *ticket receives an id for dmul_poll /
 * dmul_wait.  Thread-safe. */
int dmul_submit(dmul_ctx *ctx, const dmul_job *job, uint64_t *ticket);

/* *done = 1 when the ticket's result is in z (and *nz), else 0.  With *done = 1 the return value
 * is the ticket's own status (a request is never failed by another request of its batch) and the
 * ticket is released: later calls on it return DMUL_ERR_UNKNOWN_TICKET.  Thread-safe. */
int dmul_poll(dmul_ctx *ctx, uint64_t ticket, int *done);

/* Block until the ticket completes; returns its own status and releases the ticket (each
 * ticket's result is returned once, by dmul_wait or by the dmul_poll that reports it done; a
 * later or concurrent second call gets DMUL_ERR_UNKNOWN_TICKET).  Thread-safe. */
int dmul_wait(dmul_ctx *ctx, uint64_t ticket);

/* Serving-loop counters, a snapshot (thread-safe; all zero before the first dmul_submit). */
typedef struct {
    uint64_t queued;             /* submitted requests not yet launched                          */
    uint64_t running;            /* requests in batches on the GPU                                */
    uint64_t held;               /* tickets issued and not yet released by dmul_wait / dmul_poll  */
                                 /* (queued + running + completed but not yet claimed)            */
    uint64_t peak_running;       /* the most requests on the GPU at once so far                   */
    uint64_t admit_budget_bytes; /* device memory the loop may give to in-flight requests: the   */
                                 /* context's HBM budget minus what the context held when the    */
                                 /* loop started                                                  */
    uint64_t inflight_bytes;     /* of which in use now                                           */
} dmul_serve_info;
int dmul_serve_stats(dmul_ctx *ctx, dmul_serve_info *out);

/* ---- stage-level entry points (each step of the path on its own, for checking) --------------- */
/* The convolution residues c_k mod p_i (Sec. 3.2 + Sec. 3.3 eq. conv_theorem + Sec. 6) for
 * k in [0, nx+ny) and the three primes in ascending order: r[i*(nx+ny) + k].  x == y squares.
 * Same forward transforms, pointwise product and inverse transforms as dmul_mul. */
int dmul_conv_residues(dmul_ctx *ctx, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny,
                       uint32_t *r, void *stream);

/* The exact convolution coefficients c_k after CRT (Sec. 8.2.2): c_k = d[3k] + d[3k+1] 10^9 +
 * d[3k+2] 10^18 with every d < 10^9, k in [0, nx+ny). */
int dmul_conv_coeffs(dmul_ctx *ctx, const uint32_t *x, size_t nx, const uint32_t *y, size_t ny,
                     uint32_t *d, void *stream);

/* The carry stage alone (Sec. 3.2, eq. sigmai_and_zi): z = sum_k c_k 10^(9k) for coefficients
 * given as base-10^9 digit triples d[3k..3k+2] (each < 10^9), k in [0, L).  z_cap >= L; the
 * result must fit in L limbs, else the device status reports DMUL_ERR_INVALID.  nz as in
 * dmul_mul. */
int dmul_carry(dmul_ctx *ctx, const uint32_t *d, size_t L, uint32_t *z, size_t z_cap,
               uint64_t *nz, void *stream);

/* The carry stage of dmul_carry, for callers that cannot allocate device memory.  (The paper has
 * no counterpart: this is a deployment variant, not a step of the method.)
 *
 * Who needs it: code whose process hands the whole GPU to another allocator (a caching allocator
 * that has reserved the device), code on a latency-critical path that cannot pay for cudaMalloc's
 * implicit device-wide synchronization, and code that cannot create a context (dmul_init
 * allocates).  This function takes no context and allocates nothing: its scratch (chunk spills, the
 * lookahead control block and a status word) lives in one static device array of about 1 MiB that
 * every GPU loading the library holds until the process exits.
 *
 * Arguments as dmul_carry: d holds L base-10^9 digit triples (device), z receives L limbs (device,
 * z_cap >= L, not overlapping d), nz (device pointer or NULL) the normalized length.  L may be at
 * most DMUL_NOALLOC_MAX_LIMBS; longer inputs return DMUL_ERR_TOO_LARGE without touching the GPU.
 * Return value: DMUL_OK once the work is enqueued, or a host-side error (arguments, size, CUDA)
 * with nothing enqueued.  It never reports device-side errors (the sum does not fit L limbs, an
 * expired bounded wait): those set *nz to 0, a value no valid result has, so a caller who needs
 * to see them must pass nz; with nz = NULL they are not observable.  Asynchronous on `stream`, on
 * the current device.
 *
 * The first call on a device (and again after a device reset, which creates a new context) looks
 * up the array's device address; make that first call before any stream capture.  All calls
 * share the one array and the next call overwrites it: calls whose work overlaps on the GPU
 * (different streams, or several host threads) race and must be serialized by the caller. */
#define DMUL_NOALLOC_MAX_LIMBS (1ull << 22)
int dmul_carry_noalloc(const uint32_t *d, size_t L, uint32_t *z, size_t z_cap, uint64_t *nz,
                       void *stream);

/* In-place transpose of a rows x cols row-major uint32 matrix on the device (Sec. 7.5-7.6):
 * square matrices by tile-pair swaps (TransposeSquareSubMatrix semantics); n x 2n by the paper's
 * procedure (rho on every row, then the two n x n halves transposed in place with row stride
 * 2n); 2n x n by its inverse (the halves first, then rho^-1 on every row); n x Cn and Cn x n for
 * any integer C by the generalization the paper closes Sec. 7.6 with (rho_C: column C i + k of a
 * row to position k n + i, then the C blocks; the mirror for Cn x n).  rows and cols must each be
 * a multiple of 32, the larger a multiple of the smaller and at most 16384 when they differ.
 * The row permutation's scratch is the CTA's shared memory (C n words per row, Sec. 7.6).  A
 * 16-byte aligned matrix moves through the bulk-copy engine: 2-D tensor-map tile loads of the
 * tile pairs and one bulk copy per permuted row; otherwise plain loads. */
int dmul_transpose(dmul_ctx *ctx, uint32_t *a, size_t rows, size_t cols, void *stream);

/* ---- host-side information (no GPU work; usable without a device) ---------------------------- */
typedef struct {
    uint32_t primes[3];   /* ascending                                                     */
    uint64_t N;           /* transform length: smallest 2^k, 3*2^k or 5*2^k >= L (see DMUL_FLAG_NO_RADIX5) */
    uint32_t N1, N2;      /* N = N1 * N2: column length, row length                         */
    uint32_t col_radix[8];/* radix of each column stage, first to last (0 ends the list)   */
    uint32_t row_radix[8];/* radix of each row stage                                        */
    uint32_t sixstep;     /* 1 when the context uses the six-step form                      */
    uint32_t col_threads; /* CTA size of the column passes                                  */
    uint32_t row_threads; /* CTA size of the row pass                                       */
    uint32_t row_tma;     /* 1: persistent row pass fed by bulk async copies (TMA)          */
    uint32_t row_grid;    /* its CTAs per prime                                             */
    uint32_t col_half;    /* 1: column passes on N1 x 16 half tiles (two or more CTAs per SM) */
} dmul_plan_info;

/* Plan the transform for a product of L limbs (L >= 2).  ctx may be NULL (default plan); with a
 * context, the plan it has tuned for that length (after its first use) is reported. */
int dmul_get_plan(const dmul_ctx *ctx, uint64_t L, dmul_plan_info *out);

/* The library's prime set (ascending), found by FindPrimes(w = 31, n_min = 23, l = 3) of Sec. 4.5
 * (primes c*3*2^n + 1 < 2^30, n >= 23, c odd, the three largest).  Host-only. */
int dmul_primes(uint32_t out[3]);

/* eq. lambda of Sec. 4.2: the largest n with (10^n - 1)^2 < (2^(w-1))^l / 2^log2M, computed in
 * exact integer arithmetic; -1 on bad arguments.  The library sizes its bound checks with the
 * same arithmetic.  Host-only. */
int dmul_lambda(int w, int l, int log2M);

/* Largest min(nx, ny) (in limbs) the prime set supports: (10^9 - 1)^2 * min(nx,ny) < p1 p2 p3. */
uint64_t dmul_max_min_limbs(void);

/* ---- measurement ------------------------------------------------------------------------------ */
/* Stage timing (needs DMUL_FLAG_STAGE_TIMING): the milliseconds each pipeline stage spent on the
 * device, summed over the calls since the previous dmul_stage_times call, measured with CUDA
 * events recorded on the calls' stream.  names[i] (static strings) and ms[i] for i < *n, where
 * *n is in: capacity, out: the number of stages.  Synchronizes the context's last stream. */
int dmul_stage_times(dmul_ctx *ctx, const char **names, double *ms, uint64_t *launches, int *n);

/* Switch stage timing on (on != 0) or off for the calls that follow, whatever the context's
 * DMUL_FLAG_STAGE_TIMING said; timings already recorded stay available to dmul_stage_times.
 * With timing off, consecutive pipeline kernels overlap their launch with the predecessor's
 * drain (the event records between stages would serialize them). */
int dmul_stage_timing(dmul_ctx *ctx, int on);

/* Integer-pipe probe: runs a kernel of independent 32-bit multiply-adds (the IMAD pipe of the
 * modular arithmetic) on every SM and returns the achieved rate in operations per second. */
int dmul_probe_imad(dmul_ctx *ctx, double *imad_per_s);

/* Prime-width probe (the choice of Sec. 4.2 made by measurement on the GPU): the fused row pass
 * of the four-step form (forward row DFTs of X and Y, pointwise Montgomery product, inverse row
 * DFTs; Sec. 5.4, 6, 7.1) over N residues, once with the paper's two-prime design in 64-bit words
 * (two primes c 3 2^n + 1 < 2^62 from FindPrimes(63, 23, 2), Shoup products by constants,
 * Montgomery with R = 2^64, rows of 4096) and once as the library runs it (three primes < 2^30,
 * 32-bit words, the plan the context has for length N).  Both on resident operands; the median
 * device times of ten runs each, in ms.  N: a multiple of 4096, at most 2^23.  Allocates about
 * 32 N bytes beyond the context's plain-form scratch. */
int dmul_probe_prime_width(dmul_ctx *ctx, uint64_t N, double *ms_two_62bit, double *ms_three_30bit);

/* The two-prime probe's primes, ascending (host-only). */
int dmul_probe64_primes(uint64_t out[2]);

/* Parity hook of that probe: for each prime i (of dmul_probe64_primes) and row r < rows, the
 * cyclic convolution of length 4096 of a[i][r][.] and b[i][r][.] modulo p_i (the convolution
 * theorem, Sec. 3.3), reduced to [0, p_i), into out[i][r][.].  a, b, out: device arrays of
 * 2 x rows x 4096 uint64 residues (< p_i for a and b); rows <= 65535.  Synchronous on `stream`. */
int dmul_probe64_conv(dmul_ctx *ctx, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t rows,
                      void *stream);

#ifdef __cplusplus
}
#endif
#endif /* DMUL_H */
