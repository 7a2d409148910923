// colpass.cu -- dispatch of the specialized column passes (colpass.cuh) over the instantiating
// translation units by the plan's column length.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace dml {

#define DMUL_COLPASS_DECL(TAG)                                                                        \
    cudaError_t upload_constants_colpass_##TAG(const PrimeConst pc[kPrimes], const CrtConst &crt);   \
    bool colpass_##TAG##_matches(const PlanDev &pd);                                                   \
    cudaError_t colpass_##TAG##_fwd(const PlanDev &pd, const uint32_t *x, uint64_t nx, const uint32_t *y, \
                                   uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *status, cudaStream_t s); \
    cudaError_t colpass_##TAG##_inv(const PlanDev &pd, const uint32_t *X, uint64_t L, uint32_t *out,   \
                                   uint2 *spill, cudaStream_t s, uint64_t *zero, uint32_t nzero);     \
    cudaError_t colpass_##TAG##_fwd_b(const PlanDev &pd, const JobDev *jobs, int njobs, uint32_t *status, \
                                     cudaStream_t s);                                                  \
    cudaError_t colpass_##TAG##_inv_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s); \
    cudaError_t colpass_##TAG##_attrs();
DMUL_COLPASS_DECL(big)
DMUL_COLPASS_DECL(small)
DMUL_COLPASS_DECL(five)

static bool is_big(uint32_t n1) { return n1 >= 512; }
static bool is_five(uint32_t n1) { return n1 % 5 == 0; }

bool col_pass_specialized(const PlanDev &pd) {
    if (is_five(pd.N1)) return colpass_five_matches(pd);
    return is_big(pd.N1) ? colpass_big_matches(pd) : colpass_small_matches(pd);
}

cudaError_t launch_col_fwd_spec(const PlanDev &pd, const uint32_t *x, uint64_t nx, const uint32_t *y,
                                uint64_t ny, uint32_t *X, uint32_t *Y, uint32_t *status, cudaStream_t s) {
    if (is_five(pd.N1)) return colpass_five_fwd(pd, x, nx, y, ny, X, Y, status, s);
    return is_big(pd.N1) ? colpass_big_fwd(pd, x, nx, y, ny, X, Y, status, s)
                         : colpass_small_fwd(pd, x, nx, y, ny, X, Y, status, s);
}

cudaError_t launch_col_inv_spec(const PlanDev &pd, const uint32_t *X, uint64_t L, uint32_t *out, uint2 *spill,
                                cudaStream_t s, uint64_t *zero, uint32_t nzero) {
    if (is_five(pd.N1)) return colpass_five_inv(pd, X, L, out, spill, s, zero, nzero);
    return is_big(pd.N1) ? colpass_big_inv(pd, X, L, out, spill, s, zero, nzero)
                         : colpass_small_inv(pd, X, L, out, spill, s, zero, nzero);
}

cudaError_t launch_col_fwd_bs(const PlanDev &pd, const JobDev *jobs, int njobs, uint32_t *status,
                              cudaStream_t s) {
    if (is_five(pd.N1)) return colpass_five_fwd_b(pd, jobs, njobs, status, s);
    return is_big(pd.N1) ? colpass_big_fwd_b(pd, jobs, njobs, status, s)
                         : colpass_small_fwd_b(pd, jobs, njobs, status, s);
}

cudaError_t launch_col_inv_bs(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s) {
    if (is_five(pd.N1)) return colpass_five_inv_b(pd, jobs, njobs, s);
    return is_big(pd.N1) ? colpass_big_inv_b(pd, jobs, njobs, s) : colpass_small_inv_b(pd, jobs, njobs, s);
}

cudaError_t init_kernel_attributes_colpass() {
    cudaError_t e = colpass_big_attrs();
    if (e == cudaSuccess) e = colpass_small_attrs();
    return e != cudaSuccess ? e : colpass_five_attrs();
}

cudaError_t upload_constants_colpass(const PrimeConst pc[kPrimes], const CrtConst &crt) {
    cudaError_t e = upload_constants_colpass_big(pc, crt);
    if (e == cudaSuccess) e = upload_constants_colpass_small(pc, crt);
    return e != cudaSuccess ? e : upload_constants_colpass_five(pc, crt);
}

}  // namespace dml
