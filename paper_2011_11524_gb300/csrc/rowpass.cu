// rowpass.cu -- dispatch of the specialized row pass (rowpass.cuh) over the instantiating
// translation units by the plan's row length.
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace dml {

#define DMUL_ROWPASS_DECL(TAG)                                                                        \
    cudaError_t upload_constants_rowpass_##TAG(const PrimeConst pc[kPrimes], const CrtConst &crt);   \
    bool rowpass_##TAG##_matches(const PlanDev &pd);                                                   \
    cudaError_t rowpass_##TAG##_run(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,   \
                                   uint32_t *status, cudaStream_t s);                                  \
    cudaError_t rowpass_##TAG##_run_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s, \
                                     bool rows);                                                       \
    cudaError_t rowpass_##TAG##_attrs();                                                             \
    bool rowpass_##TAG##_dft6_matches(const PlanDev &pd);                                              \
    cudaError_t rowpass_##TAG##_dft6(const PlanDev &pd, uint32_t *A, bool inv, cudaStream_t s);
DMUL_ROWPASS_DECL(big)
DMUL_ROWPASS_DECL(small)

static bool is_big(uint32_t n2) { return n2 >= 1024; }

bool row_pass_specialized(const PlanDev &pd) {
    return is_big(pd.N2) ? rowpass_big_matches(pd) : rowpass_small_matches(pd);
}

cudaError_t launch_row_pass_ct(const PlanDev &pd, uint32_t *X, const uint32_t *Y, bool square,
                               uint32_t *status, cudaStream_t s) {
    return is_big(pd.N2) ? rowpass_big_run(pd, X, Y, square, status, s)
                         : rowpass_small_run(pd, X, Y, square, status, s);
}

cudaError_t launch_row_pass_ct_b(const PlanDev &pd, const JobDev *jobs, int njobs, cudaStream_t s, bool rows) {
    return is_big(pd.N2) ? rowpass_big_run_b(pd, jobs, njobs, s, rows) : rowpass_small_run_b(pd, jobs, njobs, s, rows);
}

bool rowdft6_specialized(const PlanDev &pd) {
    return is_big(pd.N1) ? rowpass_big_dft6_matches(pd) : rowpass_small_dft6_matches(pd);
}

cudaError_t launch_rowdft6_ct(const PlanDev &pd, uint32_t *A, bool inv, cudaStream_t s) {
    return is_big(pd.N1) ? rowpass_big_dft6(pd, A, inv, s) : rowpass_small_dft6(pd, A, inv, s);
}

cudaError_t init_kernel_attributes_rowpass() {
    cudaError_t e = rowpass_big_attrs();
    return e != cudaSuccess ? e : rowpass_small_attrs();
}

cudaError_t upload_constants_rowpass(const PrimeConst pc[kPrimes], const CrtConst &crt) {
    cudaError_t e = upload_constants_rowpass_big(pc, crt);
    return e != cudaSuccess ? e : upload_constants_rowpass_small(pc, crt);
}

}  // namespace dml
