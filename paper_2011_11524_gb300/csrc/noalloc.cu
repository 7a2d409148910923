// noalloc.cu -- dmul_carry_noalloc: the carry stage with its scratch in a static device array.
//
// Some callers cannot allocate device memory: their process hands all of HBM to another allocator
// (a caching allocator that reserved the device), or they run on a latency-critical path where
// cudaMalloc's implicit device synchronization is not acceptable, or they cannot create a library
// context (dmul_init itself allocates).  For them this entry point runs the same two kernels as
// dmul_carry (digit sums + chunk spills, then the lookahead carry scan) but takes every byte of
// scratch from one file-scope __device__ array of fixed size, so it calls no allocation routine.
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/dmul.h"
#include "kernels.cuh"

namespace dml {
namespace {

// Longest coefficient vector the static scratch can hold (and the error it returns beyond it).
constexpr uint64_t kNoAllocMaxL = DMUL_NOALLOC_MAX_LIMBS;
constexpr size_t kStatusBytes = 256;
constexpr size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kCtlBytes = align256(sizeof(CarryCtl) + ((kNoAllocMaxL + kCarryLimbs - 1) / kCarryLimbs) * 8);
constexpr size_t kSpillBytes = align256(((kNoAllocMaxL + kChunk - 1) / kChunk + 1) * sizeof(uint2));
constexpr size_t kScratchBytes = kStatusBytes + kCtlBytes + kSpillBytes;

// The scratch: [status word | carry control block | chunk spills].  Every GPU that loads the
// library holds one copy of it until the process exits.  Host code must not use this name as an
// address (it is a host-side stand-in); the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
CUcontext g_owner[kMaxDevices] = {};  // the context the cached address belongs to
CUresult (*g_ctx_current)(CUcontext *) = nullptr;

// Device address of the scratch on the current device, looked up once per device and CUDA
// context (the set-up step: a device reset or a new primary context loads the module again, and
// the array may move, so the address is looked up again for the new context).
int scratch_address(unsigned char **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DMUL_ERR_CUDA;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_ctx_current) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return DMUL_ERR_CUDA;
        g_ctx_current = (CUresult(*)(CUcontext *))fn;
    }
    // the runtime makes the device's primary context current (cudaFree(0) creates it if needed)
    if (cudaFree(nullptr) != cudaSuccess) return DMUL_ERR_CUDA;
    CUcontext cur = nullptr;
    if (g_ctx_current(&cur) != CUDA_SUCCESS || !cur) return DMUL_ERR_CUDA;
    if (!g_addr[dev] || g_owner[dev] != cur) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DMUL_ERR_CUDA;
        g_addr[dev] = p;
        g_owner[dev] = cur;
    }
    *out = (unsigned char *)g_addr[dev];
    return DMUL_OK;
}

// After the scan: a device-side error (the sum does not fit, or a bounded wait expired) turns
// the reported length into 0, which no valid result has.
__global__ void k_noalloc_finish(const uint32_t *status, uint64_t *nz) {
    if (*status) *nz = 0;
}

}  // namespace
}  // namespace dml

extern "C" int dmul_carry_noalloc(const uint32_t *d, size_t L, uint32_t *z, size_t z_cap,
                                  uint64_t *nz, void *stream) {
    using namespace dml;
    if (!d || !z || L == 0) return DMUL_ERR_INVALID;
    if (L > kNoAllocMaxL) return DMUL_ERR_TOO_LARGE;
    if (z_cap < L) return DMUL_ERR_CAPACITY;
    const uintptr_t z0 = (uintptr_t)z, z1 = z0 + L * 4, d0 = (uintptr_t)d, d1 = d0 + L * 12;
    if (z0 < d1 && d0 < z1) return DMUL_ERR_INVALID;
    unsigned char *base;
    int rc = scratch_address(&base);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    uint32_t *status = (uint32_t *)base;
    CarryCtl *ctl = (CarryCtl *)(base + kStatusBytes);
    uint2 *spill = (uint2 *)(base + kStatusBytes + kCtlBytes);
    // the status word and the control block must start at zero; the spills are overwritten
    if (cudaMemsetAsync(base, 0, kStatusBytes + carry_ctl_bytes(L), s) != cudaSuccess) return DMUL_ERR_CUDA;
    if (launch_triples_to_digits(d, L, z, spill, status, s) != cudaSuccess) return DMUL_ERR_CUDA;
    if (launch_carry(z, spill, L, ctl, nz, status, s) != cudaSuccess) return DMUL_ERR_CUDA;
    if (nz) {
        k_noalloc_finish<<<1, 1, 0, s>>>(status, nz);
        if (cudaGetLastError() != cudaSuccess) return DMUL_ERR_CUDA;
    }
    return DMUL_OK;
}
