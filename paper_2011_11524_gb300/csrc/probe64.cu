// probe64.cu -- the row pass with two 62-bit primes, for measuring the prime width on the GPU.
//
// The paper's CPU design uses two 64-bit primes (Sec. 4.2: l = 2, w = 64) with Montgomery
// multiplication (Sec. 4.4.3).  The library uses three primes below 2^30 instead; this file holds
// the alternative, so that the choice rests on a measurement: the fused row pass of the four-step
// form (forward row DFTs of X and Y, pointwise Montgomery product, inverse row DFTs, Sec. 5.4 / 6 /
// 7.1) for rows of 4096 residues modulo two primes p < 2^62 of the form c 3 2^n + 1 (FindPrimes with
// w = 63, n_min = 23, l = 2, Sec. 4.5), in 64-bit words:
//  * products by a constant use Shoup's method with w' = floor(w 2^64 / p): q = hi64(a w'),
//    r = a w - q p in [0, 2p) for any 64-bit a;
//  * the pointwise product uses subtractive Montgomery with R = 2^64: r = hi(ab) - hi(m p) + p in
//    (0, 2p) for a, b < 2p (4p < 2^64);
//  * sums stay in [0, 2p) by min(s, s - 2p).
// The layout, stage order, radix-16 network and the untwiddle-then-DFT inverse are those of the
// 32-bit row pass (rowpass.cuh), so the two differ only in word size and prime count.  The parity
// entry point finishes each row with the scale n^-1 R mod p, which turns it into the cyclic
// convolution of the two rows (the convolution theorem, Sec. 3.3); the timed form leaves it out,
// as the 32-bit row pass does (its scale sits in the column pass).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "../../include/dmul.h"
#include "ctx.h"
#include "kernels.cuh"
#include "plan.h"

namespace dml {
namespace {

constexpr int kP64 = 2;
constexpr uint32_t kRow64 = 4096;

struct Prime64 {
    uint64_t p, p2, pinv;         // p, 2p, p^-1 mod 2^64
    uint64_t w16[2][16], w16s[2][16];  // xi_16^(+-e) and Shoup companions
    uint64_t scale, scales;       // n^-1 2^64 mod p (the parity form's final scale)
};
__constant__ Prime64 c_p64[kP64];

// Per prime: stage tables {w, w'} for stages 0 and 1 of the radix-16 schedule (15 x 256 and
// 15 x 16 entries), forward then inverse.
struct Tables64 {
    const ulonglong2 *tw[kP64];
};
constexpr uint32_t kT0 = 15 * 256, kT1 = 15 * 16, kTabEntries = 2 * (kT0 + kT1);

__device__ __forceinline__ uint64_t red2p64(uint64_t a, uint64_t p2) { return a < a - p2 ? a : a - p2; }
__device__ __forceinline__ uint64_t shoup64(uint64_t a, uint64_t w, uint64_t ws, uint64_t p) {
    const uint64_t q = __umul64hi(a, ws);
    return a * w - q * p;
}
__device__ __forceinline__ uint64_t mont64(uint64_t a, uint64_t b, uint64_t p, uint64_t pinv) {
    const uint64_t lo = a * b, hi = __umul64hi(a, b);
    const uint64_t m = lo * pinv;
    return hi - __umul64hi(m, p) + p;
}

// The radix-16 DIF network of Sec. 5.3 without its final bit reversal (Sec. 5.4): output k ends in
// v[brev4(k)].  LAZY: the last level leaves every output but slot 0 unreduced in [0, 4p) for a
// twiddle product that follows.
template <int PI, int DIR, bool LAZY>
__device__ __forceinline__ void dft16_64(uint64_t (&v)[16]) {
    const uint64_t p = c_p64[PI].p, p2 = c_p64[PI].p2;
#pragma unroll
    for (int H = 8; H >= 1; H >>= 1) {
#pragma unroll
        for (int S = 0; S < 16; S += 2 * H) {
#pragma unroll
            for (int J = 0; J < H; ++J) {
                const int e = J * (8 / H);
                const bool last = H == 1;
                uint64_t x = v[S + J], y = v[S + J + H];
                uint64_t s = x + y, d = x - y + p2;
                if (!(last && LAZY && S + J != 0)) s = red2p64(s, p2);
                if (e == 0) {
                    if (!(last && LAZY)) d = red2p64(d, p2);
                } else {
                    d = shoup64(d, c_p64[PI].w16[DIR][e], c_p64[PI].w16s[DIR][e], p);
                }
                v[S + J] = s;
                v[S + J + H] = d;
            }
        }
    }
}
__device__ __forceinline__ constexpr int brev4(int k) {
    return ((k & 1) << 3) | ((k & 2) << 1) | ((k & 4) >> 1) | ((k & 8) >> 3);
}
__device__ __forceinline__ uint32_t pidx64(uint32_t a) { return a + (a >> 4); }

// forward stage t (0: m = 4096, stride 256, from global; 1: m = 256, stride 16), X and Y together
template <int PI, uint32_t M>
__device__ __forceinline__ void fwd64(const ulonglong2 *tw, uint64_t *sx, uint64_t *sy, const uint64_t *gx,
                                      const uint64_t *gy) {
    constexpr uint32_t stride = M / 16, pstride = stride + stride / 16;
    const uint64_t p = c_p64[PI].p;
    for (uint32_t g = threadIdx.x; g < kRow64 / 16; g += blockDim.x) {
        const uint32_t blk = g / stride, j = g % stride, base = blk * M + j;
        uint64_t *px = sx + pidx64(base), *py = sy + pidx64(base);
        uint64_t v[16], u[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            v[k] = gx ? gx[base + k * stride] : px[k * pstride];
            u[k] = gy ? gy[base + k * stride] : py[k * pstride];
        }
        dft16_64<PI, 0, true>(v);
        dft16_64<PI, 0, true>(u);
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            uint64_t o = v[brev4(k)], o2 = u[brev4(k)];
            if (k > 0) {
                const ulonglong2 w = tw[(k - 1) * stride + j];
                o = shoup64(o, w.x, w.y, p);
                o2 = shoup64(o2, w.x, w.y, p);
            }
            px[k * pstride] = o;
            py[k * pstride] = o2;
        }
    }
}

// inverse stage: untwiddle, inverse DFT, natural order; gout (stage 0) writes the row
template <int PI, uint32_t M, bool SCALE>
__device__ __forceinline__ void inv64(const ulonglong2 *tw, uint64_t *sx, uint64_t *gout) {
    constexpr uint32_t stride = M / 16, pstride = stride + stride / 16;
    const uint64_t p = c_p64[PI].p, p2 = c_p64[PI].p2;
    for (uint32_t g = threadIdx.x; g < kRow64 / 16; g += blockDim.x) {
        const uint32_t blk = g / stride, j = g % stride, base = blk * M + j;
        uint64_t *px = sx + pidx64(base);
        uint64_t v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = px[k * pstride];
        v[0] = red2p64(v[0], p2);
#pragma unroll
        for (int k = 1; k < 16; ++k) {
            const ulonglong2 w = tw[(k - 1) * stride + j];
            v[k] = shoup64(v[k], w.x, w.y, p);
        }
        dft16_64<PI, 1, false>(v);
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            uint64_t o = v[brev4(u)];
            if (gout) {
                if (SCALE) {
                    o = shoup64(o, c_p64[PI].scale, c_p64[PI].scales, p);
                    o = red2p64(o, p2);
                    o = o >= p ? o - p : o;
                }
                gout[base + u * stride] = o;
            } else {
                px[u * pstride] = o;
            }
        }
    }
}

template <int PI, bool SCALE>
__device__ __forceinline__ void row64_body(const Tables64 t, uint64_t *sx, uint64_t *sy, uint64_t *xr,
                                           const uint64_t *yr) {
    const ulonglong2 *tw = t.tw[PI];
    const ulonglong2 *f0 = tw, *f1 = tw + kT0, *i0 = tw + kT0 + kT1, *i1 = tw + 2 * kT0 + kT1;
    const uint64_t p = c_p64[PI].p, pinv = c_p64[PI].pinv;
    fwd64<PI, 4096>(f0, sx, sy, xr, yr);
    __syncthreads();
    fwd64<PI, 256>(f1, sx, sy, nullptr, nullptr);
    __syncthreads();
    // the center: last forward stage of both, pointwise product, first inverse stage
    for (uint32_t b = threadIdx.x; b < kRow64 / 16; b += blockDim.x) {
        uint64_t v[16], u[16], z[16];
        uint64_t *bx = sx + 17 * b, *by = sy + 17 * b;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            v[k] = bx[k];
            u[k] = by[k];
        }
        dft16_64<PI, 0, false>(v);
        dft16_64<PI, 0, false>(u);
#pragma unroll
        for (int k = 0; k < 16; ++k) z[k] = mont64(v[brev4(k)], u[brev4(k)], p, pinv);
        dft16_64<PI, 1, false>(z);
#pragma unroll
        for (int k = 0; k < 16; ++k) bx[k] = z[brev4(k)];
    }
    __syncthreads();
    inv64<PI, 256, SCALE>(i1, sx, nullptr);
    __syncthreads();
    inv64<PI, 4096, SCALE>(i0, sx, xr);
}

// one CTA per (row, prime); X, Y: [2][rows][4096] residues in [0, 2p); the result replaces X
template <bool SCALE>
__global__ void __launch_bounds__(256) k_row64(const Tables64 t, uint64_t *X, const uint64_t *Y, uint32_t rows) {
    extern __shared__ uint64_t sm64[];
    const uint32_t row = blockIdx.x, pi = blockIdx.y;
    constexpr uint32_t NP = kRow64 + kRow64 / 16;
    uint64_t *xr = X + ((uint64_t)pi * rows + row) * kRow64;
    const uint64_t *yr = Y + ((uint64_t)pi * rows + row) * kRow64;
    if (pi == 0) row64_body<0, SCALE>(t, sm64, sm64 + NP, xr, yr);
    else row64_body<1, SCALE>(t, sm64, sm64 + NP, xr, yr);
}

typedef unsigned __int128 u128;

// Miller-Rabin with the first twelve primes as bases (deterministic below 3.3e24), Sec. 4.5.
bool is_prime64(uint64_t n) {
    static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t b : bases)
        if (n % b == 0) return n == b;
    uint64_t d = n - 1;
    int s = 0;
    while (!(d & 1)) {
        d >>= 1;
        ++s;
    }
    for (uint64_t b : bases) {
        uint64_t x = powmod64(b, d, n);
        if (x == 1 || x == n - 1) continue;
        bool comp = true;
        for (int r = 1; r < s && comp; ++r) {
            x = mulmod64(x, x, n);
            if (x == n - 1) comp = false;
        }
        if (comp) return false;
    }
    return true;
}

// FindPrimes(63, 23, 2) of Sec. 4.5 (primes psi 2^n + 1 < 2^62 with psi an odd multiple of 3 and
// n >= 23; for each n the largest few, then the two largest overall), ascending.
std::vector<uint64_t> find_primes64() {
    std::vector<uint64_t> r;
    const uint64_t pmax = (1ull << 62) - 1;
    for (int n = 23; n <= 61; ++n) {
        uint64_t psi = (pmax - 1) >> n;
        if (psi % 2 == 0) psi = psi ? psi - 1 : 0;
        while (psi > 0 && psi % 3 != 0) psi = psi >= 2 ? psi - 2 : 0;
        for (int found = 0; psi > 0 && found < kP64;) {
            const uint64_t p = (psi << n) + 1;
            if (is_prime64(p)) {
                if (std::find(r.begin(), r.end(), p) == r.end()) r.push_back(p);
                ++found;
            }
            if (psi <= 6) break;
            psi -= 6;
        }
    }
    std::sort(r.begin(), r.end(), [](uint64_t a, uint64_t b) { return a > b; });
    if (r.size() > (size_t)kP64) r.resize(kP64);
    std::sort(r.begin(), r.end());
    return r;
}

uint64_t gen64(uint64_t p) {
    uint64_t n = p - 1, f[64];
    int nf = 0;
    for (uint64_t q = 2; q * q <= n; ++q)
        if (n % q == 0) {
            f[nf++] = q;
            while (n % q == 0) n /= q;
        }
    if (n > 1) f[nf++] = n;
    for (uint64_t g = 2;; ++g) {
        bool ok = true;
        for (int i = 0; i < nf && ok; ++i) ok = powmod64(g, (p - 1) / f[i], p) != 1;
        if (ok) return g;
    }
}
uint64_t comp64(uint64_t w, uint64_t p) { return (uint64_t)(((u128)w << 64) / p); }

struct Setup64 {
    bool ok = false;
    uint64_t primes[kP64] = {};
    std::vector<ulonglong2> tab[kP64];
};

// The two primes (ascending) and, per prime, the constants (uploaded) and the stage tables.
const Setup64 &setup64() {
    static Setup64 s;
    static bool done = false;
    if (done) return s;
    done = true;
    std::vector<uint64_t> pr = find_primes64();
    if (pr.size() != kP64) return s;
    Prime64 pc[kP64];
    for (int i = 0; i < kP64; ++i) {
        const uint64_t p = pr[i];
        s.primes[i] = p;
        const uint64_t g = gen64(p);
        const uint64_t w4096 = powmod64(g, (p - 1) / kRow64, p), w4096i = powmod64(w4096, p - 2, p);
        Prime64 &c = pc[i];
        c.p = p;
        c.p2 = 2 * p;
        uint64_t inv = 1;  // Newton's iteration for p^-1 mod 2^64
        for (int k = 0; k < 7; ++k) inv *= 2 - p * inv;
        c.pinv = inv;
        const uint64_t w16 = powmod64(w4096, kRow64 / 16, p), w16i = powmod64(w16, p - 2, p);
        for (int e = 0; e < 16; ++e) {
            c.w16[0][e] = powmod64(w16, e, p);
            c.w16[1][e] = powmod64(w16i, e, p);
            c.w16s[0][e] = comp64(c.w16[0][e], p);
            c.w16s[1][e] = comp64(c.w16[1][e], p);
        }
        // n^-1 R mod p with R = 2^64: undoes the Montgomery factor R^-1 and the n of the inverse
        const uint64_t R = (uint64_t)(((u128)1 << 64) % p);
        c.scale = mulmod64(R, powmod64(kRow64 % p, p - 2, p), p);
        c.scales = comp64(c.scale, p);
        // stage tables: stage 0 xi_4096^(j k) (j < 256), stage 1 xi_256^(j k) (j < 16), k = 1..15
        auto &t = s.tab[i];
        for (int dir = 0; dir < 2; ++dir) {
            const uint64_t root = dir ? w4096i : w4096;
            for (uint32_t m : {4096u, 256u}) {
                const uint64_t xm = powmod64(root, kRow64 / m, p);
                const uint32_t stride = m / 16;
                for (uint32_t k = 1; k < 16; ++k)
                    for (uint32_t j = 0; j < stride; ++j) {
                        const uint64_t w = powmod64(xm, (uint64_t)j * k, p);
                        t.push_back(make_ulonglong2(w, comp64(w, p)));
                    }
            }
        }
    }
    if (cudaMemcpyToSymbol(c_p64, pc, sizeof(pc)) != cudaSuccess) return s;
    s.ok = true;
    return s;
}

struct Dev64 {
    void *tabs = nullptr;
    Tables64 t{};
};

int upload_tables(dmul_ctx *c, const Setup64 &s, Dev64 *d) {
    const size_t per = (size_t)kTabEntries * sizeof(ulonglong2);
    int rc = dev_alloc(c, &d->tabs, kP64 * per);
    if (rc) return rc;
    for (int i = 0; i < kP64; ++i) {
        ulonglong2 *dst = (ulonglong2 *)((char *)d->tabs + i * per);
        if (cudaMemcpy(dst, s.tab[i].data(), per, cudaMemcpyHostToDevice) != cudaSuccess) return DMUL_ERR_CUDA;
        d->t.tw[i] = dst;
    }
    return DMUL_OK;
}

constexpr size_t kSmem64 = 2 * (kRow64 + kRow64 / 16) * sizeof(uint64_t);

cudaError_t launch_row64(const Tables64 &t, uint64_t *X, const uint64_t *Y, uint32_t rows, bool scale,
                         cudaStream_t s) {
    static bool attrs = false;
    if (!attrs) {
        cudaError_t e = cudaFuncSetAttribute(k_row64<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem64);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_row64<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem64);
        if (e != cudaSuccess) return e;
        attrs = true;
    }
    dim3 grid(rows, kP64);
    if (scale) k_row64<true><<<grid, 256, kSmem64, s>>>(t, X, Y, rows);
    else k_row64<false><<<grid, 256, kSmem64, s>>>(t, X, Y, rows);
    return cudaGetLastError();
}

}  // namespace
}  // namespace dml

using namespace dml;

extern "C" {

int dmul_probe64_primes(uint64_t out[2]) {
    if (!out) return DMUL_ERR_INVALID;
    std::vector<uint64_t> pr = find_primes64();
    if (pr.size() != 2) return DMUL_ERR_INVALID;
    out[0] = pr[0];
    out[1] = pr[1];
    return DMUL_OK;
}

int dmul_probe64_conv(dmul_ctx *c, const uint64_t *a, const uint64_t *b, uint64_t *out, size_t rows, void *stream) {
    if (!c || !a || !b || !out || rows == 0 || rows > 65535) return DMUL_ERR_INVALID;
    int rc = set_device(c);
    if (rc) return rc;
    const Setup64 &s = setup64();
    if (!s.ok) return DMUL_ERR_CUDA;
    Dev64 d;
    if ((rc = upload_tables(c, s, &d))) {
        dev_free(c, d.tabs, d.tabs ? kP64 * (size_t)kTabEntries * sizeof(ulonglong2) : 0);
        return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const size_t bytes = (size_t)kP64 * rows * kRow64 * sizeof(uint64_t);
    cudaError_t e = cudaMemcpyAsync(out, a, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = launch_row64(d.t, out, b, (uint32_t)rows, true, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    dev_free(c, d.tabs, kP64 * (size_t)kTabEntries * sizeof(ulonglong2));
    return e == cudaSuccess ? DMUL_OK : DMUL_ERR_CUDA;
}

int dmul_probe_prime_width(dmul_ctx *c, uint64_t N, double *ms_two_62bit, double *ms_three_30bit) {
    if (!c || !ms_two_62bit || !ms_three_30bit || N < kRow64 || N % kRow64 || N > (1ull << 23))
        return DMUL_ERR_INVALID;
    int rc = set_device(c);
    if (rc) return rc;
    const Setup64 &s = setup64();
    if (!s.ok) return DMUL_ERR_CUDA;
    PlanEntry *pe;
    if ((rc = get_plan(c, N, &pe))) return rc;
    if ((rc = ensure_scratch(c, N, N, true))) return rc;
    Dev64 d;
    uint64_t *X64 = nullptr, *Y64 = nullptr;
    const size_t b64 = (size_t)kP64 * N * sizeof(uint64_t);
    if (!(rc = upload_tables(c, s, &d))) rc = dev_alloc(c, (void **)&X64, b64);
    if (!rc) rc = dev_alloc(c, (void **)&Y64, b64);
    cudaStream_t st = c->own_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<float> t64, t32;
    uint32_t saved_status = 0;  // an error of earlier work stays for the next dmul_sync
    if (!rc && (cudaDeviceSynchronize() != cudaSuccess ||
                cudaMemcpy(&saved_status, c->status, 4, cudaMemcpyDeviceToHost) != cudaSuccess))
        rc = DMUL_ERR_CUDA;
    if (!rc) {
        // operands: valid residues of every prime (0x11 bytes: 0x1111... < 2 p for all five primes)
        cudaMemsetAsync(X64, 0x11, b64, st);
        cudaMemsetAsync(Y64, 0x11, b64, st);
        cudaMemsetAsync(c->X, 0x11, (size_t)kPrimes * N * 4, st);
        cudaMemsetAsync(c->Y, 0x11, (size_t)kPrimes * N * 4, st);
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        PlanDev pd = pe->pd;
        pd.fsync = nullptr;
        for (int it = 0; it < 12; ++it) {
            float ms = 0;
            cudaEventRecord(e0, st);
            launch_row64(d.t, X64, Y64, (uint32_t)(N / kRow64), false, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            if (it >= 2) t64.push_back(ms);
            cudaEventRecord(e0, st);
            launch_row_any(pd, c->X, c->Y, false, c->status, st);
            cudaEventRecord(e1, st);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&ms, e0, e1);
            if (it >= 2) t32.push_back(ms);
        }
        if (cudaGetLastError() != cudaSuccess) rc = DMUL_ERR_CUDA;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaStreamSynchronize(st);
        // whatever status the timing runs set is not the caller's
        cudaMemcpy(c->status, &saved_status, 4, cudaMemcpyHostToDevice);
    }
    dev_free(c, X64, X64 ? b64 : 0);
    dev_free(c, Y64, Y64 ? b64 : 0);
    dev_free(c, d.tabs, d.tabs ? kP64 * (size_t)kTabEntries * sizeof(ulonglong2) : 0);
    if (rc) return rc;
    std::sort(t64.begin(), t64.end());
    std::sort(t32.begin(), t32.end());
    *ms_two_62bit = t64[t64.size() / 2];
    *ms_three_30bit = t32[t32.size() / 2];
    return DMUL_OK;
}

}  // extern "C"
