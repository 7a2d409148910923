// modarith.cuh -- 32-bit field arithmetic mod p < 2^30 and the in-register radix-R DFTs.
//
// Representation: every value that travels between stages is an "unadjusted" residue in
// [0, 2p) (Sec. 8.3); p < 2^30 makes 4p < 2^32, so sums and differences of two such values fit a
// word without overflow checks (the p < mu/4 variant suggested in Sec. 9).
//
//  * Products by a known constant w (twiddles, DFT roots, CRT constants) use Shoup's method with
//    the precomputed companion w' = floor(w 2^32 / p): q = hi(a w'), r = a w - q p lies in
//    [0, 2p) for every 32-bit a.  Three multiplies on the IMAD pipe, no correction.
//  * Products of two variable values (the pointwise product of the convolution theorem, Sec. 3.3)
//    use Montgomery reduction (Sec. 4.4.3) in its subtractive form:  m = lo(ab) p^-1 mod 2^32,
//    r = hi(ab) - hi(m p) + p lies in (0, 2p) and equals ab 2^-32 mod p; valid for ab < p 2^32,
//    i.e. both inputs < 2p.  The factor 2^-32 it leaves behind is removed once, inside the
//    inverse transform's final scale (the linearity trick of Sec. 6).
//  * Additions and subtractions are branch-free (Sec. 8.1): the unsigned min(a, a - 2p) maps
//    [0, 4p) onto [0, 2p).
#pragma once
#include <stdint.h>
#include "common.h"

namespace dml {

// One copy of the constants per translation unit (no relocatable device code); every .cu file that
// includes this header uploads its copy through its own upload function (kernels.cuh).
static __constant__ PrimeConst c_prime[kPrimes];
static __constant__ CrtConst c_crt;

#define DMUL_DEFINE_UPLOAD(NAME)                                                             \
    cudaError_t NAME(const PrimeConst pc[kPrimes], const CrtConst &crt) {                   \
        cudaError_t e = cudaMemcpyToSymbol(c_prime, pc, sizeof(PrimeConst) * kPrimes);       \
        if (e != cudaSuccess) return e;                                                      \
        return cudaMemcpyToSymbol(c_crt, &crt, sizeof(CrtConst));                           \
    }

__device__ __forceinline__ uint32_t umin32(uint32_t a, uint32_t b) { return a < b ? a : b; }

// Programmatic dependent launch: a kernel launched with programmatic stream serialization may
// start while its predecessor in the stream drains; pdl_wait() blocks until that predecessor has
// completed and its memory is visible (a no-op without the launch attribute), pdl_trigger() lets
// the successor launch once every CTA of this grid has issued it.  Every pipeline kernel calls
// pdl_trigger() first and pdl_wait() before its first global access.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// [0, 4p) -> [0, 2p)
template <int PI>
__device__ __forceinline__ uint32_t red2p(uint32_t a) { return umin32(a, a - c_prime[PI].p2); }

// [0, 2p) -> [0, p)
template <int PI>
__device__ __forceinline__ uint32_t red1p(uint32_t a) { return umin32(a, a - c_prime[PI].p); }

// a * w mod p in [0, 2p) for any 32-bit a; w < p with companion ws.
template <int PI>
__device__ __forceinline__ uint32_t shoup(uint32_t a, uint32_t w, uint32_t ws) {
    uint32_t q = __umulhi(a, ws);
    return a * w + q * c_prime[PI].negp;
}

// a * b * 2^-32 mod p in (0, 2p) for a, b in [0, 2p).
template <int PI>
__device__ __forceinline__ uint32_t mont(uint32_t a, uint32_t b) {
    uint32_t lo = a * b;
    uint32_t hi = __umulhi(a, b);
    uint32_t m = lo * c_prime[PI].pinv;
    uint32_t t = __umulhi(m, c_prime[PI].p);
    return hi - t + c_prime[PI].p;
}

// The signed Montgomery product of the Prospects (Sec. 9) on the same unadjusted inputs: centred
// a - p, b - p in [-p, p), m = lo((a-p)(b-p)) p^-1 mod 2^32 as a signed word, and
// r = hi((a-p)(b-p)) - hi(m p) (signed high halves) lies in (-3p/4, 3p/4): |(a-p)(b-p)| <= p^2
// < p 2^30 puts the first high half within p/4 of 0 and |m p| < p 2^31 the second within p/2.
// So r + p is in (0, 2p) with no correction, congruent to ab 2^-32 mod p, as mont() returns.  It
// costs the two centring subtractions on top of mont()'s instructions, which is why the row pass
// keeps mont() (the measured comparison builds with -DDMUL_POINTWISE_SIGNED).
template <int PI>
__device__ __forceinline__ uint32_t mont_signed(uint32_t a, uint32_t b) {
    const int32_t p = (int32_t)c_prime[PI].p;
    const int32_t sa = (int32_t)a - p, sb = (int32_t)b - p;
    const int64_t t = (int64_t)sa * sb;
    const int32_t m = (int32_t)((uint32_t)t * c_prime[PI].pinv);
    const int32_t hm = __mulhi(m, p);
    return (uint32_t)((int32_t)(t >> 32) - hm + p);
}

// The pointwise product of the row pass: mont(), or mont_signed() in the comparison build.
template <int PI>
__device__ __forceinline__ uint32_t pointwise(uint32_t a, uint32_t b) {
#ifdef DMUL_POINTWISE_SIGNED
    return mont_signed<PI>(a, b);
#else
    return mont<PI>(a, b);
#endif
}

// Gentleman-Sande (DIF) butterfly of Sec. 5.3 on unadjusted values: x' = x + y,
// y' = (x - y) * xi_16^e.  e == 0 is the factor-1 butterfly of Sec. 5.6 (no multiply).
// RS / RD = false leave the sum / the factor-1 difference in [0, 4p) unreduced: allowed only
// where that output goes straight into a Shoup product (which takes any 32-bit input).
template <int PI, int DIR, int E, bool RS = true, bool RD = true>
__device__ __forceinline__ void bfly(uint32_t &x, uint32_t &y) {
    uint32_t s = RS ? red2p<PI>(x + y) : x + y;
    uint32_t d = x - y + c_prime[PI].p2;
    if constexpr (E == 0) {
        if constexpr (RD) d = red2p<PI>(d);
    } else {
        d = shoup<PI>(d, c_prime[PI].w16[DIR][E], c_prime[PI].w16s[DIR][E]);
    }
    x = s;
    y = d;
}

__host__ __device__ constexpr int brev(int v, int bits) {
    int r = 0;
    for (int i = 0; i < bits; ++i) r |= ((v >> i) & 1) << (bits - 1 - i);
    return r;
}
__host__ __device__ constexpr int ilog2c(int v) { return v <= 1 ? 0 : 1 + ilog2c(v >> 1); }

// Position of output k of an R-point DFT computed by dft<>: brev(k) for R = 2^a, k for R = 3, 5.
template <int R>
__device__ __forceinline__ constexpr int outpos(int k) {
    if constexpr (R == 3 || R == 5) return k; else return brev(k, ilog2c(R));
}

// LAZY (last level only): 0 every output reduced to [0, 2p); 1 only output k = 0 (slot 0)
// reduced, the others left in [0, 4p) for a following twiddle product; 2 no output reduced.
template <int PI, int DIR, int R, int H, int S, int J, int LAZY>
__device__ __forceinline__ void dft_level_j(uint32_t (&v)[R]) {
    if constexpr (J < H) {
        constexpr bool last = (H == 1);
        constexpr bool rs = !last || LAZY == 0 || (LAZY == 1 && S + J == 0);
        constexpr bool rd = !last || LAZY == 0;
        bfly<PI, DIR, J * (8 / H), rs, rd>(v[S + J], v[S + J + H]);
        dft_level_j<PI, DIR, R, H, S, J + 1, LAZY>(v);
    }
}
template <int PI, int DIR, int R, int H, int S, int LAZY>
__device__ __forceinline__ void dft_level_s(uint32_t (&v)[R]) {
    if constexpr (S < R) {
        dft_level_j<PI, DIR, R, H, S, 0, LAZY>(v);
        dft_level_s<PI, DIR, R, H, S + 2 * H, LAZY>(v);
    }
}
template <int PI, int DIR, int R, int H, int LAZY>
__device__ __forceinline__ void dft_levels(uint32_t (&v)[R]) {
    if constexpr (H >= 1) {
        dft_level_s<PI, DIR, R, H, 0, LAZY>(v);
        dft_levels<PI, DIR, R, H / 2, LAZY>(v);
    }
}

// In-register R-point DFT (DIR 0: root xi_R, DIR 1: xi_R^-1), no scaling.  Input in natural
// order v[0..R); output k is left in v[outpos<R>(k)].  For R = 2^a this is the radix-2 DIF
// network of Sec. 5.3 without its final bit reversal (Sec. 5.4); the butterfly at level of half
// size H and offset J uses xi_{2H}^J = xi_16^(J * 8 / H).  Outputs are in [0, 2p), except with
// LAZY (R = 2^a only; see dft_level_j) where the caller multiplies them by a twiddle next.
template <int PI, int DIR, int R, int LAZY = 0>
__device__ __forceinline__ void dft(uint32_t (&v)[R]) {
    if constexpr (R == 3) {
        // X0 = a+b+c, X1 = (a-c) + w(b-c), X2 = (a-b) - w(b-c), with w = xi_3^(+-1)
        const uint32_t p2 = c_prime[PI].p2;
        uint32_t a = v[0], b = v[1], c = v[2];
        uint32_t t = shoup<PI>(b - c + p2, c_prime[PI].w3[DIR], c_prime[PI].w3s[DIR]);
        uint32_t x0 = red2p<PI>(red2p<PI>(a + b) + c);
        uint32_t x1 = red2p<PI>(red2p<PI>(a - c + p2) + t);
        uint32_t x2 = red2p<PI>(red2p<PI>(a - b + p2) - t + p2);
        v[0] = x0; v[1] = x1; v[2] = x2;
    } else if constexpr (R == 5) {
        // With w = xi_5^(+-1), s1 = a1 + a4, d1 = a1 - a4, s2 = a2 + a3, d2 = a2 - a3:
        //   X1, X4 = a0 + c1 s1 + c2 s2 +- (e1 d1 + e2 d2)
        //   X2, X3 = a0 + c2 s1 + c1 s2 +- (e2 d1 - e1 d2)
        // where c1 = (w + w^4)/2, c2 = (w^2 + w^3)/2, e1 = (w - w^4)/2, e2 = (w^2 - w^3)/2.  Since
        // c1 + c2 = -1/2, the c-terms are b +- K2 (s1 - s2) with b = a0 - (s1 + s2)/4 and
        // K2 = (c1 - c2)/2: six constant products instead of sixteen.
        const uint32_t p2 = c_prime[PI].p2;
        const uint32_t *k = c_prime[PI].w5[DIR], *ks = c_prime[PI].w5s[DIR];
        const uint32_t a0 = v[0];
        const uint32_t s1 = red2p<PI>(v[1] + v[4]), s2 = red2p<PI>(v[2] + v[3]);
        const uint32_t d1 = v[1] - v[4] + p2, d2 = v[2] - v[3] + p2;  // (0, 4p): Shoup inputs
        const uint32_t t1 = red2p<PI>(s1 + s2);
        const uint32_t b = red2p<PI>(a0 + shoup<PI>(t1, k[0], ks[0]));
        const uint32_t m2 = shoup<PI>(s1 - s2 + p2, k[1], ks[1]);
        const uint32_t P = red2p<PI>(b + m2), Q = red2p<PI>(b - m2 + p2);
        const uint32_t e11 = shoup<PI>(d1, k[2], ks[2]), e22 = shoup<PI>(d2, k[3], ks[3]);
        const uint32_t e21 = shoup<PI>(d1, k[3], ks[3]), e12 = shoup<PI>(d2, k[2], ks[2]);
        const uint32_t E1 = red2p<PI>(e11 + e22), E2 = red2p<PI>(e21 - e12 + p2);
        v[0] = red2p<PI>(a0 + t1);
        v[1] = red2p<PI>(P + E1);
        v[4] = red2p<PI>(P - E1 + p2);
        v[2] = red2p<PI>(Q + E2);
        v[3] = red2p<PI>(Q - E2 + p2);
    } else {
        dft_levels<PI, DIR, R, R / 2, LAZY>(v);
    }
}

}  // namespace dml
