// common.h -- types shared by the host planner and the CUDA kernels of libdmul.
//
// The library multiplies base-10^9 integers through number-theoretic transforms modulo three
// primes p0 < p1 < p2 < 2^30 of the form c*3*2^n + 1 (Sec. 4.5 of the paper, FindPrimes with
// w = 31, n_min = 23, l = 3).  p < 2^30 keeps every lazily-reduced value below 4p < 2^32 (the
// "p < mu/4" variant of Sec. 9 and the unadjusted forms of Sec. 8.3).
#pragma once
#include <stdint.h>

namespace dml {

constexpr int kPrimes = 3;
constexpr uint32_t kBase = 1000000000u;  // B = 10^9
constexpr int kMaxStages = 8;
constexpr int kTile = 32;        // columns per column-pass CTA (one warp-row of 32 words)
constexpr int kChunk = 32;       // coefficients per carry chunk (one warp-row)
constexpr int kCarryLimbs = 2048;  // limbs per carry-scan CTA (256 threads x 8)
constexpr uint32_t kMaxN1 = 1536;  // longest column (tile of kMaxN1 x 32 words in shared memory)
constexpr uint32_t kMaxN2 = 8192;  // longest row (two rows of kMaxN2 words in shared memory)

// Per-prime constants, one copy in __constant__ memory per kernel translation unit.
struct PrimeConst {
    uint32_t p, p2, negp, pinv;  // p, 2p, 2^32 - p, p^-1 mod 2^32
    uint32_t w16[2][16];         // [dir][e] = xi_16^(+-e): dir 0 forward, 1 inverse
    uint32_t w16s[2][16];        // Shoup companions floor(w 2^32 / p)
    uint32_t w3[2], w3s[2];      // xi_3^(+-1) and companions
    // radix 5, w = xi_5^(+-1): [dir][0] = -1/4, [1] = (w + w^4 - w^2 - w^3) / 4,
    // [2] = (w - w^4) / 2, [3] = (w^2 - w^3) / 2 (mod p), and companions
    uint32_t w5[2][4], w5s[2][4];
};

// Constants of the three-prime Garner CRT (Sec. 8.2.2 extended to l = 3) and of the base-10^9
// digit split of the recovered coefficient.
struct CrtConst {
    uint32_t inv01, inv01s;    // p0^-1 mod p1 (and Shoup companion w.r.t. p1)
    uint32_t p0m2, p0m2s;      // p0 mod p2
    uint32_t inv012, inv012s;  // (p0 p1)^-1 mod p2
    uint32_t A0, A1;           // p0 p1 = A0 + A1 * 10^9
};

struct Stage {
    uint32_t R;       // radix of this stage (2, 3, 4, 8 or 16)
    uint32_t m;       // length of the sub-transforms this stage splits
    uint32_t tw;      // offset (in uint2 entries) of the forward inter-stage twiddle table
    uint32_t twi;     // offset of the inverse table (both unused when m == R)
};

// A transform plan for one length N = N1 * N2 (Sec. 7.1): columns of length N1, rows of length
// N2, each transformed by the listed radix stages; everything a kernel needs, passed by value.
struct PlanDev {
    uint64_t N;
    uint32_t N1, N2;
    int ncs, nrs;
    Stage cs[kMaxStages];   // column stages, first to last
    Stage rs[kMaxStages];   // row stages
    uint32_t col_threads, row_threads;  // CTA sizes of the column and row passes (autotuned)
    uint32_t row_tma;                   // 1: persistent TMA-fed row pass with row_grid CTAs/prime
    uint32_t row_grid;
    uint32_t col_half;                  // 1: column passes on N1 x 16 half tiles (colpass.cu)
    uint32_t row_rows;                  // rows per CTA of the specialized row pass (set per launch; 0: 1)
    // Per-prime hand-off from the forward column pass to the row pass (null: the row pass waits
    // for the whole column grid instead).  Column CTAs add their column count to fsync[prime] when
    // done; the row pass of a prime starts once fsync[prime] reaches ftarget (a running total).
    uint32_t *fsync;
    uint32_t ftarget;
    uint32_t spin;                      // bound of the device-side waits (polls); 0: the defaults
    uint64_t offA, offQ, offAi, offQi;  // four-step twiddle tables (uint2 offsets)
    const uint2 *tw[kPrimes];           // per-prime table buffers (device)
    // bytes of the contiguous tables at tw[0] that the forward column pass prefetches into L2
    // (a multiple of 16; 0: none)
    uint64_t tw_bytes;
};


// Whole-product-in-shared-memory plan for small lengths: one transform of length N (no
// four-step split) per prime.
constexpr uint32_t kSmallMaxN = 24576;  // 2 x 96 KB residues + spills in one CTA
constexpr uint32_t kSmallMinN = 64;
struct SmallPlanDev {
    uint32_t N;
    int ns;
    Stage st[kMaxStages];
    const uint2 *tw[kPrimes];
    uint32_t scale[kPrimes], scales[kPrimes];  // 2^32 N^-1 mod p and its Shoup companion
};

}  // namespace dml
