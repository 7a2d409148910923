// plan.h -- host-side number theory and transform planning for libdmul.
#pragma once
#include <stdint.h>
#include <vector>
#include "common.h"

namespace dml {

// Sec. 4.5 FindPrimes(w, n_min, l): the l largest primes c*3*2^n + 1 < 2^(w-1) with n >= n_min and
// c odd, largest first.  Empty when fewer than l exist.
std::vector<uint64_t> find_primes(int w, int n_min, int l);

// eq. lambda (Sec. 4.2) in exact integer arithmetic; -1 on bad arguments.
int lambda_max_digits(int w, int l, int log2M);

// Host modular arithmetic (128-bit products).
uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t p);
uint64_t powmod64(uint64_t a, uint64_t e, uint64_t p);
uint32_t smallest_generator(uint32_t p);

// The library's prime set, ascending (p0 < p1 < p2).
extern const uint32_t kPrimeSet[kPrimes];

// Constants for __constant__ memory.
void make_prime_consts(PrimeConst out[kPrimes]);
void make_crt_consts(CrtConst *out);

// Longest transform the two-pass four-step kernels support: N1 <= 1536 (column tile in shared
// memory), N2 <= 8192 (row in shared memory), N | gcd(p_i - 1).
constexpr uint64_t kMaxN = 3ull << 22;
constexpr uint64_t kMinN = 1024;

// Smallest admissible transform length >= L: N in {2^k, 3*2^k, 5*2^k} (Sec. 4.5 "smooth the
// stairs", and the smoother set suggested in Sec. 9); five = false leaves out 5*2^k.
uint64_t choose_N(uint64_t L, bool five = true);

// Split N = N1 * N2 and the radix schedules.
struct HostPlan {
    uint64_t N;
    uint32_t N1, N2;
    std::vector<uint32_t> col_radix, row_radix;
    uint32_t col_threads = 0, row_threads = 0;  // 0: the default for the split
    uint32_t row_tma = 0, row_grid = 0;         // persistent TMA-fed row pass and its CTAs/prime
    uint32_t col_half = 0;                      // column passes on N1 x 16 half tiles
};
// The column passes can run on N1 x 16 half tiles: N1 one of the specialized lengths with its
// planned schedule (last stage radix 16) and whole 32-column tiles for the six-CTA CRT clusters.
bool col_half_supported(const HostPlan &hp);
// Candidate column lengths N1 for a transform length N (the autotuner's search space).
std::vector<uint32_t> candidate_n1(uint64_t N);
bool make_host_plan(uint64_t N, HostPlan *hp, uint32_t n1_override = 0);

// Six-step form (Sec. 7.9): N = 2^k only, N1 = 2^floor(k/2), N2 = 2^ceil(k/2); both the N1-long
// and the N2-long DFTs run along contiguous rows (N1, N2 <= 8192).
uint64_t choose_N_pow2(uint64_t L);
bool make_host_plan_sixstep(uint64_t N, HostPlan *hp);

// Small lengths (whole product in one CTA per prime): N in {2^k, 3*2^k}, kSmallMinN..kSmallMaxN.
uint64_t choose_N_small(uint64_t L);
std::vector<uint32_t> small_schedule(uint64_t N);
// stage tables of one length-N transform (forward then inverse per stage) + the inverse scale
void build_small_tables(uint64_t N, SmallPlanDev *sp, std::vector<uint32_t> tables[kPrimes]);

// Build the per-prime twiddle tables of a plan (host memory): for each prime, one buffer of
// uint2 {w, w'} entries: stage tables (forward then inverse) for columns and rows, then the
// four-step tables A, Q (forward) and Ai, Qi (inverse, scaled by 2^32 N^-1).  Fills the offsets
// of `pd` (pointers left null).
void build_tables(const HostPlan &hp, PlanDev *pd, std::vector<uint32_t> tables[kPrimes]);

}  // namespace dml
