// plan.cpp -- host-side number theory and transform planning for libdmul.
#include "plan.h"

#include <algorithm>
#include <cstring>

namespace dml {

typedef unsigned __int128 u128;

uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t p) { return (uint64_t)((u128)a * b % p); }

uint64_t powmod64(uint64_t a, uint64_t e, uint64_t p) {
    uint64_t r = 1 % p;
    a %= p;
    for (; e; e >>= 1) {
        if (e & 1) r = mulmod64(r, a, p);
        a = mulmod64(a, a, p);
    }
    return r;
}

// Primality of n < 2^32 by trial division (the primality test FindPrimes needs is left open by
// Sec. 4.5; the library only searches below 2^32).
static bool is_prime_small(uint64_t n) {
    if (n < 2) return false;
    if (n % 2 == 0) return n == 2;
    for (uint64_t d = 3; d * d <= n; d += 2)
        if (n % d == 0) return false;
    return true;
}

// Sec. 4.5 FindPrimesForN: walk psi = (pmax-1) div 2^n down over odd multiples of 3.
static void find_primes_for_n(int n, uint64_t pmax, int l, std::vector<uint64_t> &r) {
    uint64_t psi = (pmax - 1) >> n;
    if (psi % 2 == 0) {
        if (psi == 0) return;
        psi -= 1;
    }
    while (psi > 0 && psi % 3 != 0) psi = psi >= 2 ? psi - 2 : 0;
    int found = 0;
    while (psi > 0 && found < l) {
        uint64_t p = (psi << n) + 1;
        if (is_prime_small(p)) {
            if (std::find(r.begin(), r.end(), p) == r.end()) r.push_back(p);
            ++found;
        }
        if (psi <= 6) break;
        psi -= 6;
    }
}

std::vector<uint64_t> find_primes(int w, int n_min, int l) {
    std::vector<uint64_t> r;
    if (w < 4 || w > 33 || l < 1 || n_min < 0) return r;
    uint64_t pmax = (1ull << (w - 1)) - 1;
    for (int n = n_min; n <= w - 2; ++n) find_primes_for_n(n, pmax, l, r);
    if ((int)r.size() < l) return {};
    std::sort(r.begin(), r.end(), [](uint64_t a, uint64_t b) { return a > b; });
    r.resize(l);
    return r;
}

// ---- eq. lambda with a few-word unsigned big integer ------------------------------------------
namespace {
struct Big {
    std::vector<uint32_t> w;  // little-endian 32-bit words
    explicit Big(uint64_t v = 0) {
        while (v) { w.push_back((uint32_t)v); v >>= 32; }
    }
    void trim() { while (!w.empty() && w.back() == 0) w.pop_back(); }
};
Big mul(const Big &a, const Big &b) {
    Big r;
    r.w.assign(a.w.size() + b.w.size() + 1, 0);
    for (size_t i = 0; i < a.w.size(); ++i) {
        uint64_t carry = 0;
        for (size_t j = 0; j < b.w.size(); ++j) {
            uint64_t t = (uint64_t)a.w[i] * b.w[j] + r.w[i + j] + carry;
            r.w[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
        size_t k = i + b.w.size();
        while (carry) {
            uint64_t t = (uint64_t)r.w[k] + carry;
            r.w[k++] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    r.trim();
    return r;
}
Big pow2(int e) {
    Big r;
    r.w.assign(e / 32 + 1, 0);
    r.w[e / 32] = 1u << (e % 32);
    return r;
}
Big sub1(Big a) {  // a - 1, a >= 1
    for (auto &x : a.w) {
        if (x) { --x; break; }
        x = 0xffffffffu;
    }
    a.trim();
    return a;
}
int cmp(const Big &a, const Big &b) {
    if (a.w.size() != b.w.size()) return a.w.size() < b.w.size() ? -1 : 1;
    for (size_t i = a.w.size(); i-- > 0;)
        if (a.w[i] != b.w[i]) return a.w[i] < b.w[i] ? -1 : 1;
    return 0;
}
}  // namespace

int lambda_max_digits(int w, int l, int log2M) {
    if (w < 2 || w > 128 || l < 1 || l > 16 || log2M < 0 || log2M > 256) return -1;
    // largest n with (10^n - 1)^2 * 2^log2M < 2^((w-1) l)
    Big lim = pow2((w - 1) * l);
    Big pm = pow2(log2M);
    int best = -1;
    Big ten_n(1);  // 10^n
    for (int n = 0; n < 200; ++n) {
        Big t = sub1(ten_n);
        Big lhs = mul(mul(t, t), pm);
        if (cmp(lhs, lim) < 0) best = n; else break;
        ten_n = mul(ten_n, Big(10));
    }
    return best;
}

// ---- prime constants -----------------------------------------------------------------------------
const uint32_t kPrimeSet[kPrimes] = {377487361u, 754974721u, 880803841u};

uint32_t smallest_generator(uint32_t p) {
    std::vector<uint64_t> f;
    uint64_t r = p - 1;
    for (uint64_t d = 2; d * d <= r; ++d)
        if (r % d == 0) {
            f.push_back(d);
            while (r % d == 0) r /= d;
        }
    if (r > 1) f.push_back(r);
    for (uint32_t g = 2; g < p; ++g) {
        bool ok = true;
        for (uint64_t q : f) ok = ok && powmod64(g, (p - 1) / q, p) != 1;
        if (ok) return g;
    }
    return 0;
}

static uint32_t shoup_companion(uint32_t w, uint32_t p) { return (uint32_t)(((uint64_t)w << 32) / p); }

static uint32_t inv_mod_2_32(uint32_t p) {
    uint32_t x = p;  // correct to 3 bits for odd p
    for (int i = 0; i < 5; ++i) x *= 2u - p * x;
    return x;
}

// Root of unity of order n in F_p from the smallest generator: xi_n = g^((p-1)/n).  All roots the
// library uses come from the same g, so xi_N^(N/m) = xi_m for every m | N.
static uint32_t root_of_unity(uint32_t p, uint64_t n) {
    uint32_t g = smallest_generator(p);
    return (uint32_t)powmod64(g, (p - 1) / n, p);
}

void make_prime_consts(PrimeConst out[kPrimes]) {
    for (int i = 0; i < kPrimes; ++i) {
        uint32_t p = kPrimeSet[i];
        PrimeConst &c = out[i];
        memset(&c, 0, sizeof(c));
        c.p = p;
        c.p2 = 2 * p;
        c.negp = 0u - p;
        c.pinv = inv_mod_2_32(p);
        uint32_t w16 = root_of_unity(p, 16);
        uint32_t w16i = (uint32_t)powmod64(w16, p - 2, p);
        for (int e = 0; e < 16; ++e) {
            c.w16[0][e] = (uint32_t)powmod64(w16, e, p);
            c.w16[1][e] = (uint32_t)powmod64(w16i, e, p);
            c.w16s[0][e] = shoup_companion(c.w16[0][e], p);
            c.w16s[1][e] = shoup_companion(c.w16[1][e], p);
        }
        uint32_t w3 = root_of_unity(p, 3);
        c.w3[0] = w3;
        c.w3[1] = (uint32_t)powmod64(w3, p - 2, p);
        c.w3s[0] = shoup_companion(c.w3[0], p);
        c.w3s[1] = shoup_companion(c.w3[1], p);
        const uint64_t w5 = root_of_unity(p, 5);
        const uint64_t inv2 = (p + 1) / 2, inv4 = mulmod64(inv2, inv2, p);
        for (int dir = 0; dir < 2; ++dir) {
            const uint64_t w = dir ? powmod64(w5, p - 2, p) : w5;
            const uint64_t w2 = mulmod64(w, w, p), w3 = mulmod64(w2, w, p), w4 = mulmod64(w3, w, p);
            uint64_t k[4];
            k[0] = p - inv4;                                           // -1/4
            k[1] = mulmod64((w + w4 + 2 * p - w2 - w3) % p, inv4, p);  // (c1 - c2) / 2
            k[2] = mulmod64((w + p - w4) % p, inv2, p);                // e1
            k[3] = mulmod64((w2 + p - w3) % p, inv2, p);               // e2
            for (int i = 0; i < 4; ++i) {
                c.w5[dir][i] = (uint32_t)k[i];
                c.w5s[dir][i] = shoup_companion((uint32_t)k[i], p);
            }
        }
    }
}

void make_crt_consts(CrtConst *o) {
    const uint64_t p0 = kPrimeSet[0], p1 = kPrimeSet[1], p2 = kPrimeSet[2];
    memset(o, 0, sizeof(*o));
    o->inv01 = (uint32_t)powmod64(p0 % p1, p1 - 2, p1);
    o->inv01s = shoup_companion(o->inv01, (uint32_t)p1);
    o->p0m2 = (uint32_t)(p0 % p2);
    o->p0m2s = shoup_companion(o->p0m2, (uint32_t)p2);
    o->inv012 = (uint32_t)powmod64(mulmod64(p0, p1, p2), p2 - 2, p2);
    o->inv012s = shoup_companion(o->inv012, (uint32_t)p2);
    uint64_t m01 = p0 * p1;
    o->A0 = (uint32_t)(m01 % kBase);
    o->A1 = (uint32_t)(m01 / kBase);
}

// ---- transform lengths and schedules ------------------------------------------------------------
uint64_t choose_N(uint64_t L, bool five) {
    uint64_t best = 0;
    for (uint64_t n = 1; n <= kMaxN; n <<= 1) {
        for (uint64_t cand : {n, 3 * n, five ? 5 * n : n}) {
            if (cand >= L && cand >= kMinN && cand <= kMaxN && (best == 0 || cand < best)) best = cand;
        }
    }
    return best;
}

static std::vector<uint32_t> pow2_schedule(uint32_t n) {
    // n = 2^a, a = 4q + r: [2^r] (when r > 0) followed by q radix-16 stages
    int a = 0;
    while ((1u << a) < n) ++a;
    std::vector<uint32_t> s;
    if (a % 4) s.push_back(1u << (a % 4));
    for (int i = 0; i < a / 4; ++i) s.push_back(16);
    return s;
}

bool make_host_plan(uint64_t N, HostPlan *hp, uint32_t n1_override) {
    if (N < kMinN || N > kMaxN) return false;
    // N = f 2^k with f in {1, 3, 5}: the odd factor is the column pass's first radix
    const uint32_t f = (N % 3 == 0) ? 3u : (N % 5 == 0) ? 5u : 1u;
    uint64_t P = N / f;
    if (P & (P - 1)) return false;
    int k = 0;
    while ((1ull << k) < P) ++k;
    uint64_t N2 = 1ull << ((k + 1) / 2);
    uint64_t N1 = N / N2;
    const uint64_t n1max = f == 3 ? kMaxN1 : f == 5 ? 1280 : 1024;
    while (N1 > n1max) { N1 /= 2; N2 *= 2; }
    while (N2 < (uint64_t)kTile) { N2 *= 2; N1 /= 2; }
    if (n1_override) {
        if (N % n1_override) return false;
        N1 = n1_override;
        N2 = N / N1;
        if (N1 > n1max || N2 < (uint64_t)kTile || (N2 & (N2 - 1))) return false;
    }
    if (N2 > kMaxN2 || N1 < 2) return false;
    hp->N = N;
    hp->N1 = (uint32_t)N1;
    hp->N2 = (uint32_t)N2;
    hp->col_radix.clear();
    if (f > 1) hp->col_radix.push_back(f);
    for (uint32_t r : pow2_schedule((uint32_t)(N1 / f))) hp->col_radix.push_back(r);
    hp->row_radix = pow2_schedule((uint32_t)N2);
    return (int)hp->col_radix.size() <= kMaxStages && (int)hp->row_radix.size() <= kMaxStages;
}

bool col_half_supported(const HostPlan &hp) {
    const uint32_t n1 = hp.N1;
    const bool spec = n1 == 64 || n1 == 80 || n1 == 96 || n1 == 128 || n1 == 160 || n1 == 192 || n1 == 256 ||
                      n1 == 320 || n1 == 384 || n1 == 512 || n1 == 640 || n1 == 768 || n1 == 1024 ||
                      n1 == 1280 || n1 == 1536;
    return spec && hp.N2 % 32 == 0 &&
           !hp.col_radix.empty() && hp.col_radix.back() == 16;
}

std::vector<uint32_t> candidate_n1(uint64_t N) {
    std::vector<uint32_t> out;
    for (uint32_t n1 = 2; n1 <= kMaxN1; n1 *= 2) {
        for (uint32_t cand : {n1, 3 * n1, 5 * n1}) {
            HostPlan hp;
            if (cand <= kMaxN1 && N % cand == 0 && make_host_plan(N, &hp, cand) && hp.N1 == cand &&
                hp.N1 >= 32 && std::find(out.begin(), out.end(), cand) == out.end())
                out.push_back(cand);
        }
    }
    std::sort(out.begin(), out.end());
    return out;
}

uint64_t choose_N_pow2(uint64_t L) {
    for (uint64_t n = kMinN; n <= (1ull << 23); n <<= 1)
        if (n >= L) return n;
    return 0;
}

bool make_host_plan_sixstep(uint64_t N, HostPlan *hp) {
    if (N < kMinN || N > (1ull << 23) || (N & (N - 1))) return false;
    int k = 0;
    while ((1ull << k) < N) ++k;
    hp->N = N;
    hp->N1 = 1u << (k / 2);
    hp->N2 = 1u << ((k + 1) / 2);
    hp->col_radix = pow2_schedule(hp->N1);
    hp->row_radix = pow2_schedule(hp->N2);
    return hp->N2 <= kMaxN2;
}

uint64_t choose_N_small(uint64_t L) {
    uint64_t best = 0;
    for (uint64_t n = 1; n <= kSmallMaxN; n <<= 1)
        for (uint64_t cand : {n, 3 * n})
            if (cand >= L && cand >= kSmallMinN && cand <= kSmallMaxN && (!best || cand < best)) best = cand;
    return best;
}

std::vector<uint32_t> small_schedule(uint64_t N) {
    std::vector<uint32_t> s;
    uint64_t P = N;
    if (N % 3 == 0) { s.push_back(3); P = N / 3; }
    for (uint32_t r : pow2_schedule((uint32_t)P)) s.push_back(r);
    return s;
}

// ---- twiddle tables ---------------------------------------------------------------------------------
static void push_pair(std::vector<uint32_t> &t, uint32_t w, uint32_t p) {
    t.push_back(w);
    t.push_back(shoup_companion(w, p));
}

// Inter-stage twiddles of one stage (m, R): entry (k-1)*(m/R) + j = xi_m^(+-j k), k in [1,R),
// j in [0, m/R).  xi_m = xi_N^(N/m).
static void stage_table(std::vector<uint32_t> &t, uint32_t p, uint32_t xiN, uint64_t N, uint32_t m,
                        uint32_t R, bool inverse) {
    uint64_t xim = powmod64(xiN, N / m, p);
    if (inverse) xim = powmod64(xim, p - 2, p);
    uint32_t cols = m / R;
    for (uint32_t k = 1; k < R; ++k) {
        uint64_t step = powmod64(xim, k, p), w = 1;
        for (uint32_t j = 0; j < cols; ++j) {
            push_pair(t, (uint32_t)w, p);
            w = mulmod64(w, step, p);
        }
    }
}

static void fill_stages(const std::vector<uint32_t> &radix, uint32_t n, Stage *st, int *ns,
                        std::vector<uint32_t> &t, uint32_t p, uint32_t xiN, uint64_t N, bool write) {
    uint32_t m = n;
    *ns = (int)radix.size();
    for (size_t i = 0; i < radix.size(); ++i) {
        uint32_t R = radix[i];
        Stage s{R, m, 0, 0};
        if (m > R) {
            s.tw = (uint32_t)(t.size() / 2);
            stage_table(t, p, xiN, N, m, R, false);
            s.twi = (uint32_t)(t.size() / 2);
            stage_table(t, p, xiN, N, m, R, true);
        }
        if (write) st[i] = s;
        m /= R;
    }
}

void build_small_tables(uint64_t N, SmallPlanDev *sp, std::vector<uint32_t> tables[kPrimes]) {
    memset(sp, 0, sizeof(*sp));
    sp->N = (uint32_t)N;
    std::vector<uint32_t> radix = small_schedule(N);
    for (int pi = 0; pi < kPrimes; ++pi) {
        const uint32_t p = kPrimeSet[pi];
        const uint32_t xiN = root_of_unity(p, N);
        tables[pi].clear();
        fill_stages(radix, (uint32_t)N, sp->st, &sp->ns, tables[pi], p, xiN, N, pi == 0);
        const uint64_t scale = mulmod64(((uint64_t)1 << 32) % p, powmod64(N % p, p - 2, p), p);
        sp->scale[pi] = (uint32_t)scale;
        sp->scales[pi] = shoup_companion((uint32_t)scale, p);
    }
}

void build_tables(const HostPlan &hp, PlanDev *pd, std::vector<uint32_t> tables[kPrimes]) {
    memset(pd, 0, sizeof(*pd));
    pd->N = hp.N;
    pd->N1 = hp.N1;
    pd->N2 = hp.N2;
    pd->col_threads = hp.col_threads ? hp.col_threads : (hp.N1 >= 512 ? 512 : 256);
    pd->row_threads = hp.row_threads ? hp.row_threads : 256;
    pd->row_tma = hp.row_tma;
    pd->row_grid = hp.row_grid;
    pd->col_half = hp.col_half;
    const uint64_t N = hp.N;
    const uint32_t N1 = hp.N1, N2 = hp.N2;
    const int s = (int)hp.col_radix.size();
    const uint32_t Rs = hp.col_radix[s - 1];
    const uint32_t nb = N1 / Rs;  // blocks of the last column stage
    // F(b): frequency of position b*Rs of the column transform's output (mixed-radix digit
    // reversal over the first s-1 radices).
    std::vector<uint64_t> F(nb);
    for (uint32_t b = 0; b < nb; ++b) {
        uint64_t rem = b, f = 0, mult = 1;
        std::vector<uint32_t> dig(s, 0);
        for (int t = s - 2; t >= 0; --t) {
            dig[t] = (uint32_t)(rem % hp.col_radix[t]);
            rem /= hp.col_radix[t];
        }
        for (int t = 0; t <= s - 2; ++t) {
            f += dig[t] * mult;
            mult *= hp.col_radix[t];
        }
        F[b] = f;
    }
    for (int pi = 0; pi < kPrimes; ++pi) {
        const uint32_t p = kPrimeSet[pi];
        const uint32_t xiN = root_of_unity(p, N);
        const uint32_t xiNi = (uint32_t)powmod64(xiN, p - 2, p);
        std::vector<uint32_t> &t = tables[pi];
        t.clear();
        fill_stages(hp.col_radix, N1, pd->cs, &pd->ncs, t, p, xiN, N, pi == 0);
        fill_stages(hp.row_radix, N2, pd->rs, &pd->nrs, t, p, xiN, N, pi == 0);
        // scale of the inverse: 2^32 N^-1 (removes the Montgomery factor and the IDFT* scale)
        const uint64_t scale = mulmod64(((uint64_t)1 << 32) % p, powmod64(N % p, p - 2, p), p);
        for (int inv = 0; inv < 2; ++inv) {
            const uint64_t root = inv ? xiNi : xiN;
            const uint64_t offA = t.size() / 2;
            for (uint32_t b = 0; b < nb; ++b) {
                uint64_t step = powmod64(root, F[b] % N, p);
                uint64_t w = inv ? scale : 1;
                for (uint32_t n2 = 0; n2 < N2; ++n2) {
                    push_pair(t, (uint32_t)w, p);
                    w = mulmod64(w, step, p);
                }
            }
            const uint64_t offQ = t.size() / 2;
            for (uint32_t k = 0; k < Rs; ++k) {
                uint64_t step = powmod64(root, ((uint64_t)nb * k) % N, p), w = 1;
                for (uint32_t n2 = 0; n2 < N2; ++n2) {
                    push_pair(t, (uint32_t)w, p);
                    w = mulmod64(w, step, p);
                }
            }
            if (pi == 0) {
                if (inv) { pd->offAi = offA; pd->offQi = offQ; }
                else { pd->offA = offA; pd->offQ = offQ; }
            }
        }
    }
}

}  // namespace dml
