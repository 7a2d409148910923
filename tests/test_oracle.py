"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: Python's own int arithmetic or
CPython's ``decimal`` (libmpdec) as library routines, sympy's primality routines, numpy's
transpose, closed forms ((10^n - 1)^2 = 10^2n - 2*10^n + 1, shifts by 10^j), invariants
(commutativity, residue fingerprints, the transpose permutation's fixed points and cycle counts
of Sec. 7.5, the identity Psi(rho'' L) = L^T of Sec. 7.6) and brute force on tiny inputs.
"""
import decimal
import math
import random

import numpy as np
import pytest

import oracle
from paper_2011_11524_gb300 import workloads as wl
from tests.limbs import from_int, to_int, to_str

B = 10**9


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rand_limbs(rng, n, top_nonzero=True):
    a = rng.integers(0, B, size=n, dtype=np.uint64).astype(np.uint32)
    if top_nonzero and n:
        a[-1] = max(1, int(a[-1]))
    return a


# ----------------------------------------------------------------------------------------------
# the product by definition vs Python ints
# ----------------------------------------------------------------------------------------------
def test_schoolbook_bruteforce_small():
    """Every shape n, m <= 24 limbs, random and extreme limbs, against Python int products."""
    rng = _rng(100)
    for n in range(1, 25):
        for m in range(1, 25):
            for kind in ("rand", "nines", "zero_top"):
                if kind == "rand":
                    x, y = _rand_limbs(rng, n), _rand_limbs(rng, m)
                elif kind == "nines":
                    x = np.full(n, B - 1, np.uint32)
                    y = np.full(m, B - 1, np.uint32)
                else:
                    x, y = _rand_limbs(rng, n, False), _rand_limbs(rng, m, False)
                    x[-1] = 0
                z = oracle.mul_schoolbook(x, y, nthreads=1)
                assert len(z) == n + m
                assert to_int(z) == to_int(x) * to_int(y)


def test_schoolbook_random_sizes_vs_python_int():
    rng = _rng(101)
    for _ in range(6):
        n = int(rng.integers(1, 4000))
        m = int(rng.integers(1, 4000))
        x, y = _rand_limbs(rng, n), _rand_limbs(rng, m)
        assert to_int(oracle.mul_schoolbook(x, y)) == to_int(x) * to_int(y)


def test_c1_size_vs_python_int():
    """The 100,000-digit configuration: schoolbook against Python's int product."""
    x, y = wl.c1_pair()
    assert len(x) == 11112 and len(y) == 11112
    z = oracle.mul_schoolbook(x, y)
    assert to_int(z) == to_int(x) * to_int(y)


def test_conv_coefficients_vs_definition_tiny():
    """c_k of the zero-padded convolution (Sec. 3.2) against a direct Python double loop."""
    rng = _rng(102)
    for n, m in ((1, 1), (3, 5), (7, 2), (16, 16)):
        x, y = _rand_limbs(rng, n), _rand_limbs(rng, m)
        c = oracle.conv_schoolbook(x, y, nthreads=1)
        ref = [0] * (n + m)
        for i in range(n):
            for j in range(m):
                ref[i + j] += int(x[i]) * int(y[j])
        assert c == ref
        # eq. ci_bound: c_i <= (B-1)^2 min(n, m)
        assert max(c) <= (B - 1) ** 2 * min(n, m)


def test_conv_at_every_k_vs_schoolbook_and_double_loop():
    """One coefficient c_k = sum_{i+j=k} x_i y_j (Sec. 3.2), which the GPU tests compare sampled
    c_k with: at every k of several shapes against the schoolbook column sums, and on tiny shapes
    against a Python double loop.  Both the i-range bounds and both ends (k = 0, k = n+m-1, where c_k = 0) are hit."""
    rng = _rng(110)
    for n, m in ((1, 1), (3, 5), (5, 3), (7, 2), (300, 17), (17, 300), (1000, 1000)):
        x, y = _rand_limbs(rng, n), _rand_limbs(rng, m)
        c = oracle.conv_schoolbook(x, y, nthreads=1)
        for k in range(n + m):
            assert oracle.conv_at(x, y, k) == c[k], (n, m, k)
        if n * m <= 64:
            for k in range(n + m):
                ref = sum(int(x[i]) * int(y[k - i]) for i in range(n) if 0 <= k - i < m)
                assert oracle.conv_at(x, y, k) == ref
    # all-nines: every c_k is (B-1)^2 times the number of index pairs, a closed form
    n, m = 40, 25
    x, y = np.full(n, B - 1, np.uint32), np.full(m, B - 1, np.uint32)
    for k in range(n + m):
        pairs = max(0, min(k, n - 1) - max(0, k - m + 1) + 1)
        assert oracle.conv_at(x, y, k) == (B - 1) ** 2 * pairs


def test_residues_vs_python_mod():
    """c_k mod p from 128-bit (lo, hi) words, against Python's int %, on hand-built words that
    exercise each half: 0, 1, 2^64 - 1, 2^64, 2^127 - 1, 2^128 - 1, multiples of p and
    neighbours."""
    ps = [377487361, 754974721, 880803841, 2**61 - 1, 3]
    vals = [0, 1, 2**32, 2**64 - 1, 2**64, 2**64 + 1, 2**96 + 12345, 2**127 - 1, 2**128 - 1,
            (10**9 - 1) ** 2 * 1864136]
    for p in ps:
        vv = vals + [p, p - 1, p + 1, p * (2**64 + 3), p * (2**64 + 3) - 1]
        vv = [v for v in vv if v < 2**128]
        words = np.array([[v & (2**64 - 1), v >> 64] for v in vv], dtype=np.uint64)
        r = oracle.residues(words, p)
        assert [int(t) for t in r] == [v % p for v in vv]


def test_normalize_cases():
    """Normalized length: strip leading zero limbs, keep at least one (zero is one limb 0)."""
    z = oracle.normalize(np.zeros(7, np.uint32))
    assert z.tolist() == [0]
    z = oracle.normalize(np.zeros(1, np.uint32))
    assert z.tolist() == [0]
    a = np.zeros(9, np.uint32)
    a[8] = 5
    assert oracle.normalize(a).tolist() == [0] * 8 + [5]
    a = np.array([3, 0, 7, 0, 0, 0], np.uint32)
    assert oracle.normalize(a).tolist() == [3, 0, 7]
    a = np.array([0, 0, 0, 1], np.uint32)
    assert len(oracle.normalize(a)) == 4
    a = np.array([B - 1], np.uint32)
    assert oracle.normalize(a).tolist() == [B - 1]
    # against Python's int: the normalized limbs are the decimal digits of the value
    rng = _rng(111)
    for n in (1, 2, 10, 100):
        for lead in (0, 1, 5):
            v = _rand_limbs(rng, n)
            w = np.concatenate([v, np.zeros(lead, np.uint32)])
            zn = oracle.normalize(w)
            assert to_int(zn) == to_int(w)
            assert zn[-1] != 0 or len(zn) == 1
            assert len(zn) == max(1, (len(str(to_int(w))) + 8) // 9) if to_int(w) else len(zn) == 1


def test_carry_vs_python_int():
    """The carry recurrence against Python's int -> decimal conversion, near-maximal c_k."""
    rng = random.Random(103)
    for L in (1, 2, 5, 64, 1000):
        for top in (2**60, 2**83):
            c = [rng.randrange(top) for _ in range(L - 1)] + [0]
            words = np.array([[v & (2**64 - 1), v >> 64] for v in c], dtype=np.uint64)
            z, fin = oracle.carry(words)
            total = sum(v * B**k for k, v in enumerate(c))
            assert fin == total // B**L
            assert to_int(z) == total % B**L


# ----------------------------------------------------------------------------------------------
# closed forms and invariants
# ----------------------------------------------------------------------------------------------
@pytest.mark.parametrize("route", ["schoolbook", "ntt"])
@pytest.mark.parametrize("ndig", [1, 8, 9, 10, 17, 18, 100, 1001, 20000])
def test_nines_square_closed_form(route, ndig):
    """(10^n - 1)^2 = 10^(2n) - 2 10^n + 1: digits '9'*(n-1) '8' '0'*(n-1) '1'."""
    x = wl.all_nines(ndig)
    z = oracle.mul_schoolbook(x, x) if route == "schoolbook" else oracle.mul_ntt(x, x)
    expect = "9" * (ndig - 1) + "8" + "0" * (ndig - 1) + "1"
    assert to_str(z) == expect


@pytest.mark.parametrize("route", ["schoolbook", "ntt"])
def test_shift_by_power_of_ten(route):
    """x * 10^j appends j zero digits to x's decimal string."""
    rng = _rng(104)
    x = _rand_limbs(rng, 300)
    xs = to_str(x)
    for j in (0, 1, 8, 9, 10, 26, 27, 500, 2000):
        y = np.zeros(j // 9 + 1, dtype=np.uint32)
        y[j // 9] = 10 ** (j % 9)
        z = oracle.mul_schoolbook(x, y) if route == "schoolbook" else oracle.mul_ntt(x, y)
        assert to_str(z) == xs + "0" * j


@pytest.mark.parametrize("route", ["schoolbook", "ntt"])
def test_commutativity(route):
    rng = _rng(105)
    f = oracle.mul_schoolbook if route == "schoolbook" else oracle.mul_ntt
    for n, m in ((1, 700), (333, 1024), (2048, 1500)):
        x, y = _rand_limbs(rng, n), _rand_limbs(rng, m)
        assert np.array_equal(f(x, y), f(y, x))


def _fp_moduli(count=4):
    out = []
    for q in wl.fingerprint_candidates():
        if oracle.is_prime_mr(q):
            out.append(q)
            if len(out) == count:
                return out


def test_fingerprint_vs_python_mod():
    rng = _rng(106)
    qs = _fp_moduli()
    sympy = pytest.importorskip("sympy")
    for q in qs:
        assert sympy.isprime(q) and (1 << 60) <= q < (1 << 61)
    for n in (1, 2, 50, 3001):
        x = _rand_limbs(rng, n)
        xi = to_int(x)
        for q in qs:
            assert oracle.fingerprint(x, q) == xi % q


def test_fingerprint_identity_on_products():
    """x*y mod q = (x mod q)(y mod q) mod q on oracle products, both routes."""
    rng = _rng(107)
    qs = _fp_moduli()
    x, y = _rand_limbs(rng, 5000), _rand_limbs(rng, 3000)
    for z in (oracle.mul_schoolbook(x, y), oracle.mul_ntt(x, y)):
        for q in qs:
            assert oracle.fingerprint(z, q) == oracle.fingerprint(x, q) * oracle.fingerprint(y, q) % q


def test_fingerprint_many_vs_python_mod():
    """The threaded many-vector form against Python's int %, vector by vector and modulus by
    modulus (a swapped index or a thread writing another vector's slot fails here)."""
    rng = _rng(108)
    qs = _fp_moduli()
    vecs = [_rand_limbs(rng, n) for n in (1, 7, 64, 999, 5000, 2, 31)] + [np.array([B - 1] * 40, np.uint32)]
    for nt in (1, 3, 8):
        out = oracle.fingerprint_many(vecs, qs, nthreads=nt)
        assert out.shape == (len(vecs), len(qs))
        for v, row in zip(vecs, out):
            vi = to_int(v)
            assert [int(t) for t in row] == [vi % q for q in qs]


# ----------------------------------------------------------------------------------------------
# the independent slow NTT route
# ----------------------------------------------------------------------------------------------
def test_ntt_route_vs_schoolbook_overlap():
    rng = _rng(108)
    for n, m in ((1, 1), (2, 3), (100, 1), (1000, 999), (4096, 4096), (20000, 7)):
        x, y = _rand_limbs(rng, n), _rand_limbs(rng, m)
        assert np.array_equal(oracle.mul_ntt(x, y), oracle.mul_schoolbook(x, y))
    x = np.full(20000, B - 1, np.uint32)
    assert np.array_equal(oracle.mul_ntt(x, x), oracle.mul_schoolbook(x, x))


@pytest.mark.slow
def test_ntt_route_vs_libmpdec_million_digits():
    """10^6 x 10^6 digits against CPython's decimal (libmpdec, the paper's comparison library)."""
    rng = _rng(109)
    x = wl.random_operand(1_000_000, rng)
    y = wl.random_operand(1_000_000, rng)
    ctx = decimal.Context(prec=decimal.MAX_PREC, Emax=decimal.MAX_EMAX, Emin=decimal.MIN_EMIN)
    dx = decimal.Decimal(to_str(x))
    dy = decimal.Decimal(to_str(y))
    dz = ctx.multiply(dx, dy)
    z = oracle.mul_ntt(x, y)
    assert to_str(z) == format(dz, "f")


def test_ntt_route_c2_shape_prefix():
    """A 2^20-digit multiply (same code path as the 2^24-digit workload) against Python int."""
    rng = _rng(110)
    x = wl.random_operand(1 << 20, rng)
    y = wl.random_operand(1 << 20, rng)
    assert to_int(oracle.mul_ntt(x, y)) == to_int(x) * to_int(y)


# ----------------------------------------------------------------------------------------------
# field transforms (Sec. 3.3, Sec. 5)
# ----------------------------------------------------------------------------------------------
P_TEST = 0x7FFFFFFFD7000001


def test_primitive_root_vs_sympy():
    sympy = pytest.importorskip("sympy")
    from sympy.ntheory import primitive_root
    for p in (7, 17, 97, 0x78000001, 0x16800001, 0x2D000001, 0x34800001):
        assert oracle.primitive_root(p) == primitive_root(p)
    assert sympy.isprime(P_TEST)
    g = oracle.primitive_root(P_TEST)
    assert sympy.n_order(g, P_TEST) == P_TEST - 1


@pytest.mark.parametrize("lg", [0, 1, 2, 3, 5, 8])
def test_radix2_transforms_vs_naive_dft(lg):
    """tau by DIF and by DIT (Sec. 5.2-5.3) equal the DFT definition; closed forms of deltas."""
    n = 1 << lg
    p = P_TEST
    g = oracle.primitive_root(p)
    w = pow(g, (p - 1) >> lg, p)
    assert pow(w, n, p) == 1 and (n == 1 or pow(w, n // 2, p) != 1)
    rng = _rng(111 + lg)
    a = rng.integers(0, p, size=n, dtype=np.uint64)
    ref = oracle.dft_naive(a, w, p)
    assert np.array_equal(oracle.tau_dif(a, w, p), ref)
    assert np.array_equal(oracle.tau_dit(a, w, p), ref)
    # closed forms: DFT(e_0) = all ones; DFT(all ones) = n e_0; DFT(e_1)[k] = w^k
    e0 = np.zeros(n, np.uint64); e0[0] = 1
    assert np.all(oracle.dft_naive(e0, w, p) == 1)
    ones = np.ones(n, np.uint64)
    exp = np.zeros(n, np.uint64); exp[0] = n % p
    assert np.array_equal(oracle.dft_naive(ones, w, p), exp)
    if n > 1:
        e1 = np.zeros(n, np.uint64); e1[1] = 1
        assert [int(v) for v in oracle.dft_naive(e1, w, p)] == [pow(w, k, p) for k in range(n)]
    # round trip f^-1(f(x)) = x with f^-1 = N^-1 tau(., w^-1)
    back = oracle.tau_dit(ref, pow(w, p - 2, p), p)
    ninv = pow(n, p - 2, p)
    assert [int(v) * ninv % p for v in back] == [int(v) for v in a]


def test_convolution_theorem_vs_direct_cyclic_sum():
    """x star y computed through the transforms equals the direct cyclic sum (Sec. 3.1, 3.3)."""
    p = P_TEST
    rng = _rng(120)
    for lg in (0, 1, 3, 6):
        n = 1 << lg
        a = rng.integers(0, 1 << 40, size=n, dtype=np.uint64)
        b = rng.integers(0, 1 << 40, size=n, dtype=np.uint64)
        direct = [sum(int(a[i]) * int(b[(k - i) % n]) for i in range(n)) % p for k in range(n)]
        assert [int(v) for v in oracle.cyclic_conv_mod(a, b, p)] == direct


# ----------------------------------------------------------------------------------------------
# primes (Sec. 4.5)
# ----------------------------------------------------------------------------------------------
def test_miller_rabin_vs_sympy():
    sympy = pytest.importorskip("sympy")
    for n in range(0, 20000):
        assert oracle.is_prime_mr(n) == sympy.isprime(n), n
    # strong pseudoprimes to several small bases and Carmichael numbers
    for n in (561, 1105, 1729, 2047, 1373653, 25326001, 3215031751, 2152302898747,
              3474749660383, 341550071728321, 3825123056546413051):
        assert oracle.is_prime_mr(n) == sympy.isprime(n), n
    rng = random.Random(121)
    for _ in range(3000):
        n = rng.randrange(1 << 62) | 1
        assert oracle.is_prime_mr(n) == sympy.isprime(n), n


def _brute_force_primes(w, n_min, l):
    sympy = pytest.importorskip("sympy")
    found = set()
    lim = 1 << (w - 1)
    for n in range(n_min, w - 1):
        c = 1
        while 3 * c * (1 << n) + 1 < lim:
            p = 3 * c * (1 << n) + 1
            if sympy.isprime(p):
                found.add(p)
            c += 2
    return sorted(found, reverse=True)[:l]


@pytest.mark.parametrize("w,n_min,l", [(31, 23, 3), (32, 23, 3), (31, 20, 4), (20, 5, 3)])
def test_find_primes_vs_brute_force(w, n_min, l):
    assert oracle.find_primes(w, n_min, l) == _brute_force_primes(w, n_min, l)


def test_find_primes_64bit_are_the_largest():
    """FindPrimes(64, 23, 2): each result is a prime c*3*2^n+1 < 2^63 (c odd, n >= 23) and no
    larger number of that form is prime."""
    sympy = pytest.importorskip("sympy")
    ps = oracle.find_primes(64, 23, 2)
    assert ps == sorted(ps, reverse=True)
    for p in ps:
        assert sympy.isprime(p) and p < (1 << 63)
        q = p - 1
        n = (q & -q).bit_length() - 1
        assert n >= 23 and (q >> n) % 3 == 0 and (q >> n) % 2 == 1
    lo = ps[-1]
    for n in range(23, 63):
        c = (lo - 1) // (3 << n) + 1
        while 3 * c * (1 << n) + 1 < (1 << 63):
            p = 3 * c * (1 << n) + 1
            if c % 2 == 1 and p > lo and sympy.isprime(p):
                assert p in ps, hex(p)
            c += 1


# ----------------------------------------------------------------------------------------------
# transposition (Sec. 7.5-7.6)
# ----------------------------------------------------------------------------------------------
def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    out = {}
    with open(path) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, *v = line.split()
            out[k] = [int(t) for t in v]
    return out


def test_transpose_worked_example():
    g = _golden("rowmajor_2x4.txt")
    t = oracle.transpose(np.array(g["flat"], np.uint32), g["rows"][0], g["cols"][0])
    assert t.tolist() == g["transposed"]


@pytest.mark.parametrize("rows,cols", [(1, 1), (2, 4), (4, 8), (8, 4), (3, 5), (16, 32), (64, 64)])
def test_transpose_vs_numpy_and_permutation_formula(rows, cols):
    a = np.arange(rows * cols, dtype=np.uint32)
    t = oracle.transpose(a, rows, cols)
    assert np.array_equal(t, a.reshape(rows, cols).T.reshape(-1))
    # Sec. 7.5: the element at index a moves to P(a) = N1 a mod (N1 N2 - 1), P(N1N2-1) = N1N2-1
    n1, n2 = rows, cols
    total = n1 * n2

    def P(i):
        return total - 1 if i == total - 1 else (n1 * i) % (total - 1) if total > 1 else 0

    for i in range(total):
        assert t[P(i)] == a[i]
    fixed = sum(1 for i in range(total) if P(i) == i)
    assert fixed == 1 + math.gcd(n1 - 1, n2 - 1)
    # cycle counts: number of cycles of length k > 1 is (1/k) sum_{d|k} mu(k/d) gcd(N1^d - 1, N1N2 - 1)
    if total > 2:
        seen = [False] * total
        counts = {}
        for i in range(total):
            if seen[i]:
                continue
            j, ln = i, 0
            while not seen[j]:
                seen[j] = True
                j = P(j)
                ln += 1
            counts[ln] = counts.get(ln, 0) + 1

        def mobius(k):
            r, d = 1, 2
            while d * d <= k:
                if k % d == 0:
                    k //= d
                    if k % d == 0:
                        return 0
                    r = -r
                d += 1
            return -r if k > 1 else r

        for k, cnt in counts.items():
            if k == 1:
                continue
            s = sum(mobius(k // d) * math.gcd(n1**d - 1, total - 1) for d in range(1, k + 1) if k % d == 0)
            assert s % k == 0 and s // k == cnt


@pytest.mark.parametrize("n,cols", [(1, 3), (2, 4), (3, 1), (4, 8), (8, 16), (32, 64)])
def test_rho_and_psi_identity(n, cols):
    """Sec. 7.6: with rho on the 2n columns, Psi(rho'' L) = L^T for an n x 2n matrix L, where Psi
    transposes the left and the right n x n halves.  rho'' on columns is rho' on the rows of
    the transpose (eq. matrix_permutation_rule)."""
    rng = _rng(130 + n)
    if cols != 2 * n:
        # rho on the rows of an arbitrary (2n) x cols matrix against the definition
        a = rng.integers(0, 1 << 30, size=2 * n * cols, dtype=np.uint64).astype(np.uint32)
        out = oracle.permute_rows_rho(a, n, cols).reshape(2 * n, cols)
        A = a.reshape(2 * n, cols)
        for i in range(2 * n):
            assert np.array_equal(out[n * (i % 2) + i // 2], A[i])
        return
    Lm = rng.integers(0, 1 << 30, size=(n, 2 * n), dtype=np.uint64).astype(np.uint32)
    # rho'' L = (rho' L^T)^T
    LT = oracle.transpose(Lm.reshape(-1), n, 2 * n)
    rhoL = oracle.transpose(oracle.permute_rows_rho(LT, n, n), 2 * n, n).reshape(n, 2 * n)
    left, right = rhoL[:, :n], rhoL[:, n:]
    psi = np.concatenate([left.T, right.T], axis=1)  # [A^T B^T], an n x 2n matrix
    assert np.array_equal(psi.reshape(-1), Lm.T.reshape(-1))
