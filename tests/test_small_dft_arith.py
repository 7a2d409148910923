"""The kernels' modular arithmetic (modarith.cuh) emulated on the CPU in exact 32-bit steps: the
Shoup and Montgomery products with their output ranges, and the odd-radix DFTs of the column pass
(radix 3 and radix 5) checked against the DFT's definition (Sec. 3.3):
every output congruent to sum_j a_j w^(jk) mod p and inside [0, 2p), for every prime, both
directions and inputs anywhere in [0, 2p) (including the extremes).  This pins the algebra of the
radix-5 decomposition (six constant products) and its range bounds, independently of the GPU."""
import numpy as np
import pytest

from paper_2011_11524_gb300 import dmul as d

M32 = (1 << 32) - 1


def smallest_generator(p):
    n, fac, q = p - 1, [], 2
    while q * q <= n:
        if n % q == 0:
            fac.append(q)
            while n % q == 0:
                n //= q
        q += 1
    if n > 1:
        fac.append(n)
    g = 2
    while any(pow(g, (p - 1) // f, p) == 1 for f in fac):
        g += 1
    return g


def companion(w, p):
    return (w << 32) // p


def shoup(a, w, ws, p):
    """a w mod p in [0, 2p) for any 32-bit a: a w - hi(a ws) p, wrapped to 32 bits."""
    q = (a * ws) >> 32
    r = (a * w - q * p) & M32
    assert r < 2 * p
    return r


def red2p(a, p):
    assert 0 <= a < 4 * p
    return min(a, (a - 2 * p) & M32)


def radix3(v, w, p):
    ws = companion(w, p)
    a, b, c = v
    t = shoup((b - c + 2 * p) & M32, w, ws, p)
    x0 = red2p(red2p(a + b, p) + c, p)
    x1 = red2p(red2p((a - c + 2 * p) & M32, p) + t, p)
    x2 = red2p((red2p((a - b + 2 * p) & M32, p) - t + 2 * p) & M32, p)
    return [x0, x1, x2]


def radix5_constants(w, p):
    inv2 = (p + 1) // 2
    inv4 = inv2 * inv2 % p
    w2, w3, w4 = w * w % p, pow(w, 3, p), pow(w, 4, p)
    k = [(p - inv4) % p, (w + w4 - w2 - w3) * inv4 % p, (w - w4) * inv2 % p, (w2 - w3) * inv2 % p]
    return k, [companion(x, p) for x in k]


def radix5(v, w, p):
    k, ks = radix5_constants(w, p)
    p2 = 2 * p
    a0 = v[0]
    s1, s2 = red2p(v[1] + v[4], p), red2p(v[2] + v[3], p)
    d1, d2 = (v[1] - v[4] + p2) & M32, (v[2] - v[3] + p2) & M32
    t1 = red2p(s1 + s2, p)
    b = red2p(a0 + shoup(t1, k[0], ks[0], p), p)
    m2 = shoup((s1 - s2 + p2) & M32, k[1], ks[1], p)
    P, Q = red2p(b + m2, p), red2p((b - m2 + p2) & M32, p)
    e11, e22 = shoup(d1, k[2], ks[2], p), shoup(d2, k[3], ks[3], p)
    e21, e12 = shoup(d1, k[3], ks[3], p), shoup(d2, k[2], ks[2], p)
    E1, E2 = red2p(e11 + e22, p), red2p((e21 - e12 + p2) & M32, p)
    return [red2p(a0 + t1, p), red2p(P + E1, p), red2p(Q + E2, p), red2p((Q - E2 + p2) & M32, p),
            red2p((P - E1 + p2) & M32, p)]


@pytest.mark.parametrize("R,fn", [(3, radix3), (5, radix5)])
def test_odd_radix_dft_matches_definition(R, fn):
    rng = np.random.Generator(np.random.PCG64(35))
    for p in d.dmul_primes():
        assert (p - 1) % R == 0
        g = smallest_generator(p)
        w_fwd = pow(g, (p - 1) // R, p)
        for w in (w_fwd, pow(w_fwd, p - 2, p)):  # forward and inverse roots
            cases = [[0] * R, [2 * p - 1] * R, [p] * R, [2 * p - 1 if j % 2 else 0 for j in range(R)]]
            cases += [[int(x) for x in rng.integers(0, 2 * p, R)] for _ in range(400)]
            for v in cases:
                out = fn(v, w, p)
                for k in range(R):
                    ref = sum(v[j] * pow(w, j * k, p) for j in range(R)) % p
                    assert 0 <= out[k] < 2 * p and out[k] % p == ref, (p, R, v, k)


def test_radix5_uses_six_products():
    """c1 + c2 = -1/2 (the four nontrivial fifth roots sum to -1), which folds the two cosine
    terms into one product by -1/4 and one by (c1 - c2)/2."""
    for p in d.dmul_primes():
        g = smallest_generator(p)
        w = pow(g, (p - 1) // 5, p)
        assert (w + pow(w, 2, p) + pow(w, 3, p) + pow(w, 4, p)) % p == p - 1


def mont(a, b, p, pinv):
    """Subtractive Montgomery: hi(ab) - hi(m p) + p with m = lo(ab) p^-1 mod 2^32."""
    ab = a * b
    lo, hi = ab & M32, ab >> 32
    m = (lo * pinv) & M32
    t = (m * p) >> 32
    return (hi - t + p) & M32


def test_shoup_and_montgomery_bounds():
    """Shoup's product takes any 32-bit input and returns a w mod p in [0, 2p) (which is what lets
    unreduced [0, 4p) sums feed it); the Montgomery product of inputs in [0, 2p) returns
    a b 2^-32 mod p in (0, 2p) with no correction step (p < 2^30)."""
    rng = np.random.Generator(np.random.PCG64(36))
    for p in d.dmul_primes():
        assert p < 1 << 30
        pinv = pow(p, -1, 1 << 32)
        r_inv = pow(1 << 32, -1, p)
        ws = [int(x) for x in rng.integers(1, p, 40)] + [1, p - 1]
        edges = [0, 1, p - 1, p, 2 * p - 1, 4 * p - 1, M32]
        for w in ws:
            wc = companion(w, p)
            for a in edges + [int(x) for x in rng.integers(0, 1 << 32, 200, dtype=np.uint64)]:
                r = shoup(a, w, wc, p)  # asserts r < 2p
                assert r % p == a * w % p
        for a in [0, 1, p, 2 * p - 1] + [int(x) for x in rng.integers(0, 2 * p, 300)]:
            for b in [0, 1, 2 * p - 1] + [int(x) for x in rng.integers(0, 2 * p, 20)]:
                r = mont(a, b, p, pinv)
                assert 0 < r < 2 * p and r % p == a * b * r_inv % p


def mont_signed(a, b, p, pinv):
    """Signed Montgomery (Sec. 9, Prospects) on centred inputs a - p, b - p: signed high halves,
    r = hi(ab') - hi(m p) + p with m the signed low word times p^-1 mod 2^32."""
    sa, sb = a - p, b - p
    t = sa * sb
    lo = t & M32
    m = (lo * pinv) & M32
    m = m - (1 << 32) if m >= 1 << 31 else m
    assert (t - m * p) % (1 << 32) == 0
    r = (t >> 32) - ((m * p) >> 32) + p  # Python's >> floors, as the arithmetic shift does
    return r


def test_signed_montgomery_bounds():
    """The signed form returns ab 2^-32 mod p in (0, 2p) for inputs in [0, 2p), like the
    subtractive form, with no correction step."""
    rng = np.random.Generator(np.random.PCG64(37))
    for p in d.dmul_primes():
        pinv = pow(p, -1, 1 << 32)
        r_inv = pow(1 << 32, -1, p)
        vals = [0, 1, p - 1, p, p + 1, 2 * p - 1] + [int(x) for x in rng.integers(0, 2 * p, 300)]
        for a in vals:
            for b in vals[:6] + [int(x) for x in rng.integers(0, 2 * p, 20)]:
                r = mont_signed(a, b, p, pinv)
                assert 0 < r < 2 * p and r % p == a * b * r_inv % p
                assert r % p == mont(a, b, p, pinv) % p
