"""Full-size parity: the benchmark workloads, in the launch configuration bench.py times.

* 2^24 x 2^24 digits (random, and all nines; multiplication and squaring): every limb against the
  oracle's independent slow NTT route; the all-nines products also against the closed form
  (10^n - 1)^2 = 10^2n - 2 10^n + 1 (maximal convolution coefficients, eq. ci_bound).
* 64M x 1M and 32M x 16M digits with 5% of the limbs 10^9 - 1: every limb against the oracle, four
  residue fingerprints (x y mod q = (x mod q)(y mod q) mod q for 61-bit primes q), and a sample of
  exact convolution coefficients c_k (after CRT) computed one by one by the oracle.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2011_11524_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

B = 10**9


@pytest.fixture(scope="module")
def d():
    from paper_2011_11524_gb300 import build as dbuild
    from paper_2011_11524_gb300 import dmul
    dbuild.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return dmul


@pytest.fixture(scope="module")
def ctx(d):
    c = d.Context(0)
    yield c
    c.close()


def _moduli(k=4):
    return list(itertools.islice((q for q in wl.fingerprint_candidates() if oracle.is_prime_mr(q)), k))


def _mul(d, ctx, x, y, square=False):
    tx = d.to_device(x)
    ty = tx if square else d.to_device(y)
    z, nz = ctx.mul(tx, ty)
    return d.to_host(z), nz


def _nines_square_limbs(ndig):
    s = "9" * (ndig - 1) + "8" + "0" * (ndig - 1) + "1"
    pad = (-len(s)) % 9
    s = "0" * pad + s
    a = np.frombuffer(s.encode(), dtype=np.uint8).astype(np.uint32) - 48
    a = a.reshape(-1, 9)
    w = np.array([10**(8 - i) for i in range(9)], dtype=np.uint64)
    limbs = (a.astype(np.uint64) * w).sum(axis=1).astype(np.uint32)
    return limbs[::-1].copy()


def test_c2_random_mul_and_sqr(d, ctx):
    x, y = wl.c2_random_pair()
    z, nz = _mul(d, ctx, x, y)
    ref = oracle.mul_ntt(x, y)
    assert np.array_equal(z, ref)
    assert nz == len(oracle.normalize(ref))
    z, nz = _mul(d, ctx, x, x, square=True)
    assert np.array_equal(z, oracle.mul_ntt(x, x))


def test_c2_all_nines(d, ctx):
    x, y = wl.c2_nines_pair()
    expect = _nines_square_limbs(wl.C2_DIGITS)
    for square in (False, True):
        z, nz = _mul(d, ctx, x, y, square=square)
        assert nz == len(expect)
        assert np.array_equal(z[:nz], expect)
        assert not z[nz:].any()
    assert np.array_equal(oracle.normalize(oracle.mul_ntt(x, y)), expect)


@pytest.mark.parametrize("which", [0, 1])
def test_c3_shapes(d, ctx, which):
    x, y = wl.c3_pairs()[which]
    z, nz = _mul(d, ctx, x, y)
    for q in _moduli():
        assert oracle.fingerprint(z, q) == oracle.fingerprint(x, q) * oracle.fingerprint(y, q) % q
    ref = oracle.mul_ntt(x, y)
    assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))
    # sampled exact coefficients after CRT
    dg = d.to_host(ctx.conv_coeffs(d.to_device(x), d.to_device(y))).reshape(-1, 3)
    rng = np.random.Generator(np.random.PCG64(300 + which))
    L = len(x) + len(y)
    ks = sorted(set(int(k) for k in rng.integers(0, L, size=200)) | {0, 1, len(y) - 1, len(y), L - 2, L - 1})
    for k in ks:
        got = int(dg[k, 0]) + int(dg[k, 1]) * B + int(dg[k, 2]) * B * B
        assert got == oracle.conv_at(x, y, k), k


@pytest.mark.parametrize("which", ["c2", "c3a"])
def test_sixstep_full_size(d, which):
    """The six-step form at the full sizes (N = 2^22 with square in-place transposes, N = 2^23 with
    the n x 2n and 2n x n ones), every limb against the oracle's slow NTT route."""
    x, y = wl.c2_random_pair() if which == "c2" else wl.c3_pairs()[0]
    with d.Context(0, flags=d.DMUL_FLAG_SIXSTEP) as c6:
        info = d.dmul_get_plan(c6.handle, len(x) + len(y))
        assert info.sixstep == 1 and info.N == (1 << 22 if which == "c2" else 1 << 23)
        z, nz = _mul(d, c6, x, y)
    ref = oracle.mul_ntt(x, y)
    assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))


def test_max_transform_length(d, ctx):
    """The longest product the planner accepts: nx + ny = 3 * 2^22 limbs (113 million digits), the
    largest transform.  Random operands against four residue fingerprints and 100 exact
    convolution coefficients (after CRT) computed one by one by the oracle; the all-nines square
    of the same length against the closed form; one limb more is refused."""
    L = 3 * 2**22
    n = L // 2
    assert d.dmul_get_plan(ctx.handle, L).N == L
    rng = np.random.Generator(np.random.PCG64(900))
    x = rng.integers(0, B, n, dtype=np.uint64).astype(np.uint32)
    y = rng.integers(0, B, n, dtype=np.uint64).astype(np.uint32)
    x[-1] = max(1, int(x[-1]))
    y[-1] = max(1, int(y[-1]))
    z, nz = _mul(d, ctx, x, y)
    for q in _moduli():
        assert oracle.fingerprint(z, q) == oracle.fingerprint(x, q) * oracle.fingerprint(y, q) % q
    assert nz == len(oracle.normalize(z)) and nz >= L - 1
    dg = d.to_host(ctx.conv_coeffs(d.to_device(x), d.to_device(y))).reshape(-1, 3)
    ks = sorted(set(int(k) for k in rng.integers(0, L, size=96)) | {0, 1, n - 1, n, L - 2, L - 1})
    for k in ks:
        got = int(dg[k, 0]) + int(dg[k, 1]) * B + int(dg[k, 2]) * B * B
        assert got == oracle.conv_at(x, y, k), k
    del dg
    # (10^(9n) - 1)^2 = 10^(18n) - 2 10^(9n) + 1 for n limbs of nines
    nines = np.full(n, B - 1, np.uint32)
    z2, nz2 = _mul(d, ctx, nines, nines, square=True)
    expect = np.zeros(2 * n, np.uint32)
    expect[0] = 1
    expect[n] = B - 2
    expect[n + 1:] = B - 1
    assert np.array_equal(z2, expect) and nz2 == 2 * n
    t = d.to_device(np.ones(n + 1, np.uint32))
    zz = torch.empty(L + 1, dtype=torch.int32, device="cuda")
    assert d.dmul_mul(ctx.handle, t, n + 1, t, n, zz, L + 1, None) == d.DMUL_ERR_TOO_LARGE
