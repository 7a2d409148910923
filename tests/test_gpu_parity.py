"""GPU parity: every result of libdmul (through its C ABI) against the CPU oracle, bit-exact.

Shapes span every transform class from the smallest (N = 1024) up to 2^17, the length families
(2^k, 3*2^k and 5*2^k), ragged tails (lengths that are not multiples of any tile), unbalanced operands,
leading zero limbs, zero, the all-nines worst case and squarings.  Each step of the path is also
checked on its own through the stage entry points: convolution residues mod each prime (forward
transforms, pointwise product, inverse transforms), exact coefficients after CRT, the carry scan
on adversarial digit patterns, and the in-place transposes.
"""
import numpy as np
import pytest

import oracle
from paper_2011_11524_gb300 import workloads as wl
from tests.limbs import to_str

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

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


@pytest.fixture(scope="module")
def ctx4(d):
    """Four-kernel pipeline for every length (the one-cluster and the cooperative one-launch paths
    for short products are off)."""
    c = d.Context(0, flags=d.DMUL_FLAG_NO_SMALL | d.DMUL_FLAG_NO_FUSED)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_tma(d):
    """Four-step path with the persistent TMA-fed row pass for every length."""
    c = d.Context(0, flags=d.DMUL_FLAG_NO_SMALL | d.DMUL_FLAG_NO_FUSED | d.DMUL_FLAG_NO_AUTOTUNE |
                  d.DMUL_FLAG_ROW_TMA)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx6(d):
    c = d.Context(0, flags=d.DMUL_FLAG_SIXSTEP)
    yield c
    c.close()


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def _rand(rng, n, top_nonzero=True):
    a = rng.integers(0, B, size=n, dtype=np.uint64).astype(np.uint32)
    if top_nonzero and n:
        a[-1] = max(1, int(a[-1]))
    return a


def _gpu_mul(d, ctx, x, y, square=False):
    tx = d.to_device(x)
    ty = tx if square else d.to_device(y)
    z, nz = ctx.mul(tx, ty)
    return d.to_host(z), nz


SHAPES = [(1, 1), (1, 2), (2, 1), (3, 5), (31, 1), (32, 32), (33, 100), (500, 524), (500, 525),
          (767, 768), (1000, 3000), (2047, 2050), (4097, 4096), (6000, 6289), (11112, 11112),
          (12000, 12577), (24575, 1), (1, 24576), (30000, 20001), (49152, 49151), (65536, 65536),
          (100000, 7), (98303, 98304)]


@pytest.mark.parametrize("n,m", SHAPES)
def test_mul_vs_oracle(d, ctx, n, m):
    rng = _rng(1000 + n + 7 * m)
    x, y = _rand(rng, n), _rand(rng, m)
    z, nz = _gpu_mul(d, ctx, x, y)
    ref = oracle.mul(x, y)
    assert np.array_equal(z, ref)
    assert nz == len(oracle.normalize(ref))


@pytest.mark.parametrize("n,m", [s for s in SHAPES if s[0] + s[1] <= 24576])
def test_mul_four_step_short(d, ctx4, n, m):
    """The short lengths (N = 1024 .. 24576) through the four-step path as well."""
    rng = _rng(1000 + n + 7 * m)
    x, y = _rand(rng, n), _rand(rng, m)
    ref = oracle.mul(x, y)
    for square in (False, True):
        z, nz = _gpu_mul(d, ctx4, x, x if square else y, square=square)
        r = oracle.mul(x, x) if square else ref
        assert np.array_equal(z, r) and nz == len(oracle.normalize(r))


@pytest.mark.parametrize("n,m", [(1, 1), (500, 525), (4097, 4096), (30000, 20001), (65536, 65536),
                                 (100000, 7), (300000, 299999)])
def test_mul_tma_row_pass(d, ctx_tma, n, m):
    """The persistent TMA-fed row pass (bulk copies into double-buffered shared memory)."""
    rng = _rng(1500 + n + 3 * m)
    x, y = _rand(rng, n), _rand(rng, m)
    for square in (False, True):
        z, nz = _gpu_mul(d, ctx_tma, x, x if square else y, square=square)
        ref = oracle.mul(x, x) if square else oracle.mul(x, y)
        assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))


@pytest.mark.parametrize("n", [1, 2, 17, 512, 513, 1536, 5000, 11112, 40000, 65536])
def test_sqr_vs_oracle(d, ctx, n):
    rng = _rng(2000 + n)
    x = _rand(rng, n)
    z, nz = _gpu_mul(d, ctx, x, x, square=True)
    ref = oracle.mul(x, x)
    assert np.array_equal(z, ref)
    assert nz == len(oracle.normalize(ref))


@pytest.mark.parametrize("ndig", [9, 100, 4609, 100_000, 500_000])
def test_nines_closed_form(d, ctx, ndig):
    """(10^n - 1)^2 = 10^2n - 2 10^n + 1, the largest convolution coefficients (eq. ci_bound)."""
    x = wl.all_nines(ndig)
    for square in (False, True):
        z, nz = _gpu_mul(d, ctx, x, x.copy() if not square else x, square=square)
        assert to_str(z[:nz]) == "9" * (ndig - 1) + "8" + "0" * (ndig - 1) + "1"


def test_zero_and_leading_zeros(d, ctx):
    rng = _rng(3000)
    y = _rand(rng, 777)
    z, nz = _gpu_mul(d, ctx, np.zeros(1, np.uint32), y)
    assert nz == 1 and not z.any()
    z, nz = _gpu_mul(d, ctx, np.zeros(5000, np.uint32), np.zeros(3, np.uint32))
    assert nz == 1 and not z.any()
    x = _rand(rng, 300)
    xp = np.concatenate([x, np.zeros(1200, np.uint32)])  # leading zero limbs (Sec. 3.2 padding)
    z, nz = _gpu_mul(d, ctx, xp, y)
    ref = oracle.mul(x, y)
    assert nz == len(oracle.normalize(ref))
    assert np.array_equal(z[:len(ref)], ref) and not z[len(ref):].any()


def test_commutative_and_repeatable(d, ctx):
    rng = _rng(3100)
    x, y = _rand(rng, 3333), _rand(rng, 9999)
    a, _ = _gpu_mul(d, ctx, x, y)
    b, _ = _gpu_mul(d, ctx, y, x)
    c, _ = _gpu_mul(d, ctx, x, y)
    assert np.array_equal(a, b) and np.array_equal(a, c)


@pytest.mark.parametrize("n,m", [(1, 1), (100, 924), (3000, 5000), (12288, 1)])
def test_conv_residues(d, ctx, n, m):
    """c_k mod p_i after forward transforms, pointwise product and inverse transforms."""
    rng = _rng(4000 + n)
    x, y = _rand(rng, n), _rand(rng, m)
    r = d.to_host(ctx.conv_residues(d.to_device(x), d.to_device(y))).reshape(3, n + m)
    c = oracle.conv_schoolbook_words(x, y)
    for i, p in enumerate(d.dmul_primes()):
        assert np.array_equal(r[i].astype(np.uint64), oracle.residues(c, p)), p


@pytest.mark.parametrize("n,m", [(1, 1), (2, 2), (1023, 1), (2500, 2600), (11112, 11112)])
def test_conv_coeffs(d, ctx, n, m):
    """exact c_k after CRT: d0 + d1 B + d2 B^2 equals the schoolbook coefficient."""
    rng = _rng(5000 + n)
    for kind in ("rand", "nines"):
        if kind == "rand":
            x, y = _rand(rng, n), _rand(rng, m)
        else:
            x, y = np.full(n, B - 1, np.uint32), np.full(m, B - 1, np.uint32)
        dg = d.to_host(ctx.conv_coeffs(d.to_device(x), d.to_device(y))).reshape(-1, 3).astype(object)
        got = dg[:, 0] + dg[:, 1] * B + dg[:, 2] * B * B
        ref = oracle.conv_schoolbook(x, y)
        assert list(got) == ref
        assert (dg < B).all()


def _triples_from_coeffs(c):
    out = np.zeros((len(c), 3), np.uint32)
    for k, v in enumerate(c):
        out[k] = (v % B, (v // B) % B, v // (B * B))
    return out


@pytest.mark.parametrize("L", [1, 2, 31, 32, 33, 2047, 2048, 2049, 10000, 70001])
def test_carry_adversarial(d, ctx, L):
    """The lookahead carry scan against the sequential recurrence (eq. sigmai_and_zi) on coefficient
    patterns that carry across chunks and tiles: long runs of 10^9-1 digits fed by a single carry,
    near-maximal coefficients, random."""
    rng = _rng(6000 + L)
    for kind in ("run", "max", "rand"):
        if kind == "run":
            c = [B - 1] * L
            c[0] = B - 1 + 1  # one carry ripples through the whole vector ...
            c[-1] = 0  # ... and stops at the top
            if L == 1:
                c = [5]
        elif kind == "max":
            c = [int(v) for v in rng.integers(0, 2**62, size=L)]
            c[-1] = 0
            if L > 1:
                c[-2] = int(rng.integers(0, B))
            if L > 2:
                c[-3] = int(rng.integers(0, B * B // 2))
            if L == 1:
                c = [int(rng.integers(0, B))]
        else:
            c = [int(v) for v in rng.integers(0, B, size=L)]
        tri = _triples_from_coeffs(c)
        z, nz = ctx.carry(d.to_device(tri.reshape(-1)), L)
        words = np.array([[v & (2**64 - 1), v >> 64] for v in c], dtype=np.uint64)
        ref, fin = oracle.carry(words)
        assert fin == 0
        assert np.array_equal(d.to_host(z), ref)
        assert nz == len(oracle.normalize(ref))


@pytest.mark.parametrize("L", [2_097_152, 2_200_001, 4_194_307, 8_400_007])
def test_carry_long(d, ctx, L):
    """Products of millions of limbs take the large carry tiles (8192 limbs; beyond 1024 tiles the
    carry-ins come from a separate scan of the tile maps): a carry rippling through every tile (no
    tile map is constant), runs of 10^9-1 across tile and chunk boundaries, near-maximal
    coefficients."""
    rng = _rng(6100 + L)
    for kind in ("run", "runs", "max", "zero_tail", "zeros"):
        if kind == "run":
            c = np.full(L, B - 1, np.uint64)
            c[0] = B
            c[-1] = 0
        elif kind == "runs":
            c = rng.integers(0, 3 * B, size=L, dtype=np.uint64)
            for start in list(range(8192 - 7, L - 40000, 8192 * 37)) + list(rng.integers(0, L - 40000, 64)):
                ln = int(rng.integers(1, 30000))
                c[int(start):int(start) + ln] = B - 1
                c[int(start)] += int(rng.integers(0, 3))
            c[-2:] = 0
        elif kind == "max":
            c = rng.integers(0, 2**62, size=L, dtype=np.uint64)
            c[-1] = 0
            c[-2] = int(rng.integers(0, B))
            c[-3] = int(rng.integers(0, B * B // 2))
        elif kind == "zero_tail":  # the top 20000 coefficients zero: the normalized length lies below the last tile
            c = rng.integers(0, 3 * B, size=L, dtype=np.uint64)
            c[L - 20000:] = 0
        else:  # a zero product: normalized length 1
            c = np.zeros(L, np.uint64)
        tri = np.stack([c % B, (c // B) % B, c // (B * B)], axis=1).astype(np.uint32)
        z, nz = ctx.carry(d.to_device(tri.reshape(-1)), L)
        words = np.stack([c, np.zeros(L, np.uint64)], axis=1)
        ref, fin = oracle.carry(words)
        assert fin == 0
        assert np.array_equal(d.to_host(z), ref), kind
        assert nz == len(oracle.normalize(ref))


@pytest.mark.parametrize("L", [100, 8192, 2_097_152, 2_097_157])
def test_carry_overflow_flagged_sizes(d, ctx, L):
    """A carry out of the top limb is reported for every tile shape (the top position at a thread's
    last limb, mid-thread, in small and large tiles), and the context stays usable."""
    tri = np.zeros((L, 3), np.uint32)
    tri[L - 1] = (5, 1, 0)  # 5 + 10^9 at the top limb
    t = d.to_device(tri.reshape(-1))
    z = torch.empty(L, dtype=torch.int32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert d.dmul_carry(ctx.handle, t, L, z, L, nz) == 0
    assert d.dmul_sync(ctx.handle) == d.DMUL_ERR_INVALID
    tri[L - 1] = (5, 0, 0)
    zz, n = ctx.carry(d.to_device(tri.reshape(-1)), L)
    assert n == L and int(d.to_host(zz)[L - 1]) == 5


def test_carry_overflow_flagged(d, ctx):
    """A coefficient vector whose value does not fit L limbs is reported, not silently truncated."""
    L = 100
    tri = np.zeros((L, 3), np.uint32)
    tri[L - 1] = (5, 1, 0)  # 5 + 10^9 at the top limb: one limb too many
    t = d.to_device(tri.reshape(-1))
    z = torch.empty(L, dtype=torch.int32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int64, device="cuda")
    assert d.dmul_carry(ctx.handle, t, L, z, L, nz) == 0
    assert d.dmul_sync(ctx.handle) == d.DMUL_ERR_INVALID
    assert d.dmul_sync(ctx.handle) == 0


def test_invalid_limb_flagged(d, ctx):
    rng = _rng(7000)
    x = _rand(rng, 5000)
    x[1234] = B  # not a base-10^9 digit
    tx, ty = d.to_device(x), d.to_device(_rand(rng, 100))
    z = torch.empty(5100, dtype=torch.int32, device="cuda")
    assert d.dmul_mul(ctx.handle, tx, 5000, ty, 100, z, 5100, None) == 0
    assert d.dmul_sync(ctx.handle) == d.DMUL_ERR_INVALID
    # the context stays usable
    x[1234] = B - 1
    zz, nz = _gpu_mul(d, ctx, x, _rand(_rng(7001), 10))


def test_error_survives_first_use_timing(d):
    """A device-side error of an asynchronous call is still reported by the next dmul_sync when a
    later call on the context first times a new length (the autotuners' timing runs keep the
    status word as they found it)."""
    rng = _rng(7050)
    with d.Context(0) as c:
        x = _rand(rng, 5000)
        x[77] = B  # not a base-10^9 digit
        tx, ty = d.to_device(x), d.to_device(_rand(rng, 100))
        z = torch.empty(5100, dtype=torch.int32, device="cuda")
        assert d.dmul_mul(c.handle, tx, 5000, ty, 100, z, 5100, None) == 0
        # new lengths: a short one (fused kernel against four-step) and a long one (split search)
        for n in (6000, 150000):
            a = d.to_device(_rand(rng, n))
            zz = torch.empty(2 * n, dtype=torch.int32, device="cuda")
            assert d.dmul_mul(c.handle, a, n, a, n, zz, 2 * n, None) == 0
        assert d.dmul_sync(c.handle) == d.DMUL_ERR_INVALID
        assert d.dmul_sync(c.handle) == 0  # reported once, then cleared


def test_argument_errors(d, ctx):
    t = d.to_device(np.ones(10, np.uint32))
    z = torch.empty(30, dtype=torch.int32, device="cuda")
    assert d.dmul_mul(ctx.handle, t, 10, t, 10, z, 19, None) == d.DMUL_ERR_CAPACITY
    assert d.dmul_mul(ctx.handle, t, 0, t, 10, z, 30, None) == d.DMUL_ERR_INVALID
    assert d.dmul_mul(ctx.handle, t, 10, t, 10, t, 20, None) == d.DMUL_ERR_INVALID  # z aliases x
    big = 3 * 2**22
    assert d.dmul_mul(ctx.handle, t, big, t, 10, z, big + 10, None) == d.DMUL_ERR_TOO_LARGE
    # transposes: sides multiples of 32, the larger a multiple of the smaller, at most 16384 apart
    for rows, cols in ((64, 96), (96, 64), (32, 32768), (33, 33), (0, 32)):
        assert d.dmul_transpose(ctx.handle, z, rows, cols) == d.DMUL_ERR_INVALID


@pytest.mark.parametrize("n,m", [(7777, 5555), (300000, 250001), (1 << 20, (1 << 20) - 3)])
def test_host_buffer_entry_point(d, ctx, n, m):
    """dmul_mul_host on pageable buffers (staged copies; y's upload overlaps x's forward pass on
    the four-step path), the normalized length and the status word returned with the product."""
    rng = _rng(7100 + n)
    x, y = _rand(rng, n), _rand(rng, m)
    z = np.zeros(len(x) + len(y), np.uint32)
    rc, nz = d.dmul_mul_host(ctx.handle, x, len(x), y, len(y), z, len(z))
    assert rc == 0
    ref = oracle.mul(x, y)
    assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))
    z2 = np.zeros(2 * len(x), np.uint32)
    rc, nz = d.dmul_mul_host(ctx.handle, x, len(x), x, len(x), z2, len(z2))
    assert rc == 0 and np.array_equal(z2, oracle.mul(x, x))
    # an invalid limb is reported through the host entry point, and the context stays usable
    bad = y.copy()
    bad[len(bad) // 2] = B
    rc, _ = d.dmul_mul_host(ctx.handle, x, len(x), bad, len(bad), z, len(z))
    assert rc == d.DMUL_ERR_INVALID
    rc, nz = d.dmul_mul_host(ctx.handle, x, len(x), y, len(y), z, len(z))
    assert rc == 0 and np.array_equal(z, ref)


def _pinned(a):
    t = torch.from_numpy(a.view(np.int32).copy()).pin_memory()
    return t


@pytest.fixture(scope="module")
def ctx_staged(d):
    c = d.Context(0, flags=d.DMUL_FLAG_HOST_STAGED_IN | d.DMUL_FLAG_HOST_STAGED_OUT)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_direct_in(d):
    c = d.Context(0, flags=d.DMUL_FLAG_HOST_DIRECT_IN)
    yield c
    c.close()


@pytest.fixture(scope="module")
def ctx_direct_out(d):
    """A page-locked z written in place by the carry scan at every length."""
    c = d.Context(0, flags=d.DMUL_FLAG_HOST_DIRECT_OUT)
    yield c
    c.close()


@pytest.mark.parametrize("n,m", [(11112, 11112), (7777, 5555), (300000, 250001), (1 << 20, (1 << 20) - 3)])
@pytest.mark.parametrize("kind", ["direct", "direct_in", "direct_out", "staged_flags", "forced_in", "forced_out"])
def test_host_pinned_in_place(d, ctx, ctx_staged, ctx_direct_in, ctx_direct_out, n, m, kind):
    """dmul_mul_host on page-locked buffers: the forward pass reads x and y in place and the carry
    scan writes z and its length in place (short products, or every length by flag), or the staged
    copies (longer products, pageable buffers, flags) -- every combination gives the oracle's
    product."""
    if n >= 1 << 20 and kind in ("direct_in", "direct_out"):
        pytest.skip("the mixed cases run at the smaller sizes")
    rng = _rng(7300 + n + m)
    x, y = _rand(rng, n), _rand(rng, m)
    L = n + m
    pinned_in = ("direct", "direct_in", "staged_flags", "forced_in", "forced_out")
    px = _pinned(x) if kind in pinned_in else x
    py = _pinned(y) if kind in pinned_in else y
    pz = (torch.zeros(L + 3, dtype=torch.int32).pin_memory()
          if kind in ("direct", "direct_out", "staged_flags", "forced_in", "forced_out")
          else np.zeros(L + 3, np.uint32))
    c = {"staged_flags": ctx_staged, "forced_in": ctx_direct_in, "forced_out": ctx_direct_out}.get(kind, ctx)
    assert d.dmul_host_direct(c.handle, px) == (kind != "direct_out")
    assert d.dmul_host_direct(c.handle, pz) == (kind != "direct_in")
    ref = oracle.mul(x, y)
    for _ in range(2):  # the second call reuses the staging / digit buffers
        rc, nz = d.dmul_mul_host(c.handle, px, n, py, m, pz, L + 3)
        assert rc == 0
        zz = pz.numpy().view(np.uint32) if hasattr(pz, "numpy") else pz
        assert np.array_equal(zz[:L], ref) and nz == len(oracle.normalize(ref))
        assert not zz[L:].any()  # nothing written past nx + ny
    # squaring in place
    z2 = torch.zeros(2 * n, dtype=torch.int32).pin_memory()
    rc, nz = d.dmul_mul_host(c.handle, px, n, px, n, z2, 2 * n)
    assert rc == 0 and np.array_equal(z2.numpy().view(np.uint32), oracle.mul(x, x))
    # an invalid limb read in place is reported, and the context stays usable
    bad = y.copy()
    bad[m // 2] = B
    pb = _pinned(bad) if kind in pinned_in else bad
    rc, _ = d.dmul_mul_host(c.handle, px, n, pb, m, pz, L + 3)
    assert rc == d.DMUL_ERR_INVALID
    rc, nz = d.dmul_mul_host(c.handle, px, n, py, m, pz, L + 3)
    zz = pz.numpy().view(np.uint32) if hasattr(pz, "numpy") else pz
    assert rc == 0 and np.array_equal(zz[:L], ref)


@pytest.mark.parametrize("n,m", [(5000, 7001), (1 << 20, 12345)])
def test_host_pinned_unaligned_product(d, ctx_direct_out, n, m):
    """A page-locked z that starts 4 bytes past a 16-byte boundary: the carry scan writes it in
    place word by word (the 16-byte stores need alignment)."""
    ctx = ctx_direct_out
    rng = _rng(7450 + m)
    x, y = _pinned(_rand(rng, n)), _pinned(_rand(rng, m))
    L = n + m
    buf = torch.zeros(L + 4, dtype=torch.int32).pin_memory()
    z = buf[1:L + 1]
    assert z.data_ptr() % 16 == 4 and d.dmul_host_direct(ctx.handle, z)
    rc, nz = d.dmul_mul_host(ctx.handle, x, n, y, m, z, L)
    ref = oracle.mul(x.numpy().view(np.uint32), y.numpy().view(np.uint32))
    assert rc == 0 and np.array_equal(z.numpy().view(np.uint32), ref) and nz == len(oracle.normalize(ref))
    assert buf[0].item() == 0 and buf[L + 1:].abs().sum().item() == 0  # nothing outside z


def test_host_pinned_zero_and_aliasing(d, ctx):
    """In place: a zero product has length 1; z overlapping an operand is rejected."""
    x = _pinned(np.zeros(5000, np.uint32))
    y = _pinned(_rand(_rng(7400), 7000))
    z = torch.full((12000,), -1, dtype=torch.int32).pin_memory()
    rc, nz = d.dmul_mul_host(ctx.handle, x, 5000, y, 7000, z, 12000)
    assert rc == 0 and nz == 1 and not z.numpy().any()
    buf = torch.zeros(30000, dtype=torch.int32).pin_memory()
    xs, zs = buf[:5000], buf[4000:16000]
    rc, _ = d.dmul_mul_host(ctx.handle, xs, 5000, y, 7000, zs, 12000)
    assert rc == d.DMUL_ERR_INVALID


# ---- six-step form (Sec. 7.2) with the in-place transposes of Sec. 7.6 -------------------------
@pytest.mark.parametrize("n,m", [(1, 1), (500, 524), (1000, 1049), (3000, 5000), (11112, 11112),
                                 (40000, 25536), (65536, 65536)])
def test_sixstep_mul(d, ctx6, n, m):
    rng = _rng(8000 + n)
    x, y = _rand(rng, n), _rand(rng, m)
    z, nz = _gpu_mul(d, ctx6, x, y)
    ref = oracle.mul(x, y)
    assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))
    z, nz = _gpu_mul(d, ctx6, x, x, square=True)
    assert np.array_equal(z, oracle.mul(x, x))


@pytest.mark.parametrize("n,m", [(1, 1), (700, 333), (3000, 5000), (40000, 25536)])
def test_sixstep_residues_and_coeffs(d, ctx6, n, m):
    """The six-step form's CRT reads the inverse's transposed tiles: the residues c_k mod p_i and
    the exact coefficients it recovers, against the oracle's schoolbook column sums."""
    rng = _rng(8100 + n)
    x, y = _rand(rng, n), _rand(rng, m)
    c = oracle.conv_schoolbook_words(x, y)
    L = n + m
    tx, ty = d.to_device(x), d.to_device(y)
    r = d.to_host(ctx6.conv_residues(tx, ty)).reshape(3, L)
    for i, p in enumerate(d.dmul_primes()):
        assert np.array_equal(r[i], oracle.residues(c, p).astype(np.uint32)), i
    dg = d.to_host(ctx6.conv_coeffs(tx, ty)).reshape(L, 3).astype(object)
    got = [int(a) + int(b) * 10**9 + int(e) * 10**18 for a, b, e in dg]
    assert got == [int(lo) | (int(hi) << 64) for lo, hi in c]


def test_sixstep_plan_shapes(d, ctx6):
    for L, (n1, n2) in ((1024, (32, 32)), (2048, (32, 64)), (2**21, (1024, 2048)), (2**22, (2048, 2048))):
        info = d.dmul_get_plan(ctx6.handle, L)
        assert (info.N1, info.N2) == (n1, n2) and info.sixstep == 1


@pytest.mark.parametrize("rows,cols", [(32, 32), (64, 64), (32, 64), (64, 32), (96, 96), (256, 512), (512, 256),
                                       (1024, 1024), (1024, 2048), (2048, 1024), (2048, 4096),
                                       (4096, 2048), (4096, 4096),
                                       # n x Cn and Cn x n, C > 2 (the generalization of Sec. 7.6)
                                       (32, 96), (96, 32), (64, 256), (256, 64), (128, 640),
                                       (640, 128), (2048, 8192), (8192, 2048), (32, 16384)])
@pytest.mark.parametrize("aligned", [True, False], ids=["tma", "unaligned"])
def test_inplace_transpose(d, ctx, rows, cols, aligned):
    """In place against the oracle's out-of-place transpose (the definition) and back.  A 16-byte aligned matrix
    takes the tensor-map tile loads (and bulk-copied rows for rho); one offset by a word takes the
    plain kernels."""
    if not aligned and rows * cols > 1 << 22:
        pytest.skip("the plain kernels are covered at the smaller sizes")
    rng = _rng(9000 + rows + cols)
    a = rng.integers(0, 2**32, size=rows * cols, dtype=np.uint64).astype(np.uint32)
    buf = torch.zeros(rows * cols + 4, dtype=torch.int32, device="cuda")
    t = buf[0:rows * cols] if aligned else buf[1:1 + rows * cols]
    t.copy_(d.to_device(a))
    ctx.transpose_(t, rows, cols)
    assert np.array_equal(d.to_host(t), oracle.transpose(a, rows, cols))
    ctx.transpose_(t, cols, rows)  # and back
    assert np.array_equal(d.to_host(t), a)
    assert int(buf[-1].item()) == 0 and (aligned or int(buf[0].item()) == 0)  # nothing outside


def test_c1_workload(d, ctx):
    """One multiplication of two 100,000-digit operands against the schoolbook oracle."""
    x, y = wl.c1_pair()
    z, nz = _gpu_mul(d, ctx, x, y)
    ref = oracle.mul_schoolbook(x, y)
    assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))


# ---- short products as one cooperative launch (N = N1 x 256, N1 in {64, 80, 96}) ----------------
@pytest.fixture(scope="module")
def ctx_fused(d):
    """Short products of N = 16384, 20480 and 24576 through the cooperative one-launch kernel (no
    first-use timing, the one-cluster kernel off), with stage timing to see which path ran."""
    c = d.Context(0, flags=d.DMUL_FLAG_NO_SMALL | d.DMUL_FLAG_NO_AUTOTUNE | d.DMUL_FLAG_STAGE_TIMING)
    yield c
    c.close()


# (n, m) with their transform lengths: full and ragged, balanced and unbalanced, one-limb operands
FUSED_SHAPES = [(8192, 8192), (7001, 8000), (16383, 1), (1, 16000), (12289 - 4000, 4000),
                (10240, 10240), (9000, 11480), (20480 - 1, 1),
                (11112, 11112), (12288, 12288), (24575, 1), (3, 24573), (12000, 12001)]


def _fused_launches(ctx):
    return ctx.stage_times().get("short_fused", (0.0, 0))[1]


@pytest.mark.parametrize("n,m", FUSED_SHAPES)
def test_fused_short_product(d, ctx_fused, n, m):
    L = n + m
    assert d.dmul_get_plan(ctx_fused.handle, L).N in (16384, 20480, 24576)
    rng = _rng(12000 + n + 3 * m)
    x, y = _rand(rng, n), _rand(rng, m)
    _fused_launches(ctx_fused)
    for square in (False, True):
        z, nz = _gpu_mul(d, ctx_fused, x, x if square else y, square=square)
        ref = oracle.mul(x, x) if square else oracle.mul(x, y)
        assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))
    # the square has length 2n: fused only when that length is one of the three
    expect = 1 + (d.dmul_get_plan(ctx_fused.handle, 2 * n).N in (16384, 20480, 24576))
    assert _fused_launches(ctx_fused) == expect


def test_fused_worst_case_and_zero(d, ctx_fused):
    """All-nines operands (the largest convolution coefficients: the prime-product bound) against
    the closed form, a zero operand, leading zero limbs, and the overflow-free top limb."""
    for h in (8192, 10240, 12288):
        nines = np.full(h, B - 1, np.uint32)
        z, nz = _gpu_mul(d, ctx_fused, nines, nines, square=True)
        expect = np.zeros(2 * h, np.uint32)
        expect[0] = 1
        expect[h] = B - 2
        expect[h + 1:] = B - 1
        assert np.array_equal(z, expect) and nz == 2 * h
    rng = _rng(12500)
    x = _rand(rng, 9000)
    zero = np.zeros(7000, np.uint32)
    z, nz = _gpu_mul(d, ctx_fused, x, zero)
    assert not z.any() and nz == 1
    y = _rand(rng, 7000)
    y[-500:] = 0  # leading zero limbs
    z, nz = _gpu_mul(d, ctx_fused, x, y)
    ref = oracle.mul(x, y)
    assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))
    assert _fused_launches(ctx_fused) == 5


def test_fused_back_to_back(d, ctx_fused):
    """Forty launches queued without a synchronization in between (the grid barrier word carries
    over from launch to launch): every product against the oracle."""
    rng = _rng(12600)
    pairs = [(_rand(rng, int(n)), _rand(rng, int(m)))
             for n, m in zip(rng.integers(6145, 12289, 40), rng.integers(6145, 12288, 40))]
    outs = []
    for x, y in pairs:
        tx, ty = d.to_device(x), d.to_device(y)
        outs.append((tx, ty) + ctx_fused.mul(tx, ty, sync=False))
    ctx_fused.sync()
    for (x, y), (_, _, z, nz) in zip(pairs, outs):
        ref = oracle.mul(x, y)
        assert np.array_equal(d.to_host(z), ref) and int(nz.item()) == len(oracle.normalize(ref))
    assert _fused_launches(ctx_fused) == 40


def test_fused_invalid_limb_flagged(d, ctx_fused):
    """A limb >= 10^9 makes dmul_sync report DMUL_ERR_INVALID, and the context stays usable."""
    rng = _rng(12700)
    x, y = _rand(rng, 8000), _rand(rng, 8000)
    bad = x.copy()
    bad[4321] = B
    with pytest.raises(d.DmulError) as e:
        _gpu_mul(d, ctx_fused, bad, y)
    assert e.value.status == d.DMUL_ERR_INVALID
    z, nz = _gpu_mul(d, ctx_fused, x, y)
    assert np.array_equal(z, oracle.mul(x, y))


def test_fused_unaligned_takes_pipeline(d, ctx_fused):
    """Operands that are not 16-byte aligned take the four-kernel pipeline (same limbs)."""
    rng = _rng(12800)
    x, y = _rand(rng, 9000), _rand(rng, 9001)
    buf = torch.zeros(9000 + 9001 + 8, dtype=torch.int32, device="cuda")
    tx = buf[1:9001]
    ty = buf[9003:9003 + 9001]
    tx.copy_(d.to_device(x))
    ty.copy_(d.to_device(y))
    _fused_launches(ctx_fused)
    z, nz = ctx_fused.mul(tx, ty)
    assert np.array_equal(d.to_host(z), oracle.mul(x, y))
    t = ctx_fused.stage_times()
    assert "short_fused" not in t and t["carry_scan"][1] == 1


def test_fused_short_waits(d):
    """With every device-side wait bounded by 2^13 polls, the cooperative kernel's grid barriers
    and carry look-back still complete: no spurious timeout, the products equal the oracle."""
    with d.Context(0, flags=d.DMUL_FLAG_NO_SMALL | d.DMUL_FLAG_NO_AUTOTUNE | d.DMUL_FLAG_SHORT_WAITS |
                   d.DMUL_FLAG_STAGE_TIMING) as c:
        rng = _rng(12950)
        for n, m in [(8192, 8192), (10000, 10480), (12288, 12288)]:
            x, y = _rand(rng, n), _rand(rng, m)
            z, nz = _gpu_mul(d, c, x, y)
            ref = oracle.mul(x, y)
            assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))
        assert c.stage_times()["short_fused"][1] == 3


def test_fused_matches_other_paths(d, ctx, ctx4):
    """The same products through the default (timed) context and the four-kernel pipeline are
    bit-identical with the oracle; the timed choice may be any of the three paths."""
    rng = _rng(12900)
    for n, m in [(11112, 11112), (8192, 8000), (10000, 10480)]:
        x, y = _rand(rng, n), _rand(rng, m)
        ref = oracle.mul(x, y)
        for c in (ctx, ctx4):
            z, nz = _gpu_mul(d, c, x, y)
            assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))


# ---- the plain form inside a CUDA graph --------------------------------------------------------
@pytest.mark.parametrize("n,m", [(3000, 4000), (11112, 11112), (300000, 250001), (1 << 20, (1 << 20) - 3)])
def test_plain_form_in_cuda_graph(d, ctx, n, m):
    """dmul_mul captured into a CUDA graph after one product of the same lengths outside the
    capture; three replays on new operands each equal the oracle, and nz follows."""
    rng = _rng(13000 + n + m)
    L = n + m
    tx, ty = d.to_device(_rand(rng, n)), d.to_device(_rand(rng, m))
    z = torch.empty(L, dtype=torch.int32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    assert d.dmul_mul(ctx.handle, tx, n, ty, m, z, L, nz, s.cuda_stream) == 0  # plans the lengths
    assert d.dmul_sync(ctx.handle, s.cuda_stream) == 0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = d.dmul_mul(ctx.handle, tx, n, ty, m, z, L, nz, s.cuda_stream)
    assert rc == 0
    for k in range(3):
        x, y = _rand(rng, n), _rand(rng, m)
        if k == 2:
            y[m // 2:] = 0  # a shorter normalized length
        tx.copy_(d.to_device(x))
        ty.copy_(d.to_device(y))
        g.replay()
        torch.cuda.synchronize()
        ref = oracle.mul(x, y)
        assert np.array_equal(d.to_host(z), ref) and int(nz.item()) == len(oracle.normalize(ref))
    assert d.dmul_sync(ctx.handle) == 0


@pytest.mark.parametrize("form", ["square", "sixstep"])
def test_graph_square_and_sixstep(d, ctx, ctx6, form):
    """A captured squaring (one forward transform) and a captured six-step product (packing
    transpose, row DFTs, in-place transposes, transposed CRT) replay exactly on new operands."""
    c = ctx6 if form == "sixstep" else ctx
    n, m = (70000, 70000) if form == "square" else (300000, 250001)
    rng = _rng(13050 + n)
    L = n + m
    tx = d.to_device(_rand(rng, n))
    ty = tx if form == "square" else d.to_device(_rand(rng, m))
    z = torch.empty(L, dtype=torch.int32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.Stream()
    call = (lambda: d.dmul_sqr(c.handle, tx, n, z, L, nz, s.cuda_stream)) if form == "square" else \
        (lambda: d.dmul_mul(c.handle, tx, n, ty, m, z, L, nz, s.cuda_stream))
    assert call() == 0
    assert d.dmul_sync(c.handle, s.cuda_stream) == 0
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        rc = call()
    assert rc == 0
    for _ in range(2):
        x = _rand(rng, n)
        tx.copy_(d.to_device(x))
        if form == "square":
            y = x
        else:
            y = _rand(rng, m)
            ty.copy_(d.to_device(y))
        g.replay()
        torch.cuda.synchronize()
        ref = oracle.mul(x, y)
        assert np.array_equal(d.to_host(z), ref) and int(nz.item()) == len(oracle.normalize(ref))
    assert d.dmul_sync(c.handle) == 0


def test_unplanned_length_refused_in_capture(d):
    """Inside a capture a product whose lengths this context has not planned is refused with
    DMUL_ERR_INVALID and enqueues nothing; the capture itself stays valid."""
    with d.Context(0) as c:
        rng = _rng(13100)
        tx, ty = d.to_device(_rand(rng, 70000)), d.to_device(_rand(rng, 70001))
        z = torch.zeros(140001, dtype=torch.int32, device="cuda")
        nz = torch.zeros(1, dtype=torch.int64, device="cuda")
        s = torch.cuda.Stream()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            rc = d.dmul_mul(c.handle, tx, 70000, ty, 70001, z, 140001, nz, s.cuda_stream)
            nz.add_(5)  # something to capture
        assert rc == d.DMUL_ERR_INVALID
        g.replay()
        torch.cuda.synchronize()
        assert int(nz.item()) == 5 and not z.any().item()
        # outside the capture the same call plans the lengths and multiplies
        zz, n_ = c.mul(tx, ty)
        ref = oracle.mul(d.to_host(tx), d.to_host(ty))
        assert np.array_equal(d.to_host(zz), ref)


# ---- compile-time specialized column passes (N1 = 2^a, 3 2^a, 5 2^a from 64 to 1536) -----------
@pytest.fixture(scope="module")
def ctx_def(d):
    """Four-step path with the planner's default split and the one-CTA-per-row pass."""
    c = d.Context(0, flags=d.DMUL_FLAG_NO_SMALL | d.DMUL_FLAG_NO_FUSED | d.DMUL_FLAG_NO_AUTOTUNE)
    yield c
    c.close()


# (n, m) whose transform length gets the default split N1 x N2 with the given N1
SPECIALIZED_COLS = [((3000, 3000), 96, 64),           # N = 3 * 2^11
                    ((4000, 4001), 64, 128),          # N = 2^13
                    ((8000, 8000), 128, 128),         # N = 2^14
                    ((12000, 12000), 192, 128),       # N = 3 * 2^13
                    ((16000, 12001), 128, 256),       # N = 2^15 (row pass specialized too)
                    ((25000, 20000), 384, 128),       # N = 3 * 2^14
                    ((33000, 32000), 256, 256),       # N = 2^16 (row pass specialized too)
                    ((50001, 45000), 384, 256),       # N = 3 * 2^15 (row pass specialized too)
                    ((180000, 180000), 768, 512),     # N = 3 * 2^17 (row pass specialized too)
                    ((262143, 200000), 512, 1024),    # N = 2^19
                    ((350000, 349999), 1536, 512),    # N = 3 * 2^18
                    ((524287, 400003), 1024, 1024),   # N = 2^20
                    ((1300, 1200), 80, 32),           # N = 5 * 2^9 (radix 5 first)
                    ((2600, 2500), 160, 32),          # N = 5 * 2^10
                    ((10000, 10000), 320, 64),        # N = 5 * 2^12
                    ((40000, 40000), 640, 128),       # N = 5 * 2^14
                    ((80001, 80000), 640, 256),       # N = 5 * 2^15 (row pass specialized too)
                    ((330000, 320000), 1280, 512)]    # N = 5 * 2^17


@pytest.fixture(scope="module")
def ctx_half(d):
    """As ctx_def, with the column passes on N1 x 16 half tiles (six-CTA CRT clusters)."""
    c = d.Context(0, flags=d.DMUL_FLAG_NO_SMALL | d.DMUL_FLAG_NO_FUSED | d.DMUL_FLAG_NO_AUTOTUNE |
                  d.DMUL_FLAG_COL_HALF)
    yield c
    c.close()


@pytest.mark.parametrize("half", [False, True], ids=["full_tiles", "half_tiles"])
@pytest.mark.parametrize("shape,n1,n2", SPECIALIZED_COLS)
def test_specialized_column_pass(d, request, half, shape, n1, n2):
    ctx_def = request.getfixturevalue("ctx_half" if half else "ctx_def")
    n, m = shape
    info = d.dmul_get_plan(ctx_def.handle, n + m)
    assert (info.N1, info.N2, info.col_half) == (n1, n2, int(half))
    rng = _rng(11000 + n1)
    x, y = _rand(rng, n), _rand(rng, m)
    for square in (False, True):
        z, nz = _gpu_mul(d, ctx_def, x, x if square else y, square=square)
        ref = oracle.mul(x, x) if square else oracle.mul(x, y)
        assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))
    # the inverse pass's other epilogues: residues and exact coefficients at sampled positions
    L = n + m
    ks = [0, 1, 31, 32, n - 1, n, m, L // 2, L - 3, L - 2, L - 1] + list(rng.integers(0, L - 1, 24))
    tx, ty = d.to_device(x), d.to_device(y)
    r = d.to_host(ctx_def.conv_residues(tx, ty)).reshape(3, L).astype(np.uint64)
    dg = d.to_host(ctx_def.conv_coeffs(tx, ty)).reshape(-1, 3).astype(object)
    primes = d.dmul_primes()
    for k in ks:
        k = int(k)
        c = oracle.conv_at(x, y, k)
        assert dg[k, 0] + dg[k, 1] * B + dg[k, 2] * B * B == c, k
        assert [int(r[i, k]) for i in range(3)] == [c % p for p in primes], k



@pytest.mark.parametrize("n,m", [(2097153, 2097152), (4194000, 1000)])
def test_five_length_long(d, ctx, n, m):
    """Long products on N = 5 2^k (here 5 2^20 = 5242880, split 1280 x 4096 or as autotuned):
    bit-exact against the oracle, plus the squaring's closed form on all-nines operands."""
    info = d.dmul_get_plan(ctx.handle, n + m)
    assert info.N == 5 * 2**20
    rng = _rng(11500 + m)
    x, y = _rand(rng, n), _rand(rng, m)
    z, nz = _gpu_mul(d, ctx, x, y)
    ref = oracle.mul(x, y)
    assert np.array_equal(z, ref) and nz == len(oracle.normalize(ref))
    # (10^(9h) - 1)^2 = 10^(18h) - 2 10^(9h) + 1 for h limbs of nines
    h = (n + m) // 2
    nines = np.full(h, B - 1, np.uint32)
    z2, nz2 = _gpu_mul(d, ctx, nines, nines, square=True)
    expect = np.zeros(2 * h, np.uint32)
    expect[0] = 1
    expect[h] = B - 2
    expect[h + 1:] = B - 1
    assert np.array_equal(z2, expect) and nz2 == 2 * h
