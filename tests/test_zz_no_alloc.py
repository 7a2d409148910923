"""dmul_carry_noalloc against dmul_carry and the oracle.

dmul_carry_noalloc is the carry stage for callers that cannot allocate device memory (their GPU
memory belongs to another allocator, or cudaMalloc's device-wide synchronization is not allowed on
their path, or they cannot create a context).  It must give exactly the limbs and length that
dmul_carry gives, and that the oracle's carry recurrence gives, call after call, although every
call reuses the same static scratch array -- including at the largest size that array holds,
where the carry runs on its 8192-limb tiles.

This file is collected last so that a run stopping at the first failure has run everything else;
it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle

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
    torch.cuda.set_device(0)
    return dmul


def _triples(rng, L, kind):
    t = rng.integers(0, B, size=(L, 3), dtype=np.uint64).astype(np.uint32)
    if kind == "ripple":  # one carry that runs through a long stretch of 10^9 - 1 digits
        t[:] = 0
        t[:, 0] = B - 1
        t[0] = (B - 1, 1, 0)
    t[L - 1] = 0  # the top coefficient of a product is 0 ...
    if L > 1:
        t[L - 2, 1:] = 0  # ... and the one below it is < 10^9, so the sum fits L limbs
    if L > 2:
        t[L - 3, 2] = 0
    return t


def _with_existing(d, ctx, tri, L):
    z, nz = ctx.carry(d.to_device(tri.reshape(-1)), L)
    return d.to_host(z), nz


def _with_noalloc(d, tri, L):
    dt = d.to_device(tri.reshape(-1))
    z = torch.full((L,), -1, dtype=torch.int32, device="cuda")
    nz = torch.full((1,), -1, dtype=torch.int64, device="cuda")
    rc = d.dmul_carry_noalloc(dt, L, z, L, nz, torch.cuda.current_stream().cuda_stream)
    assert rc == d.DMUL_OK
    torch.cuda.synchronize()
    return d.to_host(z), int(nz.item())


def _with_oracle(tri, L):
    """The carry recurrence of the oracle on the same sum: sum_k (d0_k + d1_k B + d2_k B^2) B^k
    regrouped by power of B (c'_k = d0_k + d1_(k-1) + d2_(k-2) < 3 10^9), two extra positions for
    the terms past L, which must carry nothing."""
    t = tri.astype(np.uint64)
    c = np.zeros(L + 2, dtype=np.uint64)
    c[:L] += t[:, 0]
    c[1:L + 1] += t[:, 1]
    c[2:L + 2] += t[:, 2]
    words = np.zeros((L + 2, 2), dtype=np.uint64)
    words[:, 0] = c
    z, top = oracle.carry(words)
    assert top == 0 and z[L] == 0 and z[L + 1] == 0
    return z[:L], len(oracle.normalize(z[:L]))


@pytest.mark.parametrize("cases", [((70001, "random"), (4099, "ripple")),
                                   (((1 << 22) - 5, "random"), (1 << 22, "ripple"))],
                         ids=["short", "max_size"])
def test_noalloc_matches_dmul_carry_and_oracle_twice(d, cases):
    """Two calls in a row on the shared static scratch (the second overwrites the first's), each
    equal to dmul_carry and to the oracle, limbs and normalized length.  The max_size case runs at
    L = 2^22 - 5 and at the array's limit L = 2^22 (8192-limb tiles), the second with a carry
    that ripples from position 1 through every tile to the top limb."""
    assert d.DMUL_NOALLOC_MAX_LIMBS == 1 << 22
    rng = np.random.Generator(np.random.PCG64(2024))
    with d.Context(0) as ctx:
        for L, kind in cases:
            tri = _triples(rng, L, kind)
            ref_z, ref_nz = _with_existing(d, ctx, tri, L)
            or_z, or_nz = _with_oracle(tri, L)
            got_z, got_nz = _with_noalloc(d, tri, L)
            assert np.array_equal(got_z, or_z)
            assert got_nz == or_nz
            assert np.array_equal(got_z, ref_z)
            assert got_nz == ref_nz
            if kind == "ripple":
                assert got_z[L - 1] == 1 and np.all(got_z[1:L - 1] == 0)


def test_noalloc_limits_and_errors(d):
    L = 64
    t = torch.zeros(3 * L, dtype=torch.int32, device="cuda")
    z = torch.zeros(L, dtype=torch.int32, device="cuda")
    nz = torch.zeros(1, dtype=torch.int64, device="cuda")
    big = d.DMUL_NOALLOC_MAX_LIMBS + 1
    # rejected on the host before any GPU work: the pointers are never read
    assert d.dmul_carry_noalloc(t, big, z, big, nz) == d.DMUL_ERR_TOO_LARGE
    assert d.dmul_carry_noalloc(t, L, z, L - 1, nz) == d.DMUL_ERR_CAPACITY
    # a sum that does not fit L limbs is reported through *nz = 0
    tri = np.zeros((L, 3), np.uint32)
    tri[L - 1] = (5, 1, 0)
    dt = d.to_device(tri.reshape(-1))
    assert d.dmul_carry_noalloc(dt, L, z, L, nz) == d.DMUL_OK
    torch.cuda.synchronize()
    assert int(nz.item()) == 0
