"""The prime-width probe (two 62-bit primes in 64-bit words, the paper's l = 2 design of Sec. 4.2):
its row pass computes exact cyclic convolutions (checked against the oracle's independent
radix-2 route with plain % on 128-bit products), and the timing entry point runs."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def d():
    from paper_2011_11524_gb300 import build as dbuild
    from paper_2011_11524_gb300 import dmul
    dbuild.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return dmul


def test_probe64_rows_are_cyclic_convolutions(d):
    primes = d.dmul_probe64_primes()
    rows, n = 3, 4096
    rng = np.random.Generator(np.random.PCG64(640))
    a = np.zeros((2, rows, n), dtype=np.uint64)
    b = np.zeros((2, rows, n), dtype=np.uint64)
    for i, p in enumerate(primes):
        a[i] = rng.integers(0, p, size=(rows, n), dtype=np.uint64)
        b[i] = rng.integers(0, p, size=(rows, n), dtype=np.uint64)
    # edge rows: all p - 1, and a delta (the convolution is then a cyclic shift of b)
    a[:, 1, :] = np.array(primes, dtype=np.uint64)[:, None] - 1
    a[:, 2, :] = 0
    a[:, 2, 5] = 1
    ta = torch.from_numpy(a.view(np.int64).reshape(-1)).cuda()
    tb = torch.from_numpy(b.view(np.int64).reshape(-1)).cuda()
    out = torch.zeros_like(ta)
    with d.Context(0) as ctx:
        assert d.dmul_probe64_conv(ctx.handle, ta, tb, out, rows) == d.DMUL_OK
    got = out.cpu().numpy().view(np.uint64).reshape(2, rows, n)
    for i, p in enumerate(primes):
        for r in range(rows):
            ref = oracle.cyclic_conv_mod(a[i, r], b[i, r], p)
            assert np.array_equal(got[i, r], ref), (i, r)
        assert np.array_equal(got[i, 2], np.roll(b[i, 2], 5))


def test_prime_width_probe_times_both(d):
    with d.Context(0) as ctx:
        ms64, ms32 = d.dmul_probe_prime_width(ctx.handle, 1 << 20)
        assert ms64 > 0 and ms32 > 0
        assert d.dmul_sync(ctx.handle) == d.DMUL_OK
