"""Failure detection and admission control, tested without faulting the GPU.

- A bounded device-side wait made to run out: the carry scan's tile ticket starts at 1 (fault
  injection on the host side, DMUL_FLAG_TEST_STALL_CARRY), so tile 0 never runs and tile 1's
  look-back waits for a flag that nothing sets.  With DMUL_FLAG_SHORT_WAITS the wait expires after
  a few milliseconds; the kernel ends normally, dmul_sync reports DMUL_ERR_TIMEOUT promptly, and
  the same context then multiplies correctly.
- HBM-budget admission of the serving loop: a request whose scratch exceeds the admission budget
  is refused at submission with DMUL_ERR_NOMEM, and a budget that fits one request at a time
  drains a queue of 20 with every product right and never two on the GPU at once.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2011_11524_gb300 import workloads as wl

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


def _fp_moduli(count=4):
    out = []
    for q in wl.fingerprint_candidates():
        if oracle.is_prime_mr(q):
            out.append(q)
            if len(out) == count:
                return out


def test_expired_wait_reports_timeout_and_context_recovers(d):
    flags = d.DMUL_FLAG_SHORT_WAITS | d.DMUL_FLAG_TEST_STALL_CARRY
    rng = np.random.Generator(np.random.PCG64(71))
    with d.Context(0, flags=flags) as ctx:
        L = 100_003  # 49 carry tiles of 2048 limbs
        tri = rng.integers(0, B, size=(L, 3), dtype=np.uint64).astype(np.uint32)
        tri[L - 1] = 0
        tri[L - 2, 1:] = 0
        tri[L - 3, 2] = 0
        dt = d.to_device(tri.reshape(-1))
        z = torch.zeros(L, dtype=torch.int32, device="cuda")
        nz = torch.zeros(1, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        assert d.dmul_carry(ctx.handle, dt, L, z, L, nz) == d.DMUL_OK
        assert d.dmul_sync(ctx.handle) == d.DMUL_ERR_TIMEOUT
        assert time.perf_counter() - t0 < 2.0
        # the status was cleared by that sync, and the context still computes exact products
        assert d.dmul_sync(ctx.handle) == d.DMUL_OK
        for n, m in ((11112, 11112), (300_000, 250_001)):
            x = wl.random_operand(9 * n, rng)
            y = wl.random_operand(9 * m, rng)
            zz, nzz = ctx.mul(d.to_device(x), d.to_device(y))
            ref = oracle.mul(x, y)
            assert np.array_equal(d.to_host(zz), ref)
            assert nzz == len(oracle.normalize(ref))
        assert d.dmul_sync(ctx.handle) == d.DMUL_OK


def _served_jobs(d, n, digits, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    host, dev = [], []
    for _ in range(n):
        x = wl.random_operand(digits, rng)
        y = wl.random_operand(digits, rng)
        tx, ty = d.to_device(x), d.to_device(y)
        L = len(x) + len(y)
        z = torch.full((L,), -1, dtype=torch.int32, device="cuda")
        nz = torch.zeros(1, dtype=torch.int64, device="cuda")
        host.append((x, y))
        dev.append((tx, len(x), ty, len(y), z, L, nz))
    return host, dev


def test_admission_by_hbm_budget(d):
    """Requests of 10^7 digits need about 63 MB of scratch each (two residue buffers of
    3 x 4 x 5 2^19 bytes).  A context whose budget leaves room for one of them at a time:
    a larger request is refused at submission, and 20 queued ones drain one by one, exact."""
    digits = 10_000_000
    host, dev = _served_jobs(d, 20, digits, 72)
    budget = 170 << 20
    with d.Context(0, hbm_budget_bytes=budget) as srv:
        # the plan of this length (twiddle tables, autotuned split) is built first, through the plain
        # form, so that the serving loop's admission budget is what the context leaves after it
        tx, nx, ty, ny, z, L, nz = dev[0]
        assert d.dmul_mul(srv.handle, tx, nx, ty, ny, z, L, nz) == 0
        assert d.dmul_sync(srv.handle) == 0
        ref0 = d.to_host(z).copy()
        # a product of two 2 10^7-digit operands needs twice the scratch: refused at once
        rng = np.random.Generator(np.random.PCG64(73))
        bx = d.to_device(wl.random_operand(2 * digits, rng))
        by = d.to_device(wl.random_operand(2 * digits, rng))
        bz = torch.zeros(2 * len(bx), dtype=torch.int32, device="cuda")
        big = d.make_jobs([(bx, len(bx), by, len(by), bz, len(bz), None)])
        assert d.dmul_submit(srv.handle, big[0])[0] == d.DMUL_ERR_NOMEM
        st = d.dmul_serve_stats(srv.handle)
        admit = st["admit_budget_bytes"]
        per = 2 * 3 * 4 * 5 * (1 << 19)
        assert per <= admit < 2 * per, (admit, per)
        arr = d.make_jobs(dev)
        tickets = [d.dmul_submit(srv.handle, arr[i]) for i in range(len(dev))]
        assert all(rc == 0 for rc, _ in tickets)
        for rc, t in tickets:
            assert d.dmul_wait(srv.handle, t) == 0
        st = d.dmul_serve_stats(srv.handle)
        assert st["peak_running"] == 1
        assert st["held"] == 0
    assert np.array_equal(d.to_host(dev[0][4]), ref0)
    qs = _fp_moduli()
    fx = oracle.fingerprint_many([h[0] for h in host], qs)
    fy = oracle.fingerprint_many([h[1] for h in host], qs)
    fz = oracle.fingerprint_many([d.to_host(v[4]) for v in dev], qs)
    for i in range(len(dev)):
        for j, q in enumerate(qs):
            assert int(fz[i, j]) == int(fx[i, j]) * int(fy[i, j]) % q
    # and one of them in full against the oracle's slow NTT route
    assert np.array_equal(d.to_host(dev[5][4]), oracle.mul_ntt(host[5][0], host[5][1]))
