"""Batched and served forms: every product bit-exact against the oracle, and identical to the
same product computed alone through the plain form."""
import threading

import numpy as np
import pytest

import oracle
from paper_2011_11524_gb300 import workloads as wl

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def _prep(d, jobs):
    dev = []
    for j in jobs:
        tx = d.to_device(j.x)
        ty = tx if j.square else d.to_device(j.y)
        L = len(j.x) + len(j.y)
        z = torch.full((L,), -1, dtype=torch.int32, device="cuda")
        nz = torch.zeros(1, dtype=torch.int64, device="cuda")
        dev.append((tx, len(j.x), ty, len(j.y), z, L, nz))
    return dev


def _check(d, jobs, dev):
    for j, (tx, nx, ty, ny, z, L, nz) in zip(jobs, dev):
        ref = oracle.mul(j.x, j.y)
        got = d.to_host(z)
        assert np.array_equal(got, ref)
        assert int(nz.item()) == len(oracle.normalize(ref))


@pytest.mark.parametrize("lo,hi,count,seed", [(2.0, 4.5, 300, 11), (3.0, 5.3, 120, 12)])
def test_batch_vs_oracle(d, ctx, lo, hi, count, seed):
    """Uneven sizes (log-uniform digits), 20% squarings, small and four-step jobs in one batch."""
    jobs = wl.c4_jobs(count, lo, hi, 0.2, seed=seed)
    dev = _prep(d, jobs)
    arr = d.make_jobs(dev)
    assert d.dmul_batch(ctx.handle, arr, len(dev)) == 0
    assert d.dmul_sync(ctx.handle) == 0
    _check(d, jobs, dev)


def test_batch_graph_replay_new_data(d, ctx):
    """The same batch shape twice: the second call replays the captured graph with new operands."""
    jobs1 = wl.c4_jobs(64, 2.5, 4.8, 0.25, seed=21)
    # same sizes and squaring pattern, different digits
    rng = np.random.Generator(np.random.PCG64(22))
    jobs2 = []
    for j in jobs1:
        x = rng.integers(0, 10**9, size=len(j.x), dtype=np.uint64).astype(np.uint32)
        x[-1] = max(1, int(x[-1]))
        if j.square:
            jobs2.append(wl.Job(x, x, True))
        else:
            y = rng.integers(0, 10**9, size=len(j.y), dtype=np.uint64).astype(np.uint32)
            y[-1] = max(1, int(y[-1]))
            jobs2.append(wl.Job(x, y, False))
    for jobs in (jobs1, jobs2, jobs1):
        dev = _prep(d, jobs)
        assert d.dmul_batch(ctx.handle, d.make_jobs(dev), len(dev)) == 0
        assert d.dmul_sync(ctx.handle) == 0
        _check(d, jobs, dev)


def test_batch_same_as_alone(d, ctx):
    jobs = wl.c4_jobs(40, 3.0, 5.6, 0.2, seed=31)
    dev = _prep(d, jobs)
    assert d.dmul_batch(ctx.handle, d.make_jobs(dev), len(dev)) == 0
    assert d.dmul_sync(ctx.handle) == 0
    for j, (tx, nx, ty, ny, z, L, nz) in zip(jobs, dev):
        alone, nza = ctx.mul(tx, ty)
        assert torch.equal(alone, z) and nza == int(nz.item())


def test_batch_rejects_bad_job_alone(d, ctx):
    """A job the host checks reject gets its own code at once and is not run; the others run."""
    jobs = wl.c4_jobs(3, 2.0, 3.0, 0.0, seed=41)
    dev = _prep(d, jobs)
    tx, nx, ty, ny, z, L, nz = dev[1]
    dev[1] = (tx, nx, ty, ny, z, L - 1, nz)  # capacity too small
    arr = d.make_jobs(dev)
    assert d.dmul_batch(ctx.handle, arr, len(dev)) == d.DMUL_OK
    st = d.job_statuses(arr, 3)
    assert st == [d.DMUL_PENDING, d.DMUL_ERR_CAPACITY, d.DMUL_PENDING]
    assert d.dmul_sync(ctx.handle) == d.DMUL_OK
    assert d.job_statuses(arr, 3) == [d.DMUL_OK, d.DMUL_ERR_CAPACITY, d.DMUL_OK]
    assert torch.all(dev[1][4] == -1)  # never written
    _check(d, [jobs[0], jobs[2]], [dev[0], dev[2]])


def _with_bad_limb(jobs, where, rng):
    """A copy of jobs[where] whose x has one limb equal to 10^9 (an invalid base-10^9 limb)."""
    j = jobs[where]
    x = j.x.copy()
    x[int(rng.integers(0, len(x)))] = 10**9
    return wl.Job(x, x if j.square else j.y, j.square)


@pytest.mark.parametrize("bad_kind", ["short", "four_step"])
def test_batch_bad_limb_fails_only_its_job(d, ctx, bad_kind):
    """50 valid jobs and one with a limb = 10^9 in one dmul_batch: only that job reports
    DMUL_ERR_INVALID; the 50 match the oracle and their products computed alone."""
    rng = np.random.Generator(np.random.PCG64(42))
    jobs = wl.c4_jobs(50, 2.0, 5.0, 0.2, seed=43)
    lo, hi = (2.0, 3.0) if bad_kind == "short" else (5.2, 5.4)
    extra = wl.c4_jobs(1, lo, hi, 0.0, seed=44)
    bad = _with_bad_limb(extra, 0, rng)
    where = 17
    jobs = jobs[:where] + [bad] + jobs[where:]
    dev = _prep(d, jobs)
    arr = d.make_jobs(dev)
    assert d.dmul_batch(ctx.handle, arr, len(dev)) == d.DMUL_OK
    assert d.dmul_sync(ctx.handle) == d.DMUL_ERR_INVALID
    st = d.job_statuses(arr, len(dev))
    assert st[where] == d.DMUL_ERR_INVALID
    assert all(v == d.DMUL_OK for i, v in enumerate(st) if i != where)
    good = [i for i in range(len(jobs)) if i != where]
    _check(d, [jobs[i] for i in good], [dev[i] for i in good])
    for i in good:
        tx, nx, ty, ny, z, L, nz = dev[i]
        alone, nza = ctx.mul(tx, ty)
        assert torch.equal(alone, z) and nza == int(nz.item())
    # the next sync is clean again
    assert d.dmul_sync(ctx.handle) == d.DMUL_OK


def test_served_bad_request_fails_only_itself(d):
    """50 valid requests and one with a limb = 10^9, submitted together into the serving loop: each
    ticket returns its own status, the 50 equal their alone-results and the oracle, and once every
    ticket has been waited for the server holds none of them."""
    rng = np.random.Generator(np.random.PCG64(45))
    jobs = wl.c4_jobs(50, 2.0, 5.5, 0.3, seed=46)
    where = 31
    jobs = jobs[:where] + [_with_bad_limb(jobs, where, rng)] + jobs[where:]
    with d.Context(0) as srv:
        dev = _prep(d, jobs)
        arr = d.make_jobs(dev)
        tickets = []
        for i in range(len(jobs)):
            rc, t = d.dmul_submit(srv.handle, arr[i])
            assert rc == 0
            tickets.append(t)
        rcs = [d.dmul_wait(srv.handle, t) for t in tickets]
        assert rcs[where] == d.DMUL_ERR_INVALID
        assert all(rc == d.DMUL_OK for i, rc in enumerate(rcs) if i != where)
        good = [i for i in range(len(jobs)) if i != where]
        _check(d, [jobs[i] for i in good], [dev[i] for i in good])
        with d.Context(0) as alone:
            for i in good:
                tx, nx, ty, ny, z, L, nz = dev[i]
                za, nza = alone.mul(tx, ty)
                assert torch.equal(za, z) and nza == int(nz.item())
        # every ticket was released by its wait: the table is empty and the tickets are gone
        st = d.dmul_serve_stats(srv.handle)
        assert (st["queued"], st["running"], st["held"]) == (0, 0, 0)
        for t in tickets:
            assert d.dmul_poll(srv.handle, t)[0] == d.DMUL_ERR_UNKNOWN_TICKET
            assert d.dmul_wait(srv.handle, t) == d.DMUL_ERR_UNKNOWN_TICKET


def test_served_mix_same_as_alone(d):
    """Requests submitted from several threads while others are on the GPU; every result equals the
    product computed alone and the oracle's."""
    jobs = wl.c4_jobs(120, 2.0, 5.0, 0.3, seed=51)
    with d.Context(0) as srv:
        dev = _prep(d, jobs)
        arr = d.make_jobs(dev)
        tickets = [None] * len(jobs)

        def submit(idx):
            for i in idx:
                rc, t = d.dmul_submit(srv.handle, arr[i])
                assert rc == 0
                tickets[i] = t

        th = [threading.Thread(target=submit, args=(range(k, len(jobs), 4),)) for k in range(4)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        # half the tickets collected by polling, half by waiting; each result is handed out once
        pending = list(tickets[::2])
        while pending:
            still = []
            for t in pending:
                rc, done = d.dmul_poll(srv.handle, t)
                assert rc == 0
                if not done:
                    still.append(t)
            pending = still
        for t in tickets[1::2]:
            assert d.dmul_wait(srv.handle, t) == 0
        for t in tickets:
            assert d.dmul_poll(srv.handle, t)[0] == d.DMUL_ERR_UNKNOWN_TICKET
        assert d.dmul_serve_stats(srv.handle)["held"] == 0
        _check(d, jobs, dev)
        with d.Context(0) as alone:
            for j, (tx, nx, ty, ny, z, L, nz) in zip(jobs, dev):
                za, nza = alone.mul(tx, ty)
                assert torch.equal(za, z) and nza == int(nz.item())
        assert d.dmul_wait(srv.handle, 10**9) == d.DMUL_ERR_UNKNOWN_TICKET


def test_served_short_and_long_interleaved(d):
    """Short requests (the one-cluster class, served by their own high-priority slots) and long
    ones (the general slots), alternating in one burst and then trickled in one by one: every
    result equals the oracle's, whichever queue and slot served it."""
    short = wl.c4_jobs(24, 2.5, 4.5, 0.3, seed=71)
    long_ = wl.c4_jobs(12, 5.4, 6.0, 0.3, seed=72)
    jobs = []
    for i in range(24):
        jobs.append(short[i])
        if i % 2 == 1:
            jobs.append(long_[i // 2])
    with d.Context(0) as srv:
        dev = _prep(d, jobs)
        arr = d.make_jobs(dev)
        burst = [d.dmul_submit(srv.handle, arr[i]) for i in range(len(jobs))]
        assert all(rc == 0 for rc, _ in burst)
        assert all(d.dmul_wait(srv.handle, t) == 0 for _, t in burst)
        _check(d, jobs, dev)
        for _, _, _, _, z, _, nz in dev:
            z.fill_(-1)
            nz.zero_()
        torch.cuda.synchronize()
        for i in range(len(jobs)):  # one at a time, each waited for before the next
            rc, t = d.dmul_submit(srv.handle, arr[i])
            assert rc == 0 and d.dmul_wait(srv.handle, t) == 0
        _check(d, jobs, dev)
        assert d.dmul_serve_stats(srv.handle)["held"] == 0


@pytest.mark.parametrize("half", [False, True], ids=["full_tiles", "half_tiles"])
def test_batch_specialized_splits(d, half):
    """Medium jobs whose default splits take the specialized passes (N = 2^19: 512 x 1024, both
    column and row specialized; N = 3 * 2^17: 768 x 512 and N = 5 * 2^16: 1280 x 256, column
    specialized), with squarings, and
    a group holding an operand that is not 16-byte aligned (its column passes fall back to the
    generic kernels)."""
    flags = d.DMUL_FLAG_NO_AUTOTUNE | (d.DMUL_FLAG_COL_HALF if half else 0)
    rng = np.random.Generator(np.random.PCG64(61 + half))

    def rand(n):
        a = rng.integers(0, 10**9, size=n, dtype=np.uint64).astype(np.uint32)
        a[-1] = max(1, int(a[-1]))
        return a

    shapes = [(250001, 240000, False), (262000, 262000, True), (200003, 150000, False),
              (160000, 160000, True)]
    jobs = [wl.Job(rand(nx), None, True) if sq else wl.Job(rand(nx), rand(ny), False)
            for nx, ny, sq in shapes]
    jobs = [wl.Job(j.x, j.x, True) if j.square else j for j in jobs]
    with d.Context(0, flags=flags) as c:
        for misaligned in (False, True):
            dev = _prep(d, jobs)
            if misaligned:  # job 2's x one limb into a larger buffer: 4-byte, not 16-byte aligned
                tx, nx, ty, ny, z, L, nz = dev[2]
                buf = torch.zeros(nx + 1, dtype=torch.int32, device="cuda")
                buf[1:] = tx
                dev[2] = (buf[1:], nx, ty, ny, z, L, nz)
                assert buf[1:].data_ptr() % 16 != 0
            assert d.dmul_batch(c.handle, d.make_jobs(dev), len(dev)) == 0
            assert d.dmul_sync(c.handle) == 0
            _check(d, jobs, dev)
        for nx, ny, sq in shapes[:1]:
            info = d.dmul_get_plan(c.handle, nx + ny)
            assert (info.N1, info.N2, info.col_half) == (512, 1024, int(half))


def test_few_short_jobs_take_the_measured_path(d):
    """A short job alone (or a handful of one size class) runs as a four-step group when the plain
    form measured that faster for a lone product of its length; batched and served, alone and
    again once the choice is known, the results equal the oracle's."""
    rng = np.random.Generator(np.random.PCG64(71))

    def rand(n):
        a = rng.integers(0, 10**9, size=n, dtype=np.uint64).astype(np.uint32)
        a[-1] = max(1, int(a[-1]))
        return a

    # transform lengths 24576, 16384, 8192 (size class 2) and 3072 (class 1), one squaring
    jobs = [wl.Job(rand(11112), rand(11112), False), wl.Job(rand(7000), rand(6000), False),
            wl.Job(rand(3500), rand(3000), False), wl.Job(rand(1500), rand(1200), False)]
    x = rand(9000)
    jobs.append(wl.Job(x, x, True))
    with d.Context(0) as c:
        for _ in range(2):  # first: the choices get measured; then they are known
            for k in range(1, len(jobs) + 1):
                dev = _prep(d, jobs[:k])
                assert d.dmul_batch(c.handle, d.make_jobs(dev), len(dev)) == 0
                assert d.dmul_sync(c.handle) == 0
                _check(d, jobs[:k], dev)
    with d.Context(0) as srv:
        for _ in range(2):
            dev = _prep(d, jobs)
            arr = d.make_jobs(dev)
            for i in range(len(jobs)):  # one at a time: every batch holds one job
                rc, t = d.dmul_submit(srv.handle, arr[i])
                assert rc == 0 and d.dmul_wait(srv.handle, t) == 0
            _check(d, jobs, dev)


def test_batch_status_edge_cases(d, ctx):
    """An empty batch, a batch of only rejected jobs, and the pending state before the sync."""
    arr = d.make_jobs([])
    assert d.dmul_batch(ctx.handle, arr, 0) == d.DMUL_OK
    assert d.dmul_sync(ctx.handle) == d.DMUL_OK
    jobs = wl.c4_jobs(2, 2.0, 3.0, 0.0, seed=47)
    dev = _prep(d, jobs)
    bad = [(tx, 0, ty, ny, z, L, nz) for (tx, nx, ty, ny, z, L, nz) in dev]  # nx = 0
    arr = d.make_jobs(bad)
    assert d.dmul_batch(ctx.handle, arr, 2) == d.DMUL_OK
    assert d.job_statuses(arr, 2) == [d.DMUL_ERR_INVALID] * 2
    assert d.dmul_sync(ctx.handle) == d.DMUL_OK
    # a good batch reads PENDING until the next sync fills in its statuses
    arr = d.make_jobs(dev)
    assert d.dmul_batch(ctx.handle, arr, 2) == d.DMUL_OK
    assert d.job_statuses(arr, 2) == [d.DMUL_PENDING] * 2
    assert d.dmul_sync(ctx.handle) == d.DMUL_OK
    assert d.job_statuses(arr, 2) == [d.DMUL_OK] * 2
    _check(d, jobs, dev)


def test_serve_stats_before_any_request(d):
    with d.Context(0) as c:
        st = d.dmul_serve_stats(c.handle)
        assert all(v == 0 for v in st.values())
        assert d.dmul_wait(c.handle, 1) == d.DMUL_ERR_UNKNOWN_TICKET
        assert d.dmul_poll(c.handle, 1)[0] == d.DMUL_ERR_UNKNOWN_TICKET
