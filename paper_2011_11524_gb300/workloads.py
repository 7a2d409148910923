"""Seeded synthetic operands for the multiplication workloads.

This module only draws inputs.  It holds none of the multiplication's arithmetic, so the CPU
oracle and the GPU path can both take their inputs from it without sharing any of the method.

Operands are little-endian base-10^9 ``uint32`` limb vectors.  An operand of ``d`` decimal digits
has ``ceil(d / 9)`` limbs; every limb but the top one is uniform in ``[0, 10^9 - 1]`` and the top
limb is uniform over the values with exactly ``r = d - 9 (ceil(d/9) - 1)`` digits, so the leading
decimal digit is nonzero.  The paper's own workload is random operands of ``n`` decimal digits
(Sec. 10); the functions below draw the five workload configurations.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

LIMB_DIGITS = 9
LIMB_BASE = 10**LIMB_DIGITS
NINES = LIMB_BASE - 1


def limbs_for_digits(ndigits: int) -> int:
    return max(1, -(-int(ndigits) // LIMB_DIGITS))


def top_digit_count(ndigits: int) -> int:
    r = int(ndigits) - LIMB_DIGITS * (limbs_for_digits(ndigits) - 1)
    return r


def random_operand(ndigits: int, rng: np.random.Generator) -> np.ndarray:
    """Uniformly random operand with exactly ``ndigits`` decimal digits (leading digit nonzero)."""
    n = limbs_for_digits(ndigits)
    a = rng.integers(0, LIMB_BASE, size=n, dtype=np.uint64).astype(np.uint32)
    r = top_digit_count(ndigits)
    lo = 10 ** (r - 1)
    hi = 10**r - 1
    a[-1] = np.uint32(rng.integers(lo, hi + 1))
    return a


def all_nines(ndigits: int) -> np.ndarray:
    """The operand 10^ndigits - 1 (every decimal digit a nine)."""
    n = limbs_for_digits(ndigits)
    a = np.full(n, NINES, dtype=np.uint32)
    a[-1] = np.uint32(10 ** top_digit_count(ndigits) - 1)
    return a


def with_nines(a: np.ndarray, frac: float, rng: np.random.Generator) -> np.ndarray:
    """Copy of ``a`` with a Bernoulli(frac) subset of its limbs (all but the top) set to 10^9-1."""
    a = a.copy()
    if len(a) > 1:
        mask = rng.random(len(a) - 1) < frac
        a[:-1][mask] = NINES
    return a


# ----------------------------------------------------------------------------------------------
# The five workload configurations
# ----------------------------------------------------------------------------------------------
def c1_pair():
    """One multiplication of two 100,000-digit random operands (seed 1)."""
    rng = np.random.Generator(np.random.PCG64(1))
    return random_operand(100_000, rng), random_operand(100_000, rng)


C2_DIGITS = 1 << 24


def c2_random_pair(ndigits: int = C2_DIGITS):
    """Two random 2^24-digit operands (seed 2)."""
    rng = np.random.Generator(np.random.PCG64(2))
    return random_operand(ndigits, rng), random_operand(ndigits, rng)


def c2_nines_pair(ndigits: int = C2_DIGITS):
    """The worst case: both operands 10^(2^24) - 1."""
    a = all_nines(ndigits)
    return a, a.copy()


def c3_pairs():
    """64M x 1M and 32M x 16M digits, 5% of limbs set to 10^9-1 (seeds 3 and 33)."""
    rng = np.random.Generator(np.random.PCG64(3))
    mrng = np.random.Generator(np.random.PCG64(33))
    out = []
    for nd, md in ((64_000_000, 1_000_000), (32_000_000, 16_000_000)):
        x = with_nines(random_operand(nd, rng), 0.05, mrng)
        y = with_nines(random_operand(md, rng), 0.05, mrng)
        out.append((x, y))
    return out


@dataclass
class Job:
    x: np.ndarray
    y: np.ndarray  # the same object as x for a squaring
    square: bool


def loguniform_digits(rng: np.random.Generator, lo_exp: float, hi_exp: float) -> int:
    return int(math.floor(10 ** rng.uniform(lo_exp, hi_exp)))


def c4_jobs(count: int = 4096, lo_exp: float = 3.0, hi_exp: float = 6.0, p_square: float = 0.2,
            seed: int = 4) -> list[Job]:
    """Batched workload: sizes log-uniform in [10^lo_exp, 10^hi_exp] digits, per operand."""
    rng = np.random.Generator(np.random.PCG64(seed))
    jobs = []
    for _ in range(count):
        sq = bool(rng.random() < p_square)
        x = random_operand(loguniform_digits(rng, lo_exp, hi_exp), rng)
        if sq:
            jobs.append(Job(x, x, True))
        else:
            y = random_operand(loguniform_digits(rng, lo_exp, hi_exp), rng)
            jobs.append(Job(x, y, False))
    return jobs


def c5_arrivals(rate_per_s: float, count: int, seed: int = 5) -> np.ndarray:
    """Served workload: Poisson arrival times (seconds from the start) at the given rate."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


@dataclass
class JobPool:
    """Jobs whose operands are consecutive, non-overlapping slices of one limb array, so that a
    stream of tens of thousands of requests is drawn in one call and moved in one copy."""
    pool: np.ndarray          # every operand's limbs, back to back
    jobs: list                # Job objects whose x, y are views into pool
    offsets: np.ndarray       # (count, 2) limb offsets of x and y in pool (y = x for a squaring)


def pooled_jobs(count: int, lo_exp: float, hi_exp: float, p_square: float, seed: int) -> JobPool:
    """The size law of c4_jobs (digits log-uniform per operand, a fraction p_square of
    squarings), every limb uniform in [0, 10^9) except each operand's top limb, which is uniform
    over the values with the operand's exact digit count."""
    rng = np.random.Generator(np.random.PCG64(seed))
    sq = rng.random(count) < p_square
    dx = np.floor(10.0 ** rng.uniform(lo_exp, hi_exp, size=count)).astype(np.int64)
    dy = np.floor(10.0 ** rng.uniform(lo_exp, hi_exp, size=count)).astype(np.int64)
    dy[sq] = dx[sq]
    nx = -(-dx // LIMB_DIGITS)
    ny = np.where(sq, 0, -(-dy // LIMB_DIGITS))
    starts = np.zeros(2 * count + 1, dtype=np.int64)
    starts[1:] = np.cumsum(np.stack([nx, ny], axis=1).reshape(-1))
    pool = rng.integers(0, LIMB_BASE, size=int(starts[-1]), dtype=np.uint32)
    offsets = np.stack([starts[0:-1:2], np.where(sq, starts[0:-1:2], starts[1:-1:2])], axis=1)
    # top limbs: r = digits - 9 (limbs - 1) in 1..9; uniform over [10^(r-1), 10^r - 1]
    for d, n, off, use in ((dx, nx, offsets[:, 0], np.ones(count, bool)), (dy, ny, offsets[:, 1], ~sq)):
        r = d - LIMB_DIGITS * (n - 1)
        lo = 10 ** (r - 1)
        top = lo + np.floor(rng.random(count) * (9 * lo)).astype(np.int64)
        pool[(off + n - 1)[use]] = top[use].astype(np.uint32)
    jobs = []
    for i in range(count):
        x = pool[offsets[i, 0]:offsets[i, 0] + nx[i]]
        if sq[i]:
            jobs.append(Job(x, x, True))
        else:
            jobs.append(Job(x, pool[offsets[i, 1]:offsets[i, 1] + ny[i]], False))
    return JobPool(pool, jobs, offsets)


def c5_pool(count: int, lo_exp: float = 2.0, hi_exp: float = 7.0, p_square: float = 0.3,
            seed: int = 5) -> JobPool:
    """Served workload's requests: digits log-uniform over [10^2, 10^7] per operand, 30%
    squarings (seed 5)."""
    return pooled_jobs(count, lo_exp, hi_exp, p_square, seed + 1000)


def fingerprint_candidates(seed: int = 61):
    """Endless seeded stream of odd integers in [2^60, 2^61) (candidate fingerprint moduli).

    The caller keeps the ones it accepts (the tests keep the primes); this module decides nothing.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    while True:
        yield int(rng.integers(1 << 60, 1 << 61)) | 1
