"""Seeded synthetic operands for the multiplication workloads.

This module only draws inputs.  It holds none of the multiplication's arithmetic, so the CPU
oracle and the GPU path can both take their inputs from it without sharing any of the method.

Operands are little-endian base-10^9 ``uint32`` limb vectors.  An operand of ``d`` decimal digits
has ``ceil(d / 9)`` limbs; every limb but the top one is uniform in ``[0, 10^9 - 1]`` and the top
limb is uniform over the values with exactly ``r = d - 9 (ceil(d/9) - 1)`` digits, so the leading
decimal digit is nonzero.  The paper's own workload is random operands of ``n`` decimal digits
(Sec. 10); the configurations below follow the recipe stated in the design doc.
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


def c5_stream(rate_per_s: float, count: int, lo_exp: float = 2.0, hi_exp: float = 7.0,
              p_square: float = 0.3, seed: int = 5):
    """Served workload: Poisson arrival times (seconds) and jobs, sizes log-uniform."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, size=count)
    arrivals = np.cumsum(gaps)
    jobs = c4_jobs(count, lo_exp, hi_exp, p_square, seed=seed + 1000)
    return arrivals, jobs


def fingerprint_candidates(seed: int = 61):
    """Endless seeded stream of odd integers in [2^60, 2^61) (candidate fingerprint moduli).

    The caller keeps the ones it accepts (the tests keep the primes); this module decides nothing.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    while True:
        yield int(rng.integers(1 << 60, 1 << 61)) | 1
