"""Host-side checks of libdmul (no GPU): the library loads, exports every symbol include/dmul.h
declares, and its planner's number theory agrees with the oracle and the paper's printed tables."""
import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2011_11524_gb300 import build as dbuild
from paper_2011_11524_gb300 import dmul as d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _built():
    dbuild.build()
    d.load()


def _header_symbols():
    txt = open(os.path.join(ROOT, "include", "dmul.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dmul_[a-z_0-9]+)\s*\(", txt)))


def test_exports_every_declared_symbol():
    syms = _header_symbols()
    assert len(syms) >= 20
    lib = d.load()
    for s in syms:
        assert hasattr(lib, s), s
    assert sorted(d.EXPORTS) == syms


def test_header_is_c_and_links_from_c(tmp_path):
    """include/dmul.h is a C ABI: a strict C99 program that includes it compiles without warnings
    and links against libdmul.so (no torch or C++ types cross the boundary)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use_dmul.c"
    src.write_text('#include "dmul.h"\n'
                   "int main(void) {\n"
                   "    uint32_t p[3];\n"
                   "    dmul_config cfg = {0};\n"
                   "    (void)cfg;\n"
                   "    return dmul_primes(p) == DMUL_OK && dmul_lambda(31, 3, 20) > 0 ? 0 : 1;\n"
                   "}\n")
    lib = dbuild.LIB
    exe = tmp_path / "use_dmul"
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I" + os.path.join(ROOT, "include"),
                        str(src), "-o", str(exe), "-L" + os.path.dirname(lib), "-ldmul",
                        "-Wl,-rpath," + os.path.dirname(lib)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    # host-only entry points: the program runs without a GPU
    run = subprocess.run([str(exe)], capture_output=True, text=True)
    assert run.returncode == 0, run.stderr


def test_primes_match_oracle_find_primes():
    """The GPU prime set is FindPrimes(w=31, n_min=23, l=3) (Sec. 4.5), as the oracle computes it."""
    lib_primes = d.dmul_primes()
    ref = sorted(oracle.find_primes(31, 23, 3))
    assert lib_primes == ref
    for p in ref:
        assert p < 2**30 and oracle.is_prime_mr(p)
        q = p - 1
        assert q % 3 == 0 and (q & -q) >= 2**23


def test_lambda_tables_from_paper():
    """eq. lambda against the six tables printed in Sec. 4.2."""
    path = os.path.join(ROOT, "tests", "golden", "lambda_tables.txt")
    n = 0
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        lmu, lM, l, lam = (int(t) for t in line.split())
        assert d.dmul_lambda(lmu, l, lM) == lam, (lmu, lM, l)
        n += 1
    assert n == 24


def test_product_bound():
    """(B-1)^2 min(n, m) < p0 p1 p2 exactly for min <= dmul_max_min_limbs() (eq. product_inequality)."""
    P = math.prod(d.dmul_primes())
    m = d.dmul_max_min_limbs()
    assert (10**9 - 1) ** 2 * m < P <= (10**9 - 1) ** 2 * (m + 1)
    # the configurations' worst case: two 2^24-digit operands
    assert (10**9 - 1) ** 2 * 1864136 < P


def _odd_part_admissible(n):
    """n = f 2^k with f in {1, 3, 5} (the length set {2^k, 3 2^k, 5 2^k})."""
    for f in (1, 3, 5):
        if n % f == 0 and (n // f) & (n // f - 1) == 0:
            return True
    return False


@pytest.mark.parametrize("L", [2, 3, 1000, 1024, 1025, 1280, 1281, 1536, 1537, 5000, 22224, 81920,
                               3728272, 4194305, 5242880, 5333334, 7222224, 10485761, 3 * 2**22])
def test_plan_invariants(L):
    info = d.dmul_get_plan(None, L)
    N = info.N
    assert N >= L and N >= 1024
    assert _odd_part_admissible(N)
    # smallest admissible length
    for cand in range(L, N):
        assert not (_odd_part_admissible(cand) and cand >= 1024), cand
    assert info.N1 * info.N2 == N
    cr = [r for r in info.col_radix if r]
    rr = [r for r in info.row_radix if r]
    assert math.prod(cr) == info.N1 and math.prod(rr) == info.N2
    # the odd factor is the first column radix; then powers of two, radix 16 last
    assert all(r in (2, 4, 8, 16) for r in cr[1:] + rr)
    assert cr[0] in (2, 3, 4, 5, 8, 16)
    assert info.N2 % 32 == 0 and info.N2 <= 8192 and info.N1 <= 1536
    for p in info.primes:
        assert (p - 1) % N == 0


def test_five_lengths_cut_the_staircase():
    """Between 4 2^k and 5 2^k the length set picks 5 2^k, not 6 2^k (Sec. 4.5)."""
    for k in range(9, 22):
        L = 4 * 2**k + 1
        assert d.dmul_get_plan(None, L).N == 5 * 2**k


def test_too_large_rejected():
    with pytest.raises(d.DmulError):
        d.dmul_get_plan(None, 3 * 2**22 + 1)


def test_strerror():
    for st in range(8):
        assert isinstance(d.dmul_strerror(st), str) and d.dmul_strerror(st)


def _admissible_lengths():
    out = set()
    for k in range(0, 24):
        for f in (1, 3, 5):
            n = f << k
            if 1024 <= n <= 3 * 2**22:
                out.add(n)
    return sorted(out)


@pytest.mark.parametrize("N", _admissible_lengths())
def test_every_admissible_length_plans(N):
    """Every admissible length (1024 .. 3 2^22) plans as itself: N1 N2 = N, the odd factor as the
    first column radix, power-of-two row schedules ending in radix 16, N2 in [32, 8192], N1 within
    the shared-memory tile, and N | p - 1 for every prime."""
    info = d.dmul_get_plan(None, N)
    assert info.N == N
    cr = [r for r in info.col_radix if r]
    rr = [r for r in info.row_radix if r]
    assert info.N1 * info.N2 == N and math.prod(cr) == info.N1 and math.prod(rr) == info.N2
    odd = N // (N & -N)
    assert (cr[0] == odd) if odd > 1 else cr[0] in (2, 4, 8, 16)
    assert all(r in (2, 4, 8, 16) for r in cr[1:]) and all(r in (2, 4, 8, 16) for r in rr)
    assert rr[-1] == 16 or info.N2 < 16
    assert 32 <= info.N2 <= 8192 and info.N1 <= 1536
    for p in info.primes:
        assert (p - 1) % N == 0
    # one less than the length is planned on the same N, one more on a longer one
    assert d.dmul_get_plan(None, N - 1).N == N
    if N < 3 * 2**22:
        assert d.dmul_get_plan(None, N + 1).N > N


@pytest.mark.parametrize("n,C", [(4, 2), (4, 3), (6, 4), (5, 5), (3, 8)])
def test_rho_c_then_block_transposes_is_the_transpose(n, C):
    """The generalization closing Sec. 7.6, as the library's n x Cn transpose applies it: moving
    column C i + k of every row to position k n + i, then transposing each of the C n x n blocks
    in place, gives M^T in row-major order; the mirror (blocks of the n x Cn view, then the
    inverse move on every row) undoes it.  Checked against numpy's transpose."""
    rng = np.random.default_rng(n * 10 + C)
    M = rng.integers(0, 1 << 30, size=(n, C * n))
    P = np.empty_like(M)
    for k in range(C):
        for i in range(n):
            P[:, k * n + i] = M[:, C * i + k]
    for k in range(C):
        P[:, k * n:(k + 1) * n] = P[:, k * n:(k + 1) * n].T.copy()
    assert np.array_equal(P.reshape(-1), M.T.reshape(-1))
    # inverse: the flat array seen as n x Cn again, blocks transposed, then the inverse move
    Q = P.reshape(n, C * n).copy()
    for k in range(C):
        Q[:, k * n:(k + 1) * n] = Q[:, k * n:(k + 1) * n].T.copy()
    R = np.empty_like(Q)
    for i in range(n):
        for k in range(C):
            R[:, C * i + k] = Q[:, k * n + i]
    assert np.array_equal(R, M)


def test_probe64_primes_are_findprimes_63():
    """The prime-width probe's two 62-bit primes are FindPrimes(63, 23, 2) of Sec. 4.5, as the
    oracle's independent implementation finds them."""
    assert d.dmul_probe64_primes() == sorted(oracle.find_primes(63, 23, 2))


def _pidx(a):
    return a + (a >> 4)


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096, 8192])
def test_row_center_handoffs_stay_within_a_warp(N):
    """The specialized row pass orders its last forward stage (span 256) -> center -> first inverse
    stage (span 256) hand-offs with warp barriers only: every padded word a thread reads there was
    written by its own warp.  Checked for every CTA size and rows per CTA the pass runs with, for
    squares (X only) and products (X and Y groups on the same thread)."""
    for rows in (1, 2, 4, 8, 16):
        if rows * N > 65536:
            continue
        for bd in (128, 256, 512):
            per_op = rows * (N // 16)
            g = np.arange(per_op)
            warp_of_g = (g % bd) // 32  # loop g = t, t + bd, ...: thread g mod bd
            blk, j = g // 16, g % 16
            # stage (span 256, radix 16): group g writes pidx(blk 256 + j + 16 u), u < 16
            words = _pidx(blk[:, None] * 256 + j[:, None] + 16 * np.arange(16)[None, :])
            writer = np.full(int(words.max()) + 1, -1)
            writer[words.ravel()] = np.repeat(warp_of_g, 16)
            # center: group b reads 17 b + u (X, and Y the same way), writes them
            cw = (17 * g[:, None] + np.arange(16)[None, :])
            assert (writer[cw] == warp_of_g[:, None]).all(), (N, rows, bd)
            center_writer = np.full(int(cw.max()) + 1, -1)
            center_writer[cw.ravel()] = np.repeat(warp_of_g, 16)
            # first inverse stage (span 256): group g reads its stage words
            assert (center_writer[words] == warp_of_g[:, None]).all(), (N, rows, bd)
