"""Test helpers: base-10^9 limb vectors <-> Python ints and decimal strings.

These conversions go through Python's own int and str routines (library routines), so they are
independent of both the oracle and the GPU path.
"""
import numpy as np

B = 10**9


def to_int(limbs) -> int:
    limbs = [int(v) for v in np.asarray(limbs)]
    if not limbs:
        return 0
    s = "".join(f"{v:09d}" for v in reversed(limbs))
    return int(s)


def from_int(v: int, nlimbs: int | None = None) -> np.ndarray:
    s = str(v)
    pad = (-len(s)) % 9
    s = "0" * pad + s
    out = [int(s[i:i + 9]) for i in range(0, len(s), 9)][::-1]
    if nlimbs is not None:
        assert len(out) <= nlimbs or all(o == 0 for o in out[nlimbs:])
        out = (out + [0] * nlimbs)[:nlimbs]
    return np.array(out, dtype=np.uint32)


def to_str(limbs) -> str:
    """Decimal string without leading zeros ("0" for zero)."""
    return str(to_int(limbs))
