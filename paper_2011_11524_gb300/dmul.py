"""Thin Python binding of libdmul (include/dmul.h): argument marshalling only.

Every function of the C ABI is exposed under its own name and takes the same arguments, with
torch CUDA tensors (or raw integers) in place of device pointers; all of the arithmetic runs in
the CUDA kernels of libdmul.so.  There is no fallback: if the library is missing this module
raises on import of any entry point.

``Context`` is a small convenience wrapper that allocates outputs with torch.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdmul.so")

DMUL_OK = 0
DMUL_ERR_INVALID = 1
DMUL_ERR_TOO_LARGE = 2
DMUL_ERR_NOMEM = 3
DMUL_ERR_TIMEOUT = 4
DMUL_ERR_CUDA = 5
DMUL_ERR_CAPACITY = 6
DMUL_ERR_UNKNOWN_TICKET = 7
DMUL_PENDING = -1

DMUL_FLAG_SIXSTEP = 1
DMUL_FLAG_STAGE_TIMING = 2
DMUL_FLAG_NO_SMALL = 4
DMUL_FLAG_NO_AUTOTUNE = 8
DMUL_FLAG_ROW_TMA = 16
DMUL_FLAG_COL_HALF = 32
DMUL_FLAG_HOST_STAGED_IN = 64
DMUL_FLAG_HOST_STAGED_OUT = 128
DMUL_FLAG_HOST_DIRECT_IN = 256
DMUL_FLAG_NO_RADIX5 = 512
DMUL_FLAG_SHORT_WAITS = 1024
DMUL_FLAG_TEST_STALL_CARRY = 2048
DMUL_FLAG_NO_FUSED = 4096
DMUL_FLAG_HOST_DIRECT_OUT = 8192
DMUL_HOST_IN_PLACE_LIMBS = 524288

# every symbol include/dmul.h declares
EXPORTS = [
    "dmul_init", "dmul_destroy", "dmul_strerror", "dmul_sync", "dmul_mul", "dmul_sqr",
    "dmul_mul_host", "dmul_batch", "dmul_submit", "dmul_poll", "dmul_wait", "dmul_conv_residues",
    "dmul_conv_coeffs", "dmul_carry", "dmul_transpose", "dmul_get_plan", "dmul_primes",
    "dmul_lambda", "dmul_max_min_limbs", "dmul_stage_times", "dmul_stage_timing", "dmul_probe_imad",
    "dmul_carry_noalloc", "dmul_host_direct", "dmul_serve_stats", "dmul_probe_prime_width",
    "dmul_probe64_primes", "dmul_probe64_conv",
]


class DmulError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {dmul_strerror(status)} ({status})" if what else dmul_strerror(status))


class dmul_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_uint64),
                ("max_limbs", ctypes.c_uint64), ("flags", ctypes.c_uint32)]


class dmul_job(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("nx", ctypes.c_uint64), ("y", ctypes.c_void_p),
                ("ny", ctypes.c_uint64), ("z", ctypes.c_void_p), ("z_cap", ctypes.c_uint64),
                ("nz", ctypes.c_void_p), ("status", ctypes.c_int)]


class dmul_serve_info(ctypes.Structure):
    _fields_ = [("queued", ctypes.c_uint64), ("running", ctypes.c_uint64), ("held", ctypes.c_uint64),
                ("peak_running", ctypes.c_uint64), ("admit_budget_bytes", ctypes.c_uint64),
                ("inflight_bytes", ctypes.c_uint64)]


class dmul_plan_info(ctypes.Structure):
    _fields_ = [("primes", ctypes.c_uint32 * 3), ("N", ctypes.c_uint64), ("N1", ctypes.c_uint32),
                ("N2", ctypes.c_uint32), ("col_radix", ctypes.c_uint32 * 8),
                ("row_radix", ctypes.c_uint32 * 8), ("sixstep", ctypes.c_uint32),
                ("col_threads", ctypes.c_uint32), ("row_threads", ctypes.c_uint32),
                ("row_tma", ctypes.c_uint32), ("row_grid", ctypes.c_uint32),
                ("col_half", ctypes.c_uint32)]


_lib = None


def load() -> ctypes.CDLL:
    """Load libdmul.so (built by paper_2011_11524_gb300.build); raise if it is not there."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libdmul.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, sz, u64, i32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64, ctypes.c_int
    sig = {
        "dmul_init": ([ctypes.POINTER(vp), ctypes.POINTER(dmul_config)], i32),
        "dmul_destroy": ([vp], None),
        "dmul_strerror": ([i32], ctypes.c_char_p),
        "dmul_sync": ([vp, vp], i32),
        "dmul_mul": ([vp, vp, sz, vp, sz, vp, sz, vp, vp], i32),
        "dmul_sqr": ([vp, vp, sz, vp, sz, vp, vp], i32),
        "dmul_mul_host": ([vp, vp, sz, vp, sz, vp, sz, ctypes.POINTER(sz)], i32),
        "dmul_host_direct": ([vp, vp, sz], i32),
        "dmul_batch": ([vp, ctypes.POINTER(dmul_job), sz, vp], i32),
        "dmul_submit": ([vp, ctypes.POINTER(dmul_job), ctypes.POINTER(u64)], i32),
        "dmul_poll": ([vp, u64, ctypes.POINTER(i32)], i32),
        "dmul_wait": ([vp, u64], i32),
        "dmul_serve_stats": ([vp, ctypes.POINTER(dmul_serve_info)], i32),
        "dmul_conv_residues": ([vp, vp, sz, vp, sz, vp, vp], i32),
        "dmul_conv_coeffs": ([vp, vp, sz, vp, sz, vp, vp], i32),
        "dmul_carry": ([vp, vp, sz, vp, sz, vp, vp], i32),
        "dmul_transpose": ([vp, vp, sz, sz, vp], i32),
        "dmul_carry_noalloc": ([vp, sz, vp, sz, vp, vp], i32),
        "dmul_get_plan": ([vp, u64, ctypes.POINTER(dmul_plan_info)], i32),
        "dmul_primes": ([ctypes.POINTER(ctypes.c_uint32)], i32),
        "dmul_lambda": ([i32, i32, i32], i32),
        "dmul_max_min_limbs": ([], u64),
        "dmul_stage_times": ([vp, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(u64), ctypes.POINTER(i32)], i32),
        "dmul_stage_timing": ([vp, i32], i32),
        "dmul_probe_imad": ([vp, ctypes.POINTER(ctypes.c_double)], i32),
        "dmul_probe_prime_width": ([vp, u64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)], i32),
        "dmul_probe64_primes": ([ctypes.POINTER(u64)], i32),
        "dmul_probe64_conv": ([vp, vp, vp, vp, sz, vp], i32),
    }
    for name, (args, res) in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = res
    _lib = lib
    return lib


# ---------------------------------------------------------------------------------------------
# pointer marshalling
# ---------------------------------------------------------------------------------------------
def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(s) -> int | None:
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ---------------------------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ---------------------------------------------------------------------------------------------
def dmul_strerror(status: int) -> str:
    return load().dmul_strerror(status).decode()


def dmul_init(device: int = 0, hbm_budget_bytes: int = 0, max_limbs: int = 0, flags: int = 0) -> int:
    cfg = dmul_config(device, hbm_budget_bytes, max_limbs, flags)
    h = ctypes.c_void_p()
    rc = load().dmul_init(ctypes.byref(h), ctypes.byref(cfg))
    if rc:
        raise DmulError(rc, "dmul_init")
    return h.value


def dmul_destroy(ctx: int) -> None:
    load().dmul_destroy(ctx)


def dmul_sync(ctx: int, stream=None) -> int:
    return load().dmul_sync(ctx, _stream(stream))


def dmul_mul(ctx, x, nx, y, ny, z, z_cap, nz, stream=None) -> int:
    return load().dmul_mul(ctx, _ptr(x), nx, _ptr(y), ny, _ptr(z), z_cap, _ptr(nz), _stream(stream))


def dmul_sqr(ctx, x, nx, z, z_cap, nz, stream=None) -> int:
    return load().dmul_sqr(ctx, _ptr(x), nx, _ptr(z), z_cap, _ptr(nz), _stream(stream))


def dmul_mul_host(ctx, x, nx, y, ny, z, z_cap) -> tuple[int, int]:
    """x, y, z: host buffers (numpy arrays or pinned torch CPU tensors).  Returns (status, nz)."""
    nz = ctypes.c_size_t(0)
    rc = load().dmul_mul_host(ctx, _host_ptr(x), nx, _host_ptr(y), ny, _host_ptr(z), z_cap,
                              ctypes.byref(nz))
    return rc, nz.value


def dmul_host_direct(ctx, a, nbytes=None) -> bool:
    """Whether dmul_mul_host reads / writes the host buffer `a` in place (it is page-locked)."""
    if nbytes is None:
        nbytes = a.numel() * a.element_size() if hasattr(a, "numel") else a.nbytes
    return load().dmul_host_direct(ctx, _host_ptr(a), nbytes) == 1


def _host_ptr(a) -> int:
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def make_jobs(jobs) -> ctypes.Array:
    """jobs: iterable of (x, nx, y, ny, z, z_cap, nz) with tensors or raw device pointers."""
    jobs = list(jobs)
    arr = (dmul_job * max(1, len(jobs)))()
    for i, (x, nx, y, ny, z, zc, nz) in enumerate(jobs):
        arr[i] = dmul_job(_ptr(x), nx, _ptr(y), ny, _ptr(z), zc, _ptr(nz), DMUL_PENDING)
    return arr


def job_statuses(jobs_array, count) -> list[int]:
    """The status field of the first `count` descriptors (filled by dmul_batch / dmul_sync)."""
    return [int(jobs_array[i].status) for i in range(count)]


def dmul_batch(ctx, jobs_array, count, stream=None) -> int:
    return load().dmul_batch(ctx, jobs_array, count, _stream(stream))


def dmul_submit(ctx, job: dmul_job) -> tuple[int, int]:
    t = ctypes.c_uint64(0)
    rc = load().dmul_submit(ctx, ctypes.byref(job), ctypes.byref(t))
    return rc, t.value


def dmul_poll(ctx, ticket) -> tuple[int, bool]:
    d = ctypes.c_int(0)
    rc = load().dmul_poll(ctx, ticket, ctypes.byref(d))
    return rc, bool(d.value)


def dmul_wait(ctx, ticket) -> int:
    return load().dmul_wait(ctx, ticket)


def dmul_serve_stats(ctx) -> dict:
    """The serving loop's counters as a dict (raises on error)."""
    info = dmul_serve_info()
    rc = load().dmul_serve_stats(ctx, ctypes.byref(info))
    if rc:
        raise DmulError(rc, "dmul_serve_stats")
    return {k: int(getattr(info, k)) for k, _ in dmul_serve_info._fields_}


def dmul_conv_residues(ctx, x, nx, y, ny, r, stream=None) -> int:
    return load().dmul_conv_residues(ctx, _ptr(x), nx, _ptr(y), ny, _ptr(r), _stream(stream))


def dmul_conv_coeffs(ctx, x, nx, y, ny, d, stream=None) -> int:
    return load().dmul_conv_coeffs(ctx, _ptr(x), nx, _ptr(y), ny, _ptr(d), _stream(stream))


def dmul_carry(ctx, d, L, z, z_cap, nz, stream=None) -> int:
    return load().dmul_carry(ctx, _ptr(d), L, _ptr(z), z_cap, _ptr(nz), _stream(stream))


def dmul_carry_noalloc(d, L, z, z_cap, nz, stream=None) -> int:
    """The carry stage without a context or any device allocation (see include/dmul.h)."""
    return load().dmul_carry_noalloc(_ptr(d), L, _ptr(z), z_cap, _ptr(nz), _stream(stream))


DMUL_NOALLOC_MAX_LIMBS = 1 << 22


def dmul_transpose(ctx, a, rows, cols, stream=None) -> int:
    return load().dmul_transpose(ctx, _ptr(a), rows, cols, _stream(stream))


def dmul_get_plan(ctx, L: int) -> dmul_plan_info:
    info = dmul_plan_info()
    rc = load().dmul_get_plan(ctx, L, ctypes.byref(info))
    if rc:
        raise DmulError(rc, "dmul_get_plan")
    return info


def dmul_primes() -> list[int]:
    a = (ctypes.c_uint32 * 3)()
    rc = load().dmul_primes(a)
    if rc:
        raise DmulError(rc, "dmul_primes")
    return list(a)


def dmul_lambda(w: int, l: int, log2M: int) -> int:
    return load().dmul_lambda(w, l, log2M)


def dmul_max_min_limbs() -> int:
    return int(load().dmul_max_min_limbs())


def dmul_stage_times(ctx) -> dict[str, tuple[float, int]]:
    n = ctypes.c_int(16)
    names = (ctypes.c_char_p * 16)()
    ms = (ctypes.c_double * 16)()
    la = (ctypes.c_uint64 * 16)()
    rc = load().dmul_stage_times(ctx, names, ms, la, ctypes.byref(n))
    if rc:
        raise DmulError(rc, "dmul_stage_times")
    return {names[i].decode(): (ms[i], int(la[i])) for i in range(min(n.value, 16))}


def dmul_probe_imad(ctx) -> float:
    v = ctypes.c_double(0)
    rc = load().dmul_probe_imad(ctx, ctypes.byref(v))
    if rc:
        raise DmulError(rc, "dmul_probe_imad")
    return v.value


def dmul_probe_prime_width(ctx, N: int) -> tuple[float, float]:
    """(ms of the two-prime 62-bit row pass, ms of the library's three-prime row pass) over N."""
    a, b = ctypes.c_double(0), ctypes.c_double(0)
    rc = load().dmul_probe_prime_width(ctx, N, ctypes.byref(a), ctypes.byref(b))
    if rc:
        raise DmulError(rc, "dmul_probe_prime_width")
    return a.value, b.value


def dmul_probe64_primes() -> list[int]:
    out = (ctypes.c_uint64 * 2)()
    rc = load().dmul_probe64_primes(out)
    if rc:
        raise DmulError(rc, "dmul_probe64_primes")
    return [int(v) for v in out]


def dmul_probe64_conv(ctx, a, b, out, rows, stream=None) -> int:
    return load().dmul_probe64_conv(ctx, _ptr(a), _ptr(b), _ptr(out), rows, _stream(stream))


# ---------------------------------------------------------------------------------------------
# convenience wrapper (torch for device memory and streams)
# ---------------------------------------------------------------------------------------------
class Context:
    """Owns a dmul context; multiplies torch uint32-as-int32 CUDA tensors of limbs."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_limbs: int = 0,
                 flags: int = 0):
        self.device = device
        self.handle = dmul_init(device, hbm_budget_bytes, max_limbs, flags)

    def close(self):
        if self.handle:
            dmul_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc, what):
        if rc:
            raise DmulError(rc, what)

    def sync(self, stream=None):
        self._check(dmul_sync(self.handle, stream), "dmul_sync")

    def mul(self, x, y, stream=None, sync=True):
        """x, y: int32 CUDA tensors holding uint32 limbs.  Returns (z tensor, nz int)."""
        import torch
        L = x.numel() + y.numel()
        z = torch.empty(L, dtype=torch.int32, device=x.device)
        nz = torch.zeros(1, dtype=torch.int64, device=x.device)
        if x.data_ptr() == y.data_ptr() and x.numel() == y.numel():
            rc = dmul_sqr(self.handle, x, x.numel(), z, L, nz, stream)
        else:
            rc = dmul_mul(self.handle, x, x.numel(), y, y.numel(), z, L, nz, stream)
        self._check(rc, "dmul_mul")
        if not sync:
            return z, nz
        self.sync(stream)
        return z, int(nz.item())

    def sqr(self, x, stream=None):
        return self.mul(x, x, stream)

    def conv_residues(self, x, y, stream=None):
        import torch
        L = x.numel() + y.numel()
        r = torch.empty(3 * L, dtype=torch.int32, device=x.device)
        self._check(dmul_conv_residues(self.handle, x, x.numel(), y, y.numel(), r, stream),
                    "dmul_conv_residues")
        self.sync(stream)
        return r

    def conv_coeffs(self, x, y, stream=None):
        import torch
        L = x.numel() + y.numel()
        d = torch.empty(3 * L, dtype=torch.int32, device=x.device)
        self._check(dmul_conv_coeffs(self.handle, x, x.numel(), y, y.numel(), d, stream),
                    "dmul_conv_coeffs")
        self.sync(stream)
        return d

    def carry(self, d, L, stream=None):
        import torch
        z = torch.empty(L, dtype=torch.int32, device=d.device)
        nz = torch.zeros(1, dtype=torch.int64, device=d.device)
        self._check(dmul_carry(self.handle, d, L, z, L, nz, stream), "dmul_carry")
        self.sync(stream)
        return z, int(nz.item())

    def transpose_(self, a, rows, cols, stream=None):
        self._check(dmul_transpose(self.handle, a, rows, cols, stream), "dmul_transpose")
        self.sync(stream)
        return a

    def stage_times(self):
        return dmul_stage_times(self.handle)

    def stage_timing(self, on: bool):
        rc = load().dmul_stage_timing(self.handle, 1 if on else 0)
        if rc:
            raise DmulError(rc, "dmul_stage_timing")

    def probe_imad(self) -> float:
        return dmul_probe_imad(self.handle)


def to_device(limbs, device="cuda"):
    """numpy uint32 limbs -> int32 CUDA tensor (bit-identical)."""
    import numpy as np
    import torch
    a = np.ascontiguousarray(np.asarray(limbs, dtype=np.uint32)).view(np.int32)
    return torch.from_numpy(a.copy()).to(device)


def to_host(t):
    """int32 tensor of limbs -> numpy uint32."""
    import numpy as np
    return t.detach().cpu().numpy().view(np.uint32)
