"""ctypes binding of libfitrig (include/fitrig.h), one function per C entry point.

Argument marshalling only: every step of the trigger runs in the CUDA library.
Importing this module does not load the library; the first call does, and it
raises ``FitrigError`` if the library is missing -- there is no CPU fallback.

Tensors: snapshots may be torch tensors (CUDA or CPU) or NumPy arrays; device
pointers are passed for CUDA tensors, host pointers otherwise.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import (POINTER, byref, c_char_p, c_double, c_float, c_int, c_int32, c_int64,
                    c_void_p)
from typing import Optional, Tuple

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ESTATE, ECUDA, ETIMEOUT, ETRUNC, ENONFINITE, EBUSY, EUNSUPPORTED = range(10)
BRANCH_IMAGE, BRANCH_FREQ, BRANCH_BOTH = 1, 2, 3
F32, BF16, F16 = 0, 1, 2
OPT_STORAGE, OPT_NOISE, OPT_RMODE, OPT_MMODE, OPT_EDGE, OPT_STRIDE = 1, 2, 3, 4, 5, 6
OPT_STREAM, OPT_TIMEOUT_NS = 8, 9
OPT_AUTOTUNE, OPT_MAX_SELECTED, OPT_GRAPH, OPT_ACCUMULATE, OPT_HARMONICS, OPT_REFINE = \
    10, 11, 12, 13, 14, 15
OPT_CODING = 16
CODING_VALUE, CODING_DELTA = 0, 1
REFINE_PARABOLIC, REFINE_CUBIC = 0, 1
NOISE_MEANSTD, NOISE_MEDMAD = 0, 1
RMODE_ABS, RMODE_SIGNED = 0, 1
MMODE_GLOBAL, MMODE_RUNNING = 0, 1
EDGE_PARTIAL, EDGE_DROP = 0, 1
STRIDE_TILE, STRIDE_SLIDING = 0, 1
KERNEL_STACK, KERNEL_NOISE, KERNEL_SELECT, KERNEL_SPECTRUM, KERNEL_DETECT = range(5)

# statuses that still carry valid results
SOFT = (OK, ENONFINITE)


class Candidate(ctypes.Structure):
    _fields_ = [("x", c_int32), ("y", c_int32), ("snapshot", c_int32),
                ("significance", c_float), ("branch", c_int32), ("freq_bin", c_int32),
                ("xf", c_float), ("yf", c_float)]


class Result(ctypes.Structure):
    _fields_ = [("field", c_int32), ("unit", c_int32), ("ncand", c_int32), ("status", c_int32),
                ("t_arrival_ns", c_int64), ("t_done_ns", c_int64), ("cand_offset", c_int64)]


RESULT_DTYPE = np.dtype([("field", np.int32), ("unit", np.int32), ("ncand", np.int32),
                         ("status", np.int32), ("t_arrival_ns", np.int64),
                         ("t_done_ns", np.int64), ("cand_offset", np.int64),
                         ("t_push_ns", np.int64), ("t_enqueued_ns", np.int64),
                         ("copy_ms", np.float32), ("trigger_ms", np.float32)])

CANDIDATE_DTYPE = np.dtype([("x", np.int32), ("y", np.int32), ("snapshot", np.int32),
                            ("significance", np.float32), ("branch", np.int32),
                            ("freq_bin", np.int32), ("xf", np.float32), ("yf", np.float32)])


class FitrigError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {status_string(status)} ({status})")


P = c_void_p
# ctypes signature of every entry point of include/fitrig.h
SIGNATURES = {
    "fitrig_version": (c_char_p, []),
    "fitrig_status_string": (c_char_p, [c_int]),
    "fitrig_plan_create": (c_int, [c_int, c_int, c_int, c_int, c_double, c_int, POINTER(P)]),
    "fitrig_plan_set": (c_int, [P, c_int, c_int64]),
    "fitrig_push_snapshot": (c_int, [P, P, c_int, c_int, c_int64]),
    "fitrig_push_snapshots": (c_int, [P, P, c_int32, c_int, c_int, c_int64, c_int64]),
    "fitrig_plan_reset": (c_int, [P]),
    "fitrig_detect": (c_int, [P, POINTER(c_int32)]),
    "fitrig_candidates": (c_int, [P, P, c_int32, POINTER(c_int32)]),
    "fitrig_tlisi": (c_int, [P, c_int32, P, c_int32]),
    "fitrig_unit_values": (c_int, [P, c_int32, P, c_int32]),
    "fitrig_noise_params": (c_int, [P, c_int32, POINTER(c_double), POINTER(c_double)]),
    "fitrig_spectrum": (c_int, [P, P, P, c_int32]),
    "fitrig_global_max": (c_int, [P, POINTER(c_double)]),
    "fitrig_unit_normaliser": (c_int, [P, c_int32, POINTER(c_double)]),
    "fitrig_tile_grid": (c_int, [P, POINTER(c_int32), POINTER(c_int32)]),
    "fitrig_kernel_ms": (c_int, [P, c_int, POINTER(c_float)]),
    "fitrig_stack_device_ptr": (c_int, [P, c_int32, POINTER(P), POINTER(c_int64)]),
    "fitrig_threshold_map": (c_int, [P, c_int64, c_double, c_int, c_int64,
                                     POINTER(c_int64), POINTER(c_double), POINTER(c_double)]),
    "fitrig_launch_count": (c_int, [POINTER(c_int64)]),
    "fitrig_wait_probe": (c_int, [c_int64, c_int64]),
    "fitrig_batch_create": (c_int, [POINTER(P), c_int32, POINTER(P)]),
    "fitrig_server_create": (c_int, [c_int64, c_int, POINTER(P)]),
    "fitrig_server_admit": (c_int, [P, c_int, c_int, c_int, c_double, c_int, c_int, POINTER(c_int32)]),
    "fitrig_server_admit_freq": (c_int, [P, c_int, c_int, c_int, c_double, c_int, c_int, c_int,
                                         POINTER(c_int32)]),
    "fitrig_server_push": (c_int, [P, c_int32, P, c_int, c_int64]),
    "fitrig_server_poll": (c_int, [P, P, c_int32, P, c_int32, POINTER(c_int32), POINTER(c_int32)]),
    "fitrig_server_drain": (c_int, [P]),
    "fitrig_server_retire": (c_int, [P, c_int32]),
    "fitrig_server_field_state": (c_int, [P, c_int32, POINTER(c_int32)]),
    "fitrig_server_field_export": (c_int, [P, c_int32, P, c_int64, POINTER(c_int64)]),
    "fitrig_server_field_import": (c_int, [P, P, c_int64, POINTER(c_int32)]),
    "fitrig_server_usage": (c_int, [P, POINTER(c_int64), POINTER(c_int32), POINTER(c_int32)]),
    "fitrig_server_destroy": (c_int, [P]),
    "fitrig_batch_detect": (c_int, [P, POINTER(c_int32)]),
    "fitrig_batch_ms": (c_int, [P, POINTER(c_float)]),
    "fitrig_batch_destroy": (c_int, [P]),
    "fitrig_autotune": (c_int, [c_int, c_int, POINTER(c_int32), POINTER(c_int32), POINTER(c_float)]),
    "fitrig_noise_static": (c_int, [P, c_int32, c_int64, c_int, P, c_int64]),
    "fitrig_spectrum_map": (c_int, [P, c_int32, c_int64, c_int64, c_int32, P, P, c_int32,
                                    c_int64, POINTER(c_float)]),
    "fitrig_plan_destroy": (c_int, [P]),
}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load libfitrig.so (building it first if sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or _build.LIB
    if not os.path.exists(p):
        try:
            _build.build()
        except Exception as e:  # noqa: BLE001
            raise FitrigError(ECUDA, f"libfitrig is not built and could not be built ({e})")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def status_string(s: int) -> str:
    try:
        return load().fitrig_status_string(int(s)).decode()
    except Exception:  # noqa: BLE001
        return f"status {s}"


def _check(rc: int, where: str, allow=(OK,)) -> int:
    if rc not in allow:
        raise FitrigError(rc, where)
    return rc


def _ptr_dtype(data) -> Tuple[int, int, int, int]:
    """(pointer, dtype code, on_device, row pitch in elements) of an image."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(data, torch.Tensor):
        code = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}.get(data.dtype)
        if code is None or data.dim() != 2 or data.stride(1) != 1:
            raise FitrigError(EINVAL, "push: need a 2-D float32/bfloat16/float16 tensor with unit column stride")
        return data.data_ptr(), code, int(data.is_cuda), int(data.stride(0))
    a = np.asarray(data)
    code = {np.dtype(np.float32): F32, np.dtype(np.float16): F16}.get(a.dtype)
    if code is None or a.ndim != 2 or a.strides[1] != a.itemsize:
        raise FitrigError(EINVAL, "push: need a 2-D float32/float16 array with unit column stride")
    return a.ctypes.data, code, 0, a.strides[0] // a.itemsize


# ---------------------------------------------------------------- entry points
def fitrig_version() -> str:
    return load().fitrig_version().decode()


def fitrig_status_string(status: int) -> str:
    return load().fitrig_status_string(int(status)).decode()


def fitrig_plan_create(nx: int, ny: int, nsnap: int, window: int, nsigma: float,
                       branch: int = BRANCH_IMAGE) -> c_void_p:
    h = c_void_p()
    _check(load().fitrig_plan_create(nx, ny, nsnap, window, float(nsigma), branch, byref(h)),
           "fitrig_plan_create")
    return h


def fitrig_plan_set(plan, option: int, value: int) -> None:
    _check(load().fitrig_plan_set(plan, option, int(value)), "fitrig_plan_set")


def fitrig_push_snapshot(plan, data, row_pitch_elems: Optional[int] = None) -> None:
    ptr, code, dev, pitch = _ptr_dtype(data)
    if row_pitch_elems is not None:
        pitch = row_pitch_elems
    _check(load().fitrig_push_snapshot(plan, c_void_p(ptr), code, dev, pitch),
           "fitrig_push_snapshot")


def fitrig_push_snapshots(plan, data) -> None:
    """Push a (count, ny, nx) block (torch tensor or numpy array, unit column
    stride) as `count` snapshots in one call."""
    try:
        import torch
    except ImportError:  # pragma: no cover
        torch = None
    if torch is not None and isinstance(data, torch.Tensor):
        if data.dim() != 3:
            raise FitrigError(EINVAL, "push_snapshots: need a 3-D block")
        ptr, code, dev, pitch = _ptr_dtype(data[0] if data.shape[0] else data.new_empty(1, 1))
        ptr, stride = data.data_ptr(), int(data.stride(0))
    else:
        a = np.asarray(data)
        if a.ndim != 3:
            raise FitrigError(EINVAL, "push_snapshots: need a 3-D block")
        ptr, code, dev, pitch = _ptr_dtype(a[0] if a.shape[0] else np.empty((1, 1), a.dtype))
        ptr, stride = a.ctypes.data, a.strides[0] // a.itemsize
    count = int(data.shape[0])
    if count == 0:
        stride = 0
    _check(load().fitrig_push_snapshots(plan, c_void_p(ptr), count, code, dev, pitch, stride),
           "fitrig_push_snapshots")


def fitrig_plan_reset(plan) -> None:
    _check(load().fitrig_plan_reset(plan), "fitrig_plan_reset")


def fitrig_detect(plan) -> Tuple[int, int]:
    """Returns (status, ncand); raises unless status is OK or ENONFINITE."""
    n = c_int32()
    rc = load().fitrig_detect(plan, byref(n))
    if rc == ETRUNC:
        err = FitrigError(rc, "fitrig_detect")
        err.needed = n.value   # the MAX_SELECTED that selection needed
        raise err
    _check(rc, "fitrig_detect", allow=SOFT)
    return rc, n.value


def fitrig_candidates(plan, cap: Optional[int] = None,
                      out: Optional[np.ndarray] = None) -> np.ndarray:
    """The last detect's candidates.  `out` (a CANDIDATE_DTYPE array, e.g. a
    view of pinned host memory that is reused across detects) receives them
    instead of a fresh array; then cap defaults to its length."""
    n = c_int32()
    lib = load()
    if out is not None:
        if out.dtype != CANDIDATE_DTYPE or out.ndim != 1 or not out.flags.c_contiguous:
            raise FitrigError(EINVAL, "fitrig_candidates: out must be a contiguous CANDIDATE_DTYPE vector")
        cap = len(out) if cap is None else min(cap, len(out))
    if cap is None:
        lib.fitrig_candidates(plan, None, 0, byref(n))
        cap = n.value
    if out is None:
        out = np.zeros(max(cap, 1), dtype=CANDIDATE_DTYPE)
    rc = lib.fitrig_candidates(plan, c_void_p(out.ctypes.data) if cap else None, cap, byref(n))
    _check(rc, "fitrig_candidates", allow=(OK, ETRUNC))
    return out[:min(cap, n.value)]


def fitrig_tile_grid(plan) -> Tuple[int, int]:
    ty, tx = c_int32(), c_int32()
    _check(load().fitrig_tile_grid(plan, byref(ty), byref(tx)), "fitrig_tile_grid")
    return ty.value, tx.value


def _tile_floats(fn, plan, unit) -> np.ndarray:
    ty, tx = fitrig_tile_grid(plan)
    out = np.empty(ty * tx, dtype=np.float32)
    _check(fn(plan, unit, c_void_p(out.ctypes.data), out.size), fn.__name__)
    return out.reshape(ty, tx)


def fitrig_tlisi(plan, unit: int) -> np.ndarray:
    return _tile_floats(load().fitrig_tlisi, plan, unit)


def fitrig_unit_values(plan, unit: int) -> np.ndarray:
    return _tile_floats(load().fitrig_unit_values, plan, unit)


def fitrig_noise_params(plan, unit: int) -> Tuple[float, float]:
    c, s = c_double(), c_double()
    _check(load().fitrig_noise_params(plan, unit, byref(c), byref(s)), "fitrig_noise_params")
    return c.value, s.value


def fitrig_spectrum(plan) -> Tuple[np.ndarray, np.ndarray]:
    ty, tx = fitrig_tile_grid(plan)
    eta = np.empty(ty * tx, dtype=np.float32)
    kb = np.empty(ty * tx, dtype=np.int32)
    _check(load().fitrig_spectrum(plan, c_void_p(eta.ctypes.data), c_void_p(kb.ctypes.data),
                                  eta.size), "fitrig_spectrum")
    return eta.reshape(ty, tx), kb.reshape(ty, tx)


def fitrig_global_max(plan) -> float:
    m = c_double()
    _check(load().fitrig_global_max(plan, byref(m)), "fitrig_global_max")
    return m.value


def fitrig_unit_normaliser(plan, unit: int) -> float:
    m = c_double()
    _check(load().fitrig_unit_normaliser(plan, unit, byref(m)), "fitrig_unit_normaliser")
    return m.value


def fitrig_kernel_ms(plan, kernel: int) -> float:
    ms = c_float()
    _check(load().fitrig_kernel_ms(plan, kernel, byref(ms)), "fitrig_kernel_ms")
    return ms.value


def fitrig_stack_device_ptr(plan, s: int) -> Tuple[int, int]:
    p, pitch = c_void_p(), c_int64()
    _check(load().fitrig_stack_device_ptr(plan, s, byref(p), byref(pitch)),
           "fitrig_stack_device_ptr")
    return p.value, pitch.value


def fitrig_threshold_map(dev_map, nsigma: float, noise_mode: int = NOISE_MEANSTD,
                         stream: int = 0) -> Tuple[int, float, float]:
    """dev_map: a contiguous float32 CUDA tensor; returns (nexceed, centre, scale)."""
    n, c, s = c_int64(), c_double(), c_double()
    _check(load().fitrig_threshold_map(c_void_p(dev_map.data_ptr()), dev_map.numel(),
                                       float(nsigma), noise_mode, int(stream), byref(n),
                                       byref(c), byref(s)), "fitrig_threshold_map")
    return n.value, c.value, s.value


SPECTRUM_AUTO, SPECTRUM_DIRECT, SPECTRUM_RADIX = 0, 1, 2


def fitrig_spectrum_map(dev_cube, n: int, T: int, stride: int, harmonics: int, dev_eta,
                        dev_bin, method: int = SPECTRUM_AUTO, stream: int = 0) -> float:
    """eta / bin of T series of n points (point q of series t at
    dev_cube[q * stride + t]; CUDA tensors); returns the transform's ms."""
    ms = c_float()
    _check(load().fitrig_spectrum_map(c_void_p(dev_cube.data_ptr()), n, T, stride, harmonics,
                                      c_void_p(dev_eta.data_ptr()), c_void_p(dev_bin.data_ptr()),
                                      method, int(stream), byref(ms)), "fitrig_spectrum_map")
    return ms.value


def fitrig_autotune(window: int, storage: int = F32) -> Tuple[int, int, float]:
    """(tile rows per CTA, ring depth, ms per probe launch) chosen for the window."""
    a, b, ms = c_int32(), c_int32(), c_float()
    _check(load().fitrig_autotune(window, storage, byref(a), byref(b), byref(ms)), "fitrig_autotune")
    return a.value, b.value, ms.value


NOISE_STATIC_MAX_GROUPS = 64


def fitrig_noise_static(dev_values, groups: int, n: int, noise_mode: int, dev_out,
                        stream: int = 0) -> int:
    """Noise estimate with no allocation: dev_values / dev_out are CUDA tensors
    (float32 groups*n, float64 2*groups); returns the status code."""
    return load().fitrig_noise_static(c_void_p(dev_values.data_ptr()), int(groups), int(n),
                                      int(noise_mode), c_void_p(dev_out.data_ptr()), int(stream))


def fitrig_batch_create(plans) -> c_void_p:
    """plans: a sequence of plan handles (or Plan objects) with all snapshots pushed."""
    hs = [p.h if isinstance(p, Plan) else p for p in plans]
    arr = (c_void_p * len(hs))(*[h.value if isinstance(h, c_void_p) else h for h in hs])
    b = c_void_p()
    _check(load().fitrig_batch_create(arr, len(hs), byref(b)), "fitrig_batch_create")
    return b


def fitrig_batch_detect(batch, nplans: int) -> Tuple[int, np.ndarray]:
    n = (c_int32 * nplans)()
    rc = load().fitrig_batch_detect(batch, n)
    _check(rc, "fitrig_batch_detect", allow=SOFT)
    return rc, np.array(list(n), dtype=np.int32)


def fitrig_batch_ms(batch) -> float:
    ms = c_float()
    _check(load().fitrig_batch_ms(batch, byref(ms)), "fitrig_batch_ms")
    return ms.value


def fitrig_batch_destroy(batch) -> None:
    _check(load().fitrig_batch_destroy(batch), "fitrig_batch_destroy")


FIELD_QUEUED, FIELD_ACTIVE, FIELD_RETIRED = 0, 1, 2


def fitrig_server_create(hbm_budget_bytes: int, max_fields: int) -> c_void_p:
    h = c_void_p()
    _check(load().fitrig_server_create(int(hbm_budget_bytes), int(max_fields), byref(h)),
           "fitrig_server_create")
    return h


def fitrig_server_admit(server, nx, ny, window, nsigma, storage=F32, noise=NOISE_MEANSTD):
    """Returns (status, field_id); status OK (active) or EBUSY (queued)."""
    fid = c_int32()
    rc = load().fitrig_server_admit(server, nx, ny, window, float(nsigma), storage, noise,
                                    byref(fid))
    _check(rc, "fitrig_server_admit", allow=(OK, EBUSY))
    return rc, fid.value


def fitrig_server_admit_freq(server, nx, ny, window, nsigma, storage=F32,
                             noise=NOISE_MEANSTD, freq_units=16):
    """Admit a field with the real-time frequency branch over its last
    freq_units units; returns (status, field id) (EBUSY = queued)."""
    fid = c_int32()
    rc = load().fitrig_server_admit_freq(server, int(nx), int(ny), int(window), float(nsigma),
                                         int(storage), int(noise), int(freq_units), byref(fid))
    _check(rc, "fitrig_server_admit_freq", allow=(OK, EBUSY))
    return rc, fid.value


def fitrig_server_push(server, field: int, data, t_arrival_ns: int) -> int:
    """Push one snapshot (2-D tensor or array); returns the status (OK or EBUSY)."""
    ptr, code, dev, pitch = _ptr_dtype(data)
    rc = load().fitrig_server_push(server, field, c_void_p(ptr), code, int(t_arrival_ns))
    _check(rc, "fitrig_server_push", allow=(OK, EBUSY))
    return rc


def fitrig_server_poll(server, cap: int = 4096, cand_cap: int = 1 << 20):
    """Returns (results, candidates) as structured arrays."""
    res = np.zeros(max(cap, 1), dtype=RESULT_DTYPE)
    cands = np.zeros(max(cand_cap, 1), dtype=CANDIDATE_DTYPE)
    n, nc = c_int32(), c_int32()
    _check(load().fitrig_server_poll(server, c_void_p(res.ctypes.data), cap,
                                     c_void_p(cands.ctypes.data), cand_cap, byref(n), byref(nc)),
           "fitrig_server_poll")
    return res[:n.value].copy(), cands[:nc.value].copy()


def fitrig_server_drain(server) -> None:
    _check(load().fitrig_server_drain(server), "fitrig_server_drain")


def fitrig_server_retire(server, field: int) -> None:
    _check(load().fitrig_server_retire(server, field), "fitrig_server_retire")


def fitrig_server_field_state(server, field: int) -> int:
    st = c_int32()
    _check(load().fitrig_server_field_state(server, field, byref(st)), "fitrig_server_field_state")
    return st.value


def fitrig_server_field_export(server, field: int) -> bytes:
    """Checkpoint of an active field as bytes."""
    size = c_int64()
    rc = load().fitrig_server_field_export(server, int(field), None, 0, byref(size))
    _check(rc, "fitrig_server_field_export", allow=(ETRUNC,))
    buf = ctypes.create_string_buffer(size.value)
    _check(load().fitrig_server_field_export(server, int(field), buf, size.value, byref(size)),
           "fitrig_server_field_export")
    return buf.raw


def fitrig_server_field_import(server, image: bytes) -> Tuple[int, int]:
    """A new active field from a checkpoint; returns (status, field id)."""
    fid = c_int32()
    buf = ctypes.create_string_buffer(image, len(image))
    rc = load().fitrig_server_field_import(server, buf, len(image), byref(fid))
    _check(rc, "fitrig_server_field_import", allow=(OK, EBUSY))
    return rc, fid.value


def fitrig_server_usage(server) -> Tuple[int, int, int]:
    u, a, w = c_int64(), c_int32(), c_int32()
    _check(load().fitrig_server_usage(server, byref(u), byref(a), byref(w)), "fitrig_server_usage")
    return u.value, a.value, w.value


def fitrig_server_destroy(server) -> None:
    _check(load().fitrig_server_destroy(server), "fitrig_server_destroy")


def fitrig_wait_probe(timeout_ns: int, stream: int = 0) -> int:
    """One bounded device wait that nothing completes; returns the status
    (ETIMEOUT is the expected result)."""
    return load().fitrig_wait_probe(int(timeout_ns), int(stream))


def fitrig_launch_count() -> int:
    n = c_int64()
    _check(load().fitrig_launch_count(byref(n)), "fitrig_launch_count")
    return n.value


def fitrig_plan_destroy(plan) -> None:
    _check(load().fitrig_plan_destroy(plan), "fitrig_plan_destroy")


# ---------------------------------------------------------------- convenience
class Plan:
    """Owns a plan handle; pushes a whole (L, ny, nx) stack and detects."""

    def __init__(self, nx, ny, nsnap, window, nsigma, branch=BRANCH_IMAGE, storage=F32,
                 noise=NOISE_MEANSTD, rmode=RMODE_ABS, edge=EDGE_PARTIAL, stream=None,
                 stride=STRIDE_TILE, autotune=False, max_selected=0, mmode=MMODE_GLOBAL,
                 accumulate=1, harmonics=1, refine=REFINE_PARABOLIC, coding=CODING_VALUE):
        self.h = fitrig_plan_create(nx, ny, nsnap, window, nsigma, branch)
        try:
            if coding != CODING_VALUE:
                fitrig_plan_set(self.h, OPT_CODING, coding)
            if accumulate != 1:
                fitrig_plan_set(self.h, OPT_ACCUMULATE, accumulate)
            if harmonics != 1:
                fitrig_plan_set(self.h, OPT_HARMONICS, harmonics)
            if refine != REFINE_PARABOLIC:
                fitrig_plan_set(self.h, OPT_REFINE, refine)
            if mmode != MMODE_GLOBAL:
                fitrig_plan_set(self.h, OPT_MMODE, mmode)
            if autotune:
                fitrig_plan_set(self.h, OPT_AUTOTUNE, 1)
            if max_selected:
                fitrig_plan_set(self.h, OPT_MAX_SELECTED, max_selected)
            if stride != STRIDE_TILE:
                fitrig_plan_set(self.h, OPT_STRIDE, stride)
            fitrig_plan_set(self.h, OPT_STORAGE, storage)
            fitrig_plan_set(self.h, OPT_NOISE, noise)
            fitrig_plan_set(self.h, OPT_RMODE, rmode)
            if edge != EDGE_PARTIAL:
                fitrig_plan_set(self.h, OPT_EDGE, edge)
            if stream is None:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            if stream:
                fitrig_plan_set(self.h, OPT_STREAM, stream)
        except Exception:
            fitrig_plan_destroy(self.h)
            raise
        self.nsnap = nsnap

    def push_stack(self, stack) -> None:
        for k in range(stack.shape[0]):
            fitrig_push_snapshot(self.h, stack[k])

    def detect(self) -> Tuple[int, np.ndarray]:
        rc, n = fitrig_detect(self.h)
        return rc, fitrig_candidates(self.h, n)

    def close(self):
        if self.h is not None:
            fitrig_plan_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def detect_stack(stack, window: int, nsigma: float, branch: int = BRANCH_IMAGE,
                 storage: int = F32, noise: int = NOISE_MEANSTD, rmode: int = RMODE_ABS,
                 edge: int = EDGE_PARTIAL, dumps: bool = True,
                 stride: int = STRIDE_TILE, autotune: bool = False,
                 mmode: int = MMODE_GLOBAL, accumulate: int = 1, harmonics: int = 1,
                 refine: int = REFINE_PARABOLIC, coding: int = CODING_VALUE) -> dict:
    """Push an (L*accumulate, ny, nx) stack of raw snapshots, detect (on the
    L sums of `accumulate` raw snapshots), and read back candidates and dumps."""
    Lr, ny, nx = (int(d) for d in stack.shape)
    L = Lr // accumulate
    with Plan(nx, ny, L, window, nsigma, branch, storage, noise, rmode, edge,
              stride=stride, autotune=autotune, mmode=mmode, accumulate=accumulate,
              harmonics=harmonics, refine=refine, coding=coding) as p:
        p.push_stack(stack)
        rc, cands = p.detect()
        out = {"status": rc, "candidates": cands}
        if dumps:
            ty, tx = fitrig_tile_grid(p.h)
            out["grid"] = (ty, tx)
            out["M"] = fitrig_global_max(p.h)
            out["M_units"] = np.array([fitrig_unit_normaliser(p.h, s) for s in range(L - 2)])
            if branch & BRANCH_IMAGE:
                out["values"] = np.stack([fitrig_unit_values(p.h, s) for s in range(L - 2)])
                out["noise"] = np.array([fitrig_noise_params(p.h, s) for s in range(L - 2)])
            if branch & BRANCH_FREQ:
                out["eta"], out["bin"] = fitrig_spectrum(p.h)
                out["eta_noise"] = fitrig_noise_params(p.h, -1)
            out["kernel_ms"] = {k: fitrig_kernel_ms(p.h, k) for k in range(5)}
        return out
