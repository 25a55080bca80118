"""Python binding of liblbm.so (include/lbm.h): argument marshalling only.

Every function keeps its C name and argument order; numpy arrays stand in for host pointers, and
a torch stream (or its raw handle) for the cudaStream_t of lbm_set_stream.  All arithmetic of the
time step runs in the CUDA library: if liblbm.so is missing this module raises instead of falling
back to anything else.
"""
from __future__ import annotations

import ctypes
import re
from pathlib import Path

import numpy as np

from .builder import LIB, INCLUDE

LBM_OK = 0
LBM_EINVAL = -1
LBM_ENOMEM = -2
LBM_ECUDA = -3
LBM_ETIMEOUT = -4
LBM_ENONFINITE = -5
LBM_ERANGE = -6

LBM_D2Q9, LBM_D2Q37 = 9, 37
LBM_GEOM_PLATE, LBM_GEOM_BEAM, LBM_GEOM_MASK, LBM_GEOM_NONE = 0, 1, 2, 3
LBM_DRIVE_WALL, LBM_DRIVE_BODYFORCE = 0, 1
LBM_COLL_BGK, LBM_COLL_REGULARIZED = 0, 1
LBM_STORE_F64, LBM_STORE_F32, LBM_STORE_BF16, LBM_STORE_F16 = 0, 1, 2, 3
LBM_FLUID, LBM_BODY, LBM_WALL = 0, 1, 2
LBM_BATCH_STREAMS, LBM_BATCH_PERSISTENT = 0, 1
LBM_SCHEME_BOUNCEBACK, LBM_SCHEME_DIFFUSE = 0, 1
LBM_LAYOUT_AB, LBM_LAYOUT_AA = 0, 1
STORAGE_BYTES = {LBM_STORE_F64: 8, LBM_STORE_F32: 4, LBM_STORE_BF16: 2, LBM_STORE_F16: 2}


class LbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class lbm_geometry(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("lx", ctypes.c_int),
        ("ly", ctypes.c_int),
        ("drive", ctypes.c_int),
        ("u0", ctypes.c_double),
        ("rho0", ctypes.c_double),
        ("mask", ctypes.POINTER(ctypes.c_ubyte)),
        ("eq_order", ctypes.c_int),
        ("collision", ctypes.c_int),
        ("storage", ctypes.c_int),
        ("wall_scheme", ctypes.c_int),
        ("layout", ctypes.c_int),
    ]


class lbm_info_t(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("pitch", ctypes.c_int),
        ("storage", ctypes.c_int), ("collision", ctypes.c_int), ("eq_order", ctypes.c_int), ("drive", ctypes.c_int),
        ("tau", ctypes.c_double), ("omega", ctypes.c_double), ("u0", ctypes.c_double), ("rho0", ctypes.c_double),
        ("theta", ctypes.c_double),
        ("steps_done", ctypes.c_long),
        ("n_fluid", ctypes.c_size_t), ("n_boundary", ctypes.c_size_t),
        ("bytes_per_step", ctypes.c_size_t), ("device_bytes", ctypes.c_size_t),
        ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
        ("h2d_bytes", ctypes.c_size_t), ("d2h_bytes", ctypes.c_size_t),
        ("variant", ctypes.c_int),
        ("layout", ctypes.c_int),
        ("force_1e4", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class lbm_batch_tune_entry(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("segment", ctypes.c_int), ("us_per_step", ctypes.c_double)]


class lbm_instance_desc(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("tau", ctypes.c_double), ("omega", ctypes.c_double),
        ("geom", lbm_geometry),
        ("nsteps", ctypes.c_long),
    ]


class lbm_batch_info_t(ctypes.Structure):
    _fields_ = [
        ("lattice", ctypes.c_int), ("storage", ctypes.c_int), ("collision", ctypes.c_int),
        ("live", ctypes.c_int), ("running", ctypes.c_int),
        ("fluid_running", ctypes.c_size_t), ("bytes_per_step", ctypes.c_size_t),
        ("batch_steps", ctypes.c_longlong), ("launches", ctypes.c_longlong),
        ("lattice_updates", ctypes.c_double),
        ("budget_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t),
        ("max_blocks", ctypes.c_int), ("uses_graph", ctypes.c_int),
        ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
        ("mode", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class lbm_tune_entry(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("block_x", ctypes.c_int), ("block_y", ctypes.c_int),
                ("us_per_step", ctypes.c_double)]


class lbm_request(ctypes.Structure):
    _fields_ = [("desc", lbm_instance_desc), ("skip_periods", ctypes.c_double), ("perimeter", ctypes.c_double)]


class lbm_result(ctypes.Structure):
    _fields_ = [
        ("id", ctypes.c_longlong), ("status", ctypes.c_int),
        ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
        ("f_in", ctypes.c_double), ("f_q", ctypes.c_double), ("f_0", ctypes.c_double),
        ("gamma_bar", ctypes.c_double), ("steps", ctypes.c_long), ("fluid_nodes", ctypes.c_size_t),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class lbm_server_stats_t(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("rounds", ctypes.c_longlong),
        ("lattice_updates", ctypes.c_double), ("busy_s", ctypes.c_double), ("elapsed_s", ctypes.c_double),
        ("budget_bytes", ctypes.c_size_t), ("used_bytes", ctypes.c_size_t), ("peak_used_bytes", ctypes.c_size_t),
        ("peak_running", ctypes.c_int), ("worker_error", ctypes.c_int),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)


def header_functions() -> list[str]:
    """Names of the functions include/*.h declares."""
    names = []
    for h in sorted(Path(INCLUDE).glob("*.h")):
        text = re.sub(r"/\*.*?\*/", "", h.read_text(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[a-z_]+\s*\**\s*(lbm_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return names


def lib():
    """The loaded liblbm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not Path(LIB).exists():
            raise RuntimeError(f"{LIB} is missing: build it with paper_0904_4504_gb300.builder.build()")
        L = ctypes.CDLL(str(LIB))
        sig = {
            "lbm_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.POINTER(lbm_geometry), ctypes.POINTER(_P)]),
            "lbm_step": (ctypes.c_int, [_P, ctypes.c_long]),
            "lbm_synchronize": (ctypes.c_int, [_P]),
            "lbm_force_history": (ctypes.c_int, [_P, _D, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
            "lbm_fit": (ctypes.c_int, [_P, ctypes.c_double, _D, _D, _D]),
            "lbm_gamma_bar": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_double, _D]),
            "lbm_destroy": (None, [_P]),
            "lbm_last_error": (ctypes.c_char_p, []),
            "lbm_set_stream": (ctypes.c_int, [_P, _P]),
            "lbm_get_state": (ctypes.c_int, [_P, _D, ctypes.c_size_t]),
            "lbm_set_state": (ctypes.c_int, [_P, _D, ctypes.c_size_t]),
            "lbm_get_labels": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_ubyte), ctypes.c_size_t]),
            "lbm_geometry_links": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(lbm_geometry),
                                                  ctypes.POINTER(ctypes.c_ubyte), ctypes.POINTER(ctypes.c_ulonglong),
                                                  ctypes.POINTER(ctypes.c_ulonglong), ctypes.c_size_t,
                                                  ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
            "lbm_info": (ctypes.c_int, [_P, ctypes.POINTER(lbm_info_t)]),
            "lbm_set_tile": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int]),
            "lbm_set_variant": (ctypes.c_int, [_P, ctypes.c_int]),
            "lbm_tune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(lbm_tune_entry), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int)]),
            "lbm_autotune": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(lbm_tune_entry)]),
            "lbm_lattice_velocities": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), _D, _D]),
            "lbm_params_from_tau_omega": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                         _D, _D, ctypes.POINTER(ctypes.c_int)]),
            "lbm_step_noalloc": (ctypes.c_int, [_P, ctypes.c_long, _P, _P, _P, _P]),
            "lbm_batch_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_size_t,
                                                ctypes.POINTER(_P)]),
            "lbm_batch_footprint": (ctypes.c_int, [ctypes.POINTER(lbm_instance_desc), ctypes.POINTER(ctypes.c_size_t)]),
            "lbm_batch_add": (ctypes.c_int, [_P, ctypes.POINTER(lbm_instance_desc), ctypes.POINTER(ctypes.c_int)]),
            "lbm_batch_run": (ctypes.c_int, [_P, ctypes.c_long]),
            "lbm_batch_synchronize": (ctypes.c_int, [_P]),
            "lbm_batch_status": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_long),
                                                ctypes.POINTER(ctypes.c_long)]),
            "lbm_batch_instance": (_P, [_P, ctypes.c_int]),
            "lbm_batch_remove": (ctypes.c_int, [_P, ctypes.c_int]),
            "lbm_batch_set_barrier_limit": (ctypes.c_int, [_P, ctypes.c_longlong]),
            "lbm_batch_set_mode": (ctypes.c_int, [_P, ctypes.c_int]),
            "lbm_batch_set_variant": (ctypes.c_int, [_P, ctypes.c_int]),
            "lbm_batch_set_segment": (ctypes.c_int, [_P, ctypes.c_int]),
            "lbm_batch_tune": (ctypes.c_int, [_P, ctypes.POINTER(lbm_instance_desc), ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(lbm_batch_tune_entry), ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_int)]),
            "lbm_batch_autotune": (ctypes.c_int, [_P, ctypes.POINTER(lbm_instance_desc), ctypes.c_int, ctypes.c_int,
                                                  ctypes.POINTER(lbm_batch_tune_entry)]),
            "lbm_batch_info": (ctypes.c_int, [_P, ctypes.POINTER(lbm_batch_info_t)]),
            "lbm_batch_set_stream": (ctypes.c_int, [_P, _P]),
            "lbm_batch_destroy": (None, [_P]),
            "lbm_server_create": (ctypes.c_int, [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(_P)]),
            "lbm_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(lbm_request), ctypes.POINTER(ctypes.c_longlong)]),
            "lbm_server_set_batch_mode": (ctypes.c_int, [_P, ctypes.c_int]),
            "lbm_server_set_class_kernel": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                           ctypes.c_int]),
            "lbm_server_poll": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.POINTER(lbm_result)]),
            "lbm_server_wait": (ctypes.c_int, [_P, ctypes.c_longlong, ctypes.c_double, ctypes.POINTER(lbm_result)]),
            "lbm_server_force_history": (ctypes.c_int, [_P, ctypes.c_longlong, _D, ctypes.c_size_t,
                                                        ctypes.POINTER(ctypes.c_size_t)]),
            "lbm_server_release": (ctypes.c_int, [_P, ctypes.c_longlong]),
            "lbm_server_stats": (ctypes.c_int, [_P, ctypes.POINTER(lbm_server_stats_t)]),
            "lbm_server_destroy": (None, [_P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc: int) -> int:
    if rc < 0:
        raise LbmError(rc, lib().lbm_last_error().decode())
    return rc


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_D)


# ------------------------------------------------------------------------------------------------
# the C functions, same names
# ------------------------------------------------------------------------------------------------

def lbm_last_error() -> str:
    return lib().lbm_last_error().decode()


def lbm_lattice_velocities(lattice: int):
    """(c (Q, 2) int, w (Q,), theta) in the library's direction order."""
    Q = _check(lib().lbm_lattice_velocities(lattice, None, None, None))
    c = (ctypes.c_int * (2 * Q))()
    w = np.zeros(Q)
    th = ctypes.c_double()
    _check(lib().lbm_lattice_velocities(lattice, c, _dp(w), ctypes.byref(th)))
    return np.array(c[:], dtype=np.int64).reshape(Q, 2), w, th.value


def lbm_params_from_tau_omega(lattice: int, tau_omega: float, delta_min: float = 4.0, p_min: int = 128):
    """(tau, omega, period) for a nondimensional frequency tau*omega."""
    tau, om, P = ctypes.c_double(), ctypes.c_double(), ctypes.c_int()
    _check(lib().lbm_params_from_tau_omega(lattice, tau_omega, delta_min, p_min, ctypes.byref(tau), ctypes.byref(om),
                                           ctypes.byref(P)))
    return tau.value, om.value, P.value


def make_geometry(kind=LBM_GEOM_NONE, lx=0, ly=0, drive=LBM_DRIVE_WALL, u0=0.0, rho0=1.0, mask=None, eq_order=2,
                  collision=LBM_COLL_REGULARIZED, storage=LBM_STORE_F32, wall_scheme=LBM_SCHEME_BOUNCEBACK,
                  layout=LBM_LAYOUT_AB):
    """An lbm_geometry; `mask` (ny x nx uint8) is kept alive on the returned object."""
    g = lbm_geometry(kind, lx, ly, drive, u0, rho0, None, eq_order, collision, storage, wall_scheme, layout)
    if mask is not None:
        m = np.ascontiguousarray(mask, dtype=np.uint8)
        g._mask_ref = m
        g.mask = m.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    return g


def lbm_create(lattice: int, nx: int, ny: int, tau: float, omega: float, geom: lbm_geometry) -> int:
    h = _P()
    _check(lib().lbm_create(lattice, nx, ny, tau, omega, ctypes.byref(geom), ctypes.byref(h)))
    return h.value


def lbm_step(sim: int, n: int) -> None:
    _check(lib().lbm_step(sim, n))


def lbm_synchronize(sim: int) -> None:
    _check(lib().lbm_synchronize(sim))


def lbm_force_history(sim: int, cap_steps: int | None = None) -> np.ndarray:
    """(steps, 2) FP64 array of (Fx, Fy)."""
    n = ctypes.c_size_t()
    _check(lib().lbm_force_history(sim, None, 0, ctypes.byref(n)))
    cap = n.value if cap_steps is None else min(cap_steps, n.value)
    out = np.zeros((cap, 2))
    _check(lib().lbm_force_history(sim, _dp(out), cap, ctypes.byref(n)))
    return out


def lbm_fit(sim: int, skip_periods: float):
    """(f_in, f_q, f_0)."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().lbm_fit(sim, skip_periods, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def lbm_gamma_bar(sim: int, f_in: float, perimeter: float) -> float:
    g = ctypes.c_double()
    _check(lib().lbm_gamma_bar(sim, f_in, perimeter, ctypes.byref(g)))
    return g.value


def lbm_destroy(sim: int) -> None:
    if sim:
        lib().lbm_destroy(sim)


def lbm_set_stream(sim: int, stream=None) -> None:
    """`stream`: a torch.cuda.Stream or a raw cudaStream_t handle (None or 0: the default stream)."""
    handle = getattr(stream, "cuda_stream", stream)
    _check(lib().lbm_set_stream(sim, handle or None))


def lbm_info(sim: int) -> dict:
    o = lbm_info_t()
    _check(lib().lbm_info(sim, ctypes.byref(o)))
    return o.as_dict()


def lbm_get_state(sim: int) -> np.ndarray:
    """Deviations g = f - w rho0 as a (Q, ny, nx) FP64 array."""
    i = lbm_info(sim)
    out = np.zeros((i["lattice"], i["ny"], i["nx"]))
    _check(lib().lbm_get_state(sim, _dp(out), out.size))
    return out


def lbm_set_state(sim: int, g: np.ndarray) -> None:
    g = np.ascontiguousarray(g, dtype=np.float64)
    _check(lib().lbm_set_state(sim, _dp(g), g.size))


def lbm_geometry_links(lattice: int, nx: int, ny: int, geom) -> tuple:
    """(cls, body, wall, n_fluid, n_boundary) of a geometry on the host: node classes (ny, nx) uint8
    and blocked-link masks (ny, nx) uint64 (bit i: direction i of lbm_lattice_velocities)."""
    cls = np.zeros((ny, nx), dtype=np.uint8)
    body = np.zeros((ny, nx), dtype=np.uint64)
    wall = np.zeros((ny, nx), dtype=np.uint64)
    nf, nb = ctypes.c_size_t(), ctypes.c_size_t()
    u64 = ctypes.POINTER(ctypes.c_ulonglong)
    _check(lib().lbm_geometry_links(lattice, nx, ny, ctypes.byref(geom), cls.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)),
                                    body.ctypes.data_as(u64), wall.ctypes.data_as(u64), cls.size, ctypes.byref(nf),
                                    ctypes.byref(nb)))
    return cls, body, wall, nf.value, nb.value


def lbm_get_labels(sim: int) -> np.ndarray:
    i = lbm_info(sim)
    out = np.zeros((i["ny"], i["nx"]), dtype=np.uint8)
    _check(lib().lbm_get_labels(sim, out.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)), out.size))
    return out


def lbm_set_tile(sim: int, block_x: int, block_y: int) -> None:
    _check(lib().lbm_set_tile(sim, block_x, block_y))


def lbm_set_variant(sim: int, variant: int) -> None:
    _check(lib().lbm_set_variant(sim, variant))


def lbm_tune(sim: int, steps: int = 20) -> list[dict]:
    """Time every kernel candidate on a clone; list of {variant, block_x, block_y, us_per_step}."""
    out = (lbm_tune_entry * 32)()
    n = ctypes.c_int()
    _check(lib().lbm_tune(sim, steps, out, 32, ctypes.byref(n)))
    return [{f: getattr(out[k], f) for f, _ in lbm_tune_entry._fields_} for k in range(n.value)]


def lbm_autotune(sim: int, steps: int = 20) -> dict:
    best = lbm_tune_entry()
    _check(lib().lbm_autotune(sim, steps, ctypes.byref(best)))
    return {f: getattr(best, f) for f, _ in lbm_tune_entry._fields_}


def lbm_step_noalloc(sim: int, n: int, g_in: int, g_out: int, force_out: int, stream=None) -> None:
    """One step between caller-owned device buffers (raw device addresses, e.g. tensor.data_ptr()),
    with the force written to force_out (2 doubles); allocates nothing."""
    handle = getattr(stream, "cuda_stream", stream)
    _check(lib().lbm_step_noalloc(sim, n, g_in, g_out, force_out, handle or None))


# ------------------------------------------------------------------------------------------------
# batches
# ------------------------------------------------------------------------------------------------

def make_instance(lattice, nx, ny, tau, omega, nsteps, **geometry) -> lbm_instance_desc:
    g = make_geometry(**geometry)
    d = lbm_instance_desc(lattice, nx, ny, tau, omega, g, nsteps)
    d._geom_ref = g
    return d


def lbm_batch_create(lattice: int, storage: int, collision: int, device_budget_bytes: int = 0) -> int:
    h = _P()
    _check(lib().lbm_batch_create(lattice, storage, collision, device_budget_bytes, ctypes.byref(h)))
    return h.value


def lbm_batch_footprint(desc: lbm_instance_desc) -> int:
    n = ctypes.c_size_t()
    _check(lib().lbm_batch_footprint(ctypes.byref(desc), ctypes.byref(n)))
    return n.value


def lbm_batch_add(batch: int, desc: lbm_instance_desc) -> int:
    slot = ctypes.c_int()
    _check(lib().lbm_batch_add(batch, ctypes.byref(desc), ctypes.byref(slot)))
    return slot.value


def lbm_batch_run(batch: int, steps: int) -> None:
    _check(lib().lbm_batch_run(batch, steps))


def lbm_batch_synchronize(batch: int) -> None:
    _check(lib().lbm_batch_synchronize(batch))


def lbm_batch_status(batch: int, slot: int):
    done, total = ctypes.c_long(), ctypes.c_long()
    _check(lib().lbm_batch_status(batch, slot, ctypes.byref(done), ctypes.byref(total)))
    return done.value, total.value


def lbm_batch_instance(batch: int, slot: int) -> int:
    h = lib().lbm_batch_instance(batch, slot)
    if not h:
        raise LbmError(LBM_ERANGE, f"no instance in slot {slot}")
    return h


def lbm_batch_remove(batch: int, slot: int) -> None:
    _check(lib().lbm_batch_remove(batch, slot))


def lbm_batch_set_mode(batch: int, mode: int) -> None:
    _check(lib().lbm_batch_set_mode(batch, mode))


def lbm_batch_set_variant(batch: int, variant: int) -> None:
    _check(lib().lbm_batch_set_variant(batch, variant))


def lbm_batch_tune(batch: int, descs, steps: int = 20) -> list:
    """Time the batch's kernel candidates on clones of the instance descriptions (see lbm.h)."""
    arr = (lbm_instance_desc * len(descs))(*descs)
    out = (lbm_batch_tune_entry * 64)()
    n = ctypes.c_int()
    _check(lib().lbm_batch_tune(batch, arr, len(descs), steps, out, 64, ctypes.byref(n)))
    return [{"variant": out[k].variant, "segment": out[k].segment, "us_per_step": out[k].us_per_step}
            for k in range(n.value)]


def lbm_batch_autotune(batch: int, descs, steps: int = 20) -> dict:
    arr = (lbm_instance_desc * len(descs))(*descs)
    best = lbm_batch_tune_entry()
    _check(lib().lbm_batch_autotune(batch, arr, len(descs), steps, ctypes.byref(best)))
    return {"variant": best.variant, "segment": best.segment, "us_per_step": best.us_per_step}


def lbm_batch_set_segment(batch: int, tiles: int) -> None:
    _check(lib().lbm_batch_set_segment(batch, tiles))


def lbm_batch_set_barrier_limit(batch: int, cycles: int) -> None:
    _check(lib().lbm_batch_set_barrier_limit(batch, cycles))


def lbm_batch_info(batch: int) -> dict:
    o = lbm_batch_info_t()
    _check(lib().lbm_batch_info(batch, ctypes.byref(o)))
    return o.as_dict()


def lbm_batch_set_stream(batch: int, stream=None) -> None:
    handle = getattr(stream, "cuda_stream", stream)
    _check(lib().lbm_batch_set_stream(batch, handle or None))


def lbm_batch_destroy(batch: int) -> None:
    if batch:
        lib().lbm_batch_destroy(batch)


# ------------------------------------------------------------------------------------------------
# serving
# ------------------------------------------------------------------------------------------------

def lbm_server_create(device_budget_bytes: int = 0, steps_per_round: int = 64) -> int:
    h = _P()
    _check(lib().lbm_server_create(device_budget_bytes, steps_per_round, ctypes.byref(h)))
    return h.value


def make_request(desc: lbm_instance_desc, skip_periods: float, perimeter: float = 0.0) -> lbm_request:
    r = lbm_request(desc, skip_periods, perimeter)
    r._desc_ref = desc
    return r


def lbm_server_set_batch_mode(server: int, mode: int) -> None:
    _check(lib().lbm_server_set_batch_mode(server, mode))


def lbm_server_set_class_kernel(server: int, lattice: int, storage: int, collision: int, variant: int,
                                segment: int = 0) -> None:
    _check(lib().lbm_server_set_class_kernel(server, lattice, storage, collision, variant, segment))


def lbm_server_submit(server: int, req: lbm_request) -> int:
    i = ctypes.c_longlong()
    _check(lib().lbm_server_submit(server, ctypes.byref(req), ctypes.byref(i)))
    return i.value


def lbm_server_poll(server: int, rid: int):
    """(finished, result dict)."""
    r = lbm_result()
    done = _check(lib().lbm_server_poll(server, rid, ctypes.byref(r)))
    return bool(done), r.as_dict()


def lbm_server_wait(server: int, rid: int, timeout_s: float = 60.0):
    r = lbm_result()
    done = _check(lib().lbm_server_wait(server, rid, timeout_s, ctypes.byref(r)))
    return bool(done), r.as_dict()


def lbm_server_force_history(server: int, rid: int) -> np.ndarray:
    n = ctypes.c_size_t()
    _check(lib().lbm_server_force_history(server, rid, None, 0, ctypes.byref(n)))
    out = np.zeros((n.value, 2))
    _check(lib().lbm_server_force_history(server, rid, _dp(out), n.value, ctypes.byref(n)))
    return out


def lbm_server_release(server: int, rid: int) -> None:
    _check(lib().lbm_server_release(server, rid))


def lbm_server_stats(server: int) -> dict:
    o = lbm_server_stats_t()
    _check(lib().lbm_server_stats(server, ctypes.byref(o)))
    return o.as_dict()


def lbm_server_destroy(server: int) -> None:
    if server:
        lib().lbm_server_destroy(server)


class Simulation:
    """Owning handle: ``with Simulation(...) as s: lbm_step(s.handle, n)``."""

    def __init__(self, lattice, nx, ny, tau, omega, **geometry):
        self.geom = make_geometry(**geometry)
        self.handle = lbm_create(lattice, nx, ny, tau, omega, self.geom)

    def close(self):
        if self.handle:
            lbm_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
