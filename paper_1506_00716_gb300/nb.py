"""Thin ctypes binding of the C ABI in include/nb.h.

Argument marshalling only: every step of the method runs in the CUDA
library libnbgb.so.  There is no fallback; if the library is missing or no
GPU is present the calls raise.

Buffers may be numpy arrays (host memory) or torch tensors (host or CUDA);
the library moves data with cudaMemcpyAsync on the context's stream.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

NB_OK = 0
NB_COUL_RF = 0
NB_COUL_EWALD = 1
NB_F_ENERGY = 1
NB_F_VIRIAL = 2
NB_F_PME = 4

STATUS = {0: "NB_OK", 1: "NB_ERR_ARG", 2: "NB_ERR_BOX", 3: "NB_ERR_OOM", 4: "NB_ERR_BUDGET",
          5: "NB_ERR_CUDA", 6: "NB_ERR_NOT_READY", 7: "NB_ERR_TIMEOUT", 8: "NB_ERR_STATE",
          9: "NB_ERR_CAPACITY"}

# the exported functions declared in include/nb.h
EXPORTS = ["nb_last_error", "nb_ctx_create", "nb_ctx_destroy", "nb_ctx_memory", "nb_sys_footprint",
           "nb_sys_create", "nb_sys_create_box", "nb_sys_destroy", "nb_set_exclusions", "nb_grid_put",
           "nb_pairlist_build",
           "nb_pairlist_info", "nb_pairlist_prune", "nb_forces", "nb_pairlist_export", "nb_pairlist_export_slots",
           "nb_batch_create",
           "nb_batch_destroy", "nb_sys_set_coords", "nb_batch_submit", "nb_batch_poll",
           "nb_sys_results", "nb_ctx_set_timing", "nb_ctx_set_timing_stages", "nb_ctx_timing", "nb_eval_info",
           "nb_eval_noalloc", "nb_ctx_set_tuning", "nb_ctx_get_tuning", "nb_server_create",
           "nb_server_destroy", "nb_server_submit", "nb_server_wait", "nb_pme_init", "nb_pme_forces",
           "nb_ctx_inject_alloc_failures", "nb_ewald_force_table", "nb_ewald_energy_table"]
NB_NSTAGE = 11
NB_MOD_LJ_SHIFT = 1
NB_MOD_EWALD_SHIFT = 2
NB_MOD_RF_EXCL = 4
STAGES = ["grid", "search", "prune", "coord", "zero", "forces", "final", "energy", "pme_spread", "pme_fft",
          "pme_gather"]


class NbError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class nb_params(ctypes.Structure):
    _fields_ = [("rc", ctypes.c_double), ("rlist", ctypes.c_double), ("coul", ctypes.c_int),
                ("eps_r", ctypes.c_double), ("eps_rf", ctypes.c_double),
                ("ewald_beta", ctypes.c_double), ("fcoul", ctypes.c_double),
                ("ntypes", ctypes.c_int), ("c6", ctypes.POINTER(ctypes.c_float)),
                ("c12", ctypes.POINTER(ctypes.c_float)), ("modifiers", ctypes.c_uint)]


class nb_pme_params(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_int * 3), ("order", ctypes.c_int)]


class nb_tuning(ctypes.Structure):
    _fields_ = [("max_entries", ctypes.c_int), ("force_min_blocks", ctypes.c_int), ("search_mode", ctypes.c_int),
                ("energy_mode", ctypes.c_int), ("jcluster", ctypes.c_int)]


class nb_request_stats(ctypes.Structure):
    _fields_ = [("latency_s", ctypes.c_double), ("queue_s", ctypes.c_double),
                ("n_pairs", ctypes.c_longlong), ("wave_size", ctypes.c_int)]


class nb_list_info(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_longlong), ("n_items", ctypes.c_longlong),
                ("n_entries", ctypes.c_longlong), ("n_entries_raw", ctypes.c_longlong),
                ("n_slots", ctypes.c_longlong), ("n_entries_inner", ctypes.c_longlong)]


_lib = None
_vp = ctypes.c_void_p
_st = ctypes.c_int


def lib_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libnbgb.so (raise if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or _build.LIB
    if not os.path.exists(path):
        raise NbError(5, f"{path} not found: build it with paper_1506_00716_gb300.build.build()")
    lib = ctypes.CDLL(path)
    sig = {
        "nb_last_error": ([], ctypes.c_char_p),
        "nb_ctx_create": ([ctypes.c_int, _vp, ctypes.c_size_t, ctypes.POINTER(_vp)], _st),
        "nb_ctx_destroy": ([_vp], _st),
        "nb_ctx_memory": ([_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)], _st),
        "nb_ctx_inject_alloc_failures": ([_vp, ctypes.c_int], _st),
        "nb_sys_footprint": ([ctypes.POINTER(nb_params), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_size_t)], _st),
        "nb_sys_create": ([_vp, ctypes.POINTER(nb_params), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(_vp)], _st),
        "nb_sys_create_box": ([_vp, ctypes.POINTER(nb_params), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                               ctypes.POINTER(_vp)], _st),
        "nb_sys_destroy": ([_vp], _st),
        "nb_set_exclusions": ([_vp, _vp, _vp], _st),
        "nb_grid_put": ([_vp, _vp, _vp], _st),
        "nb_pairlist_build": ([_vp], _st),
        "nb_pairlist_info": ([_vp, ctypes.POINTER(nb_list_info)], _st),
        "nb_pairlist_prune": ([_vp, ctypes.c_double], _st),
        "nb_forces": ([_vp, _vp, _vp, _vp, _vp, ctypes.c_uint], _st),
        "nb_pme_init": ([_vp, ctypes.POINTER(nb_pme_params)], _st),
        "nb_pme_forces": ([_vp, _vp, _vp, _vp, _vp, ctypes.c_uint], _st),
        "nb_pairlist_export": ([_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_longlong)], _st),
        "nb_pairlist_export_slots": ([_vp, _vp, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_longlong)], _st),
        "nb_ewald_energy_table": ([ctypes.c_double, ctypes.c_double, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_double)], _st),
        "nb_ewald_force_table": ([ctypes.c_double, ctypes.c_double, _vp, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                  ctypes.POINTER(ctypes.c_double)], _st),
        "nb_batch_create": ([_vp, ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp)], _st),
        "nb_batch_destroy": ([_vp], _st),
        "nb_sys_set_coords": ([_vp, _vp, _vp], _st),
        "nb_batch_submit": ([_vp, ctypes.c_uint, ctypes.POINTER(ctypes.c_ulonglong)], _st),
        "nb_batch_poll": ([_vp, ctypes.c_ulonglong, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int)], _st),
        "nb_sys_results": ([_vp, _vp, _vp, _vp], _st),
        "nb_ctx_set_timing": ([_vp, ctypes.c_int], _st),
        "nb_ctx_set_timing_stages": ([_vp, ctypes.c_uint], _st),
        "nb_ctx_set_tuning": ([_vp, ctypes.POINTER(nb_tuning)], _st),
        "nb_ctx_get_tuning": ([_vp, ctypes.POINTER(nb_tuning)], _st),
        "nb_server_create": ([_vp, ctypes.POINTER(nb_params), ctypes.c_size_t, ctypes.c_int,
                              ctypes.POINTER(_vp)], _st),
        "nb_server_destroy": ([_vp], _st),
        "nb_server_submit": ([_vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double), _vp, _vp, _vp, _vp,
                              ctypes.c_uint, ctypes.POINTER(ctypes.c_ulonglong)], _st),
        "nb_server_wait": ([_vp, ctypes.c_ulonglong, ctypes.c_longlong, _vp, _vp, _vp,
                            ctypes.POINTER(nb_request_stats)], _st),
        "nb_ctx_timing": ([_vp, _vp, _vp, ctypes.c_int], _st),
        "nb_eval_info": ([_vp, ctypes.POINTER(ctypes.c_longlong)], _st),
        "nb_eval_noalloc": ([ctypes.POINTER(nb_params), ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                             _vp, _vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_uint, _vp], _st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def last_error() -> str:
    return load().nb_last_error().decode()


def check(status: int) -> int:
    if status != NB_OK:
        raise NbError(status, last_error())
    return status


def ptr(x):
    """Address of a numpy array or torch tensor (None -> NULL)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return ctypes.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        return ctypes.c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError(f"cannot take the address of {type(x)}")


def make_params(p) -> tuple[nb_params, tuple]:
    """nb_params from an object with rc, rlist, coul, eps_r, eps_rf, beta, fcoul, ntypes, c6, c12."""
    import numpy as np

    c6 = np.ascontiguousarray(p.c6, dtype=np.float32)
    c12 = np.ascontiguousarray(p.c12, dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    s = nb_params(float(p.rc), float(p.rlist), int(p.coul), float(p.eps_r), float(p.eps_rf),
                  float(p.beta), float(p.fcoul), int(p.ntypes), c6.ctypes.data_as(fp),
                  c12.ctypes.data_as(fp), int(getattr(p, "modifiers", 0)))
    return s, (c6, c12)


# ----------------------------------------------------------------- wrappers

def nb_ctx_create(device: int = 0, stream=None, budget: int = 0) -> int:
    out = _vp()
    st = None
    if stream is not None:
        st = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    check(load().nb_ctx_create(device, st, budget, ctypes.byref(out)))
    return out.value


def nb_ctx_destroy(ctx) -> None:
    check(load().nb_ctx_destroy(ctx))


def nb_ctx_memory(ctx) -> tuple[int, int]:
    a, b = ctypes.c_size_t(), ctypes.c_size_t()
    check(load().nb_ctx_memory(ctx, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def nb_ctx_inject_alloc_failures(ctx, count: int) -> None:
    """Test hook: the next `count` device allocations of ctx fail with NB_ERR_OOM."""
    check(load().nb_ctx_inject_alloc_failures(ctx, count))


def nb_sys_footprint(params, natoms: int, box) -> int:
    ps, keep = make_params(params)
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    out = ctypes.c_size_t()
    check(load().nb_sys_footprint(ctypes.byref(ps), natoms, b, ctypes.byref(out)))
    del keep
    return out.value


def nb_sys_create(ctx, params, natoms: int, box, skew=None) -> int:
    """A system in a rectangular box (box = edges), or in a triclinic one when
    skew = (bx, cx, cy) is given and nonzero (box = (ax, by, cz))."""
    ps, keep = make_params(params)
    out = _vp()
    if skew is not None and any(float(v) != 0.0 for v in skew):
        ax, by, cz = (float(v) for v in box)
        bx, cx, cy = (float(v) for v in skew)
        m = (ctypes.c_double * 9)(ax, 0.0, 0.0, bx, by, 0.0, cx, cy, cz)
        check(load().nb_sys_create_box(ctx, ctypes.byref(ps), natoms, m, ctypes.byref(out)))
    else:
        b = (ctypes.c_double * 3)(*[float(v) for v in box])
        check(load().nb_sys_create(ctx, ctypes.byref(ps), natoms, b, ctypes.byref(out)))
    del keep
    return out.value


def nb_sys_destroy(sys) -> None:
    check(load().nb_sys_destroy(sys))


def nb_set_exclusions(sys, excl_index, excl_atoms) -> None:
    import numpy as np

    ei = np.ascontiguousarray(excl_index, dtype=np.int32)
    ea = np.ascontiguousarray(excl_atoms, dtype=np.int32)
    if ea.size == 0:
        ea = np.zeros(1, dtype=np.int32)
    check(load().nb_set_exclusions(sys, ptr(ei), ptr(ea)))


def nb_grid_put(sys, xq, type_) -> None:
    check(load().nb_grid_put(sys, ptr(xq), ptr(type_)))


def nb_pairlist_build(sys) -> None:
    check(load().nb_pairlist_build(sys))


def nb_pairlist_info(sys) -> dict:
    info = nb_list_info()
    check(load().nb_pairlist_info(sys, ctypes.byref(info)))
    return {k: getattr(info, k) for k, _ in nb_list_info._fields_}


def nb_pairlist_prune(sys, r_inner: float) -> None:
    check(load().nb_pairlist_prune(sys, float(r_inner)))


def nb_forces(sys, x_new=None, f=None, energy=None, virial=None, flags: int = 0) -> None:
    check(load().nb_forces(sys, ptr(x_new), ptr(f), ptr(energy), ptr(virial), flags))


def nb_pme_init(sys, grid, order: int = 4) -> None:
    """Enable the long-range (PME) part: grid = (Kx, Ky, Kz), B-spline order."""
    pp = nb_pme_params((ctypes.c_int * 3)(*[int(k) for k in grid]), int(order))
    check(load().nb_pme_init(sys, ctypes.byref(pp)))


def nb_pme_forces(sys, x_new=None, f=None, energy=None, virial=None, flags: int = 0) -> None:
    """Long-range part alone: energy = (E_rec, E_self, E_excl)."""
    check(load().nb_pme_forces(sys, ptr(x_new), ptr(f), ptr(energy), ptr(virial), flags))


def nb_ewald_energy_table(beta: float, rc: float):
    """The energy kernels' Ewald table: (float32 [K, 8] coefficients, h)."""
    import numpy as np

    n = ctypes.c_int()
    h = ctypes.c_double()
    check(load().nb_ewald_energy_table(float(beta), float(rc), None, 0, ctypes.byref(n), ctypes.byref(h)))
    coef = np.zeros((n.value, 8), dtype=np.float32)
    check(load().nb_ewald_energy_table(float(beta), float(rc), coef.ctypes.data_as(_vp), n.value, ctypes.byref(n),
                                       ctypes.byref(h)))
    return coef, h.value


def nb_ewald_force_table(beta: float, rc: float):
    """The force kernel's Ewald table: (float32 [K, 4] coefficients, h)."""
    import numpy as np

    n = ctypes.c_int()
    h = ctypes.c_double()
    check(load().nb_ewald_force_table(float(beta), float(rc), None, 0, ctypes.byref(n), ctypes.byref(h)))
    coef = np.zeros((n.value, 4), dtype=np.float32)
    check(load().nb_ewald_force_table(float(beta), float(rc), coef.ctypes.data_as(_vp), n.value, ctypes.byref(n),
                                      ctypes.byref(h)))
    return coef, h.value


def nb_pairlist_export(sys, perm=None, items=None, cj=None, mask=None) -> int:
    n = ctypes.c_longlong()
    check(load().nb_pairlist_export(sys, ptr(perm), ptr(items), ptr(cj), ptr(mask), ctypes.byref(n)))
    return n.value


def nb_pairlist_export_slots(sys, perm=None, items=None, jslot=None, mask=None) -> int:
    n = ctypes.c_longlong()
    check(load().nb_pairlist_export_slots(sys, ptr(perm), ptr(items), ptr(jslot), ptr(mask), ctypes.byref(n)))
    return n.value


def nb_batch_create(ctx, systems) -> int:
    arr = (_vp * len(systems))(*systems)
    out = _vp()
    check(load().nb_batch_create(ctx, arr, len(systems), ctypes.byref(out)))
    return out.value


def nb_batch_destroy(batch) -> None:
    check(load().nb_batch_destroy(batch))


def nb_sys_set_coords(sys, xq, type_) -> None:
    check(load().nb_sys_set_coords(sys, ptr(xq), ptr(type_)))


def nb_batch_submit(batch, flags: int = 0) -> int:
    t = ctypes.c_ulonglong()
    check(load().nb_batch_submit(batch, flags, ctypes.byref(t)))
    return t.value


def nb_batch_poll(batch, ticket: int, timeout_us: int = 0) -> bool:
    """True once the submission finished; raises NbError on NB_ERR_TIMEOUT and other failures."""
    done = ctypes.c_int()
    check(load().nb_batch_poll(batch, ticket, timeout_us, ctypes.byref(done)))
    return bool(done.value)


def nb_sys_results(sys, f=None, energy=None, virial=None) -> None:
    check(load().nb_sys_results(sys, ptr(f), ptr(energy), ptr(virial)))


def nb_ctx_set_timing(ctx, enable: bool) -> None:
    check(load().nb_ctx_set_timing(ctx, 1 if enable else 0))


def nb_ctx_set_timing_stages(ctx, stages) -> None:
    """Time only the named stages (names from STAGES)."""
    mask = 0
    for name in stages:
        mask |= 1 << STAGES.index(name)
    check(load().nb_ctx_set_timing_stages(ctx, mask))


def nb_ctx_timing(ctx, reset: bool = False) -> dict:
    """{stage: (total ms, launches)} of the stages timed since the last reset."""
    ms = (ctypes.c_double * NB_NSTAGE)()
    n = (ctypes.c_longlong * NB_NSTAGE)()
    check(load().nb_ctx_timing(ctx, ctypes.cast(ms, _vp), ctypes.cast(n, _vp), 1 if reset else 0))
    return {name: (ms[k], n[k]) for k, name in enumerate(STAGES)}


def nb_eval_info(sys) -> dict:
    n = ctypes.c_longlong()
    check(load().nb_eval_info(sys, ctypes.byref(n)))
    return {"n_pairs": n.value}


def nb_eval_noalloc(params, natoms: int, box, excl_index, excl_atoms, xq, type_, f=None, energy=None,
                    virial=None, flags: int = 0, stream=None) -> None:
    """Allocation-free evaluation through a fixed scratch array (see include/nb.h)."""
    import numpy as np

    ps, keep = make_params(params)
    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    ei = ea = None
    if excl_index is not None:
        ei = np.ascontiguousarray(excl_index, dtype=np.int32)
        ea = np.ascontiguousarray(excl_atoms, dtype=np.int32)
        if ea.size == 0:
            ea = np.zeros(1, dtype=np.int32)
    st = None
    if stream is not None:
        st = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    check(load().nb_eval_noalloc(ctypes.byref(ps), natoms, b, ptr(ei), ptr(ea), ptr(xq), ptr(type_),
                                 ptr(f), ptr(energy), ptr(virial), flags, st))
    del keep


def nb_ctx_set_tuning(ctx, max_entries: int = 32, force_min_blocks: int = 3, search_mode: int = 0,
                      energy_mode: int = 0, jcluster: int = 8) -> None:
    t = nb_tuning(int(max_entries), int(force_min_blocks), int(search_mode), int(energy_mode), int(jcluster))
    check(load().nb_ctx_set_tuning(ctx, ctypes.byref(t)))


def nb_ctx_get_tuning(ctx) -> dict:
    t = nb_tuning()
    check(load().nb_ctx_get_tuning(ctx, ctypes.byref(t)))
    return {"max_entries": t.max_entries, "force_min_blocks": t.force_min_blocks, "search_mode": t.search_mode,
            "energy_mode": t.energy_mode, "jcluster": t.jcluster or 8}


def nb_server_create(ctx, params, budget: int = 0, max_wave: int = 64) -> int:
    ps, keep = make_params(params)
    out = _vp()
    check(load().nb_server_create(ctx, ctypes.byref(ps), budget, max_wave, ctypes.byref(out)))
    del keep
    return out.value


def nb_server_destroy(srv) -> None:
    check(load().nb_server_destroy(srv))


def nb_server_submit(srv, natoms: int, box, xq, type_, excl_index=None, excl_atoms=None, flags: int = 0) -> int:
    import numpy as np

    b = (ctypes.c_double * 3)(*[float(v) for v in box])
    ei = ea = None
    if excl_index is not None:
        ei = np.ascontiguousarray(excl_index, dtype=np.int32)
        ea = np.ascontiguousarray(excl_atoms, dtype=np.int32)
        if ea.size == 0:
            ea = np.zeros(1, dtype=np.int32)
    t = ctypes.c_ulonglong()
    check(load().nb_server_submit(srv, natoms, b, ptr(xq), ptr(type_), ptr(ei), ptr(ea), flags,
                                  ctypes.byref(t)))
    return t.value


def nb_server_wait(srv, ticket: int, timeout_us: int = -1, f=None, energy=None, virial=None) -> dict:
    st = nb_request_stats()
    check(load().nb_server_wait(srv, ticket, timeout_us, ptr(f), ptr(energy), ptr(virial), ctypes.byref(st)))
    return {k: getattr(st, k) for k, _ in nb_request_stats._fields_}
