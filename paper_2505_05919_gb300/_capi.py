"""ctypes binding of ``include/cvf.h`` -- argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: the work runs in ``libcvf.so``'s CUDA kernels.  The
library must have been built (``paper_2505_05919_gb300.build.build()``);
without it every call raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

CVF_OK, CVF_EINVAL, CVF_ENOMEM, CVF_ECUDA, CVF_ETIMEOUT, CVF_EBUSY, CVF_EOVERFLOW = range(7)
CVF_INIT_RANDOM, CVF_INIT_ORDERED = 0, 1
CVF_SCHED_CHECKERBOARD, CVF_SCHED_LAYERED = 0, 1

_ERRNAMES = {1: "CVF_EINVAL", 2: "CVF_ENOMEM", 3: "CVF_ECUDA", 4: "CVF_ETIMEOUT",
             5: "CVF_EBUSY", 6: "CVF_EOVERFLOW", 7: "CVF_EBOUNDS"}


class CvfError(RuntimeError):
    def __init__(self, code: int, func: str, text: str):
        self.code = code
        super().__init__("%s returned %s: %s" % (func, _ERRNAMES.get(code, str(code)), text))


class cvf_params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("q", ctypes.c_int32),
                ("epsilon", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("J", ctypes.c_double), ("J_sigma", ctypes.c_double),
                ("v_HB", ctypes.c_double), ("kT", ctypes.c_double),
                ("P", ctypes.c_double), ("v_iso_init", ctypes.c_double),
                ("dv_max_frac", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("init", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("volume_moves", ctypes.c_int32), ("rng_words", ctypes.c_int32),
                ("eta_moves", ctypes.c_int32), ("pad", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class cvf_obs(ctypes.Structure):
    _fields_ = [("sweep", ctypes.c_int64), ("n_hb", ctypes.c_int64),
                ("n_hb_raw", ctypes.c_int64), ("n_coop", ctypes.c_int64),
                ("acc_sigma", ctypes.c_int64), ("acc_volume", ctypes.c_int64),
                ("V_iso", ctypes.c_double), ("V", ctypes.c_double),
                ("U_LJ", ctypes.c_double), ("H", ctypes.c_double),
                ("g", ctypes.c_int32), ("status", ctypes.c_int32),
                ("n_state", ctypes.c_int64 * 8)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f != "n_state"}
        d["n_state"] = list(self.n_state)
        return d


_P = ctypes.POINTER
_vp = ctypes.c_void_p
_SIGS = {
    "cvf_last_error": (ctypes.c_char_p, []),
    "cvf_params_default": (ctypes.c_int, [_P(cvf_params)]),
    "cvf_params_physical": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _P(cvf_params)]),
    "cvf_threshold_table": (ctypes.c_int, [_P(cvf_params), _P(ctypes.c_uint64)]),
    "cvf_create": (ctypes.c_int, [_P(cvf_params), _vp, _vp, _P(_vp)]),
    "cvf_sweep": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int32]),
    "cvf_observables": (ctypes.c_int, [_vp, _P(cvf_obs)]),
    "cvf_drain_series": (ctypes.c_int, [_vp, _P(cvf_obs), ctypes.c_int64, _P(ctypes.c_int64)]),
    "cvf_get_state": (ctypes.c_int, [_vp, _P(ctypes.c_uint16), ctypes.c_size_t]),
    "cvf_set_state": (ctypes.c_int, [_vp, _P(ctypes.c_uint16), ctypes.c_size_t, ctypes.c_double,
                                     ctypes.c_int64]),
    "cvf_recount": (ctypes.c_int, [_vp, _P(ctypes.c_int64), _P(ctypes.c_int64)]),
    "cvf_state_device_ptr": (ctypes.c_int, [_vp, _P(_vp)]),
    "cvf_destroy": (ctypes.c_int, [_vp]),
    "cvf_set_tiles": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "cvf_get_tiles": (ctypes.c_int, [_vp, _P(ctypes.c_int32), _P(ctypes.c_int32), _P(ctypes.c_int32)]),
    "cvf_philox_probe": (ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64, _vp, _vp]),
    "cvf_sweep_noalloc": (ctypes.c_int, [_P(cvf_params), _vp, ctypes.c_double, ctypes.c_int64,
                                         ctypes.c_int64, ctypes.c_int32, _P(cvf_obs), ctypes.c_int64,
                                         _P(ctypes.c_int64), _P(cvf_obs), _vp]),
    "cvf_batch_create": (ctypes.c_int, [_P(cvf_params), ctypes.c_int32, _vp, _P(_vp)]),
    "cvf_batch_add": (ctypes.c_int, [_vp, _P(cvf_params), _P(ctypes.c_int32)]),
    "cvf_batch_remove": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "cvf_batch_size": (ctypes.c_int, [_vp, _P(ctypes.c_int32), _P(ctypes.c_int32)]),
    "cvf_batch_sweep": (ctypes.c_int, [_vp, _P(ctypes.c_int64), ctypes.c_int32]),
    "cvf_batch_sync": (ctypes.c_int, [_vp]),
    "cvf_batch_observables": (ctypes.c_int, [_vp, ctypes.c_int32, _P(cvf_obs)]),
    "cvf_batch_memory": (ctypes.c_int, [_vp, _P(ctypes.c_uint64), _P(ctypes.c_uint64)]),
    "cvf_batch_observables_many": (ctypes.c_int, [_vp, _P(ctypes.c_int32), ctypes.c_int32,
                                                  _P(cvf_obs)]),
    "cvf_batch_observables_enqueue": (ctypes.c_int, [_vp, _P(ctypes.c_int32), ctypes.c_int32,
                                                     _P(ctypes.c_int64)]),
    "cvf_batch_observables_collect": (ctypes.c_int, [_vp, ctypes.c_int64, _P(cvf_obs),
                                                     ctypes.c_int32]),
    "cvf_batch_get_state": (ctypes.c_int, [_vp, ctypes.c_int32, _P(ctypes.c_uint16), ctypes.c_size_t]),
    "cvf_batch_set_tiles": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "cvf_batch_get_tiles": (ctypes.c_int, [_vp, _P(ctypes.c_int32), _P(ctypes.c_int32)]),
    "cvf_batch_tile_config": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_int32), _P(ctypes.c_int32)]),
    "cvf_batch_config_threads": (ctypes.c_int, [ctypes.c_int32, _P(ctypes.c_int32)]),
    "cvf_batch_destroy": (ctypes.c_int, [_vp]),
    # cubic lattice (the paper's 3D model)
    "cvf3_params_physical": (ctypes.c_int, [ctypes.c_double, ctypes.c_double, _P(cvf_params)]),
    "cvf3_threshold_table": (ctypes.c_int, [_P(cvf_params), _P(ctypes.c_uint64)]),
    "cvf3_create": (ctypes.c_int, [_P(cvf_params), _vp, _vp, _P(_vp)]),
    "cvf3_sweep": (ctypes.c_int, [_vp, ctypes.c_int64, ctypes.c_int32]),
    "cvf3_observables": (ctypes.c_int, [_vp, _P(cvf_obs)]),
    "cvf3_drain_series": (ctypes.c_int, [_vp, _P(cvf_obs), ctypes.c_int64, _P(ctypes.c_int64)]),
    "cvf3_get_state": (ctypes.c_int, [_vp, _P(ctypes.c_uint32), ctypes.c_size_t]),
    "cvf3_set_state": (ctypes.c_int, [_vp, _P(ctypes.c_uint32), ctypes.c_size_t, ctypes.c_double,
                                      ctypes.c_int64]),
    "cvf3_recount": (ctypes.c_int, [_vp, _P(ctypes.c_int64), _P(ctypes.c_int64)]),
    "cvf3_get_eta": (ctypes.c_int, [_vp, _P(ctypes.c_uint8), ctypes.c_size_t]),
    "cvf3_set_eta": (ctypes.c_int, [_vp, _P(ctypes.c_uint8), ctypes.c_size_t]),
    "cvf3_state_device_ptr": (ctypes.c_int, [_vp, _P(_vp)]),
    "cvf3_destroy": (ctypes.c_int, [_vp]),
    "cvf3_set_resident": (ctypes.c_int, [_vp, ctypes.c_int32]),
    "cvf3_get_resident": (ctypes.c_int, [_vp, _P(ctypes.c_int32)]),
    "cvf_get_window": (ctypes.c_int, [_vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, _P(ctypes.c_uint16)]),
    "cvf3_get_window": (ctypes.c_int, [_vp] + [ctypes.c_int32] * 6 + [_P(ctypes.c_uint32)]),
    "cvf_debug_checks": (ctypes.c_int, []),
    "cvf_copy_probe": (ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _vp]),
    "cvf_wait_probe": (ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_uint32, _vp]),
}

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """The loaded libcvf.so; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_build.LIB):
        if build_if_missing:
            _build.build()
        else:
            raise RuntimeError("libcvf.so is not built (run __graft_entry__.build() or "
                               "paper_2505_05919_gb300.build.build()); there is no fallback")
    L = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def declared_symbols():
    return list(_SIGS)


def _check(rc: int, func: str) -> int:
    if rc != CVF_OK:
        raise CvfError(rc, func, cvf_last_error())
    return rc


def cvf_last_error() -> str:
    return load().cvf_last_error().decode(errors="replace")


def cvf_params_default() -> cvf_params:
    p = cvf_params()
    _check(load().cvf_params_default(ctypes.byref(p)), "cvf_params_default")
    return p


def cvf_params_physical(T_kelvin: float, P_MPa: float) -> cvf_params:
    p = cvf_params()
    _check(load().cvf_params_physical(T_kelvin, P_MPa, ctypes.byref(p)), "cvf_params_physical")
    return p


def cvf_threshold_table(p: cvf_params):
    out = (ctypes.c_uint64 * 42)()
    _check(load().cvf_threshold_table(ctypes.byref(p), out), "cvf_threshold_table")
    return list(out)


def cvf_create(p: cvf_params, stream: int | None = None, dev_state: int | None = None) -> int:
    h = _vp()
    _check(load().cvf_create(ctypes.byref(p), stream or None, dev_state or None, ctypes.byref(h)),
           "cvf_create")
    return h.value


def cvf_sweep(h: int, n_sweeps: int, record_every: int = 0) -> None:
    _check(load().cvf_sweep(h, n_sweeps, record_every), "cvf_sweep")


def cvf_observables(h: int) -> cvf_obs:
    o = cvf_obs()
    _check(load().cvf_observables(h, ctypes.byref(o)), "cvf_observables")
    return o


def cvf_drain_series(h: int, cap: int):
    """Returns (records, overflowed)."""
    buf = (cvf_obs * max(cap, 1))()
    n = ctypes.c_int64()
    rc = load().cvf_drain_series(h, buf, cap, ctypes.byref(n))
    if rc not in (CVF_OK, CVF_EOVERFLOW):
        _check(rc, "cvf_drain_series")
    return [buf[i] for i in range(n.value)], rc == CVF_EOVERFLOW


def cvf_get_state(h: int, host_ptr: int, n: int) -> None:
    _check(load().cvf_get_state(h, ctypes.cast(host_ptr, _P(ctypes.c_uint16)), n), "cvf_get_state")


def cvf_set_state(h: int, host_ptr: int, n: int, V_iso: float, sweep: int) -> None:
    _check(load().cvf_set_state(h, ctypes.cast(host_ptr, _P(ctypes.c_uint16)), n, V_iso, sweep),
           "cvf_set_state")


def cvf_recount(h: int):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().cvf_recount(h, ctypes.byref(a), ctypes.byref(b)), "cvf_recount")
    return a.value, b.value


def cvf_state_device_ptr(h: int) -> int:
    p = _vp()
    _check(load().cvf_state_device_ptr(h, ctypes.byref(p)), "cvf_state_device_ptr")
    return p.value


def cvf_destroy(h: int) -> None:
    _check(load().cvf_destroy(h), "cvf_destroy")


def cvf_set_tiles(h: int, config: int) -> None:
    _check(load().cvf_set_tiles(h, config), "cvf_set_tiles")


def cvf_get_tiles(h: int):
    c, r, w = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().cvf_get_tiles(h, ctypes.byref(c), ctypes.byref(r), ctypes.byref(w)),
           "cvf_get_tiles")
    return c.value, r.value, w.value


def cvf_sweep_noalloc(p: cvf_params, dev_state: int, V_iso: float, sweep: int, n_sweeps: int,
                      record_every: int = 0, series_cap: int = 0, stream: int | None = None):
    """Returns (observables, records).  Allocates nothing on the device."""
    series = (cvf_obs * max(series_cap, 1))()
    n = ctypes.c_int64()
    out = cvf_obs()
    _check(load().cvf_sweep_noalloc(ctypes.byref(p), dev_state, V_iso, sweep, n_sweeps, record_every,
                                    series, series_cap, ctypes.byref(n), ctypes.byref(out),
                                    stream or None), "cvf_sweep_noalloc")
    return out, [series[i] for i in range(n.value)]


# ---------------------------------------------------------------- batches --
def cvf_batch_create(params_list, stream: int | None = None) -> int:
    n = len(params_list)
    arr = (cvf_params * max(n, 1))(*params_list)
    b = _vp()
    _check(load().cvf_batch_create(arr, n, stream or None, ctypes.byref(b)), "cvf_batch_create")
    return b.value


def cvf_batch_add(b: int, p: cvf_params) -> int:
    rid = ctypes.c_int32()
    _check(load().cvf_batch_add(b, ctypes.byref(p), ctypes.byref(rid)), "cvf_batch_add")
    return rid.value


def cvf_batch_remove(b: int, replica: int) -> None:
    _check(load().cvf_batch_remove(b, replica), "cvf_batch_remove")


def cvf_batch_size(b: int):
    a, c = ctypes.c_int32(), ctypes.c_int32()
    _check(load().cvf_batch_size(b, ctypes.byref(a), ctypes.byref(c)), "cvf_batch_size")
    return a.value, c.value


def cvf_batch_sweep(b: int, sweeps) -> None:
    n = len(sweeps)
    arr = (ctypes.c_int64 * max(n, 1))(*[int(x) for x in sweeps])
    _check(load().cvf_batch_sweep(b, arr, n), "cvf_batch_sweep")


def cvf_batch_sync(b: int) -> None:
    _check(load().cvf_batch_sync(b), "cvf_batch_sync")


def cvf_batch_observables(b: int, replica: int) -> cvf_obs:
    o = cvf_obs()
    _check(load().cvf_batch_observables(b, replica, ctypes.byref(o)), "cvf_batch_observables")
    return o


def cvf_batch_observables_many(b: int, replicas) -> list:
    ids = [int(r) for r in replicas]
    n = len(ids)
    arr = (ctypes.c_int32 * max(n, 1))(*ids)
    out = (cvf_obs * max(n, 1))()
    _check(load().cvf_batch_observables_many(b, arr, n, out), "cvf_batch_observables_many")
    return [out[i] for i in range(n)]


def cvf_batch_observables_enqueue(b: int, replicas) -> int:
    ids = [int(r) for r in replicas]
    arr = (ctypes.c_int32 * max(len(ids), 1))(*ids)
    t = ctypes.c_int64(-1)
    _check(load().cvf_batch_observables_enqueue(b, arr, len(ids), ctypes.byref(t)),
           "cvf_batch_observables_enqueue")
    return t.value


def cvf_batch_observables_collect(b: int, ticket: int, n: int) -> list:
    out = (cvf_obs * max(n, 1))()
    _check(load().cvf_batch_observables_collect(b, ticket, out, n), "cvf_batch_observables_collect")
    return [out[i] for i in range(n)]


def cvf_batch_memory(b: int) -> tuple:
    r, u = ctypes.c_uint64(0), ctypes.c_uint64(0)
    _check(load().cvf_batch_memory(b, ctypes.byref(r), ctypes.byref(u)), "cvf_batch_memory")
    return r.value, u.value


def cvf_batch_get_state(b: int, replica: int, host_ptr: int, n: int) -> None:
    _check(load().cvf_batch_get_state(b, replica, ctypes.cast(host_ptr, _P(ctypes.c_uint16)), n),
           "cvf_batch_get_state")


def cvf_batch_set_tiles(b: int, config: int) -> None:
    _check(load().cvf_batch_set_tiles(b, config), "cvf_batch_set_tiles")


def cvf_batch_get_tiles(b: int) -> tuple:
    """(setting, shape the last call used): -1 = automatic / no call yet."""
    c, u = ctypes.c_int32(), ctypes.c_int32()
    _check(load().cvf_batch_get_tiles(b, ctypes.byref(c), ctypes.byref(u)), "cvf_batch_get_tiles")
    return c.value, u.value


def cvf_batch_tile_config(config: int):
    """(rows, words, block threads) of a batched-kernel configuration."""
    r, w, t = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
    _check(load().cvf_batch_tile_config(config, ctypes.byref(r), ctypes.byref(w)),
           "cvf_batch_tile_config")
    _check(load().cvf_batch_config_threads(config, ctypes.byref(t)), "cvf_batch_config_threads")
    return r.value, w.value, t.value


def cvf_batch_destroy(b: int) -> None:
    _check(load().cvf_batch_destroy(b), "cvf_batch_destroy")


# ----------------------------------------------------------- cubic lattice --
def cvf3_params_physical(T_kelvin: float, P_MPa: float) -> cvf_params:
    p = cvf_params()
    _check(load().cvf3_params_physical(T_kelvin, P_MPa, ctypes.byref(p)), "cvf3_params_physical")
    return p


def cvf3_threshold_table(p: cvf_params):
    out = (ctypes.c_uint64 * 66)()
    _check(load().cvf3_threshold_table(ctypes.byref(p), out), "cvf3_threshold_table")
    return list(out)


def cvf3_create(p: cvf_params, stream: int | None = None, dev_state: int | None = None) -> int:
    h = _vp()
    _check(load().cvf3_create(ctypes.byref(p), stream or None, dev_state or None, ctypes.byref(h)),
           "cvf3_create")
    return h.value


def cvf3_sweep(h: int, n_sweeps: int, record_every: int = 0) -> None:
    _check(load().cvf3_sweep(h, n_sweeps, record_every), "cvf3_sweep")


def cvf3_observables(h: int) -> cvf_obs:
    o = cvf_obs()
    _check(load().cvf3_observables(h, ctypes.byref(o)), "cvf3_observables")
    return o


def cvf3_drain_series(h: int, cap: int):
    """Returns (records, overflowed)."""
    buf = (cvf_obs * max(cap, 1))()
    n = ctypes.c_int64()
    rc = load().cvf3_drain_series(h, buf, cap, ctypes.byref(n))
    if rc not in (CVF_OK, CVF_EOVERFLOW):
        _check(rc, "cvf3_drain_series")
    return [buf[i] for i in range(n.value)], rc == CVF_EOVERFLOW


def cvf3_get_state(h: int, host_ptr: int, n: int) -> None:
    _check(load().cvf3_get_state(h, ctypes.cast(host_ptr, _P(ctypes.c_uint32)), n), "cvf3_get_state")


def cvf3_set_state(h: int, host_ptr: int, n: int, V_iso: float, sweep: int) -> None:
    _check(load().cvf3_set_state(h, ctypes.cast(host_ptr, _P(ctypes.c_uint32)), n, V_iso, sweep),
           "cvf3_set_state")


def cvf3_get_eta(h: int, host_ptr: int, n: int) -> None:
    _check(load().cvf3_get_eta(h, ctypes.cast(host_ptr, _P(ctypes.c_uint8)), n), "cvf3_get_eta")


def cvf3_set_eta(h: int, host_ptr: int, n: int) -> None:
    _check(load().cvf3_set_eta(h, ctypes.cast(host_ptr, _P(ctypes.c_uint8)), n), "cvf3_set_eta")


def cvf3_recount(h: int):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(load().cvf3_recount(h, ctypes.byref(a), ctypes.byref(b)), "cvf3_recount")
    return a.value, b.value


def cvf3_state_device_ptr(h: int) -> int:
    p = _vp()
    _check(load().cvf3_state_device_ptr(h, ctypes.byref(p)), "cvf3_state_device_ptr")
    return p.value


def cvf3_destroy(h: int) -> None:
    _check(load().cvf3_destroy(h), "cvf3_destroy")


def cvf3_set_resident(h: int, mode: int) -> None:
    _check(load().cvf3_set_resident(h, mode), "cvf3_set_resident")


def cvf3_get_resident(h: int) -> int:
    r = ctypes.c_int32()
    _check(load().cvf3_get_resident(h, ctypes.byref(r)), "cvf3_get_resident")
    return r.value


def cvf_copy_probe(dst_ptr: int, src_ptr: int, nbytes: int, stream_ptr: int = 0) -> None:
    """Enqueue one 16-byte-vector copy of nbytes between device buffers."""
    _check(load().cvf_copy_probe(dst_ptr, src_ptr, nbytes, stream_ptr or None), "cvf_copy_probe")


def cvf_philox_probe(seed: int, n_cells: int, step: int, out_ptr: int, stream_ptr: int = 0) -> None:
    """Enqueue the Philox draws of one checkerboard step over n_cells cells
    (nothing else); their words are XOR-folded into the device word out_ptr."""
    _check(load().cvf_philox_probe(seed, n_cells, step, out_ptr, stream_ptr or None),
           "cvf_philox_probe")


def cvf_wait_probe(flag_ptr: int, target: int, polls: int, stream_ptr: int = 0) -> None:
    """Run the library's bounded device wait on a device word (CvfError with
    code CVF_ETIMEOUT when it gives up)."""
    _check(load().cvf_wait_probe(flag_ptr, target, polls, stream_ptr or None), "cvf_wait_probe")


def cvf_get_window(h: int, x0: int, y0: int, W: int, H: int, host_ptr: int) -> None:
    """Copy the H x W rectangle of cell words at (x0, y0) to host_ptr."""
    _check(load().cvf_get_window(h, x0, y0, W, H, ctypes.cast(host_ptr, _P(ctypes.c_uint16))),
           "cvf_get_window")


def cvf3_get_window(h: int, x0: int, y0: int, z0: int, W: int, H: int, D: int,
                    host_ptr: int) -> None:
    """Copy the D x H x W box of cell words at (x0, y0, z0) to host_ptr."""
    _check(load().cvf3_get_window(h, x0, y0, z0, W, H, D,
                                  ctypes.cast(host_ptr, _P(ctypes.c_uint32))), "cvf3_get_window")


def cvf_debug_checks() -> bool:
    """Whether the loaded library is the debug build with device index checks."""
    return load().cvf_debug_checks() == 1
