"""CPU oracle of the CVF Metropolis hot path (2D and 3D) -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU legs of ``bench.py``
(``cpu_baseline`` and ``--impl reference``) may import this package.  The
product library (``paper_2505_05919_gb300``) never does; the two share no code.

The arithmetic lives in ``cvf_oracle.c`` (2D) and ``cvf_oracle3.c`` (the 3D
cubic-lattice variant), plain single-threaded C; this module only builds them
with gcc and marshals arguments through ctypes.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field, asdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cvf_oracle.c")
_SRC3 = os.path.join(_HERE, "cvf_oracle3.c")
_LIB = os.path.join(_HERE, "libcvf_oracle.so")

INIT_RANDOM, INIT_ORDERED = 0, 1
SCHED_CHECKERBOARD, SCHED_LAYERED = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC), os.path.getmtime(_SRC3),
                                              os.path.getmtime(os.path.join(_HERE, "cvf_oracle.h")))):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, _SRC3, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("L", ctypes.c_int32), ("q", ctypes.c_int32),
                ("epsilon", ctypes.c_double), ("cutoff", ctypes.c_double),
                ("J", ctypes.c_double), ("J_sigma", ctypes.c_double),
                ("v_HB", ctypes.c_double), ("kT", ctypes.c_double),
                ("P", ctypes.c_double), ("v_iso_init", ctypes.c_double),
                ("dv_max_frac", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("init", ctypes.c_int32), ("schedule", ctypes.c_int32),
                ("volume_moves", ctypes.c_int32), ("rng_words", ctypes.c_int32),
                ("eta_moves", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Obs(ctypes.Structure):
    _fields_ = [("sweep", ctypes.c_int64), ("n_hb", ctypes.c_int64),
                ("n_hb_raw", ctypes.c_int64), ("n_coop", ctypes.c_int64),
                ("acc_sigma", ctypes.c_int64), ("acc_volume", ctypes.c_int64),
                ("V_iso", ctypes.c_double), ("V", ctypes.c_double),
                ("U_LJ", ctypes.c_double), ("H", ctypes.c_double),
                ("g", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("n_state", ctypes.c_int64 * 8)]

    def as_dict(self) -> dict:
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("pad", "n_state")}
        d["n_state"] = list(self.n_state)
        return d


class State(ctypes.Structure):
    _fields_ = [("p", Params), ("N", ctypes.c_int64),
                ("w", ctypes.POINTER(ctypes.c_uint16)),
                ("V_iso", ctypes.c_double), ("dV_max", ctypes.c_double),
                ("sweep", ctypes.c_int64), ("n_hb_raw", ctypes.c_int64),
                ("n_coop", ctypes.c_int64), ("acc_sigma", ctypes.c_int64),
                ("acc_volume", ctypes.c_int64), ("g", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("table", ctypes.c_uint64 * 42)]


class State3(ctypes.Structure):
    _fields_ = [("p", Params), ("N", ctypes.c_int64),
                ("w", ctypes.POINTER(ctypes.c_uint32)),
                ("V_iso", ctypes.c_double), ("dV_max", ctypes.c_double),
                ("sweep", ctypes.c_int64), ("n_hb_raw", ctypes.c_int64),
                ("n_coop", ctypes.c_int64), ("acc_sigma", ctypes.c_int64),
                ("acc_volume", ctypes.c_int64), ("g", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("table", ctypes.c_uint64 * 66),
                ("eta", ctypes.POINTER(ctypes.c_uint8)), ("ncube", ctypes.c_int64),
                ("acc_eta", ctypes.c_int64), ("eta_table", ctypes.c_uint64 * 18)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        u16p, u32p, u64p = P(ctypes.c_uint16), P(ctypes.c_uint32), P(ctypes.c_uint64)
        u8p = P(ctypes.c_uint8)
        i32p, i64p, dp = P(ctypes.c_int32), P(ctypes.c_int64), P(ctypes.c_double)
        sigs = {
            "orc_philox4x32_10": (None, [u32p, u32p, u32p]),
            "orc_lj_cell_energy": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double]),
            "orc_shell_table": (ctypes.c_int, [ctypes.c_double, i64p, i64p, ctypes.c_int]),
            "orc_threshold_table": (None, [P(Params), u64p]),
            "orc_recount": (None, [P(Params), u16p, i64p, i64p]),
            "orc_check_params": (ctypes.c_int, [P(Params)]),
            "orc_bond_partner": (None, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int, i64p,
                                        P(ctypes.c_int)]),
            "orc_init": (ctypes.c_int, [P(State), P(Params), u16p]),
            "orc_set": (ctypes.c_int, [P(State), P(Params), u16p, ctypes.c_double, ctypes.c_int64]),
            "orc_volume_move": (None, [P(State)]),
            "orc_step": (None, [P(State)]),
            "orc_observables": (None, [P(State), P(Obs)]),
            "orc_run": (ctypes.c_int64, [P(State), ctypes.c_int64, ctypes.c_int32, P(Obs), ctypes.c_int64]),
            "orc_layer_order": (None, [P(Params), ctypes.c_int64, P(ctypes.c_int)]),
            "orc_arm_probe": (None, [P(Params), u16p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                                     ctypes.c_int32, u32p, i32p, i32p, u64p]),
            "orc_arm_probe_all": (None, [P(Params), u16p, ctypes.c_int64, ctypes.c_int32, u32p, u64p]),
            "orc_init_window": (None, [P(Params), u16p, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.c_int32, ctypes.c_int32]),
            "orc_window_run": (None, [P(Params), u16p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_int64, ctypes.c_int64, i32p]),
            "orc_volume_chain": (ctypes.c_int64, [P(Params), ctypes.c_double, ctypes.c_int64,
                                                  ctypes.c_int64, dp, i32p, i64p]),
            # 3D variant
            "orc3_neighbour": (ctypes.c_int64, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int]),
            "orc3_shell_table": (ctypes.c_int, [ctypes.c_double, i64p, i64p, ctypes.c_int]),
            "orc3_lj_cell_energy": (ctypes.c_double, [ctypes.c_double, ctypes.c_double, ctypes.c_double]),
            "orc3_threshold_table": (None, [P(Params), u64p]),
            "orc3_recount": (None, [P(Params), u32p, i64p, i64p]),
            "orc3_check_params": (ctypes.c_int, [P(Params)]),
            "orc3_init": (ctypes.c_int, [P(State3), P(Params), u32p, u8p]),
            "orc3_set": (ctypes.c_int, [P(State3), P(Params), u32p, u8p, ctypes.c_double,
                                        ctypes.c_int64]),
            "orc3_matchings": (ctypes.c_int, [P(ctypes.c_uint16)]),
            "orc3_cube_corner_cells": (None, [ctypes.c_int32, ctypes.c_int64, i64p]),
            "orc3_edge_of": (None, [ctypes.c_int32, ctypes.c_int64, ctypes.c_int, i64p,
                                    P(ctypes.c_int)]),
            "orc3_eta_of": (ctypes.c_int, [P(Params), u8p, ctypes.c_int64, ctypes.c_int]),
            "orc3_eta_table": (None, [P(Params), u64p]),
            "orc3_eta_moves": (None, [P(State3)]),
            "orc3_eta_probe": (None, [P(Params), u32p, u8p, ctypes.c_int64, ctypes.c_uint32,
                                      ctypes.c_int32, u32p, i32p, u64p]),
            "orc3_recount_eta": (None, [P(Params), u32p, u8p, i64p, i64p]),
            "orc3_volume_move": (None, [P(State3)]),
            "orc3_permutation": (None, [ctypes.c_int, P(ctypes.c_int)]),
            "orc3_layer_order": (None, [P(Params), ctypes.c_int64, P(ctypes.c_int)]),
            "orc3_step": (None, [P(State3)]),
            "orc3_observables": (None, [P(State3), P(Obs)]),
            "orc3_run": (ctypes.c_int64, [P(State3), ctypes.c_int64, ctypes.c_int32, P(Obs), ctypes.c_int64]),
            "orc3_arm_probe": (None, [P(Params), u32p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32,
                                      ctypes.c_int32, u32p, u64p]),
            "orc3_volume_chain": (ctypes.c_int64, [P(Params), ctypes.c_double, ctypes.c_int64,
                                                   ctypes.c_int64, ctypes.c_int64, dp]),
            "orc3_init_window": (None, [P(Params), u32p, u8p] + [ctypes.c_int32] * 6),
            "orc3_window_run": (None, [P(Params), u32p, u8p] + [ctypes.c_int32] * 6 +
                                [ctypes.c_int64, ctypes.c_int64, i32p]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


# --------------------------------------------------------------------------
# Parameter record (reduced units: eps, r0, v0 = r0^3; Table 1 defaults)
# --------------------------------------------------------------------------
@dataclass
class OracleParams:
    L: int = 64
    q: int = 6
    epsilon: float = 1.0
    cutoff: float = 6.0
    J: float = 2.0          # J / (4 eps) = 0.5
    J_sigma: float = 0.32   # J_sigma / (4 eps) = 0.08
    v_HB: float = 0.6
    kT: float = 0.4535
    P: float = 2.6704e-4
    v_iso_init: float = math.cbrt(2.0)
    dv_max_frac: float = 0.01
    seed: int = 1
    init: int = INIT_RANDOM
    schedule: int = SCHED_CHECKERBOARD
    volume_moves: int = 1
    rng_words: int = 1
    eta_moves: int = 0      # 3D only: the eta update of App. A

    def c(self) -> Params:
        return Params(**asdict(self))


# Table 1 units: eps = 5.5 kJ/mol, r0 = 2.9 Angstrom, v0 = r0^3.
R_KJ_PER_MOL_K = 8.31446261815324e-3
EPS_KJ_PER_MOL = 5.5
R0_M = 2.9e-10
N_AVOGADRO = 6.02214076e23


def physical_params(T_kelvin: float, P_MPa: float, **kw) -> OracleParams:
    """Reduced kT/eps and P v0/eps of a physical state point (Table 1)."""
    kT = T_kelvin * R_KJ_PER_MOL_K / EPS_KJ_PER_MOL
    P = (P_MPa * 1.0e6) * (R0_M ** 3) * N_AVOGADRO / (EPS_KJ_PER_MOL * 1.0e3)
    return OracleParams(kT=kT, P=P, **kw)


def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32).copy()
    k = np.asarray(key, dtype=np.uint32).copy()
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c, ctypes.c_uint32), _ptr(k, ctypes.c_uint32),
                            _ptr(out, ctypes.c_uint32))
    return out


def lj_cell_energy(v_iso: float, epsilon: float = 1.0, cutoff: float = 6.0) -> float:
    return lib().orc_lj_cell_energy(v_iso, epsilon, cutoff)


def shell_table(cutoff: float = 6.0):
    d2 = np.zeros(4096, np.int64)
    m = np.zeros(4096, np.int64)
    n = lib().orc_shell_table(cutoff, _ptr(d2, ctypes.c_int64), _ptr(m, ctypes.c_int64), 4096)
    return d2[:n].copy(), m[:n].copy()


def threshold_table(p: OracleParams) -> np.ndarray:
    out = np.zeros(42, np.uint64)
    cp = p.c()
    lib().orc_threshold_table(ctypes.byref(cp), _ptr(out, ctypes.c_uint64))
    return out.reshape(2, 3, 7)


def recount(p: OracleParams, w: np.ndarray):
    a = np.ascontiguousarray(w, dtype=np.uint16)
    hb, co = ctypes.c_int64(), ctypes.c_int64()
    cp = p.c()
    lib().orc_recount(ctypes.byref(cp), _ptr(a, ctypes.c_uint16), ctypes.byref(hb), ctypes.byref(co))
    return hb.value, co.value


def bond_partner(L: int, cell: int, arm: int):
    c, a = ctypes.c_int64(), ctypes.c_int()
    lib().orc_bond_partner(L, cell, arm, ctypes.byref(c), ctypes.byref(a))
    return c.value, a.value


def layer_order(p: OracleParams, step: int):
    out = (ctypes.c_int * 4)()
    cp = p.c()
    lib().orc_layer_order(ctypes.byref(cp), step, out)
    return list(out)


def arm_probe_all(p: OracleParams, cfgs: np.ndarray, g: int):
    """Proposed value and threshold of every (configuration, cell, arm, k)."""
    cfgs = np.ascontiguousarray(cfgs, dtype=np.uint16)
    n = cfgs.shape[0]
    N = p.L * p.L
    shape = (n, N, 4, p.q - 1)
    s_new = np.zeros(shape, np.uint32)
    T = np.zeros(shape, np.uint64)
    cp = p.c()
    lib().orc_arm_probe_all(ctypes.byref(cp), _ptr(cfgs, ctypes.c_uint16), n, g,
                            _ptr(s_new, ctypes.c_uint32), _ptr(T, ctypes.c_uint64))
    return s_new, T


def window_run(p: OracleParams, w_full: np.ndarray, x0: int, y0: int, W: int, H: int,
               step0: int, gates) -> np.ndarray:
    a = np.ascontiguousarray(w_full, dtype=np.uint16).copy()
    g = np.ascontiguousarray(gates, dtype=np.int32)
    cp = p.c()
    lib().orc_window_run(ctypes.byref(cp), _ptr(a, ctypes.c_uint16), x0, y0, W, H, step0,
                         len(g), _ptr(g, ctypes.c_int32))
    return a


def window_init_run(p: OracleParams, w_full: np.ndarray, x0: int, y0: int, W: int, H: int,
                    step0: int, gates) -> None:
    """In place on the L x L array w_full (which may be a lazily zeroed
    array far larger than memory could hold written out): initialise the
    window's cells by the init rule, then run len(gates) checkerboard steps
    over the window alone.  Cells more than 2 len(gates) inside the window
    are then exact; the window may run across the periodic edges (cells
    taken mod L, 0 <= x0, y0 < L, W, H <= L)."""
    assert w_full.dtype == np.uint16 and w_full.flags.c_contiguous
    assert w_full.size == p.L * p.L
    assert 0 <= x0 < p.L and 0 < W <= p.L and 0 <= y0 < p.L and 0 < H <= p.L
    g = np.ascontiguousarray(gates, dtype=np.int32)
    cp = p.c()
    ptr = w_full.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16))
    lib().orc_init_window(ctypes.byref(cp), ptr, x0, y0, W, H)
    lib().orc_window_run(ctypes.byref(cp), ptr, x0, y0, W, H, step0, len(g),
                         _ptr(g, ctypes.c_int32))


def volume_chain(p: OracleParams, V_iso: float, step0: int, K: int):
    V = np.zeros(K, np.float64)
    g = np.zeros(K, np.int32)
    acc = ctypes.c_int64()
    cp = p.c()
    done = lib().orc_volume_chain(ctypes.byref(cp), V_iso, step0, K, _ptr(V, ctypes.c_double),
                                  _ptr(g, ctypes.c_int32), ctypes.byref(acc))
    return done, V, g, acc.value


class Oracle:
    """One lattice advanced by the oracle, step by step."""

    def __init__(self, p: OracleParams, state: np.ndarray | None = None,
                 V_iso: float | None = None, sweep: int = 0):
        self.p = p
        self._cp = p.c()
        self.w = np.zeros(p.L * p.L, np.uint16)
        self.st = State()
        if state is None:
            rc = lib().orc_init(ctypes.byref(self.st), ctypes.byref(self._cp), _ptr(self.w, ctypes.c_uint16))
        else:
            self.w[:] = np.asarray(state, dtype=np.uint16).reshape(-1)
            if V_iso is None:
                V_iso = p.L * p.L * p.v_iso_init
            rc = lib().orc_set(ctypes.byref(self.st), ctypes.byref(self._cp),
                               _ptr(self.w, ctypes.c_uint16), V_iso, sweep)
        if rc != 0:
            raise ValueError("oracle rejected the parameters (code %d)" % rc)

    def step(self) -> None:
        lib().orc_step(ctypes.byref(self.st))

    def run(self, n: int, record_every: int = 0) -> list:
        cap = (n // record_every + 1) if record_every > 0 else 0
        ring = (Obs * max(cap, 1))()
        k = lib().orc_run(ctypes.byref(self.st), n, record_every, ring, cap)
        return [ring[i].as_dict() for i in range(k)]

    def volume_move(self) -> None:
        lib().orc_volume_move(ctypes.byref(self.st))

    def observables(self) -> dict:
        o = Obs()
        lib().orc_observables(ctypes.byref(self.st), ctypes.byref(o))
        return o.as_dict()

    def state(self) -> np.ndarray:
        return self.w.reshape(self.p.L, self.p.L).copy()

    def recount(self):
        return recount(self.p, self.w)


# --------------------------------------------------------------------------
# 3D variant: cubic lattice, six arms per cell, layered schedule
# --------------------------------------------------------------------------
def params3(**kw) -> OracleParams:
    """3D defaults: v_iso0 = sqrt(2) (the pair minimum r = 2^(1/6) r0 with
    v = r^3), the layered schedule, one random word per update and the eta
    moves of App. A (they need an even L; eta_moves=0 gives eta = 1)."""
    base = dict(L=16, v_iso_init=math.sqrt(2.0), schedule=SCHED_LAYERED, rng_words=1,
                eta_moves=1)
    base.update(kw)
    return OracleParams(**base)


def physical_params3(T_kelvin: float, P_MPa: float, **kw) -> OracleParams:
    p = physical_params(T_kelvin, P_MPa)
    return params3(kT=p.kT, P=p.P, **kw)


def neighbour3(L: int, cell: int, arm: int) -> int:
    return lib().orc3_neighbour(L, cell, arm)


def shell_table3(cutoff: float = 6.0):
    d2 = np.zeros(4096, np.int64)
    m = np.zeros(4096, np.int64)
    n = lib().orc3_shell_table(cutoff, _ptr(d2, ctypes.c_int64), _ptr(m, ctypes.c_int64), 4096)
    return d2[:n].copy(), m[:n].copy()


def lj_cell_energy3(v_iso: float, epsilon: float = 1.0, cutoff: float = 6.0) -> float:
    return lib().orc3_lj_cell_energy(v_iso, epsilon, cutoff)


def threshold_table3(p: OracleParams) -> np.ndarray:
    out = np.zeros(66, np.uint64)
    cp = p.c()
    lib().orc3_threshold_table(ctypes.byref(cp), _ptr(out, ctypes.c_uint64))
    return out.reshape(2, 3, 11)


def recount3(p: OracleParams, w: np.ndarray):
    a = np.ascontiguousarray(w, dtype=np.uint32).reshape(-1)
    hb, co = ctypes.c_int64(), ctypes.c_int64()
    cp = p.c()
    lib().orc3_recount(ctypes.byref(cp), _ptr(a, ctypes.c_uint32), ctypes.byref(hb), ctypes.byref(co))
    return hb.value, co.value


def permutation3(idx: int):
    out = (ctypes.c_int * 6)()
    lib().orc3_permutation(idx, out)
    return list(out)


def layer_order3(p: OracleParams, step: int):
    out = (ctypes.c_int * 6)()
    cp = p.c()
    lib().orc3_layer_order(ctypes.byref(cp), step, out)
    return list(out)


def arm_probe3(p: OracleParams, w: np.ndarray, cell: int, arm: int, k: int, g: int):
    a = np.ascontiguousarray(w, dtype=np.uint32).reshape(-1)
    s_new, T = ctypes.c_uint32(), ctypes.c_uint64()
    cp = p.c()
    lib().orc3_arm_probe(ctypes.byref(cp), _ptr(a, ctypes.c_uint32), cell, arm, k, g,
                         ctypes.byref(s_new), ctypes.byref(T))
    return s_new.value, T.value


def matchings3():
    out = (ctypes.c_uint16 * 9)()
    n = lib().orc3_matchings(out)
    return n, list(out)


def cube_corner_cells3(L: int, cube: int):
    out = np.zeros(8, np.int64)
    lib().orc3_cube_corner_cells(L, cube, _ptr(out, ctypes.c_int64))
    return list(out)


def edge_of3(L: int, cell: int, arm: int):
    cube, e = ctypes.c_int64(), ctypes.c_int()
    lib().orc3_edge_of(L, cell, arm, ctypes.byref(cube), ctypes.byref(e))
    return cube.value, e.value


def eta_of3(p: OracleParams, eta: np.ndarray, cell: int, arm: int) -> int:
    a = np.ascontiguousarray(eta, dtype=np.uint8).reshape(-1)
    cp = p.c()
    return lib().orc3_eta_of(ctypes.byref(cp), _ptr(a, ctypes.c_uint8), cell, arm)


def eta_table3(p: OracleParams) -> np.ndarray:
    out = np.zeros(18, np.uint64)
    cp = p.c()
    lib().orc3_eta_table(ctypes.byref(cp), _ptr(out, ctypes.c_uint64))
    return out.reshape(2, 9)


def eta_probe3(p: OracleParams, w: np.ndarray, eta: np.ndarray, cube: int, k: int, g: int):
    a = np.ascontiguousarray(w, dtype=np.uint32).reshape(-1)
    e = np.ascontiguousarray(eta, dtype=np.uint8).reshape(-1)
    nw, dhb, T = ctypes.c_uint32(), ctypes.c_int32(), ctypes.c_uint64()
    cp = p.c()
    lib().orc3_eta_probe(ctypes.byref(cp), _ptr(a, ctypes.c_uint32), _ptr(e, ctypes.c_uint8), cube,
                         k, g, ctypes.byref(nw), ctypes.byref(dhb), ctypes.byref(T))
    return nw.value, dhb.value, T.value


def recount3_eta(p: OracleParams, w: np.ndarray, eta: np.ndarray):
    a = np.ascontiguousarray(w, dtype=np.uint32).reshape(-1)
    e = np.ascontiguousarray(eta, dtype=np.uint8).reshape(-1)
    hb, co = ctypes.c_int64(), ctypes.c_int64()
    cp = p.c()
    lib().orc3_recount_eta(ctypes.byref(cp), _ptr(a, ctypes.c_uint32), _ptr(e, ctypes.c_uint8),
                           ctypes.byref(hb), ctypes.byref(co))
    return hb.value, co.value


def volume_chain3(p: OracleParams, V_iso: float, n_hb_raw: int, step0: int, K: int):
    V = np.zeros(K, np.float64)
    cp = p.c()
    acc = lib().orc3_volume_chain(ctypes.byref(cp), V_iso, n_hb_raw, step0, K,
                                  _ptr(V, ctypes.c_double))
    return V, acc


def window_init_run3(p: OracleParams, w_full: np.ndarray, x0: int, y0: int, z0: int, W: int,
                     H: int, D: int, step0: int, gates, eta_full: np.ndarray | None = None) -> None:
    """In place on the L^3 array w_full (possibly lazily zeroed) and, with eta
    moves, the L^3/4 cube configurations eta_full: initialise the box's cells
    (and the cubes with a corner in it) by the init rule, then run len(gates)
    layered steps over the box alone.  Cells more than 3 len(gates) (2
    len(gates) without eta moves) inside the box are then exact; the box
    must lie inside the cube."""
    L = p.L
    assert w_full.dtype == np.uint32 and w_full.flags.c_contiguous and w_full.size == L ** 3
    assert 0 <= x0 and x0 + W <= L and 0 <= y0 and y0 + H <= L and 0 <= z0 and z0 + D <= L
    eptr = None
    if p.eta_moves:
        assert eta_full is not None and eta_full.dtype == np.uint8 and eta_full.size == L ** 3 // 4
        eptr = eta_full.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
    g = np.ascontiguousarray(gates, dtype=np.int32)
    cp = p.c()
    ptr = w_full.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    lib().orc3_init_window(ctypes.byref(cp), ptr, eptr, x0, y0, z0, W, H, D)
    lib().orc3_window_run(ctypes.byref(cp), ptr, eptr, x0, y0, z0, W, H, D, step0, len(g),
                          _ptr(g, ctypes.c_int32))


class Oracle3:
    """One cubic lattice advanced by the 3D oracle, step by step."""

    def __init__(self, p: OracleParams, state: np.ndarray | None = None,
                 V_iso: float | None = None, sweep: int = 0, eta: np.ndarray | None = None):
        self.p = p
        self._cp = p.c()
        self.N = p.L ** 3
        self.w = np.zeros(self.N, np.uint32)
        # cube configurations (App. A), one byte per checkerboard cube
        self.eta_cfg = np.zeros(max(self.N // 4, 1) if p.eta_moves else 1, np.uint8)
        eptr = _ptr(self.eta_cfg, ctypes.c_uint8) if p.eta_moves else None
        self.st = State3()
        if state is None:
            rc = lib().orc3_init(ctypes.byref(self.st), ctypes.byref(self._cp),
                                 _ptr(self.w, ctypes.c_uint32), eptr)
        else:
            self.w[:] = np.asarray(state, dtype=np.uint32).reshape(-1)
            if p.eta_moves and eta is not None:
                self.eta_cfg[:] = np.asarray(eta, dtype=np.uint8).reshape(-1)
            if V_iso is None:
                V_iso = self.N * p.v_iso_init
            rc = lib().orc3_set(ctypes.byref(self.st), ctypes.byref(self._cp),
                                _ptr(self.w, ctypes.c_uint32), eptr, V_iso, sweep)
        if rc != 0:
            raise ValueError("oracle rejected the parameters (code %d)" % rc)

    def step(self) -> None:
        lib().orc3_step(ctypes.byref(self.st))

    def run(self, n: int, record_every: int = 0) -> list:
        cap = (n // record_every + 1) if record_every > 0 else 0
        ring = (Obs * max(cap, 1))()
        k = lib().orc3_run(ctypes.byref(self.st), n, record_every, ring, cap)
        return [ring[i].as_dict() for i in range(k)]

    def volume_move(self) -> None:
        lib().orc3_volume_move(ctypes.byref(self.st))

    def observables(self) -> dict:
        o = Obs()
        lib().orc3_observables(ctypes.byref(self.st), ctypes.byref(o))
        return o.as_dict()

    def state(self) -> np.ndarray:
        L = self.p.L
        return self.w.reshape(L, L, L).copy()

    def eta(self) -> np.ndarray:
        """The cube configurations 0..8 (empty without eta moves)."""
        return self.eta_cfg.copy() if self.p.eta_moves else np.zeros(0, np.uint8)

    def eta_moves(self) -> None:
        lib().orc3_eta_moves(ctypes.byref(self.st))

    @property
    def acc_eta(self) -> int:
        return self.st.acc_eta

    def recount(self):
        if self.p.eta_moves:
            return recount3_eta(self.p, self.w, self.eta_cfg)
        return recount3(self.p, self.w)
