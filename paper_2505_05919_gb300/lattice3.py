"""Python face of one cubic lattice (the paper's 3D model) on the GPU.

PyTorch supplies the device memory (L^3 uint32 words, updated in place) and
the stream; the layered Metropolis passes, the counts and the volume move
run in ``libcvf.so`` through the C ABI (``_capi``, ``cvf3_*``).
"""
from __future__ import annotations

import numpy as np

from . import _capi
from ._capi import cvf_params


def params3(T_kelvin: float = 300.0, P_MPa: float = 0.1, **overrides) -> cvf_params:
    """Table 1 parameters at (T, P) for the cubic lattice (L = 16,
    v_iso0 = 2^(1/2), layered schedule, eta moves), with field overrides."""
    p = _capi.cvf3_params_physical(T_kelvin, P_MPa)
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError("cvf_params has no field %r" % k)
        setattr(p, k, v)
    return p


class Lattice3:
    """One cubic lattice: create, sweep, read observables and state."""

    def __init__(self, p: cvf_params, stream=None, use_torch_memory: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Lattice3 needs a CUDA device (no CPU fallback)")
        self.p = p
        self.L = p.L
        self.N = p.L ** 3
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._state = None
        dev_ptr = None
        if use_torch_memory:
            self._state = torch.empty(self.N + 4, dtype=torch.int32, device="cuda")
            dev_ptr = self._state.data_ptr()
            dev_ptr += (-dev_ptr) % 16
        self.h = _capi.cvf3_create(p, self.stream.cuda_stream, dev_ptr)

    def sweep(self, n: int, record_every: int = 0) -> None:
        _capi.cvf3_sweep(self.h, n, record_every)

    def observables(self) -> dict:
        return _capi.cvf3_observables(self.h).as_dict()

    def drain(self, cap: int = 1 << 16):
        recs, overflow = _capi.cvf3_drain_series(self.h, cap)
        return [r.as_dict() for r in recs], overflow

    def state(self) -> np.ndarray:
        out = np.empty(self.N, np.uint32)
        _capi.cvf3_get_state(self.h, out.ctypes.data, self.N)
        return out.reshape(self.L, self.L, self.L)

    def window(self, x0: int, y0: int, z0: int, W: int, H: int, D: int) -> np.ndarray:
        """The D x H x W box of cell words at (x0, y0, z0), without copying
        the rest of the cube."""
        out = np.empty((D, H, W), np.uint32)
        _capi.cvf3_get_window(self.h, x0, y0, z0, W, H, D, out.ctypes.data)
        return out

    def set_state(self, words, V_iso: float, sweep: int = 0) -> None:
        a = np.ascontiguousarray(np.asarray(words, dtype=np.uint32).reshape(-1))
        _capi.cvf3_set_state(self.h, a.ctypes.data, a.size, float(V_iso), int(sweep))

    def eta(self) -> np.ndarray:
        """The cube configurations 0..8 of the eta update (L^3 / 4 bytes;
        empty without eta moves)."""
        if not self.p.eta_moves:
            return np.zeros(0, np.uint8)
        out = np.empty(self.N // 4, np.uint8)
        _capi.cvf3_get_eta(self.h, out.ctypes.data, out.size)
        return out

    def set_eta(self, cfg) -> None:
        a = np.ascontiguousarray(np.asarray(cfg, dtype=np.uint8).reshape(-1))
        _capi.cvf3_set_eta(self.h, a.ctypes.data, a.size)

    def recount(self):
        return _capi.cvf3_recount(self.h)

    def set_resident(self, mode: int) -> None:
        """1: the cube resident in one thread-block cluster during each call
        (L a multiple of 8, 16 <= L <= 64); 0: four launches per step; -1: choose."""
        _capi.cvf3_set_resident(self.h, mode)

    def resident(self) -> bool:
        return bool(_capi.cvf3_get_resident(self.h))

    def close(self) -> None:
        if getattr(self, "h", None):
            _capi.cvf3_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
