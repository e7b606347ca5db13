"""Python face of one CVF lattice on the GPU.

PyTorch supplies the device memory (the state pair) and the stream; every
step of the method runs in ``libcvf.so`` through the C ABI (``_capi``).
"""
from __future__ import annotations

import numpy as np

from . import _capi
from ._capi import cvf_params


def params(T_kelvin: float = 300.0, P_MPa: float = 0.1, **overrides) -> cvf_params:
    """Table 1 parameters at (T, P) with field overrides (L=..., q=..., ...)."""
    p = _capi.cvf_params_physical(T_kelvin, P_MPa)
    for k, v in overrides.items():
        if not hasattr(p, k):
            raise AttributeError("cvf_params has no field %r" % k)
        setattr(p, k, v)
    return p


def params_from_dict(d: dict) -> cvf_params:
    p = cvf_params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


class Lattice:
    """One lattice: create, sweep, read observables and state."""

    def __init__(self, p: cvf_params, stream=None, use_torch_memory: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Lattice needs a CUDA device (no CPU fallback)")
        self.p = p
        self.L = p.L
        self.N = p.L * p.L
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._state = None
        dev_ptr = None
        if use_torch_memory:
            # the lattice and its double buffer, owned by torch
            self._state = torch.empty(2 * self.N + 8, dtype=torch.int16, device="cuda")
            dev_ptr = self._state.data_ptr()
            dev_ptr += (-dev_ptr) % 16
        self.h = _capi.cvf_create(p, self.stream.cuda_stream, dev_ptr)

    def sweep(self, n: int, record_every: int = 0) -> None:
        _capi.cvf_sweep(self.h, n, record_every)

    def observables(self) -> dict:
        return _capi.cvf_observables(self.h).as_dict()

    def drain(self, cap: int = 1 << 16):
        recs, overflow = _capi.cvf_drain_series(self.h, cap)
        return [r.as_dict() for r in recs], overflow

    def state(self) -> np.ndarray:
        out = np.empty(self.N, np.uint16)
        _capi.cvf_get_state(self.h, out.ctypes.data, self.N)
        return out.reshape(self.L, self.L)

    def window(self, x0: int, y0: int, W: int, H: int) -> np.ndarray:
        """The H x W rectangle of cell words at (x0, y0), without copying the
        rest of the lattice."""
        out = np.empty((H, W), np.uint16)
        _capi.cvf_get_window(self.h, x0, y0, W, H, out.ctypes.data)
        return out

    def set_state(self, words, V_iso: float, sweep: int = 0) -> None:
        a = np.ascontiguousarray(np.asarray(words, dtype=np.uint16).reshape(-1))
        _capi.cvf_set_state(self.h, a.ctypes.data, a.size, float(V_iso), int(sweep))

    def recount(self):
        return _capi.cvf_recount(self.h)

    def set_tiles(self, config: int) -> None:
        """Tile shape of the sweep (0: 64x64, 1: 32x32, 2: 16x32 words; 3: the
        whole lattice resident in one thread-block cluster; 4, 5, 6: the
        shapes of 0, 1, 2 in the wavefront sweep, one persistent launch per
        call; -1: automatic)."""
        _capi.cvf_set_tiles(self.h, config)

    def tiles(self):
        """(config, rows, words) of the sweep's tile shape."""
        return _capi.cvf_get_tiles(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            _capi.cvf_destroy(self.h)
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
