"""Python face of a batch of replicas (one persistent launch per call).

Device memory is allocated by the library per replica (one stream-ordered
allocation each, from the batch's own pool); the stream comes from PyTorch.
Adding, removing and sweeping enqueue work without waiting for the GPU.  All
method steps run in ``libcvf.so``.
"""
from __future__ import annotations

import numpy as np

from . import _capi
from ._capi import cvf_params


def tile_configs():
    """The (rows, words, block threads) configurations the batched kernel can
    use; the first four are the ones the automatic per-call choice takes."""
    out = []
    c = 0
    while True:
        try:
            out.append(_capi.cvf_batch_tile_config(c))
        except _capi.CvfError:
            return out
        c += 1


class Batch:
    def __init__(self, params_list=(), stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("Batch needs a CUDA device (no CPU fallback)")
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.b = _capi.cvf_batch_create(list(params_list), self.stream.cuda_stream)
        self.L = {i: p.L for i, p in enumerate(params_list)}

    # replicas --------------------------------------------------------------
    def add(self, p: cvf_params) -> int:
        rid = _capi.cvf_batch_add(self.b, p)
        self.L[rid] = p.L
        return rid

    def remove(self, rid: int) -> None:
        _capi.cvf_batch_remove(self.b, rid)
        self.L.pop(rid, None)

    def pool_bytes(self) -> tuple:
        """(mapped, in use) bytes of the batch's memory pool."""
        return _capi.cvf_batch_memory(self.b)

    def slots(self) -> int:
        return _capi.cvf_batch_size(self.b)[0]

    # work ------------------------------------------------------------------
    def sweep(self, sweeps) -> None:
        """sweeps: a list over slots, or a dict {replica: steps}."""
        if isinstance(sweeps, dict):
            lst = [0] * self.slots()
            for k, v in sweeps.items():
                lst[k] = v
            sweeps = lst
        _capi.cvf_batch_sweep(self.b, sweeps)

    def sync(self) -> None:
        _capi.cvf_batch_sync(self.b)

    def set_tiles(self, config: int) -> None:
        """Kernel configuration (index into tile_configs()), or -1 (the
        default) to let each call choose the largest 256-thread tile that
        still gives every co-resident block a tile (the smallest tile, with
        512-thread blocks when its tiles are under a quarter of the
        blocks)."""
        _capi.cvf_batch_set_tiles(self.b, config)

    def tiles(self) -> tuple:
        """(setting, configuration the last call used)."""
        return _capi.cvf_batch_get_tiles(self.b)

    # results ---------------------------------------------------------------
    def observables(self, rid: int) -> dict:
        return _capi.cvf_batch_observables(self.b, rid).as_dict()

    def observables_many(self, rids) -> list:
        """Observables of several replicas with one synchronisation."""
        return [o.as_dict() for o in _capi.cvf_batch_observables_many(self.b, rids)]

    def observables_enqueue(self, rids) -> int:
        """Ticket for the observables of rids at this point of the stream
        (returns without waiting)."""
        return _capi.cvf_batch_observables_enqueue(self.b, rids)

    def observables_collect(self, ticket: int, n: int) -> list:
        """Waits for a ticket's point of the stream and returns its n records."""
        return [o.as_dict() for o in _capi.cvf_batch_observables_collect(self.b, ticket, n)]

    def state(self, rid: int) -> np.ndarray:
        L = self.L[rid]
        out = np.empty(L * L, np.uint16)
        _capi.cvf_batch_get_state(self.b, rid, out.ctypes.data, L * L)
        return out.reshape(L, L)

    def close(self) -> None:
        if getattr(self, "b", None):
            _capi.cvf_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
