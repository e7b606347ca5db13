"""Parity cases run against the debug build of the library (libcvf_debug.so,
compiled with CVF_DEBUG: every kernel checks its shared- and global-memory
indices and the TMA alignment rule, records the first failing site in the
lattice's status word and skips the access).  Run as a separate process by
tests/test_gpu_debug_build.py, so that this process loads the debug library
instead of the release one.  Every case must match the oracle bit for bit
and every observables call must return CVF_OK (a failed check would make it
raise CvfError with CVF_EBOUNDS and the site).
"""
import os
import sys
from dataclasses import asdict

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import paper_2505_05919_gb300.build as _build  # noqa: E402

_build.LIB = _build.build(debug=True)

import oracle  # noqa: E402
from paper_2505_05919_gb300 import Batch, Lattice, Lattice3, params_from_dict  # noqa: E402


def square(L, steps, tiles=-1, **kw):
    op = oracle.physical_params(300.0, 0.1, L=L, seed=L + 7, **kw)
    ref = oracle.Oracle(op)
    ref.run(steps)
    with Lattice(params_from_dict(asdict(op))) as lat:
        if tiles >= 0:
            lat.set_tiles(tiles)
        lat.sweep(steps)
        assert np.array_equal(lat.state(), ref.state()), ("square", L, tiles, kw)
        o = lat.observables()                      # raises on a failed check
    assert o["n_hb_raw"] == ref.observables()["n_hb_raw"]


def cubic(L, steps, resident=-1):
    # eta moves where they apply (even side)
    eta = 0 if L % 2 else 1
    op = oracle.physical_params3(300.0, 0.1, L=L, seed=L + 3, dv_max_frac=0.05, eta_moves=eta)
    ref = oracle.Oracle3(op)
    ref.run(steps)
    with Lattice3(params_from_dict(asdict(op))) as lat:
        if resident >= 0:
            lat.set_resident(resident)
        lat.sweep(steps)
        assert np.array_equal(lat.state(), ref.state()), ("cubic", L, resident)
        assert np.array_equal(lat.eta(), ref.eta()), ("cubic eta", L, resident)
        lat.observables()


def batch(sizes, steps, config=-1):
    ops = [oracle.physical_params(300.0, 0.1, L=L, seed=100 + L) for L in sizes]
    with Batch([params_from_dict(asdict(op)) for op in ops]) as b:
        b.set_tiles(config)
        b.sweep([steps] * len(ops))
        for i, op in enumerate(ops):
            ref = oracle.Oracle(op)
            ref.run(steps)
            assert np.array_equal(b.state(i), ref.state()), ("batch", sizes[i])
            b.observables(i)


def noalloc(L, steps):
    """The allocation-free entry point on a caller-owned state pair (a torch
    tensor), so its launches run the debug build's index checks too."""
    import torch
    from paper_2505_05919_gb300 import _capi
    op = oracle.physical_params(300.0, 0.1, L=L, seed=L + 11)
    ref = oracle.Oracle(op)
    start = ref.state().copy()
    V0 = ref.observables()["V_iso"]
    ref.run(steps)
    N = L * L
    buf = torch.zeros(2 * N + 8, dtype=torch.int16, device="cuda")
    base = buf.data_ptr() + (-buf.data_ptr()) % 16
    off = (base - buf.data_ptr()) // 2
    buf[off:off + N].copy_(torch.from_numpy(start.reshape(-1).view(np.int16)))
    torch.cuda.synchronize()
    _capi.cvf_sweep_noalloc(params_from_dict(asdict(op)), base, V0, 0, steps,
                            stream=torch.cuda.current_stream().cuda_stream)  # raises on a check
    h = (steps & 1) * N
    got = buf[off + h:off + h + N].cpu().numpy().view(np.uint16).reshape(L, L)
    assert np.array_equal(got, ref.state()), ("noalloc", L)


def main():
    from paper_2505_05919_gb300 import _capi
    assert _capi.lib_path() == _build.DEBUG_LIB and _capi.cvf_debug_checks()
    for L in (2, 16, 64):
        square(L, 9)                               # resident cluster form where it applies
    square(130, 6)                                 # odd number of words per row
    for t in (0, 1, 2):
        square(258, 5, tiles=t)                    # ragged tiles, periodic staging
    square(1024, 4, tiles=0)                       # TMA staging
    for L, t in ((392, 4), (200, 5), (136, 6)):
        square(L, 6, tiles=t)                      # the wavefront sweep, ragged tiles
    square(96, 7, rng_words=2)
    square(64, 8, schedule=oracle.SCHED_LAYERED)
    square(34, 8, schedule=oracle.SCHED_LAYERED)
    for L, res in ((8, 0), (9, 0), (12, 0), (16, 1), (24, 1), (16, 0), (130, 0)):
        cubic(L, 5, res)
    batch([16, 34, 64, 130, 2], 12)
    for config in (0, 4, 7, 8, 11):   # 256-, 128- and 512-thread blocks
        batch([16, 34, 130, 2], 7, config)
    noalloc(64, 7)
    noalloc(130, 6)
    print("debug build: all cases match, no index check failed")


if __name__ == "__main__":
    main()
