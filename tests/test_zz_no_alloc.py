"""The allocation-free entry point, cvf_sweep_noalloc.

It exists for callers that cannot let a library allocate device memory --
applications that own every byte through their own pool, or that must not
allocate mid-run because an allocation can synchronise the device or fail
under memory pressure.  These tests hand it caller-owned memory (a torch
tensor) and check, over two calls in a row, that its lattice and
observables equal those of the allocating path (cvf_create + cvf_sweep) run
from the same start: the lattice bit for bit, counters exactly, FP64
observables within the relative 1e-12 the other tests use.  The file is
collected last so a failure here comes after every other test has run; it
also passes on its own in a fresh process.
"""
from dataclasses import asdict

import numpy as np
import pytest

import oracle
from paper_2505_05919_gb300 import Lattice, params_from_dict, _capi

pytestmark = pytest.mark.gpu

FP_REL = 1e-12


def _compare(got, want, counts_too=True):
    keys = ["sweep", "n_hb", "n_hb_raw", "n_coop", "g"]
    if counts_too:
        keys += ["acc_sigma", "acc_volume"]
    for k in keys:
        assert got[k] == want[k], (k, got[k], want[k])
    assert list(got["n_state"]) == list(want["n_state"])
    for k in ("V_iso", "V", "U_LJ", "H"):
        assert abs(got[k] - want[k]) <= FP_REL * abs(want[k]), (k, got[k], want[k])


@pytest.mark.parametrize("L,extra", [(64, {}), (130, dict(q=5, T=330.0, P=40.0)), (6, dict(rng_words=2))])
def test_noalloc_matches_allocating_path_two_calls(L, extra):
    import torch
    extra = dict(extra)
    T, P = extra.pop("T", 300.0), extra.pop("P", 0.1)
    p = params_from_dict(asdict(oracle.physical_params(T, P, L=L, seed=77, dv_max_frac=0.03, **extra)))
    N = L * L
    with Lattice(p) as ref:
        start = ref.state()
        V0 = ref.observables()["V_iso"]
        ref.sweep(40, 8)
        s1, o1 = ref.state(), ref.observables()
        r1, _ = ref.drain()
        ref.sweep(35, 7)
        s2, o2 = ref.state(), ref.observables()
        r2, _ = ref.drain()
    # caller-owned state pair; the lattice starts in half (sweep & 1) = 0
    buf = torch.zeros(2 * N + 8, dtype=torch.int16, device="cuda")
    base = buf.data_ptr() + (-buf.data_ptr()) % 16
    off = (base - buf.data_ptr()) // 2
    buf[off:off + N].copy_(torch.from_numpy(start.reshape(-1).view(np.int16)))
    stream = torch.cuda.current_stream().cuda_stream
    torch.cuda.synchronize()

    obs1, rec1 = _capi.cvf_sweep_noalloc(p, base, V0, 0, 40, record_every=8, series_cap=64,
                                         stream=stream)
    half = 40 & 1
    got1 = buf[off + half * N: off + half * N + N].cpu().numpy().view(np.uint16).reshape(L, L)
    assert np.array_equal(got1, s1)
    _compare(obs1.as_dict(), o1)
    assert len(rec1) == len(r1) == 5
    for a, b in zip(rec1, r1):
        _compare(a.as_dict(), b)

    # second call continues from the first call's output
    obs2, rec2 = _capi.cvf_sweep_noalloc(p, base, obs1.V_iso, 40, 35, record_every=7, series_cap=64,
                                         stream=stream)
    half = 75 & 1
    got2 = buf[off + half * N: off + half * N + N].cpu().numpy().view(np.uint16).reshape(L, L)
    assert np.array_equal(got2, s2)
    # acceptance counters restart at each call; everything else continues
    _compare(obs2.as_dict(), o2, counts_too=False)
    assert obs2.acc_sigma == o2["acc_sigma"] - o1["acc_sigma"]
    assert len(rec2) == len(r2) == 5
    for a, b in zip(rec2, r2):
        _compare(a.as_dict(), b, counts_too=False)


def test_noalloc_rejects_too_many_records():
    import torch
    p = params_from_dict(asdict(oracle.physical_params(300.0, 0.1, L=8, seed=1)))
    buf = torch.zeros(2 * 64 + 8, dtype=torch.int16, device="cuda")
    base = buf.data_ptr() + (-buf.data_ptr()) % 16
    with pytest.raises(_capi.CvfError) as e:
        _capi.cvf_sweep_noalloc(p, base, 64 * 1.3, 0, 300, record_every=1, series_cap=300)
    assert e.value.code == _capi.CVF_EINVAL and "256" in str(e.value)


def test_noalloc_reports_invalid_cells():
    """A caller lattice holding a word that is not a valid cell for q is
    reported as CVF_EINVAL once the call has run (the check runs on the
    device: the library never copies the caller's buffer to the host)."""
    import torch
    L = 8
    p = params_from_dict(asdict(oracle.physical_params(300.0, 0.1, L=L, seed=1, q=5)))
    buf = torch.zeros(2 * L * L + 8, dtype=torch.int16, device="cuda")
    base = buf.data_ptr() + (-buf.data_ptr()) % 16
    off = (base - buf.data_ptr()) // 2
    buf[off + 9] = 0x0500  # nibble 2 = 5 >= q
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(_capi.CvfError) as e:
        _capi.cvf_sweep_noalloc(p, base, L * L * 1.3, 0, 3, stream=stream)
    assert e.value.code == _capi.CVF_EINVAL
    # the shared array is cleared by the next call: a valid lattice runs clean
    buf.zero_()
    torch.cuda.synchronize()
    obs, _ = _capi.cvf_sweep_noalloc(p, base, L * L * 1.3, 0, 3, stream=stream)
    assert obs.status == 0 and obs.sweep == 3
