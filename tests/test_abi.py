"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every entry point include/cvf.h declares, and its host-only functions agree
with the oracle on the same inputs."""
import os
import re
from dataclasses import asdict

import numpy as np
import pytest

import oracle
from paper_2505_05919_gb300 import _capi, build as libbuild, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return _capi.load()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(cvf3?_[a-z0-9_]+)\s*\(", text))
    return names


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert "cvf_create" in names and "cvf_sweep" in names and "cvf_destroy" in names
    assert "cvf3_create" in names and "cvf3_sweep" in names and "cvf3_destroy" in names
    for n in sorted(names):
        assert hasattr(lib, n), n
    # and the binding wraps each of them under the same name
    assert names <= set(_capi.declared_symbols())


def test_params_physical_matches_oracle_units(lib):
    for T, P in ((270.0, 0.1), (300.0, 0.1), (330.0, 50.0), (285.5, 12.3)):
        got = _capi.cvf_params_physical(T, P)
        want = oracle.physical_params(T, P)
        assert got.kT == pytest.approx(want.kT, rel=1e-15)
        assert got.P == pytest.approx(want.P, rel=1e-15)
        assert (got.J, got.J_sigma, got.v_HB, got.q, got.cutoff) == (2.0, 0.32, 0.6, 6, 6.0)


@pytest.mark.parametrize("T,P", [(270, 0.1), (300, 0.1), (330, 50.0)])
@pytest.mark.parametrize("q", [2, 6, 8])
def test_threshold_table_equals_oracle(lib, T, P, q):
    op = oracle.physical_params(T, P, q=q)
    got = np.array(_capi.cvf_threshold_table(_capi.cvf_params(**asdict(op))), dtype=np.uint64)
    want = oracle.threshold_table(op).reshape(-1)
    assert np.array_equal(got, want)


def test_threshold_table_limits(lib):
    hot = oracle.OracleParams(kT=1e300)
    assert set(_capi.cvf_threshold_table(_capi.cvf_params(**asdict(hot)))) == {2 ** 32}
    cold = oracle.OracleParams(kT=1e-3)
    t = np.array(_capi.cvf_threshold_table(_capi.cvf_params(**asdict(cold)))).reshape(2, 3, 7)
    assert t[1, 0, 0] == 0 and t[1, 2, 6] == 2 ** 32


@pytest.mark.parametrize("bad", [dict(L=3), dict(L=0), dict(q=1), dict(q=9), dict(kT=0.0),
                                 dict(kT=-1.0), dict(v_iso_init=0.5), dict(rng_words=3),
                                 dict(schedule=7), dict(init=5), dict(cutoff=0.0),
                                 dict(dv_max_frac=-0.1), dict(volume_moves=2)])
def test_invalid_params_rejected_on_host(lib, bad):
    p = _capi.cvf_params(**asdict(oracle.OracleParams(**bad)))
    with pytest.raises(_capi.CvfError) as e:
        _capi.cvf_threshold_table(p)
    assert e.value.code == _capi.CVF_EINVAL


def test_workloads_are_deterministic():
    a, b = workloads.c4(), workloads.c4()
    assert a == b and len(a) == 256
    assert {r["L"] for r in a} <= {32, 64, 128, 256, 512}
    w = workloads.random_words(8, 6, 3)
    assert w.shape == (8, 8) and np.array_equal(w, workloads.random_words(8, 6, 3))
    assert int(((w >> 0) & 7).max()) < 6
    jobs = workloads.c5(n_jobs=50)
    assert all(jobs[i]["arrival"] <= jobs[i + 1]["arrival"] for i in range(49))


# ------------------------------------------------------------ cubic lattice --
def test_cvf3_params_physical(lib):
    for T, P in ((270.0, 0.1), (330.0, 50.0)):
        got = _capi.cvf3_params_physical(T, P)
        want = oracle.physical_params3(T, P)
        assert got.kT == pytest.approx(want.kT, rel=1e-15)
        assert got.P == pytest.approx(want.P, rel=1e-15)
        assert got.v_iso_init == want.v_iso_init == 2 ** 0.5
        assert (got.schedule, got.rng_words, got.L) == (_capi.CVF_SCHED_LAYERED, 1, 16)


@pytest.mark.parametrize("T,P", [(270, 0.1), (300, 0.1), (330, 50.0)])
@pytest.mark.parametrize("q", [2, 6, 8])
def test_cvf3_threshold_table_equals_oracle(lib, T, P, q):
    op = oracle.physical_params3(T, P, q=q)
    got = np.array(_capi.cvf3_threshold_table(_capi.cvf_params(**asdict(op))), dtype=np.uint64)
    assert np.array_equal(got, oracle.threshold_table3(op).reshape(-1))


@pytest.mark.parametrize("field,value", [("schedule", 0), ("rng_words", 2), ("L", 1025), ("L", 1),
                                         ("q", 9), ("kT", 0.0), ("v_iso_init", 0.9)])
def test_cvf3_rejects_bad_params(lib, field, value):
    p = _capi.cvf3_params_physical(300.0, 0.1)
    setattr(p, field, value)
    with pytest.raises(_capi.CvfError) as e:
        _capi.cvf3_threshold_table(p)
    assert e.value.code == _capi.CVF_EINVAL


@pytest.mark.parametrize("dst,src,n", [(0, 4096, 16), (4096, 0, 16), (4096, 8192, 24),
                                       (4100, 8192, 16), (4096, 8200, 16)])
def test_copy_probe_rejects_bad_arguments_on_host(lib, dst, src, n):
    # NULL or misaligned arguments are refused before any launch (no GPU here)
    with pytest.raises(_capi.CvfError):
        _capi.cvf_copy_probe(dst, src, n, 0)


@pytest.mark.parametrize("flag,polls", [(0, 16), (4098, 16), (4096, 0), (4096, (1 << 22) + 1)])
def test_wait_probe_rejects_bad_arguments_on_host(lib, flag, polls):
    with pytest.raises(_capi.CvfError) as e:
        _capi.cvf_wait_probe(flag, 1, polls, 0)
    assert e.value.code == 1  # CVF_EINVAL, before any device work


@pytest.mark.parametrize("out,step", [(0, 0), (4098, 0), (4096, -1)])
def test_philox_probe_rejects_bad_arguments_on_host(lib, out, step):
    with pytest.raises(_capi.CvfError) as e:
        _capi.cvf_philox_probe(1, 64, step, out, 0)
    assert e.value.code == 1  # CVF_EINVAL, before any device work


def test_batch_tile_configs_and_cells_per_thread(lib):
    from paper_2505_05919_gb300.autotune import cells_per_thread
    from paper_2505_05919_gb300.batch import tile_configs
    cfgs = tile_configs()
    assert len(cfgs) == 12 and cfgs[0] == (64, 64, 256) and cfgs[4] == (64, 64, 128)
    # the same four tiles with 256-, 128- and 512-thread blocks
    assert [c[:2] for c in cfgs[:4]] == [c[:2] for c in cfgs[4:8]] == [c[:2] for c in cfgs[8:]]
    assert [{c[2] for c in cfgs[k:k + 4]} for k in (0, 4, 8)] == [{256}, {128}, {512}]
    assert [cells_per_thread(c) for c in range(len(cfgs))] == [2 * r * w // t for r, w, t in cfgs]
    assert [cells_per_thread(c) for c in range(12)] == [32, 8, 4, 2, 64, 16, 8, 4, 16, 4, 2, 1]
    with pytest.raises(_capi.CvfError):
        _capi.cvf_batch_tile_config(12)


def test_release_build_has_no_debug_checks(lib):
    assert not _capi.cvf_debug_checks()


def test_eta_moves_only_on_an_even_cubic_lattice(lib):
    p = _capi.cvf_params_physical(300.0, 0.1)
    assert p.eta_moves == 0
    p.eta_moves = 1   # the square lattice has eta = 1 on every edge
    with pytest.raises(_capi.CvfError) as e:
        _capi.cvf_threshold_table(p)
    assert e.value.code == _capi.CVF_EINVAL
    p3 = _capi.cvf3_params_physical(300.0, 0.1)
    assert p3.eta_moves == 1
    _capi.cvf3_threshold_table(p3)
    p3.L = 5
    with pytest.raises(_capi.CvfError):
        _capi.cvf3_threshold_table(p3)
    p3.eta_moves = 0
    _capi.cvf3_threshold_table(p3)
