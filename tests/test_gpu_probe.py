"""The byte-roofline probe (cvf_copy_probe) copies exactly: the L2 and DRAM
copy bandwidths reported beside the sweep come from a kernel that moves the
bytes it is timed on."""
import pytest
import torch

from paper_2505_05919_gb300 import _capi

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("nbytes", [16, 4096 + 16, 1 << 20, (32 << 20) + 48])
def test_copy_probe_copies(nbytes):
    g = torch.Generator(device="cuda").manual_seed(nbytes)
    a = torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device="cuda", generator=g)
    b = torch.zeros(nbytes + 64, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())   # the fills above run on torch's stream
    _capi.cvf_copy_probe(b.data_ptr(), a.data_ptr(), nbytes, s.cuda_stream)
    s.synchronize()
    assert torch.equal(b[:nbytes], a)
    assert not b[nbytes:].any()          # nothing written past the end


def test_copy_probe_zero_bytes_is_a_no_op():
    a = torch.ones(64, dtype=torch.uint8, device="cuda")
    b = torch.zeros(64, dtype=torch.uint8, device="cuda")
    _capi.cvf_copy_probe(b.data_ptr(), a.data_ptr(), 0, 0)
    torch.cuda.synchronize()
    assert not b.any()


def test_wait_probe_gives_up_with_a_status_and_the_context_survives():
    """The bounded wait of the persistent batched sweep, on a flag that
    nothing sets, ends with CVF_ETIMEOUT; afterwards the device still runs a
    sweep that matches the oracle."""
    from dataclasses import asdict

    import numpy as np

    import oracle
    from paper_2505_05919_gb300 import Lattice, params_from_dict

    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(_capi.CvfError) as e:
        _capi.cvf_wait_probe(flag.data_ptr(), 1, 1 << 14)
    assert e.value.code == 4  # CVF_ETIMEOUT
    # far from the target the wait polls less often and still gives up
    with pytest.raises(_capi.CvfError) as e:
        _capi.cvf_wait_probe(flag.data_ptr(), 1000, 1 << 14)
    assert e.value.code == 4
    op = oracle.physical_params(300.0, 0.1, L=16, seed=9)
    ref = oracle.Oracle(op)
    ref.run(12)
    with Lattice(params_from_dict(asdict(op))) as lat:
        lat.sweep(12)
        assert np.array_equal(lat.state(), ref.state())


def test_wait_probe_returns_when_the_flag_is_set():
    flag = torch.full((1,), 7, dtype=torch.int32, device="cuda")
    _capi.cvf_wait_probe(flag.data_ptr(), 5, 1 << 14)   # already >= target
    _capi.cvf_wait_probe(flag.data_ptr(), 7, 1)


@pytest.mark.parametrize("n,step,seed", [(1, 0, 3), (4097, 5, 3), (256 * 152 * 8 + 33, 1 << 33, 0xDEADBEEF12345)])
def test_philox_probe_draws_the_sweep_words(n, step, seed):
    """The random-number ceiling probe computes the very words a step draws:
    the XOR fold of Philox((c, step, 0), seed) over every cell c < n equals
    the fold of the oracle's own Philox4x32-10 (an independent
    implementation, pinned by the published known-answer vectors); every
    block enters the fold, so no draw is skipped."""
    import numpy as np

    import oracle
    key = [seed & 0xFFFFFFFF, seed >> 32]
    want = 0
    for c in range(n):
        r = oracle.philox([c, step & 0xFFFFFFFF, step >> 32, 0], key)
        want ^= int(r[0]) ^ int(r[1]) ^ int(r[2]) ^ int(r[3])
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    _capi.cvf_philox_probe(seed, n, step, out.data_ptr(), s.cuda_stream)
    s.synchronize()
    assert int(out.cpu().numpy().view(np.uint32)[0]) == want
