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
