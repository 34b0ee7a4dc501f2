"""The measured rate of the scatter's shared-memory atomic add.

erpp_shared_add_rate times the add that accumulates every stencil node's
contribution (Sec. 2.4, Eq. ns_regularized_filtered) with nothing else
limiting it; bench.py sets the scatter phase against it.  Checked here: both
kinds return a positive rate below what the GPU could issue at all (four
instructions per clock per SM at 3 GHz, 32 lanes each), the 32-bit integer
add is faster than the FP32 add (the reason the scatter accumulates in fixed
point), and a call with an unknown kind is refused without a launch.
"""

import ctypes

import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def erpp():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1405_6969_gb300 as pkg
    return pkg


def test_shared_add_rates(erpp):
    import torch
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    bound = 32 * 4 * nsm * 3.0e9
    s32 = erpp.shared_add_rate("s32")
    f32 = erpp.shared_add_rate("f32")
    assert 0.0 < f32 < bound
    assert 0.0 < s32 < bound
    assert s32 > f32


def test_shared_add_rate_refuses_unknown_kind(erpp):
    so = erpp.load()
    out = ctypes.c_double(-1.0)
    assert so.erpp_shared_add_rate(2, ctypes.byref(out)) == 1  # ERPP_EINVAL
    assert out.value == -1.0
