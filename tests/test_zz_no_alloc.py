"""The conserved-totals entry point that allocates nothing (strm_conserved_totals_static).

It serves callers that must not allocate device memory, such as a monitor attached to a
running solver whose allocator already holds the device memory. It keeps its scratch in a
static array of the library instead of a workspace. The checks go through the C ABI: the
totals must equal those of strm_conserved_totals (within the 1e-12 bar of the parity tests)
on two calls in a row, the second on a smaller grid, so that partial sums left in the shared
array by the first call cannot leak into the second. Grids above the stated maximum must be
refused with a clear error.

This file is named to be collected last, so a run that stops at the first failure has already
run every other test.
"""
import numpy as np
import pytest
import torch

from paper_2004_02276_gb300 import binding, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12
MAX_NODES = 67108864  # STRM_STATIC_MAX_NODES in include/strm.h


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)


def reference_totals(case, w):
    s = binding.Solver(case)
    try:
        return np.array(s.totals(w))
    finally:
        s.close()


def test_static_totals_match_context_totals_on_two_calls():
    calls = [
        (inputs.Case(nx=96, ny=64, nz=48), 1),                          # tanh channel, 72 blocks
        (inputs.Case(nx=37, ny=29, nz=11, beta=0.0, y_wall=False), 2),  # uniform, ragged, 3 blocks
    ]
    for case, seed in calls:
        w = torch.from_numpy(inputs.channel_state(case, seed)).cuda()
        want = reference_totals(case, w)
        got = np.array(binding.conserved_totals_static(case, w))
        np.testing.assert_allclose(got, want, rtol=TOL, atol=0)


def test_static_totals_refuse_oversized_grid():
    case = inputs.Case(nx=1024, ny=256, nz=257)  # 67,371,008 nodes > the static maximum
    assert case.npts > MAX_NODES
    w = torch.zeros(8, dtype=torch.float64, device="cuda")  # never read: refused first
    with pytest.raises(binding.StrmError) as e:
        binding.conserved_totals_static(case, w)
    assert e.value.code == -1 and "at most" in str(e.value)
