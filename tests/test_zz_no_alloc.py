"""The conserved-totals entry point that allocates nothing (strm_conserved_totals_static).

It serves callers that must not allocate device memory, such as a monitor attached to a
running solver whose allocator already holds the device memory. It keeps its scratch in a
static array of the library instead of a workspace. The checks go through the C ABI: the
totals must equal those of strm_conserved_totals and of the FP64 oracle (within the 1e-12 bar
of the parity tests) on calls in a row, each on a different grid and wall-normal map, so that
partial sums left in the shared array by one call cannot leak into the next. Grids above the
stated maximum must be refused with a clear error.

This file is named to be collected last, so a run that stops at the first failure has already
run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
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


CALLS = [
    (inputs.Case(nx=96, ny=64, nz=48), "channel", 1),                           # tanh, 72 blocks
    (inputs.Case(nx=37, ny=29, nz=11, beta=0.0, y_wall=False), "channel", 2),   # uniform, ragged
    (inputs.PAPER_CHANNEL, "channel", 3),                                       # erf map
    (inputs.bl_case("bl-sinh-48x40x12", 48, 40, 12, 7.0, 6.0, 1.5, y_map="sinh1", beta=4.0), "bl", 4),
    (inputs.bl_case("bl-48x40x12", 48, 40, 12, 7.0, 6.0, 1.5), "bl", 5),        # one-sided tanh
]


def test_static_totals_match_context_and_oracle_on_calls_in_a_row():
    for case, kind, seed in CALLS:
        w0 = inputs.channel_state(case, seed) if kind == "channel" else inputs.bl_state(case, seed)
        w = torch.from_numpy(w0).cuda()
        want = reference_totals(case, w)
        oracle = O.totals(O.make_cfg(case), w0)
        for _ in range(2):  # a repeated call must not see the previous call's partial sums
            got = np.array(binding.conserved_totals_static(case, w))
            np.testing.assert_allclose(got, want, rtol=TOL, atol=1e-15 * np.abs(want).max())
            np.testing.assert_allclose(got, oracle, rtol=TOL, atol=1e-15 * np.abs(oracle).max())


def test_static_totals_refuse_oversized_grid():
    case = inputs.Case(nx=1024, ny=256, nz=257)  # 67,371,008 nodes > the static maximum
    assert case.npts > MAX_NODES
    w = torch.zeros(8, dtype=torch.float64, device="cuda")  # never read: refused first
    g, _, _ = binding.structs(case)
    out = (ctypes.c_double * 5)()
    rc = binding.lib().strm_conserved_totals_static(ctypes.byref(g), binding._ptr(w), out, None)
    assert rc == -1  # STRM_EINVAL
    assert "at most" in binding.lib().strm_last_error().decode()
    # the binding refuses a state of the wrong shape before calling the library
    with pytest.raises(ValueError):
        binding.conserved_totals_static(case, w)
