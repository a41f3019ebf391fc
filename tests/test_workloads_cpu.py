"""The seeded workloads carry the benchmark configurations' parameters (no GPU): grid, domain,
gas, scheme and boundary kinds of the channel, boundary-layer and shock/boundary-layer cases,
and the ranges of the batched ensemble draws."""
import math

from paper_2004_02276_gb300 import inputs


def test_channel_workloads():
    for c, grid, re, steps in ((inputs.C1, (64, 48, 32), 3000.0, 20),
                               (inputs.C2, (256, 192, 128), 7000.0, 200)):
        assert (c.nx, c.ny, c.nz) == grid and c.kind == "channel"
        assert math.isclose(c.lx, 2 * math.pi) and c.ly == 2.0 and math.isclose(c.lz, math.pi)
        assert c.y_map == "tanh" and c.beta == 1.5 and c.y_wall and c.bc_xmin is None
        assert (c.mach, c.reynolds, c.prandtl, c.gamma, c.visc_exp) == (1.5, re, 0.72, 1.4, 0.76)
        assert c.visc_law == "power" and c.forcing
        assert (c.L, c.weno_mode, c.theta_thr, c.cfl, c.steps) == (3, "sensor", 0.05, 0.8, steps)
        assert c.noise == 0.05 and c.precision == "fp64"


def test_boundary_layer_workloads():
    c3, c4 = inputs.C3, inputs.C4
    assert (c3.nx, c3.ny, c3.nz) == (1024, 256, 256)
    assert (c4.nx, c4.ny, c4.nz) == (2048, 384, 256)
    for c in (c3, c4):
        assert c.kind == "bl" and c.mach == 2.0 and c.t_wall == 1.7
        assert (c.bc_xmin, c.bc_xmax, c.bc_ymin, c.bc_ymax) == ("recycle", "char", "wall", "char")
        assert c.weno_mode == "sensor" and c.L == 3 and not c.forcing
    assert not c3.shock
    assert c4.shock and math.isclose(c4.shock_theta, math.radians(8.0))
    assert c3.npts == 67_108_864 and c4.npts == 201_326_592


def test_ensemble_draws_in_range():
    cases = inputs.ensemble_cases(seed=0)
    assert len(cases) == 64
    for c in cases:
        assert 32 <= c.nx <= 192 and 32 <= c.ny <= 128 and 32 <= c.nz <= 128
        assert 0.3 <= c.mach <= 3.0 and 2000.0 <= c.reynolds <= 8000.0
    assert abs(sum(c.npts for c in cases) - 44.7e6) < 0.1e6
    # the same seed gives the same ensemble; another seed another one
    assert [c.nx for c in inputs.ensemble_cases(seed=0)] == [c.nx for c in cases]
    assert [c.nx for c in inputs.ensemble_cases(seed=1)] != [c.nx for c in cases]


def test_bl_state_does_not_depend_on_its_chunking():
    """The boundary-layer initial state is built a few z planes at a time (to keep the memory of
    the 201 M-point workload low); the values are those of the whole-array recipe: the same
    SplitMix64 outputs per (component, k, j, i) and the same arithmetic per element."""
    import numpy as np

    c = inputs.bl_case("bl-40x24x11", 40, 24, 11, 5.0, 6.0, 1.0, noise=0.05)
    ref = inputs.bl_state(c, seed=4, planes_per_chunk=1000)
    for ch in (1, 3, 11):
        assert np.array_equal(inputs.bl_state(c, seed=4, planes_per_chunk=ch), ref)
    # the noise field of component m at node (k, j, i) is output (m nz + k) ny nx + j nx + i
    r = inputs.uniform(4, (3, c.nz, c.ny, c.nx))
    blk = inputs.uniform_block(4, (2 * c.nz + 5) * c.ny * c.nx, c.ny * c.nx).reshape(c.ny, c.nx)
    assert np.array_equal(blk, r[2, 5])
