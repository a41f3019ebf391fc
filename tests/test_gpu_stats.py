"""Flow statistics on the GPU (Section 3: Reynolds and Favre averages over the homogeneous
directions and in time) against the oracle's per-sample statistics of the oracle's own states,
through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2004_02276_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


def rel_max(a, b):
    scale = np.abs(b).reshape(b.shape[0], -1).max(axis=1)
    return (np.abs(a - b).reshape(b.shape[0], -1).max(axis=1) / np.maximum(scale, 1e-300)).max()


def oracle_mean(case, w0, nsteps, mode, every=1, include_initial=True):
    cfg = O.make_cfg(case)
    samples = [O.stats(cfg, w0, mode)] if include_initial else []
    w = w0
    for n in range(1, nsteps + 1):
        w, _ = O.rk_step(cfg, w, 0.0, case.cfl)
        if n % every == 0:
            samples.append(O.stats(cfg, w, mode))
    return np.mean(samples, axis=0), len(samples)


def test_channel_xz_statistics_match_oracle():
    case = inputs.C1
    w0 = inputs.channel_state(case, seed=0)
    ref, nref = oracle_mean(case, w0, 4, 0)
    s = binding.Solver(case)
    w = torch.from_numpy(w0).cuda()
    r_old = torch.zeros_like(w)
    s.stats_bind("xz", every=1)
    s.stats_sample(w)
    s.advance_n(w, r_old, 4, cfl=case.cfl)  # graph replay path
    got, ns = s.stats_read()
    s.close()
    assert ns == nref == 5
    assert rel_max(got, ref) <= 1e-12


def test_boundary_layer_z_statistics_match_oracle():
    case = inputs.bl_case("bl-48x40x12", 48, 40, 12, 7.0, 6.0, 1.5)
    w0 = inputs.bl_state(case, seed=3)
    ref, nref = oracle_mean(case, w0, 4, 1, every=2, include_initial=False)
    s = binding.Solver(case)
    w = torch.from_numpy(w0).cuda()
    r_old = torch.zeros_like(w)
    s.stats_bind("z", every=2)
    for _ in range(4):
        s.rk_step(w, r_old, dt=0.0, cfl=case.cfl)  # eager path
    got, ns = s.stats_read()
    s.close()
    assert ns == nref == 2 and got.shape == (24, case.ny, case.nx)
    assert rel_max(got, ref) <= 1e-12


def test_favre_and_reynolds_stress_profiles_are_consistent():
    """Derived profiles from the accumulated means: the Favre mean velocity and the density-
    weighted turbulent stress tau_11 = mean(rho uu) - mean(rho) u~^2 >= 0."""
    case = inputs.C1
    s = binding.Solver(case)
    w = torch.from_numpy(inputs.channel_state(case, seed=1)).cuda()
    r_old = torch.zeros_like(w)
    s.stats_bind("xz", every=1)
    s.advance_n(w, r_old, 3, cfl=case.cfl)
    m, ns = s.stats_read()
    s.close()
    N = binding.Solver.STAT_NAMES
    rho, rho_u, rho_uu = m[N.index("rho")], m[N.index("rho_u")], m[N.index("rho_uu")]
    u_favre = rho_u / rho
    tau11 = rho_uu - rho * u_favre ** 2
    assert ns == 3 and np.all(tau11 >= -1e-14) and np.all(np.isfinite(u_favre))


def test_statistics_errors():
    case = inputs.Case(nx=8, ny=6, nz=4)
    s = binding.Solver(case)
    w = torch.from_numpy(inputs.channel_state(case, 0)).cuda()
    with pytest.raises(binding.StrmError):
        s.stats_sample(w)  # no buffer bound
    L = binding.lib()
    assert L.strm_stats_bytes(s.ctx, 7) == 0
    buf = torch.empty(16, dtype=torch.uint8, device="cuda")
    assert L.strm_stats_bind(s.ctx, 0, buf.data_ptr(), 16) == -4  # too small
    assert L.strm_stats_every(s.ctx, -1) == -1
    s.stats_bind("xz")
    m, ns = s.stats_read()
    assert ns == 0 and not m.any()
    s.close()
