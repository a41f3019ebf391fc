"""Overlap modes (strm_set_overlap): the ghost fill concurrent with the inner part of the
Ducros sensor (bit 1), and the x, y, z face stages as concurrent branches (bit 2). Only the order of
independent kernels changes, so every result must equal the sequential order bit for bit:
eager right-hand sides, eager RK steps and graph-replayed steps, in FP64 and mixed precision,
for the channel, the recycling shock/boundary layer, the digital-filter inflow and a grid too
thin for an interior region. The overlapped modes are also checked against the FP64 oracle
directly, so that parity does not rest on the sequential order alone."""
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


CH = inputs.C1
SBLI = inputs.bl_case("sbli-64x40x12", 64, 40, 12, 12.0, 6.0, 1.5, shock=True, noise=0.003)
DF = inputs.bl_case("bl-df-48x40x16", 48, 40, 16, 7.0, 6.0, 1.5, bc_xmin="df", df_ny=3, df_nz=2,
                    df_tau=0.5, df_seed=12345)
THIN = inputs.Case(name="thin-32x24x5", nx=32, ny=24, nz=5, reynolds=3000.0)  # nz < 2L + 1

CASES = [(c, p) for c in (CH, SBLI, DF, THIN) for p in ("fp64", "mixed")]


def state(case):
    w = inputs.channel_state(case, seed=0) if case.kind == "channel" else inputs.bl_state(case, seed=0)
    return torch.from_numpy(w).cuda()


def solver(case, overlap):
    s = binding.Solver(case, inflow=inputs.df_profiles(case) if case.bc_xmin == "df" else None)
    s.set_overlap(overlap)
    return s


@pytest.mark.parametrize("case,prec", CASES, ids=lambda v: v if isinstance(v, str) else v.name)
def test_overlap_is_bitwise_sequential(case, prec):
    case = case.replace(precision=prec)
    w0 = state(case)
    out = {}
    for ov in (0, 1, 2, 3):
        s = solver(case, ov)
        r = s.compute_rhs(w0.clone())
        w, r_old = w0.clone(), torch.zeros_like(w0)
        s.rk_step(w, r_old, dt=0.0, cfl=case.cfl)   # eager step
        s.advance_n(w, r_old, 4, cfl=case.cfl)       # captured graph
        torch.cuda.synchronize()
        out[ov] = (r.cpu(), w.cpu(), s.time())
        s.close()
    for ov in (1, 2, 3):
        assert torch.equal(out[0][0], out[ov][0]), ov
        assert torch.equal(out[0][1], out[ov][1]), ov
        assert out[0][2] == out[ov][2], ov


def test_overlap_toggle_rebuilds_graph():
    w0 = state(CH)
    ref = solver(CH, False)
    s = solver(CH, True)
    wa, ra = w0.clone(), torch.zeros_like(w0)
    wb, rb = w0.clone(), torch.zeros_like(w0)
    for ov in (True, False, True):
        s.set_overlap(ov)
        s.advance_n(wb, rb, 2, cfl=CH.cfl)
        ref.advance_n(wa, ra, 2, cfl=CH.cfl)
    torch.cuda.synchronize()
    assert torch.equal(wa, wb)
    assert binding.lib().strm_set_overlap(None, 1) == -1  # STRM_EINVAL
    assert binding.lib().strm_set_overlap(s.ctx, 4) == -1
    ref.close()
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_overlap_full_size_rhs_bitwise(prec):
    """The 256x192x128 benchmark channel: right-hand side with both overlap bits equals the
    sequential one bit for bit."""
    case = inputs.C2.replace(precision=prec)
    w = state(case)
    out = []
    for ov in (0, 3):
        s = solver(case, ov)
        out.append(s.compute_rhs(w).cpu())
        s.close()
    assert torch.equal(out[0], out[1])


def rel_max(a, b):
    return np.array([np.abs(a[m] - b[m]).max() / max(np.abs(b[m]).max(), 1e-300) for m in range(5)])


def rel_l2(a, b):
    return np.array([np.linalg.norm(a[m] - b[m]) / max(np.linalg.norm(b[m]), 1e-300) for m in range(5)])


@pytest.mark.parametrize("case", [CH, SBLI], ids=lambda c: c.name)
def test_overlap_modes_match_oracle(case):
    """Each overlap mode (ghost fill beside the inner sensor, concurrent face branches, both):
    the right-hand side element-wise within 1e-12 of each field's largest value and 4
    graph-replayed CFL steps within relative L2 1e-12 per field of the oracle, same time."""
    w0 = inputs.channel_state(case, seed=0) if case.kind == "channel" else inputs.bl_state(case, seed=0)
    cfg = O.make_cfg(case)
    r_ref = O.rhs(cfg, w0)
    w_ref, t_ref, _ = O.advance(cfg, w0, 4, cfl=case.cfl)
    for ov in (1, 2, 3):
        s = solver(case, ov)
        r = s.compute_rhs(torch.from_numpy(w0).cuda()).cpu().numpy()
        w = torch.from_numpy(w0).cuda()
        s.advance_n(w, torch.zeros_like(w), 4, cfl=case.cfl)
        t, _ = s.time()
        wg = w.cpu().numpy()
        s.close()
        e_r, e_w = rel_max(r, r_ref), rel_l2(wg, w_ref)
        assert e_r.max() <= 1e-12, (ov, e_r)
        assert e_w.max() <= 1e-12, (ov, e_w)
        assert abs(t - t_ref) <= 1e-13 * t_ref, (ov, t, t_ref)
