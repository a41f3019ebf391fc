"""Checkpoint and resume: everything a run carries between steps is caller-owned (the state w,
the simulated time, and with a digital-filter inflow the inflow buffer holding the fluctuation
plane and the draw counter), so saving those and restoring them in a fresh context continues
the run bit for bit: 10 steps, save, 10 steps in a new context equals 20 steps."""
import numpy as np
import pytest
import torch

from paper_2004_02276_gb300 import binding, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__

    __graft_entry__.build()
    torch.cuda.set_device(0)


CASES = [
    (inputs.C1, None),
    (inputs.bl_case("bl-df-48x40x16", 48, 40, 16, 7.0, 6.0, 1.5, bc_xmin="df", df_ny=3, df_nz=2,
                    df_tau=0.5, df_seed=99), "df"),
    (inputs.bl_case("sbli-64x40x12", 64, 40, 12, 12.0, 6.0, 1.5, shock=True, noise=0.003), None),
]


def make_solver(case, kind):
    return binding.Solver(case, inflow=inputs.df_profiles(case) if kind == "df" else None)


def initial(case):
    return inputs.channel_state(case, 0) if case.kind == "channel" else inputs.bl_state(case, 0)


@pytest.mark.parametrize("case,kind", CASES, ids=lambda v: getattr(v, "name", str(v)))
def test_resume_is_bitwise(case, kind):
    w0 = torch.from_numpy(initial(case)).cuda()
    # uninterrupted
    s = make_solver(case, kind)
    w = w0.clone()
    r = torch.zeros_like(w)
    s.advance_n(w, r, 20, cfl=case.cfl)
    full, t_full = w.cpu().numpy(), s.time()[0]
    s.close()
    # 10 steps, checkpoint to host, fresh context, restore, 10 steps
    s = make_solver(case, kind)
    w = w0.clone()
    r = torch.zeros_like(w)
    s.advance_n(w, r, 10, cfl=case.cfl)
    torch.cuda.synchronize()
    saved_w, saved_t = w.cpu().clone(), s.time()[0]
    saved_df = s._df_buf.cpu().clone() if kind == "df" else None
    s.close()
    del w, r
    s = make_solver(case, kind)
    w = saved_w.cuda()
    r = torch.zeros_like(w)
    s.set_time(saved_t)
    if kind == "df":
        s._df_buf.copy_(saved_df.cuda())
    s.advance_n(w, r, 10, cfl=case.cfl)
    resumed, t_res = w.cpu().numpy(), s.time()[0]
    s.close()
    assert np.array_equal(resumed, full)
    assert t_res == t_full
