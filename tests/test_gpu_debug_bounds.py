"""The bounds-checking build (-DSTRM_DEBUG, libstrm_debug.so) on the GPU: every kernel checks the
extreme nodes of each stencil, each ghost source and each list entry before using them and
records a violation in the context's error word instead of faulting. Run on every code path
(FP64 and mixed channels, the paper's L = 2 settings, boundary layers with each face kind,
the digital-filter inflow, statistics, the overlap modes and the batched ensemble), it must record nothing and
give the oracle's right-hand sides."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, {root!r})
from oracle import oracle as O
from paper_2004_02276_gb300 import binding, inputs
assert binding.lib().strm_debug_build() == 1
bl = lambda name, *a, **k: inputs.bl_case(name, *a, **k)
cases = {{
    "channel-fp64": inputs.C1,
    "channel-mixed": inputs.C1.replace(precision="mixed"),
    "paper-channel": inputs.PAPER_CHANNEL,
    "bl-recycle": bl("bl", 48, 40, 12, 7.0, 6.0, 1.5),
    "sbli": bl("sbli", 64, 40, 12, 12.0, 6.0, 1.5, shock=True, noise=0.003),
    "bl-sinh-mixed": bl("bls", 48, 40, 12, 7.0, 6.0, 1.5, y_map="sinh1", beta=4.0, precision="mixed"),
    "open-char": bl("open", 40, 24, 10, 6.0, 6.0, 1.5, bc_xmin="char", bc_ymin="char", weno_mode="all"),
    "bl-df": bl("bldf", 36, 30, 10, 5.0, 6.0, 1.5, bc_xmin="df", df_ny=2, df_nz=2, df_tau=0.3, df_seed=3),
    # overlap: the sensor's inner-box and shell regions, concurrent face branches
    "channel-fp64-overlap": inputs.C1,
    "sbli-mixed-overlap": bl("sblim", 64, 40, 12, 12.0, 6.0, 1.5, shock=True, noise=0.003, precision="mixed"),
}}
out = {{}}
for name, c in cases.items():
    prof = inputs.df_profiles(c) if c.bc_xmin == "df" else None
    w0 = inputs.channel_state(c, 0) if c.kind == "channel" else inputs.bl_state(c, 0)
    s = binding.Solver(c, inflow=prof)
    if name.endswith("-overlap"):
        s.set_overlap(3)
    w = torch.from_numpy(w0).cuda()
    r = s.compute_rhs(w).cpu().numpy()
    cfg = O.make_cfg(c, df=O.DFState(c, prof) if prof is not None else None)
    ref = O.rhs(cfg, w0)
    err = max(float(np.abs(r[m] - ref[m]).max() / np.abs(ref[m]).max()) for m in range(5))
    s.stats_bind("xz" if c.kind == "channel" else "z", every=1)
    s.advance_n(w, torch.zeros_like(w), 3, cfl=c.cfl)
    s.stats_read()
    out[name] = {{"flags": s.debug_flags(), "rhs_err": err, "mixed": c.precision == "mixed"}}
    s.close()
for prec in ("fp64", "mixed"):
    bag = [inputs.Case(nx=40, ny=24, nz=18, precision=prec),
           bl("e1", 48, 40, 12, 7.0, 6.0, 1.5, precision=prec),
           bl("e2", 36, 30, 10, 5.0, 6.0, 1.5, bc_xmin="df", df_ny=2, df_nz=2, df_tau=0.3, df_seed=3, precision=prec)]
    E = binding.Ensemble(bag, inflows={{2: inputs.df_profiles(bag[2])}})
    ws = [torch.from_numpy(inputs.channel_state(c, 0) if c.kind == "channel" else inputs.bl_state(c, 0)).cuda() for c in bag]
    rs = [torch.zeros_like(x) for x in ws]
    E.tune(ws, rs)
    E.advance(ws, rs, 3, cfl=0.8)
    out["ensemble-" + prec] = {{"flags": E.debug_flags(), "rhs_err": 0.0, "mixed": prec == "mixed"}}
    E.close()
print(json.dumps(out))
"""


def test_bounds_checking_build_records_no_violation():
    sys.path.insert(0, ROOT)
    from paper_2004_02276_gb300 import build

    build.build(debug=True)
    env = dict(os.environ, STRM_LIBRARY="debug")
    res = subprocess.run([sys.executable, "-c", SCRIPT.format(root=ROOT)], env=env,
                         capture_output=True, text=True, timeout=900)
    assert res.returncode == 0, res.stderr[-3000:]
    out = json.loads(res.stdout.strip().splitlines()[-1])
    for name, r in out.items():
        assert r["flags"] == 0, (name, r)
        assert r["rhs_err"] <= (1e-4 if r["mixed"] else 1e-12), (name, r)
