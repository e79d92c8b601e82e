"""Runs a few small cases through the library and saves the results (used by
tests/test_gpu_debug_build.py with NB_DEBUG=0 and NB_DEBUG=1)."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from paper_2604_09184_b300 import ics, nb  # noqa: E402


def main(out):
    res = {"lib": np.array(os.path.basename(nb.LIB_PATH))}
    d = ics.make_disk(64, 2.0, 0.97, 1.03, 0.01, 0.005, 6.0, seed=964, f_radius=400.0)
    s = nb.NBodySystem(nb.params(dt_rcrit=d.dt), d.x, d.v, d.m, d.R)
    s.step(60, d.dt)
    st = s.state()
    res["sys_x"], res["sys_v"], res["sys_m"] = st["x"], st["v"], st["m"]
    res["sys_stats"] = np.array([s.stats()[k] for k in ("groups", "merges", "bs_substeps")])
    s2 = nb.NBodySystem(nb.params(dt_rcrit=d.dt, ml_levels=2), d.x, d.v, d.m, d.R)
    s2.step(20, d.dt)
    res["ml_x"] = s2.state()["x"]
    import torch
    x, m = torch.tensor(d.x, device="cuda"), torch.tensor(d.m, device="cuda")
    rc = torch.tensor(st["rc"][:1].repeat(d.n) * 3, device="cuda")
    a, p, code = nb.kick(x, m, rc, precision=nb.NB_PREC_DS, rows=(5, 77))
    res["kick_a"], res["kick_code"] = a.cpu().numpy(), np.array(code)
    b = nb.NBodyBatch(nb.params(dt_rcrit=3.0), ics.ensemble(n_systems=16))
    b.step(6, 3.0)
    res["batch_x"] = b.state()["x"]
    dd = ics.make_disk(24, 2.0, 0.97, 1.03, 0.02, 0.01, 6.0, seed=6)
    rcd = np.full(dd.n, 3e-3)
    adj = nb.NBodyAdjoint(nb.params(dt_rcrit=dd.dt), dd.x, dd.v, dd.m, dd.R, rcd, 12, 5)
    adj.forward(dd.dt)
    g = adj.backward(np.ones((dd.n, 3)), np.ones((dd.n, 3)), np.ones(dd.n))
    res["adj_dx"], res["adj_dv"], res["adj_dm"] = g
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
