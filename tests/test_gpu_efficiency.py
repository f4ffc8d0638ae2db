"""The BF / BFE / sigma efficiency comparison (Sec. 4.4.1, Table
fig:s4_s_time) on the hydrostatic sine + slope tank: the three models share
the vertical spacing at the shallowest point, so BFE and sigma need ~2/5 and
~1/4 of BF's particles.  On the GPU each model runs 20 steps (mixed form):
the pressure stays hydrostatic in all three (relative L2 error of a few
percent at most, comparable across the models as in Fig. s4_s_l2).  The time
per step is reported: at these sizes (8k-32k particles) the GPU step is bound
by the pressure solve's per-iteration latency, not by the particle count, so
the paper's 1 : 1/3 : 1/6 time ratios (a CPU code) are not expected here
(timed over 40 further steps)."""
import numpy as np
import pytest

from paper_2607_28872_b300 import scenarios as S

pytestmark = pytest.mark.gpu


def test_bf_bfe_sigma_efficiency():
    import torch
    from paper_2607_28872_b300 import vct as V
    rows = {}
    for kind in ("BF", "BFE", "SIGMA"):
        sc = S.efficiency_tank(kind)
        s = V.Solver(sc)
        st = V.DeviceState(sc)
        s.vct_step(st, 20)
        g = st.numpy()
        f = sc.type == S.FLUID
        hyd = sc.params["rho"] * sc.params["g"] * (sc.params["H"] - g["z"])
        deep = f & (g["p"] > 0)
        err = np.linalg.norm((g["p"] - hyd)[deep]) / np.linalg.norm(hyd[deep])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.vct_step(st, 40)
        e1.record()
        e1.synchronize()
        rows[kind] = (sc.n_fluid, e0.elapsed_time(e1) / 40, err)
        print(f"PARITY efficiency {kind}: n_fluid={sc.n_fluid} ms/step={rows[kind][1]:.3f} "
              f"p_rel_l2={err:.3e}")
    nb, tb, _ = rows["BF"]
    assert 0.35 < rows["BFE"][0] / nb < 0.45 and 0.2 < rows["SIGMA"][0] / nb < 0.3
    for kind in rows:
        assert rows[kind][2] < 0.05, rows
