"""The paper's 1D Euler examples with discontinuities (Examples 3.5-3.7),
full runs on the GPU against full runs of the oracle (shocked tolerance,
relative L-inf 1e-8), plus the linear-weight study of Example 3.7 on a
reduced grid."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2207_05258_gb300 import workloads as W
from _util import oracle_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hw():
    from paper_2207_05258_gb300 import build
    build.build()
    from paper_2207_05258_gb300 import hweno
    return hweno


def both(hw, w, **opts):
    s = hw.Solver.from_workload(w, **opts)
    U, V = torch.from_numpy(w.U.copy()).cuda(), torch.from_numpy(w.V.copy()).cuda()
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    s.run(U, V, None, t, w.t_end)
    g = U.cpu().numpy().reshape(w.m, -1), V.cpu().numpy().reshape(w.m, -1), float(t.item())
    s.close()
    o = O.run(oracle_problem(w, **opts), w.U, w.V, None, 0.0, w.t_end)
    return g, o


def check(g, o, tol=1e-8):
    assert g[2] == o[3]
    eu = np.max(np.abs(g[0] - o[0])) / np.max(np.abs(o[0]))
    ev = np.max(np.abs(g[1] - o[1])) / max(np.max(np.abs(o[1])), 1.0)
    assert eu <= tol and ev <= tol, (eu, ev)
    rho, m, E = g[0]
    p = 0.4 * (E - 0.5 * m * m / rho)
    assert np.all(rho > 0) and np.all(p > 0)


@pytest.mark.parametrize("make", [lambda: W.lax(200), lambda: W.shu_osher(400),
                                  lambda: W.blast_waves(800)],
                         ids=["lax", "shu_osher", "blast_waves"])
def test_example_full_run(hw, make):
    g, o = both(hw, make())
    check(g, o)


@pytest.mark.parametrize("G,D", [("G1", "D1"), ("G1", "D3"), ("G3", "D1")])
def test_weight_study_blast_waves(hw, G, D):
    w = W.blast_waves(200, t_end=0.01)
    g, o = both(hw, w, lin_w=W.WEIGHT_SETS[G], lim_d=W.WEIGHT_SETS[D])
    check(g, o)
