"""Paper-scale 3D spreading inputs on the GPU (Sec. 3-4): the geodesic /
truncated-sphere meshes against the oracle on a small lattice, and a short
run of the 250 x 250 x 150 case with its ~120 000-triangle drop."""
import numpy as np
import pytest

from paper_2604_17463_gb300 import iblb
from paper_2604_17463_gb300 import workloads as W
from helpers import fluid_mask, oracle_from_workload, rel_l2

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", ["cap", "sphere"])
def test_small_geodesic_drop_matches_oracle(shape):
    R, xi = 6.0, 1.0
    if shape == "cap":
        q, tri = W.truncated_sphere(6, R, 90.0, W.WALL_PLANE + xi, (12.3, 11.8))
        theta = 60.0
    else:
        q, tri = W.geodesic_sphere(6, R, (12.3, 11.8, W.WALL_PLANE + xi + R))
        theta = 45.0
    wl = W.Workload("geo", 19, 24, 24, 18, 0.56, 2e-3, xi, theta, 9, 3, 10, q, tri)
    o = oracle_from_workload(wl)
    g = iblb.Simulation.from_workload(wl)
    assert o.step(10) == 0
    g.step(10)
    ro, uo, qo = o.fields()
    rg, ug, qg = g.fields()
    m = fluid_mask(o.shape, 3)
    assert rel_l2(rg[m] - 1.0, ro[m] - 1.0) < 1e-9
    assert rel_l2(ug[:, m], uo[:, m]) < 1e-10
    assert np.max(np.abs(qg - qo)) < 1e-11
    g.close()


def test_paper_scale_cap_short_run():
    case = W.spread3d_cap(0.59, t_mu_count=1.0)
    wl = case.work
    g = iblb.Simulation.from_workload(wl, storage=iblb.FP32_DEV)
    o0 = g.observables()
    g.step(300)
    o1 = g.observables()
    g.close()
    assert abs(o1["volume"] / o0["volume"] - 1.0) < 1e-3
    assert abs(o0["height"] / (2.0 ** (1.0 / 3.0) * case.R0) - 1.0) < 2e-3   # hemisphere
    assert abs(o1["height"] / o0["height"] - 1.0) < 0.05
    assert 80.0 < o0["theta_deg"] < 100.0
