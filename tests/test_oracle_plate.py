"""Oracle pin on the elliptic plate (Section 4.3.2), CPU only: the oracle's own stepping
with the boundary rules converges to the manufactured solution at first order, the
character of the printed EOCs (displacement 1.06 / 1.07, stress 1.01 in L2; fixture
tests/golden/plate_primal_eoc.txt).  The paper's boundary rules are not given, so the
order is pinned, not the printed error values.  Protocol as printed: 40 N_x^2 sweeps
from f_S = 0, errors on the active nodes, E = 0.1, nu = 0.7; N_x = 16, 32 and 48 keep
the run to seconds (the GPU parity suite repeats it at N_x = 32 ... 256)."""
import numpy as np

import oracle
from paper_2609_31347_b300 import inputs as I
from tests.conftest import golden


def test_plate_primal_converges_at_first_order():
    gd = golden("plate_primal_eoc.txt")
    nxs, ed2, es2 = [16, 32, 48], [], []
    for Nx in nxs:
        geo = I.plate_geometry(Nx)
        dstar, sigma, F = I.plate_manufactured(geo.X, geo.Y)
        F = F * geo.active
        wd, wT = I.plate_wall_data(geo)
        g = oracle.Grid(geo.nx, geo.nx, geo.dx, I.PLATE_NU, periodic=False,
                        node_type=geo.node_type, link=geo.link, wall_d=wd, wall_T=wT,
                        wall_n=geo.normal)
        fS = oracle.primal(g, I.PLATE_E, F, 40 * Nx * Nx)
        act = geo.active == 1
        d = oracle.displacement(g, fS, F)
        ed2.append(oracle.norm_L2((d - dstar)[:, act], geo.dx) /
                   oracle.norm_L2(dstar[:, act], geo.dx))
        fro = oracle.stress_frobenius_rows
        s = oracle.stress(g, I.PLATE_E, fS, F)
        es2.append(oracle.norm_L2(fro(s - sigma)[:, act], geo.dx) /
                   oracle.norm_L2(fro(sigma)[:, act], geo.dx))
    eoc_d, eoc_s = oracle.eoc(nxs, ed2), oracle.eoc(nxs, es2)
    # measured: 0.682, 0.310, 0.197 (EOC 1.13) and 0.346, 0.153, 0.115 (EOC 1.02)
    assert abs(eoc_d - gd["eoc_d_L2"][0]) < 0.15, eoc_d
    assert abs(eoc_s - gd["eoc_sigma_L2"][0]) < 0.15, eoc_s
    # and not second order, as on the periodic domain: the boundary rules are first order
    assert eoc_d < 1.6 and eoc_s < 1.6
    assert np.all(np.diff(ed2) < 0) and np.all(np.diff(es2) < 0)
