"""Pin of the energy objective's normalisation (Eq. 9's energy term as the
nanoparticle workload states it: (E_d + E_ex)(m_N) / (K_d V_domain), K_d =
mu0 Ms^2 / 2).

For a uniformly magnetised prism with psi = 1 everywhere, E_ex = 0 and
E_d = (mu0/2) Ms^2 V sum_ij m.N_ij m = K_d V_domain N_m, with N_m the
prism's demagnetising factor along m.  So the energy term equals Aharoni's
closed-form factor (written out in test_oracle_demag) along each axis; a
wrong V_domain, K_d or energy sign would move it.
"""
import numpy as np
import pytest

import workloads as W
from oracle import llg
from tests.test_oracle_demag import aharoni_factor


@pytest.mark.parametrize("cells,h", [((6, 4, 1), (3e-9, 4e-9, 2.5e-9)), ((4, 3, 2), (5e-9, 2e-9, 3e-9))])
def test_uniform_prism_energy_is_demag_factor(cells, h):
    nx, ny, nz = cells
    dx, dy, dz = h
    p = W.Problem(nx=nx, ny=ny, nz=nz, dx=dx, dy=dy, dz=dz, Ms=8e5, A=1.3e-11, objective=W.J_ENERGY_AREA,
                  area_target=0.3, penalty_w=0.7, nsteps=0)
    model = llg.Model(p, np.ones((nz, ny, nx)))       # psi = 1/(1 + e^-50) = 1 in FP64
    assert np.all(model.psi == 1.0)
    a, b, c = nx * dx / 2, ny * dy / 2, nz * dz / 2
    factors = [aharoni_factor(b, c, a), aharoni_factor(c, a, b), aharoni_factor(a, b, c)]
    penalty = p.penalty_w * (1.0 - p.area_target) ** 2
    for axis in range(3):
        m = np.zeros((3, nz, ny, nx))
        m[axis] = 1.0
        J = model.terminal(m)
        assert J - penalty == pytest.approx(factors[axis], rel=1e-10)
        Ed, Ee = model.energy_terms(m)
        assert Ee == 0.0
