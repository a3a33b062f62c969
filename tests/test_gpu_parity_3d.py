"""3D grids (nz > 1: z exchange, full 3D demag with a 6-component tensor and
a zero-padded z transform) through the C ABI against the FP64 oracle, and
at the thick-film size (512 x 512 x 4, padded 1024 x 1024 x 8) against the
magnetometric demagnetising factors of the prism in closed form.

Tolerances are those of the film tests: FP64 rounding order only, FP32
1e-5 on m and 1e-4 on dJ/dPhi."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_run, gpu_solver, oracle_run, rel_l2
from tests.test_oracle_demag import aharoni_factor

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MU0 = 4e-7 * np.pi


@pytest.fixture(scope="module", autouse=True)
def _needs_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2411_19109_gb300 import load
    load()


# (nx, ny, nz): padded z lengths 4, 8 and 16, ragged column tiles, ny = 1
FIELD_CASES_3D = [(8, 4, 2), (12, 7, 3), (16, 9, 4), (8, 5, 5), (4, 3, 8), (20, 1, 2), (32, 12, 3)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-6)])
@pytest.mark.parametrize("shape", FIELD_CASES_3D)
def test_field_parity_3d(shape, precision, tol):
    from oracle import llg
    inst = W.random_small(*shape, seed=sum(shape) * 5 + shape[2])
    s = gpu_solver([inst], precision)
    try:
        phi = s.pack_scalar([inst.phi])
        m = s.pack_vector([inst.m0])
        model = llg.Model(inst.problem, inst.phi)
        Bd = s.unpack_vector(s.field(phi, m, 0.0, demag_only=True))[0].double().cpu().numpy()
        assert rel_l2(Bd, model.demag(inst.m0)) < tol
        t = 2.9e-11
        B = s.unpack_vector(s.field(phi, m, t))[0].double().cpu().numpy()
        assert rel_l2(B, model.field(inst.m0, t)) < tol
    finally:
        s.close()


@pytest.mark.parametrize("precision,tol_m,tol_g", [("fp64", 1e-10, 1e-9), ("fp32", 1e-5, 1e-4)])
@pytest.mark.parametrize("shape,objective", [((12, 8, 2), W.J_PORT), ((8, 6, 3), W.J_ENERGY_AREA),
                                             ((16, 5, 4), W.J_PORT)])
def test_forward_adjoint_parity_3d(shape, objective, precision, tol_m, tol_g):
    inst = W.random_small(*shape, seed=7, nsteps=30, objective=objective)
    g = gpu_run([inst], precision, want_dm0=True)
    o = oracle_run(inst)
    assert rel_l2(g["mT"][0], o["mT"]) < tol_m
    assert abs(g["J"][0] - o["J"]) <= tol_g * max(abs(o["J"]), 1e-30)
    assert rel_l2(g["dphi"][0], o["dphi"]) < tol_g
    assert rel_l2(g["dm0"][0], o["dm0"]) < tol_g


def test_batch_of_films_and_3d_grids_matches_single_runs():
    insts = [W.random_small(12, 8, 2, seed=11, nsteps=20),
             W.random_small(16, 6, 1, seed=12, nsteps=20, objective=W.J_ENERGY_AREA),
             W.random_small(8, 4, 3, seed=13, nsteps=20)]
    b = gpu_run(insts, "fp64")
    for k, inst in enumerate(insts):
        o = oracle_run(inst)
        assert rel_l2(b["mT"][k], o["mT"]) < 1e-10
        assert rel_l2(b["dphi"][k], o["dphi"]) < 1e-9
        single = gpu_run([inst], "fp64")
        np.testing.assert_array_equal(single["dphi"][0], b["dphi"][k])
        assert single["J"][0] == b["J"][k]


@pytest.mark.parametrize("axis", [0, 2])
def test_thick_film_mean_demag_field_is_the_prism_factor(axis):
    """Uniform magnetisation of the full 512 x 512 x 4 film (psi = 1): the
    node-averaged demag field is -mu0 Ms N_axis m with N the magnetometric
    factor of the 2.56 um x 2.56 um x 20 nm prism (Aharoni's closed form),
    because the Newell tensor is the exact cell-pair average."""
    base = W.thick512(nsteps=2)
    p = base.problem
    phi = np.ones((p.nz, p.ny, p.nx))
    m0 = np.zeros((3, p.nz, p.ny, p.nx))
    m0[axis] = 1.0
    inst = W.Instance(p, phi, m0, base.mask, "uniform")
    s = gpu_solver([inst], "fp32")
    try:
        B = s.field(s.pack_scalar([phi]), s.pack_vector([m0]), 0.0, demag_only=True)
        Bm = s.unpack_vector(B)[0].double().cpu().numpy()
    finally:
        s.close()
    a, b, c = p.nx * p.dx / 2, p.ny * p.dy / 2, p.nz * p.dz / 2
    N = {0: aharoni_factor(b, c, a), 2: aharoni_factor(a, b, c)}[axis]
    expect = -MU0 * p.Ms * N
    got = Bm[axis].mean()
    assert abs(got - expect) <= 1e-5 * abs(expect)
    # the transverse components average to zero by symmetry
    for k in range(3):
        if k != axis:
            assert abs(Bm[k].mean()) <= 1e-6 * abs(expect)


def test_thick_film_forward_adjoint_runs_at_full_size():
    """The 512 x 512 x 4 film (1,048,576 nodes) for 6 RK4 steps, FP32 and
    checkpointed: J and dJ/dPhi finite and |m| kept to 1e-5.  (The FP64
    column tile of this grid does not fit in shared memory; the FP64 path is
    held to the oracle on the smaller 3D grids above.)"""
    inst = W.thick512(nsteps=6)
    g = gpu_run([inst], "fp32")
    assert np.isfinite(g["J"][0]) and np.isfinite(g["dphi"][0]).all()
    m = g["mT"][0]
    nrm = np.sqrt((m ** 2).sum(axis=0))
    assert np.abs(nrm - 1.0).max() < 1e-5
    assert np.abs(g["dphi"][0]).max() > 0
