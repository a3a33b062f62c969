"""GPU path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances: FP64 path 1e-9 relative (rounding order only); FP32
path 1e-5 relative L2 on m after 1000 steps and 1e-4 relative L2 on dJ/dPhi
(the targets the method's FP32 build is held to)."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_run, gpu_solver, oracle_run, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _needs_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2411_19109_gb300 import load
    load()


# column lengths 8..64 (8-element FFT lanes) and 128, 256, 1024 (16-element
# lanes in FP32: ny = 64, 100, 400)
FIELD_CASES = [(4, 1), (8, 5), (12, 7), (16, 9), (32, 32), (36, 20), (64, 3), (8, 64), (4, 100), (4, 400)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("fp32", 2e-6)])
@pytest.mark.parametrize("shape", FIELD_CASES)
def test_field_parity(shape, precision, tol):
    from oracle import llg
    inst = W.random_small(*shape, 1, seed=shape[0] * 7 + shape[1])
    s = gpu_solver([inst], precision)
    try:
        phi = s.pack_scalar([inst.phi])
        m = s.pack_vector([inst.m0])
        model = llg.Model(inst.problem, inst.phi)
        Bd = s.unpack_vector(s.field(phi, m, 0.0, demag_only=True))[0].double().cpu().numpy()
        assert rel_l2(Bd, model.demag(inst.m0)) < tol
        t = 3.7e-11
        B = s.unpack_vector(s.field(phi, m, t))[0].double().cpu().numpy()
        assert rel_l2(B, model.field(inst.m0, t)) < tol
    finally:
        s.close()


# "fp32-df": FP32 with the double-float frequency domain in the adjoint
@pytest.mark.parametrize("precision,tol_m,tol_g", [("fp64", 1e-10, 1e-9), ("fp32", 1e-5, 1e-4),
                                                   ("fp32-df", 1e-5, 1e-4)])
@pytest.mark.parametrize("shape,objective", [((12, 8), W.J_PORT), ((16, 12), W.J_ENERGY_AREA),
                                             ((8, 5), W.J_PORT), ((20, 3), W.J_ENERGY_AREA),
                                             ((8, 64), W.J_PORT)])
def test_forward_adjoint_parity_small(shape, objective, precision, tol_m, tol_g):
    inst = W.random_small(*shape, 1, seed=3, nsteps=40, objective=objective)
    kw = {"adj_spectral": "dfloat"} if precision == "fp32-df" else {}
    g = gpu_run([inst], precision[:4], want_dm0=True, **kw)
    o = oracle_run(inst)
    assert rel_l2(g["mT"][0], o["mT"]) < tol_m
    assert abs(g["J"][0] - o["J"]) <= tol_g * max(abs(o["J"]), 1e-30)
    assert rel_l2(g["dphi"][0], o["dphi"]) < tol_g
    assert rel_l2(g["dm0"][0], o["dm0"]) < tol_g


# The unit vector m at air nodes (psi -> 0) carries no magnetisation and its
# motion is ill-conditioned: in the oracle a 1e-9 perturbation of m0 grows to
# 3e-2 at nodes with psi ~ 1e-16 within 1000 steps while the magnetisation
# M/Ms = psi m moves by 2e-9.  Parity on m is therefore measured on psi m.
# FP64: rounding-order differences (FMA on the GPU, none in the oracle) stay
# far below 1e-8 on psi m.
@pytest.mark.parametrize("precision,tol_m,tol_g", [("fp64", 1e-8, 1e-7), ("fp32", 1e-5, 1e-4)])
def test_film32_1000_steps(precision, tol_m, tol_g):
    from oracle import llg
    inst = W.film32()
    psi = llg.psi_map(inst.phi, inst.problem.sigmoid_a)
    g = gpu_run([inst], precision)
    o = oracle_run(inst)
    em = rel_l2(psi * g["mT"][0], psi * o["mT"])
    ej = abs(g["J"][0] - o["J"]) / abs(o["J"])
    eg = rel_l2(g["dphi"][0], o["dphi"])
    print(f"film32 {precision}: psi*m {em:.2e}  J {ej:.2e}  dJ/dPhi {eg:.2e}")
    assert em < tol_m
    assert ej < tol_g
    assert eg < tol_g


def test_batch_of_uneven_grids_matches_single_runs():
    insts = [W.random_small(12, 8, 1, seed=1, nsteps=30),
             W.random_small(32, 5, 1, seed=2, nsteps=30, objective=W.J_ENERGY_AREA),
             W.random_small(8, 16, 1, seed=3, nsteps=30)]
    b = gpu_run(insts, "fp64")
    for k, inst in enumerate(insts):
        o = oracle_run(inst)
        assert rel_l2(b["mT"][k], o["mT"]) < 1e-10
        assert rel_l2(b["dphi"][k], o["dphi"]) < 1e-9
        single = gpu_run([inst], "fp64")
        np.testing.assert_array_equal(single["dphi"][0], b["dphi"][k])


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32-df"])
def test_schedules_give_identical_gradients(precision):
    inst = W.random_small(12, 8, 1, seed=5, nsteps=23)
    kw = {"adj_spectral": "dfloat"} if precision == "fp32-df" else {}
    ref = gpu_run([inst], precision[:4], ckpt="store_all", **kw)
    for ckpt, seg in (("periodic", 0), ("periodic", 1), ("periodic", 4), ("periodic", 23), ("periodic", 40),
                      ("binomial", 0), ("binomial", 1), ("binomial", 2), ("binomial", 6)):
        g = gpu_run([inst], precision[:4], ckpt=ckpt, seg_len=seg, want_dm0=True, **kw)
        np.testing.assert_array_equal(g["dphi"][0], ref["dphi"][0])
        assert g["J"][0] == ref["J"][0]


def test_levelset_step_matches_oracle():
    from oracle import llg
    insts = [W.random_small(12, 8, 1, seed=1), W.random_small(8, 4, 1, seed=2)]
    rng = np.random.default_rng(0)
    s = gpu_solver(insts, "fp64")
    try:
        phi = s.pack_scalar([i.phi for i in insts])
        grads = [rng.standard_normal(i.phi.shape) for i in insts]
        masks = []
        for i in insts:
            mk = (rng.uniform(size=i.phi.shape) < 0.6).astype(np.uint8)
            masks.append(mk)
        grad = s.pack_scalar(grads)
        mask = torch.cat([torch.as_tensor(mk.reshape(-1)) for mk in masks]).cuda()
        s.levelset_step(phi, grad, mask, 0.07)
        out = s.unpack_scalar(phi)
        for k, inst in enumerate(insts):
            ref = llg.levelset_step(inst.phi, grads[k], masks[k], 0.07)
            np.testing.assert_allclose(out[k].cpu().numpy(), ref, rtol=1e-15, atol=1e-15)
    finally:
        s.close()


def test_zero_steps_and_late_window():
    inst = W.random_small(8, 4, 1, seed=4, nsteps=0, objective=W.J_ENERGY_AREA)
    g = gpu_run([inst], "fp64")
    o = oracle_run(inst)
    assert abs(g["J"][0] - o["J"]) < 1e-9 * abs(o["J"])
    assert rel_l2(g["dphi"][0], o["dphi"]) < 1e-9
    inst = W.random_small(8, 4, 1, seed=4, nsteps=5, n_from=9)
    g = gpu_run([inst], "fp64")
    assert g["J"][0] == 0.0
    assert np.abs(g["dphi"][0]).max() == 0.0


def test_autograd_function():
    from paper_2411_19109_gb300 import llg_function
    inst = W.random_small(12, 8, 1, seed=6, nsteps=20)
    s = gpu_solver([inst], "fp64")
    try:
        phi = s.pack_scalar([inst.phi]).requires_grad_(True)
        m0 = s.pack_vector([inst.m0]).requires_grad_(True)
        J = llg_function().apply(phi, m0, s)
        (3.0 * J.sum()).backward()
        o = oracle_run(inst)
        assert rel_l2(phi.grad.cpu().numpy(), 3.0 * o["dphi"]) < 1e-9
        assert rel_l2(m0.grad.cpu().numpy(), 3.0 * o["dm0"]) < 1e-9
    finally:
        s.close()


def test_invalid_sizes_are_rejected():
    from paper_2411_19109_gb300 import LLGError
    bad = W.random_small(6, 4, 1).problem        # nx % 4 != 0
    with pytest.raises(LLGError):
        gpu_solver([type("I", (), {"problem": bad})()])


def test_contexts_of_different_sizes_coexist():
    """A context for a small grid created after one for a large grid must not
    restrict the large one's launches (kernel attributes are process-wide)."""
    big = W.random_small(256, 24, 1, seed=31, nsteps=3)
    small = W.random_small(8, 4, 1, seed=32, nsteps=3)
    ref = gpu_run([big], "fp32")
    s_big = gpu_solver([big], "fp32")
    s_small = gpu_solver([small], "fp32")
    try:
        phi = s_small.pack_scalar([small.phi])
        m0 = s_small.pack_vector([small.m0])
        s_small.forward(phi, m0)
        phi = s_big.pack_scalar([big.phi])
        m0 = s_big.pack_vector([big.m0])
        J, _ = s_big.forward(phi, m0)
        g, _ = s_big.adjoint()
        assert J[0] == ref["J"][0]
        np.testing.assert_array_equal(s_big.unpack_scalar(g)[0].double().cpu().numpy(), ref["dphi"][0])
    finally:
        s_small.close()
        s_big.close()


def test_graph_replay_matches_direct_launches():
    """Segments replayed from captured CUDA graphs give bit-identical J,
    dJ/dPhi and m_N to the same launches issued one by one, over a schedule
    whose segments have two different lengths (37 steps, K = 6)."""
    insts = [W.random_small(24, 10, 1, seed=41, nsteps=37), W.random_small(16, 12, 1, seed=42, nsteps=37)]
    direct = gpu_run(insts, "fp32", seg_len=6, use_graph=False)
    for _ in range(2):   # the second run replays the graphs captured by the first
        s = gpu_solver(insts, "fp32", seg_len=6, use_graph=True)
        try:
            for rep in range(2):
                phi = s.pack_scalar([i.phi for i in insts])
                m0 = s.pack_vector([i.m0 for i in insts])
                J, mT = s.forward(phi, m0, want_mT=True)
                g, _ = s.adjoint()
                np.testing.assert_array_equal(J, direct["J"])
                for k, x in enumerate(s.unpack_vector(mT)):
                    np.testing.assert_array_equal(x.double().cpu().numpy(), direct["mT"][k])
                for k, x in enumerate(s.unpack_scalar(g)):
                    np.testing.assert_array_equal(x.double().cpu().numpy(), direct["dphi"][k])
        finally:
            s.close()


def test_batch_with_both_column_kernels_matches_single_runs():
    """Column lengths 64 and 128 in one FP32 context: one instance on each
    column kernel, each identical bit for bit to its run alone."""
    insts = [W.random_small(12, 32, 1, seed=51, nsteps=12), W.random_small(8, 64, 1, seed=52, nsteps=12)]
    b = gpu_run(insts, "fp32")
    for k, inst in enumerate(insts):
        single = gpu_run([inst], "fp32")
        np.testing.assert_array_equal(single["dphi"][0], b["dphi"][k])
        np.testing.assert_array_equal(single["mT"][0], b["mT"][k])
        assert single["J"][0] == b["J"][k]


# The widest rows llg_create accepts: nx = 1024 in FP32 (row FFT length 1024,
# one row per tile, 128-lane FFT groups on named barriers) and nx = 780 in
# FP64 (the adjoint's row tile at its shared-memory limit; the same FFT
# length), plus the double-float adjoint spectrum at nx = 1024.
@pytest.mark.parametrize("precision,nx,tol", [("fp32", 1024, 2e-6), ("fp64", 780, 1e-11), ("fp32", 780, 2e-6)])
def test_widest_rows_field(precision, nx, tol):
    from oracle import llg
    inst = W.random_small(nx, 3, 1, seed=nx)
    s = gpu_solver([inst], precision)
    try:
        phi = s.pack_scalar([inst.phi])
        m = s.pack_vector([inst.m0])
        model = llg.Model(inst.problem, inst.phi)
        B = s.unpack_vector(s.field(phi, m, 2.0e-11))[0].double().cpu().numpy()
        assert rel_l2(B, model.field(inst.m0, 2.0e-11)) < tol
    finally:
        s.close()


@pytest.mark.parametrize("precision,nx,tol_m,tol_g", [("fp32", 1024, 1e-5, 1e-4), ("fp32-df", 1024, 1e-5, 1e-4),
                                                      ("fp64", 780, 1e-10, 1e-9)])
def test_widest_rows_forward_adjoint(precision, nx, tol_m, tol_g):
    inst = W.random_small(nx, 2, 1, seed=nx + 1, nsteps=12)
    kw = {"adj_spectral": "dfloat"} if precision == "fp32-df" else {}
    g = gpu_run([inst], precision[:4], want_dm0=True, **kw)
    o = oracle_run(inst)
    assert rel_l2(g["mT"][0], o["mT"]) < tol_m
    assert abs(g["J"][0] - o["J"]) <= tol_g * max(abs(o["J"]), 1e-30)
    assert rel_l2(g["dphi"][0], o["dphi"]) < tol_g
    assert rel_l2(g["dm0"][0], o["dm0"]) < tol_g


@pytest.mark.parametrize("precision", ["fp32", "fp64", "fp32-df"])
def test_state_records_match_stage_records(precision):
    """LLG_RECORD_STATES (m per step; each reverse step recomputes its
    stages) gives bit-identical J and gradients to LLG_RECORD_STAGES in
    every schedule, batched over two uneven grids with two instance-group
    chains and graph replays, and holds less memory on a long segment."""
    insts = [W.random_small(12, 8, 1, seed=5, nsteps=23), W.random_small(16, 5, 1, seed=6, nsteps=23,
                                                                           objective=W.J_ENERGY_AREA)]
    kw = {"adj_spectral": "dfloat"} if precision == "fp32-df" else {}
    for ckpt, seg in (("periodic", 0), ("periodic", 23), ("binomial", 2), ("store_all", 0)):
        ref = gpu_run(insts, precision[:4], ckpt=ckpt, seg_len=seg, want_dm0=True, **kw)
        for graphs in (True, False):
            g = gpu_run(insts, precision[:4], ckpt=ckpt, seg_len=seg, want_dm0=True, record="states",
                        use_graph=graphs, **kw)
            np.testing.assert_array_equal(g["J"], ref["J"])
            for k in range(len(insts)):
                np.testing.assert_array_equal(g["dphi"][k], ref["dphi"][k])
                np.testing.assert_array_equal(g["dm0"][k], ref["dm0"][k])
        if ckpt == "periodic" and seg == 23:
            assert g["bytes"] < ref["bytes"]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-5)])
@pytest.mark.parametrize("cells,h", [((64, 16), (3e-9, 4e-9, 2.5e-9)), ((48, 8), (5e-9, 5e-9, 5e-9))])
def test_film_mean_demag_field_is_the_prism_factor(cells, h, precision, tol):
    """A check of the GPU-built demag tensor independent of the oracle: the
    uniformly magnetised film (psi = 1) of 64 x 16 or 48 x 8 cells -- long
    enough that the tensor's far-field branch carries a share of the sum --
    has node-averaged demag field -mu0 Ms N_axis m, with N Aharoni's closed
    form for the prism along each axis (the Newell tensor is the exact
    cell-pair average)."""
    from tests.test_oracle_demag import aharoni_factor
    nx, ny = cells
    dx, dy, dz = h
    base = W.random_small(nx, ny, 1, seed=7)
    p = base.problem.replace(dx=dx, dy=dy, dz=dz)
    phi = np.ones((1, ny, nx))
    a, b, c = nx * dx / 2, ny * dy / 2, dz / 2
    factors = [aharoni_factor(b, c, a), aharoni_factor(c, a, b), aharoni_factor(a, b, c)]
    for axis in range(3):
        m = np.zeros((3, 1, ny, nx))
        m[axis] = 1.0
        inst = W.Instance(p, phi, m, base.mask, "uniform")
        s = gpu_solver([inst], precision)
        try:
            B = s.unpack_vector(s.field(s.pack_scalar([phi]), s.pack_vector([m]), 0.0, demag_only=True))[0]
            Bm = B.double().cpu().numpy()
        finally:
            s.close()
        expect = -4e-7 * np.pi * p.Ms * factors[axis]
        assert abs(Bm[axis].mean() - expect) <= tol * abs(expect)
        for k in range(3):
            if k != axis:
                assert abs(Bm[k].mean()) <= tol * abs(expect)
