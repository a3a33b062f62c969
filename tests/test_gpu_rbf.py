"""RBF level-set map (Eq. 2, Eq. 3, renormalised), its gradient and Adam
through the C ABI against the FP64 oracle, alone and chained with the LLG
forward and adjoint (s -> Phi -> J and dJ/dPhi -> dJ/ds)."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_solver, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

H = 5e-9
# (nx, ny, design box, nrx, nry): a small box and the paper's 20 x 20 RBFs on a
# 60 x 60-node design region of the 256 x 64 demultiplexer
CASES = [(20, 12, (2, 14, 1, 10), 4, 3), (256, 64, (98, 158, 2, 62), 20, 20)]


@pytest.fixture(scope="module", autouse=True)
def _needs_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2411_19109_gb300 import load
    load()


def _layout(case):
    from oracle import rbf
    nx, ny, box, nrx, nry = case
    xk, yk, c = rbf.centres(nx, ny, H, H, box, nrx, nry)
    xj, yj = rbf.design_nodes(nx, ny, H, H, box)
    return xk, yk, c, xj, yj


def _design(a, box):
    x0, x1, y0, y1 = box
    return a[y0:y1, x0:x1].ravel()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-7)])
@pytest.mark.parametrize("case", CASES)
def test_phi_and_gradient_match_the_oracle(case, precision, tol):
    from oracle import rbf
    from paper_2411_19109_gb300 import LLG_FP32, LLG_FP64, llg_rbf_grad, llg_rbf_phi, llg_rbf_workspace_bytes, make_rbf
    nx, ny, box, nrx, nry = case
    xk, yk, c, xj, yj = _layout(case)
    rng = np.random.default_rng(nx + nrx)
    s = rng.uniform(-60e-9, 60e-9, xk.size)
    r = make_rbf(nx, ny, H, H, box, nrx, nry, 90.0)
    dt = torch.float32 if precision == "fp32" else torch.float64
    prec = LLG_FP32 if precision == "fp32" else LLG_FP64
    work = torch.empty(llg_rbf_workspace_bytes(r), dtype=torch.uint8, device="cuda")
    s_d = torch.as_tensor(s, device="cuda")
    phi = torch.full((ny, nx), 7.0, dtype=dt, device="cuda")
    llg_rbf_phi(r, s_d.data_ptr(), phi.data_ptr(), prec, work.data_ptr())
    torch.cuda.synchronize()
    got = phi.double().cpu().numpy()
    expect, _ = rbf.phi_map(s, xk, yk, c, xj, yj, 90)
    assert rel_l2(_design(got, box), expect) < tol
    inside = np.zeros((ny, nx), bool)
    inside[box[2]:box[3], box[0]:box[1]] = True
    assert (got[~inside] == 7.0).all()                 # nodes outside the box untouched
    g = torch.as_tensor(rng.standard_normal((ny, nx)), dtype=dt, device="cuda")
    dJds = torch.empty(xk.size, dtype=torch.float64, device="cuda")
    llg_rbf_grad(r, s_d.data_ptr(), g.data_ptr(), prec, dJds.data_ptr(), work.data_ptr())
    torch.cuda.synchronize()
    ref = rbf.phi_grad(s, xk, yk, c, xj, yj, 90, _design(g.double().cpu().numpy(), box))
    assert rel_l2(dJds.cpu().numpy(), ref) < 1e-10


def test_adam_matches_the_oracle():
    from oracle import rbf
    from paper_2411_19109_gb300 import llg_adam_step
    rng = np.random.default_rng(5)
    n = 400
    s = rng.standard_normal(n)
    m, v = np.zeros(n), np.zeros(n)
    sd, md, vd = (torch.as_tensor(a, device="cuda") for a in (s, m, v))
    for t in (1, 2, 3):
        g = rng.standard_normal(n)
        gd = torch.as_tensor(g, device="cuda")
        llg_adam_step(sd.data_ptr(), gd.data_ptr(), md.data_ptr(), vd.data_ptr(), n, t, 0.01)
        s, m, v = rbf.adam(s, g, m, v, t, 0.01)
    torch.cuda.synchronize()
    np.testing.assert_allclose(sd.cpu().numpy(), s, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(vd.cpu().numpy(), v, rtol=1e-13, atol=1e-30)


def test_chain_through_the_llg_adjoint_matches_the_oracle():
    """s -> Phi (RBF map) -> LLG forward and discrete adjoint -> dJ/dPhi ->
    dJ/ds, FP64 on both sides."""
    from oracle import llg, rbf
    from paper_2411_19109_gb300 import LLG_FP64, llg_rbf_grad, llg_rbf_phi, llg_rbf_workspace_bytes, make_rbf
    inst = W.random_small(16, 12, 1, seed=9, nsteps=20)
    box, nrx, nry = (3, 13, 2, 10), 3, 2
    xk, yk, c, xj, yj = _layout((16, 12, box, nrx, nry))
    s = np.random.default_rng(11).uniform(-20e-9, 20e-9, xk.size)
    # oracle chain
    phi_o = inst.phi.copy()
    phi_o[0, box[2]:box[3], box[0]:box[1]] = rbf.phi_map(s, xk, yk, c, xj, yj, 90)[0].reshape(8, 10)
    inst_o = W.Instance(inst.problem, phi_o, inst.m0, inst.mask, "rbf")
    _, dphi_o, _ = llg.gradient(inst_o)
    dJds_o = rbf.phi_grad(s, xk, yk, c, xj, yj, 90, _design(dphi_o[0], box))
    # GPU chain
    r = make_rbf(16, 12, H, H, box, nrx, nry, 90.0)
    work = torch.empty(llg_rbf_workspace_bytes(r), dtype=torch.uint8, device="cuda")
    s_d = torch.as_tensor(s, device="cuda")
    sv = gpu_solver([inst], "fp64")
    try:
        phi = sv.pack_scalar([inst.phi])
        llg_rbf_phi(r, s_d.data_ptr(), phi.data_ptr(), LLG_FP64, work.data_ptr())
        m0 = sv.pack_vector([inst.m0])
        sv.forward(phi, m0)
        g, _ = sv.adjoint()
        dJds = torch.empty(xk.size, dtype=torch.float64, device="cuda")
        llg_rbf_grad(r, s_d.data_ptr(), g.data_ptr(), LLG_FP64, dJds.data_ptr(), work.data_ptr())
        torch.cuda.synchronize()
    finally:
        sv.close()
    assert rel_l2(dJds.cpu().numpy(), dJds_o) < 1e-8
