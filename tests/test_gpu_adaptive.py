"""Adaptive Dormand-Prince 5(4) integrator through the C ABI against the
FP64 oracle: in FP64 the step schedule, m_T, J, dJ/dPhi and dJ/dm0 follow
the oracle's own step control; in FP32 the oracle replays the GPU's accepted
steps and the gradient over that schedule is compared.  Films of both
column-kernel families and a 3D grid, a batch of uneven instances against
single runs, periodic checkpoints with schedule replay against one
checkpoint per accepted step, and the argument checks."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_solver, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

RTOL, ATOL = 1e-5, 1e-8


@pytest.fixture(scope="module", autouse=True)
def _needs_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2411_19109_gb300 import load
    load()


def _case(nx, ny, nz=1, seed=51, N=60):
    return W.random_small(nx, ny, nz, seed=seed, nsteps=N, objective=W.J_ENERGY_AREA)


def _gpu(insts, precision, **kw):
    s = gpu_solver(insts, precision, integrator="dopri5", rtol=RTOL, atol=ATOL, **kw)
    try:
        phi = s.pack_scalar([i.phi for i in insts])
        m0 = s.pack_vector([i.m0 for i in insts])
        J, mT = s.forward(phi, m0, want_mT=True)
        sched = [s.adaptive_steps(k) for k in range(len(insts))]
        g, dm0 = s.adjoint(want_dm0=True)
        return dict(J=J, mT=[x.double().cpu().numpy() for x in s.unpack_vector(mT)],
                    dphi=[x.double().cpu().numpy() for x in s.unpack_scalar(g)],
                    dm0=[x.double().cpu().numpy() for x in s.unpack_vector(dm0)], sched=sched)
    finally:
        s.close()


@pytest.mark.parametrize("shape", [(12, 8, 1), (8, 64, 1), (8, 6, 2)])
def test_fp64_follows_the_oracle_step_control(shape):
    from oracle import adaptive as AD
    from oracle import llg
    inst = _case(*shape)
    p = inst.problem
    mod = llg.Model(p, inst.phi)
    mT, sched, _ = AD.integrate(mod, inst.m0, p.nsteps * p.dt, p.dt, RTOL, ATOL)
    J, dphi, dm0 = AD.adjoint(mod, inst.m0, sched)
    g = _gpu([inst], "fp64")
    t, h = g["sched"][0]
    assert len(t) == len(sched) and 3 < len(sched) < p.nsteps
    np.testing.assert_allclose(h, [hh for _, hh in sched], rtol=1e-9)
    np.testing.assert_allclose(t, [tt for tt, _ in sched], rtol=1e-9, atol=1e-22)
    assert rel_l2(g["mT"][0], mT) < 1e-10
    assert abs(g["J"][0] - J) <= 1e-9 * abs(J)
    assert rel_l2(g["dphi"][0], dphi) < 1e-9
    assert rel_l2(g["dm0"][0], dm0) < 1e-9


@pytest.mark.parametrize("shape", [(12, 8, 1), (8, 64, 1), (8, 6, 2), (20, 3, 1)])
def test_fp32_gradient_over_its_own_schedule(shape):
    from oracle import adaptive as AD
    from oracle import llg
    inst = _case(*shape, seed=52)
    p = inst.problem
    g = _gpu([inst], "fp32")
    t, h = g["sched"][0]
    assert abs(h.sum() - p.nsteps * p.dt) <= 1e-12 * p.nsteps * p.dt
    sched = list(zip(t.tolist(), h.tolist()))
    mod = llg.Model(p, inst.phi)
    traj = AD.replay(mod, inst.m0, sched)
    J, dphi, dm0 = AD.adjoint(mod, inst.m0, sched)
    assert rel_l2(g["mT"][0], traj[-1]) < 1e-5
    assert abs(g["J"][0] - J) <= 1e-4 * abs(J)
    assert rel_l2(g["dphi"][0], dphi) < 1e-4
    assert rel_l2(g["dm0"][0], dm0) < 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_of_adaptive_instances_matches_single_runs(precision):
    insts = [_case(12, 8, seed=53, N=40), _case(16, 12, seed=54, N=40), _case(8, 6, 2, seed=55, N=40)]
    both = _gpu(insts, precision)
    for k, inst in enumerate(insts):
        one = _gpu([inst], precision)
        assert both["J"][k] == one["J"][0]
        np.testing.assert_array_equal(both["sched"][k][1], one["sched"][0][1])
        np.testing.assert_array_equal(both["dphi"][k], one["dphi"][0])


def test_invalid_adaptive_setups_are_rejected():
    from paper_2411_19109_gb300 import LLGError
    ok = _case(12, 8, N=10)
    bad_problems = [ok.problem.replace(objective=W.J_PORT),
                    ok.problem.replace(drive=(0.0,) * 33)]
    for p in bad_problems:
        with pytest.raises(LLGError):
            gpu_solver([type("I", (), {"problem": p})()], "fp32", integrator="dopri5", rtol=RTOL, atol=ATOL)
    with pytest.raises(LLGError):
        gpu_solver([ok], "fp32", integrator="dopri5", rtol=0.0, atol=ATOL)


def test_checkpoint_slots_cap_the_accepted_steps():
    from paper_2411_19109_gb300 import LLGError
    inst = _case(12, 8, seed=56, N=40)
    ref = _gpu([inst], "fp32")
    K = len(ref["sched"][0][1])
    assert K > 3
    same = _gpu([inst], "fp32", seg_len=K)                 # exactly enough slots
    assert same["J"][0] == ref["J"][0]
    np.testing.assert_array_equal(same["dphi"][0], ref["dphi"][0])
    s = gpu_solver([inst], "fp32", integrator="dopri5", rtol=RTOL, atol=ATOL, seg_len=K - 1)
    try:
        with pytest.raises(LLGError):
            s.forward(s.pack_scalar([inst.phi]), s.pack_vector([inst.m0]))
    finally:
        s.close()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_periodic_checkpoints_replay_the_accepted_steps(precision):
    """Periodic checkpoints (m every K = ceil(sqrt(seg_len)) accepted steps,
    each reverse block replaying the recorded steps) give bit-identical J and
    gradients to one checkpoint per accepted step, on a batch whose instances
    accept different numbers of steps, and hold fewer states."""
    insts = [_case(12, 8, seed=57, N=80), _case(16, 12, seed=58, N=80), _case(8, 6, 2, seed=59, N=80)]
    ref = _gpu(insts, precision, ckpt="store_all")
    counts = [len(x[1]) for x in ref["sched"]]
    assert len(set(counts)) > 1 and max(counts) > 9
    for seg in (0, max(counts), 2 * max(counts)):      # seg_len caps the accepted steps; K = ceil(sqrt(.))
        per = _gpu(insts, precision, ckpt="periodic", seg_len=seg)
        np.testing.assert_array_equal(per["J"], ref["J"])
        for k in range(len(insts)):
            np.testing.assert_array_equal(per["sched"][k][1], ref["sched"][k][1])
            np.testing.assert_array_equal(per["dphi"][k], ref["dphi"][k])
            np.testing.assert_array_equal(per["dm0"][k], ref["dm0"][k])
    big = [_case(12, 8, seed=57, N=400)]
    s_all = gpu_solver(big, precision, integrator="dopri5", rtol=RTOL, atol=ATOL, ckpt="store_all")
    s_per = gpu_solver(big, precision, integrator="dopri5", rtol=RTOL, atol=ATOL, ckpt="periodic")
    try:
        assert s_per.query()[0] < s_all.query()[0]
    finally:
        s_all.close()
        s_per.close()
