"""Magnetisation-curve objective (Eq. 8 sampled per field level, size and
centre terms of Eq. 9) and the tabulated drive through the C ABI against the
FP64 oracle: J, m_N, dJ/dPhi and dJ/dm0 on films of both column-kernel
families and a 3D grid, the Stoner-Wohlfarth workload at a reduced number of
steps, a batch with port-objective instances, every checkpoint schedule, and
the argument checks."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_run, gpu_solver, oracle_run, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def curve_case(nx, ny, nz=1, seed=31, N=40):
    drive = tuple(np.repeat(0.02 * (np.arange(N + 1) // 10), 3).tolist())
    return W.random_small(nx, ny, nz, seed=seed, nsteps=N, objective=W.J_CURVE, comp=0, drive=drive,
                          rf_dir=(1.0, 0.0, 0.0), src=(0, nx, 0, ny),
                          sample_steps=(N // 4, N // 2, 3 * N // 4, N),
                          sample_targets=(1.7, -0.5, 1.9, 0.1), sample_weights=(1.0, 0.5, 2.0, 1.0),
                          penalty_w=0.3, area_target=0.2, centre_w=0.7, centre_target=(1.2, 3.9))


@pytest.fixture(scope="module", autouse=True)
def _needs_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2411_19109_gb300 import load
    load()


@pytest.mark.parametrize("precision,tol_m,tol_g", [("fp64", 1e-10, 1e-9), ("fp32", 1e-5, 1e-4)])
@pytest.mark.parametrize("shape", [(12, 8, 1), (8, 64, 1), (8, 6, 2), (20, 3, 1)])
def test_curve_forward_adjoint_parity(shape, precision, tol_m, tol_g):
    inst = curve_case(*shape)
    g = gpu_run([inst], precision, want_dm0=True)
    o = oracle_run(inst)
    assert rel_l2(g["mT"][0], o["mT"]) < tol_m
    assert abs(g["J"][0] - o["J"]) <= tol_g * abs(o["J"])
    assert rel_l2(g["dphi"][0], o["dphi"]) < tol_g
    assert rel_l2(g["dm0"][0], o["dm0"]) < tol_g


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_sw_particle_reduced_steps(precision, tol):
    """The hysteresis workload (32 x 30 mesh, 3 levels held 20 steps each,
    regularised) against the oracle; the gradient is compared on the
    design mask, where the level-set step uses it."""
    inst = W.sw_particle(levels=3, hold=20, regularised=True)
    g = gpu_run([inst], precision, want_dm0=True)
    o = oracle_run(inst)
    mask = inst.mask.astype(bool)
    assert abs(g["J"][0] - o["J"]) <= tol * abs(o["J"])
    assert rel_l2(g["dphi"][0][mask], o["dphi"][mask]) < tol
    assert rel_l2(g["dm0"][0], o["dm0"]) < tol


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_of_curve_and_port_instances_matches_single_runs(precision):
    insts = [curve_case(12, 8, seed=32, N=30),
             W.random_small(16, 12, 1, seed=33, nsteps=30, objective=W.J_PORT, n_from=1),
             curve_case(8, 6, 2, seed=34, N=30)]
    both = gpu_run(insts, precision)
    for k, inst in enumerate(insts):
        one = gpu_run([inst], precision)
        assert both["J"][k] == one["J"][0]
        np.testing.assert_array_equal(both["dphi"][k], one["dphi"][0])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_curve_schedules_give_identical_gradients(precision):
    inst = curve_case(12, 8, seed=35, N=40)
    ref = gpu_run([inst], precision, ckpt="store_all")
    for ckpt, seg in (("periodic", 1), ("periodic", 7), ("binomial", 2), ("binomial", 5)):
        g = gpu_run([inst], precision, ckpt=ckpt, seg_len=seg, want_dm0=True)
        np.testing.assert_array_equal(g["dphi"][0], ref["dphi"][0])
        assert g["J"][0] == ref["J"][0]


def test_invalid_curve_problems_are_rejected():
    from paper_2411_19109_gb300 import LLGError
    base = curve_case(12, 8, N=40)
    bad = [dict(sample_steps=(), sample_targets=(), sample_weights=()),
           dict(sample_steps=(20, 10, 30, 40)),                       # not increasing
           dict(sample_steps=(0, 20, 30, 40)),                        # step 0
           dict(sample_steps=(10, 20, 30, 41)),                       # beyond nsteps
           dict(sample_targets=(1.0, float("nan"), 1.0, 1.0)),
           dict(comp=3),
           dict(drive=(0.0,) * 3 * 40 + (float("inf"),) * 3)]
    for over in bad:
        with pytest.raises(LLGError):
            gpu_solver([type("I", (), {"problem": base.problem.replace(**over)})()])
