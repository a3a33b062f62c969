"""Spectral port objective (Eq. 10 at the window's frequencies) through the C
ABI against the FP64 oracle: J, m_N, dJ/dPhi and dJ/dm0 on films of both
column-kernel families and on a 3D grid, in a batch with port-objective
instances, under every checkpoint schedule, and the argument checks."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_run, gpu_solver, oracle_run, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SPEC = dict(objective=W.J_SPECTRAL, freqs=(8e9, 9.5e9, 12e9), n_from=10)


@pytest.fixture(scope="module", autouse=True)
def _needs_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2411_19109_gb300 import load
    load()


@pytest.mark.parametrize("precision,tol_m,tol_g", [("fp64", 1e-10, 1e-9), ("fp32", 1e-5, 1e-4)])
@pytest.mark.parametrize("shape", [(12, 8, 1), (8, 64, 1), (8, 6, 2), (20, 3, 1)])
def test_spectral_forward_adjoint_parity(shape, precision, tol_m, tol_g):
    inst = W.random_small(*shape, seed=13, nsteps=40, **SPEC)
    g = gpu_run([inst], precision, want_dm0=True)
    o = oracle_run(inst)
    assert rel_l2(g["mT"][0], o["mT"]) < tol_m
    assert abs(g["J"][0] - o["J"]) <= tol_g * abs(o["J"])
    assert rel_l2(g["dphi"][0], o["dphi"]) < tol_g
    assert rel_l2(g["dm0"][0], o["dm0"]) < tol_g


def test_one_box_one_frequency_and_window_at_the_last_step():
    # w_1 = 0 (second box unused) and a window holding only step N
    for over in (dict(weights=(1.0, 0.0), freqs=(9e9,)), dict(n_from=30, freqs=(9e9,))):
        inst = W.random_small(12, 8, 1, seed=14, nsteps=30, **{**SPEC, **over})
        g = gpu_run([inst], "fp64", want_dm0=True)
        o = oracle_run(inst)
        assert abs(g["J"][0] - o["J"]) <= 1e-9 * abs(o["J"])
        assert rel_l2(g["dphi"][0], o["dphi"]) < 1e-9
        assert rel_l2(g["dm0"][0], o["dm0"]) < 1e-9


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_batch_of_spectral_and_port_instances_matches_single_runs(precision):
    insts = [W.random_small(12, 8, 1, seed=15, nsteps=25, **SPEC),
             W.random_small(16, 12, 1, seed=16, nsteps=25, objective=W.J_PORT, n_from=10),
             W.random_small(8, 6, 2, seed=17, nsteps=25, **{**SPEC, "freqs": (5e9,)})]
    both = gpu_run(insts, precision)
    for k, inst in enumerate(insts):
        one = gpu_run([inst], precision)
        assert both["J"][k] == one["J"][0]
        np.testing.assert_array_equal(both["dphi"][k], one["dphi"][0])


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_spectral_schedules_give_identical_gradients(precision):
    inst = W.random_small(12, 8, 1, seed=18, nsteps=23, **SPEC)
    ref = gpu_run([inst], precision, ckpt="store_all")
    for ckpt, seg in (("periodic", 1), ("periodic", 5), ("binomial", 2), ("binomial", 4)):
        g = gpu_run([inst], precision, ckpt=ckpt, seg_len=seg, want_dm0=True)
        np.testing.assert_array_equal(g["dphi"][0], ref["dphi"][0])
        assert g["J"][0] == ref["J"][0]


def test_invalid_spectral_problems_are_rejected():
    from paper_2411_19109_gb300 import LLGError
    for over in (dict(freqs=()), dict(freqs=tuple(1e9 * (k + 1) for k in range(9))), dict(n_from=0),
                 dict(comp=3), dict(freqs=(float("nan"),))):
        bad = W.random_small(12, 8, 1, seed=19, nsteps=5, **{**SPEC, **over})
        with pytest.raises(LLGError):
            gpu_solver([bad])
