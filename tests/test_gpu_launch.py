"""Launch configurations and the adjoint's per-instance cotangents, through
the C ABI.

* Every launch-configuration candidate (llg_launch: register-cap variants of
  the double-float column and adjoint kernels, the fused or split
  double-float adjoint stage, one or two instance-group chains) gives
  bit-identical J and gradients to the default; the FP32
  column pass with 8- instead of 16-element FFT lanes (a different radix
  order) meets the oracle bars.  The configuration the timing search picks
  (LLG_TUNE_MEASURE) meets them too, and a second context of the same batch
  takes it from the process cache without timing.
* dJ_dextra (the cotangent of each instance's J under a combination made
  outside the library): the gradients of sum_i w_i J_i, checked against the
  oracle for two frequency runs of one candidate that share Phi (Eq. 10 as
  the sum of the two runs' objectives), and through the autograd wrapper.
"""
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


def _batch():
    # two uneven film shapes with 128- and 256-point columns (the 16-element
    # lane lengths), two instances each
    return [W.random_small(12, 64, 1, seed=41, nsteps=12), W.random_small(32, 100, 1, seed=42, nsteps=12),
            W.random_small(16, 64, 1, seed=43, nsteps=12, objective=W.J_ENERGY_AREA),
            W.random_small(8, 100, 1, seed=44, nsteps=12)]


DEFAULT = {"col_lanes": 16, "col_blocks": 2, "adj_blocks": 2, "groups": 2, "adj_split": 1}


@pytest.mark.parametrize("precision,spec", [("fp32", "dfloat"), ("fp32", "working"), ("fp64", "working")])
def test_launch_candidates_are_bit_identical(precision, spec):
    insts = _batch()
    ref = gpu_run(insts, precision, adj_spectral=spec, tune="given", launch=DEFAULT, want_dm0=True)
    for alt in ({"col_blocks": 1}, {"adj_blocks": 3}, {"adj_split": 0}, {"adj_split": 0, "adj_blocks": 1},
                {"groups": 1}):
        cfg = dict(DEFAULT, **alt)
        g = gpu_run(insts, precision, adj_spectral=spec, tune="given", launch=cfg, want_dm0=True)
        np.testing.assert_array_equal(g["J"], ref["J"])
        for k in range(len(insts)):
            np.testing.assert_array_equal(g["dphi"][k], ref["dphi"][k])
            np.testing.assert_array_equal(g["dm0"][k], ref["dm0"][k])


@pytest.mark.parametrize("lanes", [8, 16])
def test_column_lane_widths_meet_the_oracle(lanes):
    insts = _batch()
    g = gpu_run(insts, "fp32", adj_spectral="dfloat", tune="given", launch=dict(DEFAULT, col_lanes=lanes))
    for k, inst in enumerate(insts):
        o = oracle_run(inst)
        assert rel_l2(g["mT"][k], o["mT"]) < 1e-5
        assert rel_l2(g["dphi"][k], o["dphi"]) < 1e-4


def test_measured_configuration_meets_the_oracle_and_is_cached():
    insts = _batch()
    s = gpu_solver(insts, "fp32", adj_spectral="dfloat", tune="measure")
    try:
        cfg, ms = s.launch_config()
        assert cfg["col_lanes"] in (8, 16) and cfg["col_blocks"] in (1, 2)
        assert cfg["adj_blocks"] in (1, 2, 3) and cfg["groups"] in (1, 2) and cfg["adj_split"] in (0, 1)
    finally:
        s.close()
    s2 = gpu_solver(insts, "fp32", adj_spectral="dfloat", tune="measure")
    try:
        cfg2, ms2 = s2.launch_config()
        assert cfg2 == cfg and ms2 == 0.0          # from the process cache
    finally:
        s2.close()
    g = gpu_run(insts, "fp32", adj_spectral="dfloat", tune="measure")
    for k, inst in enumerate(insts):
        o = oracle_run(inst)
        assert rel_l2(g["dphi"][k], o["dphi"]) < 1e-4


def test_default_configuration_is_reported():
    s = gpu_solver(_batch()[:1], "fp64")
    try:
        cfg, ms = s.launch_config()
        assert cfg == DEFAULT and ms == 0.0
    finally:
        s.close()


def test_invalid_launch_configuration_is_rejected():
    from paper_2411_19109_gb300 import LLGError
    with pytest.raises(LLGError, match="launch"):
        gpu_solver(_batch()[:1], "fp32", tune="given", launch=dict(DEFAULT, col_lanes=4))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 1e-4)])
def test_cotangents_combine_two_frequency_runs(precision, tol):
    """Eq. 10 across the two drive frequencies of one candidate: J = J_f1 +
    J_f2 with both runs sharing Phi and m0; dJ/dPhi is the sum of the
    instances' gradients of w_1 J_1 + w_2 J_2 at w = (1, 1); other weights
    scale each run.  A non-finite cotangent is rejected."""
    a = W.demux(64, 32, 3.0e9, 1.0, config=4, instance=0, nsteps=30)
    b = W.demux(64, 32, 3.4e9, -1.0, config=4, instance=0, nsteps=30)
    b.phi, b.m0, b.mask = a.phi, a.m0, a.mask
    oa, ob = oracle_run(a), oracle_run(b)
    s = gpu_solver([a, b], precision, adj_spectral="dfloat" if precision == "fp32" else "working")
    try:
        phi = s.pack_scalar([a.phi, b.phi])
        m0 = s.pack_vector([a.m0, b.m0])
        for w in ((1.0, 1.0), (0.5, -2.0)):
            s.forward(phi, m0)
            g, dm0 = s.adjoint(want_dm0=True, dJ_dextra=list(w))
            ga, gb = [x.double().cpu().numpy() for x in s.unpack_scalar(g)]
            ma, mb = [x.double().cpu().numpy() for x in s.unpack_vector(dm0)]
            # the two runs nearly cancel at this horizon (J_b ~ -J_a), so the
            # sum is compared normwise: against the sum of the terms' norms
            ref = w[0] * oa["dphi"] + w[1] * ob["dphi"]
            scale = np.linalg.norm(w[0] * oa["dphi"]) + np.linalg.norm(w[1] * ob["dphi"])
            assert np.linalg.norm(ga + gb - ref) < tol * scale
            assert rel_l2(ga, w[0] * oa["dphi"]) < tol and rel_l2(gb, w[1] * ob["dphi"]) < tol
            assert rel_l2(ma, w[0] * oa["dm0"]) < tol and rel_l2(mb, w[1] * ob["dm0"]) < tol
        with pytest.raises(Exception):
            s.forward(phi, m0)
            s.adjoint(dJ_dextra=[1.0, float("nan")])
    finally:
        s.close()


def test_autograd_combined_objective():
    """torch autograd over a combination of the instances' J: the backward
    seeds the adjoint with each instance's cotangent (dJ_dextra)."""
    from paper_2411_19109_gb300 import llg_function
    insts = [W.random_small(12, 8, 1, seed=6, nsteps=20), W.random_small(8, 4, 1, seed=7, nsteps=20)]
    s = gpu_solver(insts, "fp64")
    try:
        phi = s.pack_scalar([i.phi for i in insts]).requires_grad_(True)
        m0 = s.pack_vector([i.m0 for i in insts]).requires_grad_(True)
        J = llg_function().apply(phi, m0, s)
        (3.0 * J[0] - 0.25 * J[1] ** 2).backward()
        o = [oracle_run(i) for i in insts]
        w = [3.0, -0.5 * o[1]["J"]]
        gp = s.unpack_scalar(phi.grad)
        gm = s.unpack_vector(m0.grad)
        for k in range(2):
            assert rel_l2(gp[k].cpu().numpy(), w[k] * o[k]["dphi"]) < 1e-9
            assert rel_l2(gm[k].cpu().numpy(), w[k] * o[k]["dm0"]) < 1e-9
    finally:
        s.close()
