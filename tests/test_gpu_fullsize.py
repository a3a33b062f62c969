"""Parity at the workloads' full grid sizes over a number of steps the FP64
oracle can follow in seconds to a minute: one instance of each of the four
batch64 shapes, in the launch configurations the benchmark times (the FP32
checkpointed path with CUDA graphs over all 64 instances and the double-float
adjoint spectrum, and the plain FP64 store-all path), the nanoparticle
(64 x 64), the single demultiplexer (256 x 64), and two demultiplexer shapes
over 1000 steps.  m is compared as psi m (the magnetisation; m at air nodes
carries none), J against the sum of the magnitudes of its terms (the port
objective is a difference of two ports), dJ/dPhi over the whole grid and over
the design mask (the nodes the level-set step updates).

Why the demultiplexer's FP32 gradient needs the double-float spectrum: the
adjoint field starts at the output ports, and the design region sees only its
tail, partly through the demag far field.  An FP32 FFT perturbs every node by
about 1e-7 of the whole field's norm, which is the size of that tail, so the
plain FP32 gradient is 1e-3 off after 100 steps (2e-2 after 20) while m and
J hold 1e-5 and 1e-4.  Rounding the oracle's own adjoint demag FFT to complex64
reproduces it; rounding its forward FFT, or every stored state, field and
slope, gives below 1e-6 (tests/test_oracle_precision.py).  With the adjoint's
frequency domain in double-float (about 48 bits) the gradient meets 1e-4."""
import numpy as np
import pytest

import workloads as W
from tests.gpu_util import gpu_run, rel_l2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _needs_gpu():
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    from paper_2411_19109_gb300 import load
    load()


def _oracle(inst, f32_inputs=False):
    """The oracle on the instance's inputs, or on those inputs rounded to
    FP32 -- the values an FP32 context receives."""
    from oracle import llg
    p = inst.problem
    phi, m0 = inst.phi, inst.m0
    if f32_inputs:
        phi = phi.astype(np.float32).astype(np.float64)
        m0 = m0.astype(np.float32).astype(np.float64)
    mod = llg.Model(p, phi)
    J, mN, traj = mod.forward(m0, keep=True)
    dphi, dm0, _ = mod.adjoint(m0, traj)
    if p.objective == W.J_PORT:
        scale = 0.0
        for n in range(max(p.n_from, 0), p.nsteps + 1):
            for b, box in enumerate(p.boxes):
                bm = mod._box_mask(box)
                if bm.any():
                    v = traj[n][p.comp][bm]
                    scale += abs(p.weights[b]) * float(np.mean(v * v if p.power == 2 else np.abs(v)))
    else:
        scale = abs(J)
    return dict(J=J, mT=mN, dphi=dphi, psi=mod.psi, scale=scale, mask=inst.mask.astype(bool))


def _check(g, k, o, tol_m, tol_J, tol_g, tag=""):
    psi = o["psi"]
    em = rel_l2(psi * g["mT"][k].reshape(o["mT"].shape), psi * o["mT"])
    ej = abs(g["J"][k] - o["J"]) / o["scale"]
    eg = rel_l2(g["dphi"][k], o["dphi"])
    mk = o["mask"]
    egm = rel_l2(g["dphi"][k].reshape(mk.shape)[mk], o["dphi"][mk])
    print(f"{tag}: psi m {em:.2e}, J {ej:.2e}, dJ/dPhi {eg:.2e} (design mask {egm:.2e})")
    assert em < tol_m
    assert ej <= tol_J
    assert eg < tol_g
    assert egm < tol_g


def test_batch64_full_sizes_in_both_benchmark_configurations():
    insts = W.batch64(nsteps=100)
    g32 = gpu_run(insts, "fp32", ckpt="periodic", use_graph=True, adj_spectral="dfloat")
    g64 = gpu_run(insts, "fp64", ckpt="store_all", use_graph=True)
    for k in (0, 16, 32, 48):                   # 128x64, 256x64, 256x128, 512x128
        o = _oracle(insts[k])
        _check(g64, k, o, 1e-10, 1e-9, 1e-9, f"fp64 {insts[k].tag}")
        _check(g32, k, o, 1e-5, 1e-4, 1e-4, f"fp32 + double-float adjoint {insts[k].tag}")


def test_nanoparticle_full_size():
    inst = W.particle64(nsteps=200)
    o = _oracle(inst)
    _check(gpu_run([inst], "fp32", ckpt="periodic", use_graph=True), 0, o, 1e-5, 1e-4, 1e-4, "fp32")
    _check(gpu_run([inst], "fp32", ckpt="periodic", use_graph=True, adj_spectral="dfloat"), 0, o, 1e-5, 1e-4, 1e-4,
           "fp32 + double-float adjoint")
    _check(gpu_run([inst], "fp64", ckpt="store_all", use_graph=True), 0, o, 1e-10, 1e-9, 1e-9, "fp64")


def test_demultiplexer_full_size():
    inst = W.demux256(0, nsteps=100)
    o = _oracle(inst)
    _check(gpu_run([inst], "fp32", ckpt="periodic", use_graph=True, adj_spectral="dfloat"), 0, o, 1e-5, 1e-4, 1e-4,
           "fp32 + double-float adjoint")
    _check(gpu_run([inst], "fp64", ckpt="store_all", use_graph=True), 0, o, 1e-10, 1e-9, 1e-9, "fp64")


def test_plain_fp32_adjoint_spectrum_error_on_the_demultiplexer():
    """The documented FP32-spectrum rounding of the adjoint (see above): m and
    J meet their bars, the gradient is held only to 3e-3."""
    inst = W.demux256(0, nsteps=100)
    o = _oracle(inst)
    _check(gpu_run([inst], "fp32", ckpt="periodic", use_graph=True), 0, o, 1e-5, 1e-4, 3e-3, "fp32")


# 128x64 and 256x64 shapes of batch64 over 1000 steps, against the oracle
# on the same FP32-rounded inputs.  On the 256x64 shape the exact gradient at
# this horizon is ill-conditioned (the motion of m at air nodes is chaotic):
# in the oracle, rounding the stage inputs, fields and slopes at which the
# adjoint is linearised to FP32 moves dJ/dPhi by 1.9e-4 even with m carried
# exactly (2.0e-4 with m rounded too), and a 1e-7 perturbation of m0 moves it
# by 2.4e-4.  Any FP32-state evaluation lands at a few 1e-4 depending on its
# rounding pattern (the GPU: 3.9e-4), so that case is held to 1e-3; the
# 128x64 shape (1.1e-5) and every 100-step case (<= 2.7e-6) meet 1e-4.
@pytest.mark.parametrize("k,tol_g", [(0, 1e-4), (2, 1e-3)])
def test_demultiplexer_shapes_1000_steps(k, tol_g):
    inst = W.batch64(nsteps=1000, candidates=1)[k]
    assert (inst.problem.nx, inst.problem.ny) == ((128, 64) if k == 0 else (256, 64))
    o = _oracle(inst, f32_inputs=True)
    _check(gpu_run([inst], "fp32", ckpt="periodic", use_graph=True, adj_spectral="dfloat"), 0, o, 1e-5, 1e-4, tol_g,
           f"fp32 + double-float adjoint, 1000 steps, {inst.tag}")
