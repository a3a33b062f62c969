"""Parity at the workloads' full grid sizes over a number of steps the FP64
oracle can follow in seconds: one instance of each of the four batch64
shapes, in the launch configurations the benchmark times (the FP32
checkpointed path with CUDA graphs over all 64 instances, and the plain FP64
store-all path), and the nanoparticle (64 x 64) and single demultiplexer
(256 x 64) workloads.  m is compared as psi m (the magnetisation; m at air
nodes carries none), J against the sum of the magnitudes of its terms (the
port objective is a difference of two ports).

FP32 and the demultiplexer's gradient: it is 1e-3 off the oracle after 100
steps (2e-2 after 20), while m and J hold 1e-5 and 1e-4 and the same kernels
in FP64 hold 1e-9.  The source is the FP32 FFT of the adjoint's demag
transpose: the adjoint field starts at the output ports and the design region
sees only its tail, which FFT rounding (relative to the whole field's norm)
cannot resolve.  Rounding the oracle's own adjoint demag FFT to FP32 (complex64)
reproduces it (1e-2 after 20 steps, 5e-4 after 100), while FP32 rounding of
the forward FFT or of every stored state, field and slope gives below 1e-6.
Every rounding in the frequency domain contributes (the Newell tensor
spectrum stored in FP32 alone gives 2e-3 after 20 steps, the row spectrum
stored in FP32 5e-4), rounding in space does not.  On the largest batch64
shape (512 x 128) the emulated error stays near 1e-3 up to 1000 steps.
The nanoparticle and the random test grids, whose adjoint fields cover the
grid, hold 1e-4 on the gradient in FP32."""
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


def _oracle(inst):
    from oracle import llg
    p = inst.problem
    mod = llg.Model(p, inst.phi)
    J, mN, traj = mod.forward(inst.m0, keep=True)
    dphi, dm0, _ = mod.adjoint(inst.m0, traj)
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
    return dict(J=J, mT=mN, dphi=dphi, psi=mod.psi, scale=scale)


def _check(g, k, o, tol_m, tol_J, tol_g):
    psi = o["psi"]
    assert rel_l2(psi * g["mT"][k].reshape(o["mT"].shape), psi * o["mT"]) < tol_m
    assert abs(g["J"][k] - o["J"]) <= tol_J * o["scale"]
    if tol_g is not None:
        assert rel_l2(g["dphi"][k], o["dphi"]) < tol_g


def test_batch64_full_sizes_in_both_benchmark_configurations():
    insts = W.batch64(nsteps=20)
    g32 = gpu_run(insts, "fp32", ckpt="periodic", use_graph=True)
    g64 = gpu_run(insts, "fp64", ckpt="store_all", use_graph=True)
    for k in (0, 16, 32, 48):                   # 128x64, 256x64, 256x128, 512x128
        o = _oracle(insts[k])
        _check(g64, k, o, 1e-10, 1e-9, 1e-9)
        _check(g32, k, o, 1e-5, 1e-4, None)     # gradient: FP32 rounding-bound here (see above)


def test_nanoparticle_full_size():
    inst = W.particle64(nsteps=200)
    o = _oracle(inst)
    _check(gpu_run([inst], "fp32", ckpt="periodic", use_graph=True), 0, o, 1e-5, 1e-4, 1e-4)
    _check(gpu_run([inst], "fp64", ckpt="store_all", use_graph=True), 0, o, 1e-10, 1e-9, 1e-9)


def test_demultiplexer_full_size():
    inst = W.demux256(0, nsteps=100)
    o = _oracle(inst)
    _check(gpu_run([inst], "fp32", ckpt="periodic", use_graph=True), 0, o, 1e-5, 1e-4, 3e-3)
    _check(gpu_run([inst], "fp64", ckpt="store_all", use_graph=True), 0, o, 1e-10, 1e-9, 1e-9)
