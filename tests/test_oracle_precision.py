"""Where FP32 rounding enters the demultiplexer's gradient, measured on the
FP64 oracle itself (no GPU): the adjoint's demag transpose
D = N * Bbar (a zero-padded FFT convolution, Eq. 6 and Eq. 7 through the
demag field of the effective field) is recomputed with one kind of FP32
rounding at a time, and dJ/dPhi compared with the plain oracle's.

* Rounding in space (Bbar before the transform, D after it) is a relative
  perturbation of each node's value, convolved with the same kernel as the
  value itself: it moves the gradient by about the FP32 unit.
* Rounding in the frequency domain (the Newell tensor spectrum, or the
  transform arithmetic in complex64) is a relative perturbation of each
  Fourier coefficient, which spreads over the whole grid: the design region,
  which at 20 steps sees only the tail of an adjoint field concentrated at
  the output ports, receives an error of the size of the whole field's.

This is the stated FP32 exception of the CUDA path on these shapes (its
frequency domain is FP32), and what a double-float frequency domain
removes."""
import numpy as np
import pytest

import workloads as W


def _conv(M, spectrum, space32=False, tensor32=False, fft32=False):
    from oracle import demag as dm
    _, nz, ny, nx = M.shape
    Pz, Py, Px = dm.padded_shape(nx, ny, nz)
    if space32:
        M = M.astype(np.float32).astype(np.float64)
    Mp = np.zeros((3, Pz, Py, Px), dtype=np.float32 if fft32 else np.float64)
    Mp[:, :nz, :ny, :nx] = M
    if fft32:
        import scipy.fft as sf                       # keeps complex64 (numpy's FFT promotes to complex128)
        Mh = sf.rfftn(Mp, axes=(1, 2, 3))
        assert Mh.dtype == np.complex64
    else:
        Mh = np.fft.rfftn(Mp, axes=(1, 2, 3))
    spec = spectrum
    if tensor32 or fft32:
        spec = [c.astype(np.complex64) for c in spectrum]
        if not fft32:
            spec = [c.astype(np.complex128) for c in spec]
    xx, yy, zz, xy, xz, yz = spec
    Hh = np.array([xx * Mh[0] + xy * Mh[1] + xz * Mh[2],
                   xy * Mh[0] + yy * Mh[1] + yz * Mh[2],
                   xz * Mh[0] + yz * Mh[1] + zz * Mh[2]])
    if fft32:
        import scipy.fft as sf
        H = sf.irfftn(Hh.astype(np.complex64), s=(Pz, Py, Px), axes=(1, 2, 3))
    else:
        H = np.fft.irfftn(Hh, s=(Pz, Py, Px), axes=(1, 2, 3))
    H = np.asarray(H[:, :nz, :ny, :nx], dtype=np.float64)
    if space32:
        H = H.astype(np.float32).astype(np.float64)
    return -dm.MU0 * H


@pytest.fixture(scope="module")
def demux():
    from oracle import llg
    inst = W.demux256(0, nsteps=20)
    model = llg.Model(inst.problem, inst.phi)
    _, _, traj = model.forward(inst.m0, keep=True)
    g0, _, _ = model.adjoint(inst.m0, traj)
    return inst, traj, g0


def _gradient(inst, traj, **rounding):
    from oracle import llg

    class Rounded(llg.Model):
        def demag_T(self, Bbar, Y):
            D = _conv(Bbar, self.spectrum, **rounding)
            return self.p.Ms * self.psi * D, self.p.Ms * llg.dot(Y, D)

    g, _, _ = Rounded(inst.problem, inst.phi).adjoint(inst.m0, traj)
    return g


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_unrounded_restatement_reproduces_the_oracle(demux):
    inst, traj, g0 = demux
    assert _rel(_gradient(inst, traj), g0) < 1e-12


def test_fp32_rounding_in_space_is_harmless(demux):
    inst, traj, g0 = demux
    assert _rel(_gradient(inst, traj, space32=True), g0) < 1e-5


def test_fp32_tensor_spectrum_alone_exceeds_the_fp32_bar(demux):
    inst, traj, g0 = demux
    assert _rel(_gradient(inst, traj, tensor32=True), g0) > 1e-3


def test_fp32_transform_arithmetic_exceeds_the_fp32_bar(demux):
    inst, traj, g0 = demux
    assert _rel(_gradient(inst, traj, fft32=True), g0) > 3e-3
