"""Seeded synthetic workloads for the level-set / adjoint LLG solver.

This module is shared by the CUDA path and by the FP64 oracle.  It holds
problem descriptions (grid, material constants, drive, geometry, objective
selection) and seeded generators for the level-set function Phi, the initial
magnetisation m0 and the design mask.  It holds none of the method's
arithmetic: no field, no integrator, no objective evaluation, no gradient.

Workloads (the paper uses no dataset; every input here is synthetic):
  film32      32x32x1 Permalloy film, 5 nm cells, 50 mT bias along x,
              J = time-integrated mean m_y over a 4x4 patch, 1000 steps.
  particle64  64x64x1 nanoparticle at 2 nm, alpha=0.5 relaxation, no field,
              J = (demag + exchange energy) + area penalty at 30 %, 5000 steps.
  demux256    256x64x1 YIG demultiplexer at 5 nm, absorbing x-ends, 100 mT
              bias, 1 mT RF line source at 3.0 / 3.4 GHz, J = port contrast of
              time-averaged m_y^2, 20000 steps.
  batch64     8 candidates x 4 shapes (128x64, 256x64, 256x128, 512x128) x
              2 drive frequencies of the demux geometry, 10000 steps each.
  thick512    512x512x4 YIG film, full 3D demag, 50000 steps.

Geometry of the material follows the level-set convention of Eq. 1 with
Phi > 0 = magnetic (psi -> 1) and Phi < 0 = air.
"""
from __future__ import annotations

import dataclasses
from dataclasses import dataclass
from typing import List, Optional, Tuple

import numpy as np

# objective kinds (mirrors include/llg.h)
J_PORT = 0      # sum_{n>=n_from} sum_b w_b mean_{box b}(m_c,n ^ p)
J_ENERGY_AREA = 1  # (E_demag + E_exchange)(m_N)/(K_d V_dom) + xi (mean psi - s_t)^2
J_SPECTRAL = 2   # sum_b w_b sum_q |DFT of the port-mean series at f_q| (Eq. 10, windowed)
J_CURVE = 3      # sum_j w_j |P(m_{n_j}) - T_j| + size and centre penalties (Eq. 8, Eq. 9)

Box = Tuple[int, int, int, int]  # x0, x1, y0, y1 (half open, node indices)


@dataclass
class Problem:
    """One LLG instance: grid, material, drive, time stepping, objective."""
    nx: int
    ny: int
    nz: int = 1
    dx: float = 5e-9
    dy: float = 5e-9
    dz: float = 5e-9
    Ms: float = 8e5           # A/m
    A: float = 1.3e-11        # J/m
    Ku: float = 0.0           # J/m^3, uniaxial
    ku: Tuple[float, float, float] = (0.0, 0.0, 1.0)
    alpha: float = 0.02
    alpha_edge: float = 0.5
    absorb_nodes: int = 0     # ramp width W in nodes (0 = no absorbing edges)
    absorb_x: int = 1         # ramp on the two x ends
    absorb_y: int = 0         # ramp on the two y ends
    B_bias: Tuple[float, float, float] = (0.0, 0.0, 0.0)   # T
    b_rf: float = 0.0         # T
    f_rf: float = 0.0         # Hz
    rf_dir: Tuple[float, float, float] = (0.0, 1.0, 0.0)
    src: Box = (0, 0, 0, 0)   # RF source box (all z layers)
    dt: float = 1e-13
    nsteps: int = 1000
    sigmoid_a: float = 50.0
    objective: int = J_PORT
    comp: int = 1             # sampled component of m (J_PORT)
    power: int = 1            # 1 or 2 (J_PORT)
    boxes: Tuple[Box, Box] = ((0, 0, 0, 0), (0, 0, 0, 0))
    weights: Tuple[float, float] = (0.0, 0.0)
    n_from: int = 1           # first step index n included in the running sum
    area_target: float = 0.3
    penalty_w: float = 1.0
    freqs: Tuple[float, ...] = ()   # J_SPECTRAL: frequencies of the windowed spectral sum (Hz)
    # applied drive b(t) on the source box along rf_dir, tabulated per step n
    # at t = n dt, n dt + dt/2, n dt + dt (3 nsteps + 3 values, tesla); None:
    # the sine b_rf sin(2 pi f_rf t)
    drive: Optional[Tuple[float, ...]] = None
    # J_CURVE: J = sum_j w_j |P(m_{n_j}) - T_j|, P = sum psi m_comp / sum psi
    sample_steps: Tuple[int, ...] = ()
    sample_targets: Tuple[float, ...] = ()
    sample_weights: Tuple[float, ...] = ()
    # J_CURVE penalties (Eq. 9): penalty_w (mean psi - area_target)^2 and
    # centre_w (|x_c - x_0| + |y_c - y_0|), the psi-weighted centre of the
    # (first) layer's nodes in node-index units
    centre_w: float = 0.0
    centre_target: Tuple[float, float] = (0.0, 0.0)

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)

    @property
    def nodes(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class Instance:
    """A problem plus its seeded inputs."""
    problem: Problem
    phi: np.ndarray            # [nz][ny][nx] float64
    m0: np.ndarray             # [3][nz][ny][nx] float64
    mask: np.ndarray           # [nz][ny][nx] uint8 design region
    tag: str = ""


# --------------------------------------------------------------------------
# seeded field generators (input synthesis only)
# --------------------------------------------------------------------------

def _rng(config: int, instance: int) -> np.random.Generator:
    return np.random.default_rng(1000 * config + instance)


def gaussian_bumps(rng, nx, ny, dx, dy, n, sigma, region: Box | None = None):
    """Sum of n Gaussians with centres uniform in `region` and amplitudes in
    [-1, 1], divided by its max |.|.  Returns [ny][nx]."""
    x0, x1, y0, y1 = region if region is not None else (0, nx, 0, ny)
    X, Y = np.meshgrid(np.arange(nx) * dx, np.arange(ny) * dy)
    out = np.zeros((ny, nx))
    for _ in range(n):
        cx = rng.uniform(x0 * dx, (x1 - 1) * dx)
        cy = rng.uniform(y0 * dy, (y1 - 1) * dy)
        amp = rng.uniform(-1.0, 1.0)
        out += amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * sigma * sigma))
    mx = np.abs(out).max()
    return out / mx if mx > 0 else out


def noisy_uniform_m0(rng, nx, ny, nz, direction=(1.0, 0.0, 0.0), noise=1e-3):
    m = np.zeros((3, nz, ny, nx))
    for c in range(3):
        m[c] = direction[c]
    m += noise * rng.standard_normal(m.shape)
    m /= np.sqrt((m * m).sum(axis=0, keepdims=True))
    return m


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def film32(instance: int = 0, nsteps: int = 1000) -> Instance:
    """Plain-method film: 32x32x1, 5 nm, Permalloy, 50 mT along x."""
    rng = _rng(1, instance)
    nx = ny = 32
    p = Problem(nx=nx, ny=ny, nz=1, dx=5e-9, dy=5e-9, dz=5e-9,
                Ms=8e5, A=1.3e-11, alpha=0.02, B_bias=(0.05, 0.0, 0.0),
                dt=1e-13, nsteps=nsteps, objective=J_PORT, comp=1, power=1,
                boxes=((24, 28, 14, 18), (0, 0, 0, 0)), weights=(1e-13, 0.0),
                n_from=1)
    phi = gaussian_bumps(rng, nx, ny, p.dx, p.dy, 8, 20e-9)[None]
    m0 = noisy_uniform_m0(rng, nx, ny, 1)
    mask = np.ones((1, ny, nx), np.uint8)
    return Instance(p, phi, m0, mask, "film32")


def particle64(instance: int = 0, nsteps: int = 5000) -> Instance:
    """Nanoparticle shape problem: 64x64x1 at 2 nm, disc of 40 nm radius."""
    rng = _rng(2, instance)
    nx = ny = 64
    h = 2e-9
    p = Problem(nx=nx, ny=ny, nz=1, dx=h, dy=h, dz=h, Ms=8e5, A=1.3e-11,
                alpha=0.5, dt=5e-14, nsteps=nsteps, objective=J_ENERGY_AREA,
                area_target=0.3, penalty_w=1.0)
    X, Y = np.meshgrid((np.arange(nx) - (nx - 1) / 2) * h, (np.arange(ny) - (ny - 1) / 2) * h)
    r = np.sqrt(X * X + Y * Y)
    phi = (40e-9 - r) / 40e-9 + 0.05 * rng.standard_normal((ny, nx))
    phi /= np.abs(phi).max()
    m0 = noisy_uniform_m0(rng, nx, ny, 1)
    mask = np.ones((1, ny, nx), np.uint8)
    return Instance(p, phi[None], m0, mask, "particle64")


def demux_geometry(nx: int, ny: int):
    """Guides, design region, source line and ports of the demultiplexer,
    laid out on a 256x64 reference grid and scaled to nx x ny."""
    sx, sy = nx / 256.0, ny / 64.0
    X = lambda v: int(round(v * sx))
    Y = lambda v: int(round(v * sy))
    return dict(
        guide_in=(0, X(98), Y(22), Y(42)),
        design=(X(98), X(158), Y(2), Y(62)),
        out_bottom=(X(158), nx, Y(4), Y(24)),
        out_top=(X(158), nx, Y(40), Y(60)),
        src=(X(30), X(30) + 1, Y(22), Y(42)),
        port_top=(X(220), X(224), Y(40), Y(60)),
        port_bottom=(X(220), X(224), Y(4), Y(24)),
    )


def _fill(a, box, v):
    x0, x1, y0, y1 = box
    a[y0:y1, x0:x1] = v


def demux(nx: int = 256, ny: int = 64, f_rf: float = 3.0e9, sign: float = 1.0,
          config: int = 3, instance: int = 0, nsteps: int = 20000) -> Instance:
    """YIG demultiplexer instance.  `sign`=+1 gives the f1 term of the port
    contrast (top - bottom), -1 the f2 term (bottom - top)."""
    rng = _rng(config, instance)
    g = demux_geometry(nx, ny)
    n_from = nsteps // 2 + 1
    n_avg = nsteps - nsteps // 2
    p = Problem(nx=nx, ny=ny, nz=1, dx=5e-9, dy=5e-9, dz=5e-9,
                Ms=1.4e5, A=3.5e-12, alpha=2e-4, alpha_edge=0.5, absorb_nodes=20,
                absorb_x=1, absorb_y=0, B_bias=(0.1, 0.0, 0.0), b_rf=1e-3,
                f_rf=f_rf, rf_dir=(0.0, 1.0, 0.0), src=g["src"], dt=1e-13,
                nsteps=nsteps, objective=J_PORT, comp=1, power=2,
                boxes=(g["port_top"], g["port_bottom"]),
                weights=(sign / n_avg, -sign / n_avg), n_from=n_from)
    phi = -np.ones((ny, nx))
    for k in ("guide_in", "out_bottom", "out_top"):
        _fill(phi, g[k], 1.0)
    dx0, dx1, dy0, dy1 = g["design"]
    bumps = gaussian_bumps(rng, dx1 - dx0, dy1 - dy0, p.dx, p.dy, 16, 40e-9 * min(1.0, nx / 256.0))
    phi[dy0:dy1, dx0:dx1] = bumps
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[0, dy0:dy1, dx0:dx1] = 1
    m0 = noisy_uniform_m0(rng, nx, ny, 1)
    return Instance(p, phi[None], m0, mask, f"demux{nx}x{ny}@{f_rf/1e9:.1f}GHz")


def demux256(freq_index: int = 0, instance: int = 0, nsteps: int = 20000) -> Instance:
    f = (3.0e9, 3.4e9)[freq_index]
    sign = (1.0, -1.0)[freq_index]
    inst = demux(256, 64, f, sign, config=3, instance=instance, nsteps=nsteps)
    # both frequency runs share the same seeded design
    if freq_index == 1:
        base = demux(256, 64, 3.0e9, 1.0, config=3, instance=instance, nsteps=nsteps)
        inst.phi, inst.m0, inst.mask = base.phi, base.m0, base.mask
    return inst


BATCH_SHAPES = ((128, 64), (256, 64), (256, 128), (512, 128))


def batch64(nsteps: int = 10000, candidates: int = 8) -> List[Instance]:
    """8 candidates x 4 shapes x 2 frequencies = 64 instances.  The two
    frequency runs of one candidate share Phi and m0."""
    out = []
    for s, (nx, ny) in enumerate(BATCH_SHAPES):
        for c in range(candidates):
            seed_inst = s * candidates + c
            a = demux(nx, ny, 3.0e9, 1.0, config=4, instance=seed_inst, nsteps=nsteps)
            b = demux(nx, ny, 3.4e9, -1.0, config=4, instance=seed_inst, nsteps=nsteps)
            b.phi, b.m0, b.mask = a.phi, a.m0, a.mask
            out += [a, b]
    return out


def thick512(nsteps: int = 50000, nx: int = 512, ny: int = 512, nz: int = 4) -> Instance:
    """Thick YIG film with full 3D demag; the whole film is the design."""
    rng = _rng(5, 0)
    n_from = nsteps // 2 + 1
    n_avg = nsteps - nsteps // 2
    sx = nx / 512.0
    src = (int(30 * sx), int(30 * sx) + 1, 0, ny)
    top = (int(440 * sx), int(444 * sx), ny // 2, ny)
    bot = (int(440 * sx), int(444 * sx), 0, ny // 2)
    p = Problem(nx=nx, ny=ny, nz=nz, dx=5e-9, dy=5e-9, dz=5e-9,
                Ms=1.4e5, A=3.5e-12, alpha=2e-4, alpha_edge=0.5, absorb_nodes=20,
                absorb_x=1, absorb_y=0, B_bias=(0.1, 0.0, 0.0), b_rf=1e-3,
                f_rf=3.0e9, rf_dir=(0.0, 1.0, 0.0), src=src, dt=1e-13,
                nsteps=nsteps, objective=J_PORT, comp=1, power=2,
                boxes=(top, bot), weights=(1.0 / n_avg, -1.0 / n_avg), n_from=n_from)
    plane = gaussian_bumps(rng, nx, ny, p.dx, p.dy, 64, 40e-9)
    phi = np.repeat(plane[None], nz, axis=0)
    m0 = noisy_uniform_m0(rng, nx, ny, nz)
    mask = np.ones((nz, ny, nx), np.uint8)
    return Instance(p, phi, m0, mask, "thick512")


def sw_particle(instance: int = 0, levels: int = 30, hold: int = 500, regularised: bool = False,
                nx: int = 32, ny: int = 30, design: int = 30) -> Instance:
    """Stoner-Wohlfarth hysteresis task (Eq. 8; Eq. 9 when `regularised`):
    a 30 x 30 x 1 Permalloy design region of 3 nm cells (the mesh is nx = 32
    wide, a multiple of 4 as the row FFTs need; columns x >= 30 are air,
    Phi = -1, outside the design mask) holding an initially circular particle
    (radius 10 cells), a uniform field along x raised in `levels`
    equal steps from 0 to 0.3 Ms (mu0 H), each level held `hold` RK4 steps
    (alpha 0.5, so the particle relaxes), and M_x/Ms = sum psi m_x / sum psi
    sampled at the end of levels j = 1..levels against the target 2 H_j/Ms
    with weights 1/(levels T_j) (zeta/(levels T_j), zeta = 10, with the size
    penalty xi = 0.05 toward a one-cell-wide wire across the design region
    and the centre penalty nu = 1 toward the design region's centre when
    `regularised`).  m0 = +y with 1e-3 seeded noise."""
    rng = _rng(6, instance)
    h = 3e-9
    Ms = 8e5
    N = (levels + 1) * hold
    b_max = 4e-7 * np.pi * 0.3 * Ms                      # mu0 * 0.3 Ms (T)
    level_of_step = np.minimum(np.arange(N + 1) // hold, levels)
    b = (b_max * level_of_step / levels).astype(float)
    drive = tuple(np.repeat(b, 3)[:3 * N + 3].tolist())  # constant within each step
    js = np.arange(1, levels + 1)
    targets = 2.0 * 0.3 * js / levels
    zeta = 10.0 if regularised else 1.0
    p = Problem(nx=nx, ny=ny, nz=1, dx=h, dy=h, dz=h, Ms=Ms, A=1.3e-11, alpha=0.5, alpha_edge=0.5,
                B_bias=(0.0, 0.0, 0.0), b_rf=0.0, f_rf=0.0, rf_dir=(1.0, 0.0, 0.0), src=(0, nx, 0, ny),
                dt=1e-13, nsteps=N, objective=J_CURVE, comp=0, n_from=1, drive=drive,
                sample_steps=tuple(int(v) for v in (js + 1) * hold),
                sample_targets=tuple(targets.tolist()),
                sample_weights=tuple((zeta / (levels * targets)).tolist()),
                area_target=design / (nx * ny), penalty_w=0.05 if regularised else 0.0,
                centre_w=1.0 if regularised else 0.0, centre_target=((design - 1) / 2.0, (ny - 1) / 2.0))
    yy, xx = np.mgrid[0:ny, 0:nx]
    r = np.hypot(xx - (design - 1) / 2.0, yy - (ny - 1) / 2.0) * h
    R = 10 * h
    phi = (R - r) / R + 0.05 * rng.standard_normal((ny, nx))
    phi = phi / np.abs(phi[:, :design]).max()
    phi[:, design:] = -1.0
    m0 = noisy_uniform_m0(rng, nx, ny, 1, direction=(0.0, 1.0, 0.0))
    mask = np.zeros((1, ny, nx), np.uint8)
    mask[:, :, :design] = 1
    return Instance(p, phi[None], m0, mask, "sw_particle" + ("_reg" if regularised else ""))


def random_small(nx: int, ny: int, nz: int = 1, seed: int = 0, nsteps: int = 50,
                 objective: int = J_PORT, **over) -> Instance:
    """Small seeded instance with every field term switched on (bias, RF,
    anisotropy, absorbing ramp), for parity and finite-difference checks."""
    rng = np.random.default_rng(90000 + seed)
    h = 5e-9
    bx = (nx // 2, nx // 2 + max(1, nx // 4), ny // 4, ny // 4 + max(1, ny // 4))
    by = (max(0, nx // 4 - 1), nx // 4 + 1, ny // 2, min(ny, ny // 2 + 2))
    p = Problem(nx=nx, ny=ny, nz=nz, dx=h, dy=h, dz=h, Ms=8e5, A=1.3e-11,
                Ku=2e4, ku=(0.0, 0.6, 0.8), alpha=0.05, alpha_edge=0.3,
                absorb_nodes=min(3, max(1, nx // 4)), absorb_x=1, absorb_y=1,
                B_bias=(0.05, 0.01, 0.0), b_rf=5e-3, f_rf=8e9, rf_dir=(0.0, 1.0, 0.0),
                src=(0, 1, 0, ny), dt=1e-13, nsteps=nsteps, objective=objective,
                comp=1, power=2, boxes=(bx, by), weights=(1.0, -0.5), n_from=1,
                area_target=0.3, penalty_w=1.0)
    p = p.replace(**over)
    phi = np.stack([gaussian_bumps(rng, nx, ny, h, h, 4, 2 * h) for _ in range(nz)])
    phi = 0.04 * np.sign(phi) + 0.06 * phi   # keep psi in (0.05, 0.95): interfaces everywhere
    m0 = noisy_uniform_m0(rng, nx, ny, nz, noise=0.2)
    mask = np.ones((nz, ny, nx), np.uint8)
    return Instance(p, phi, m0, mask, f"small{nx}x{ny}x{nz}")


def by_name(name: str, **kw):
    return {"film32": film32, "particle64": particle64, "demux256": demux256, "sw_particle": sw_particle,
            "batch64": batch64, "thick512": thick512}[name](**kw)
