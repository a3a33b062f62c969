"""FP64 oracle of the LLG forward pass and its exact discrete adjoint
(test infrastructure only; see the package docstring).

Discretisation (node-as-cell, one cuboid V = dx dy dz per node):
  material   psi_i = 1/(1 + exp(-a Phi_i))                      (Eq. 4)
             Ms_i = Ms psi_i, A_i = A psi_i                     (Results, level-set mapping)
  exchange   E_ex = sum_edges A_ij V |m_j - m_i|^2 / h^2 with the harmonic
             edge mean A_ij = 2 A_i A_j/(A_i + A_j); its field
             B_ex,i = -(1/(Ms_i V)) dE_ex/dm_i
                    = (2A/Ms) sum_j w_ij (m_j - m_i)/h^2,  w_ij = 2 psi_j/(psi_i + psi_j)
  anisotropy B_an = (2 Ku/Ms)(m.u) u   (Ku scaled by psi like Ms, so psi cancels)
  Zeeman     B_z = B_bias + b(t) e_rf on the source box, b(t) = b_rf sin(2 pi f t)
             or a tabulated drive b(n dt + c dt), c = 0, 1/2, 1, per step n
  demag      B_d = -mu0 N * (Ms psi m)   (oracle.demag)
  dynamics   LL form of Eq. 11: f(m) = -gamma/(1+alpha^2) [m x B + alpha m x (m x B)]
             alpha_i ramps linearly from alpha_edge at an absorbing edge to
             alpha over `absorb_nodes` nodes
  time       classic fixed-step RK4, no renormalisation of m
  objective  J_PORT:        sum_{n >= n_from} sum_b w_b mean_{box b}(m_c,n ^ p)
             J_ENERGY_AREA: (E_d + E_ex)(m_N)/(K_d V_dom) + xi (mean psi - s_t)^2,
                            the size term of Eq. 9 on the area fraction
             J_SPECTRAL:    sum_b w_b sum_q |X_b(f_q)|, X_b(f) = sum_{n >= n_from}
                            P_b[n] exp(-2 pi i f n dt), P_b[n] = mean_{box b} m_c,n:
                            Eq. 10's port spectra summed over a frequency window,
                            evaluated at the window's frequencies f_q
             J_CURVE:       sum_j w_j |P(m_{n_j}) - T_j| with P = sum psi m_c / sum psi,
                            the magnetisation curve of Eq. 8 sampled at the end of
                            each field level, + xi (mean psi - s_t)^2 + nu (|x_c - x_0|
                            + |y_c - y_0|), the size and centre terms of Eq. 9
                            (centre = psi-weighted mean node index)
  gradient   the exact derivative of this discrete map (discretise, then
             differentiate): the adjoint recursion of Eq. 6 taken through the
             four RK4 stages, and the parameter integral of Eq. 7 as the sum
             over steps and stages of (df/dpsi)^T u_s, then
             dJ/dPhi = a psi (1 - psi) dJ/dpsi.
  level set  Phi <- Phi - lr g on the design mask (Eq. 5), then divided by the
             largest |Phi| on the mask (renormalisation to [-1, 1]).
"""
from __future__ import annotations

import numpy as np

from . import demag as dm

GAMMA = 1.76085963023e11   # rad s^-1 T^-1 (electron gyromagnetic ratio)
MU0 = dm.MU0

J_PORT = 0
J_ENERGY_AREA = 1
J_SPECTRAL = 2
J_CURVE = 3


def psi_map(phi, a):
    """Eq. 4."""
    return 1.0 / (1.0 + np.exp(-a * phi))


def cross(a, b):
    return np.array([a[1] * b[2] - a[2] * b[1],
                     a[2] * b[0] - a[0] * b[2],
                     a[0] * b[1] - a[1] * b[0]])


def dot(a, b):
    return (a * b).sum(axis=0)


def _edges(shape):
    """Directed edges (i receives from j) as (index_i, index_j, axis) slices
    over [nz][ny][nx] arrays."""
    nz, ny, nx = shape
    out = []
    for axis, n in ((2, nx), (1, ny), (0, nz)):
        if n < 2:
            continue
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, n - 1)
        hi[axis] = slice(1, n)
        out.append((tuple(lo), tuple(hi), axis))   # i = lower node, j = upper node
        out.append((tuple(hi), tuple(lo), axis))   # i = upper node, j = lower node
    return out


class Model:
    """A problem with its material map and demag spectrum prepared."""

    def __init__(self, problem, phi):
        p = problem
        self.p = p
        self.shape = (p.nz, p.ny, p.nx)
        self.phi = np.asarray(phi, float).reshape(self.shape)
        self.psi = psi_map(self.phi, p.sigmoid_a)
        self.h = {2: p.dx, 1: p.dy, 0: p.dz}
        self.V = p.dx * p.dy * p.dz
        self.spectrum = dm.tensor_spectrum(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
        self.alpha = self._alpha_map()
        u = np.array(p.ku, float)
        self.ku = u / np.linalg.norm(u) if np.linalg.norm(u) > 0 else u
        self.src = np.zeros(self.shape, bool)
        x0, x1, y0, y1 = p.src
        self.src[:, y0:y1, x0:x1] = True

    # ---- material / geometry ------------------------------------------
    def _alpha_map(self):
        p = self.p
        a = np.full(self.shape, p.alpha)
        W = p.absorb_nodes
        if W <= 0:
            return a
        iz, iy, ix = np.meshgrid(np.arange(p.nz), np.arange(p.ny), np.arange(p.nx), indexing="ij")
        d = np.full(self.shape, np.inf)
        if p.absorb_x:
            d = np.minimum(d, np.minimum(ix, p.nx - 1 - ix))
        if p.absorb_y:
            d = np.minimum(d, np.minimum(iy, p.ny - 1 - iy))
        ramp = np.maximum(0.0, (W - d) / W)
        return p.alpha + (p.alpha_edge - p.alpha) * ramp

    # ---- field terms ---------------------------------------------------
    def exchange(self, m):
        p, psi = self.p, self.psi
        B = np.zeros_like(m)
        for I, Jn, ax in _edges(self.shape):
            c = 2.0 * p.A / (p.Ms * self.h[ax] ** 2)
            w = 2.0 * psi[Jn] / (psi[I] + psi[Jn])
            B[(slice(None),) + I] += c * w * (m[(slice(None),) + Jn] - m[(slice(None),) + I])
        return B

    def demag(self, m):
        return dm.demag_field_fft(self.p.Ms * self.psi * m, self.p.dx, self.p.dy, self.p.dz,
                                  self.spectrum)

    def anisotropy(self, m):
        if self.p.Ku == 0.0:
            return np.zeros_like(m)
        u = self.ku.reshape(3, 1, 1, 1)
        return (2.0 * self.p.Ku / self.p.Ms) * dot(m, u) * u

    def drive(self, n, ci):
        """b at t = n dt + (ci/2) dt: the tabulated drive, else the sine."""
        p = self.p
        if p.drive is not None:
            return p.drive[3 * n + ci]
        if p.b_rf == 0.0:
            return 0.0
        return p.b_rf * np.sin(2.0 * np.pi * p.f_rf * (n * p.dt + 0.5 * ci * p.dt))

    def _zeeman_of(self, s):
        p = self.p
        B = np.zeros((3,) + self.shape)
        for c in range(3):
            B[c] += p.B_bias[c]
        if s != 0.0:
            for c in range(3):
                B[c][self.src] += s * p.rf_dir[c]
        return B

    def zeeman_stage(self, n, ci):
        """Zeeman field at the stage time n dt + (ci/2) dt of step n."""
        return self._zeeman_of(self.drive(n, ci))

    def zeeman(self, t):
        """Zeeman field at time t (sine drive; a tabulated drive is defined at
        stage times only, see zeeman_stage)."""
        p = self.p
        if p.drive is not None:
            raise ValueError("a tabulated drive is defined at stage times only")
        return self._zeeman_of(p.b_rf * np.sin(2.0 * np.pi * p.f_rf * t) if p.b_rf != 0.0 else 0.0)

    def stage_field(self, m, n, ci):
        return self.exchange(m) + self.demag(m) + self.anisotropy(m) + self.zeeman_stage(n, ci)

    def field(self, m, t):
        return self.exchange(m) + self.demag(m) + self.anisotropy(m) + self.zeeman(t)

    def rhs(self, m, B):
        a = self.alpha
        g = GAMMA / (1.0 + a * a)
        mxB = cross(m, B)
        return -g * (mxB + a * cross(m, mxB))

    # ---- time stepping ---------------------------------------------------
    def stages(self, m, n):
        """RK4 stage inputs Y_s, fields B_s and slopes k_s for step n."""
        dt = self.p.dt
        Y, B, K = [], [], []
        y = m
        for s, (ci, c_next) in enumerate(((0, 0.5), (1, 0.5), (1, 1.0), (2, None))):
            b = self.stage_field(y, n, ci)
            k = self.rhs(y, b)
            Y.append(y)
            B.append(b)
            K.append(k)
            if c_next is not None:
                y = m + c_next * dt * k
        return Y, B, K

    def step(self, m, n):
        _, _, K = self.stages(m, n)
        return m + self.p.dt / 6.0 * (K[0] + 2.0 * K[1] + 2.0 * K[2] + K[3])

    # ---- objectives ------------------------------------------------------
    def _box_mask(self, box):
        x0, x1, y0, y1 = box
        b = np.zeros(self.shape, bool)
        b[:, y0:y1, x0:x1] = True
        return b

    def port_term(self, m):
        """sum_b w_b mean_{box b}(m_c^p) at one step."""
        p = self.p
        v = 0.0
        for box, w in zip(p.boxes, p.weights):
            b = self._box_mask(box)
            if w == 0.0 or not b.any():
                continue
            v += w * (m[p.comp][b] ** p.power).mean()
        return v

    def port_term_grad(self, m):
        p = self.p
        g = np.zeros_like(m)
        for box, w in zip(p.boxes, p.weights):
            b = self._box_mask(box)
            if w == 0.0 or not b.any():
                continue
            g[p.comp][b] += w * p.power * m[p.comp][b] ** (p.power - 1) / b.sum()
        return g

    def port_means(self, m):
        """(P_0, P_1): mean of m_comp over each port box (0 for an empty box)."""
        p = self.p
        out = []
        for box in p.boxes:
            b = self._box_mask(box)
            out.append(m[p.comp][b].mean() if b.any() else 0.0)
        return np.array(out)

    def spectral_value(self, series):
        """Eq. 10 in discrete form for the port series [n][b] of steps
        n_from..N: sum_b w_b sum_q |sum_n P_b[n] exp(-2 pi i f_q n dt)|."""
        p = self.p
        n = np.arange(p.n_from, p.nsteps + 1)
        J = 0.0
        for b in range(2):
            if p.weights[b] == 0.0:
                continue
            for f in p.freqs:
                th = 2.0 * np.pi * f * n * p.dt
                J += p.weights[b] * abs((series[:, b] * np.exp(-1j * th)).sum())
        return J

    def spectral_weights(self, series):
        """dJ/dP_b[n] for the series of spectral_value ([n][b], n = n_from..N)."""
        p = self.p
        n = np.arange(p.n_from, p.nsteps + 1)
        W = np.zeros_like(series)
        for b in range(2):
            if p.weights[b] == 0.0:
                continue
            for f in p.freqs:
                th = 2.0 * np.pi * f * n * p.dt
                xr = (series[:, b] * np.cos(th)).sum()
                xi = -(series[:, b] * np.sin(th)).sum()
                a = np.hypot(xr, xi)
                if a > 0.0:
                    W[:, b] += p.weights[b] * (xr * np.cos(th) - xi * np.sin(th)) / a
        return W

    def spectral_source(self, w):
        """Adjoint source of one step: w_b / |box b| on m_comp over box b."""
        p = self.p
        g = np.zeros((3,) + self.shape)
        for b, box in enumerate(p.boxes):
            bm = self._box_mask(box)
            if bm.any() and w[b] != 0.0:
                g[p.comp][bm] += w[b] / bm.sum()
        return g

    def curve_point(self, m):
        """P = sum psi m_c / sum psi, the particle's mean magnetisation
        component (M_c / Ms) in Eq. 8."""
        psi = self.psi
        return float((psi * m[self.p.comp]).sum() / psi.sum())

    def curve_samples(self):
        """{step n_j: (target T_j, weight w_j)} of J_CURVE (steps 1..N)."""
        p = self.p
        out = {}
        for n, T, w in zip(p.sample_steps, p.sample_targets, p.sample_weights):
            if not 1 <= n <= p.nsteps:
                raise ValueError("curve samples must lie in steps 1..nsteps")
            out[int(n)] = (float(T), float(w))
        return out

    def curve_source(self, m, T, w):
        """(dJ/dm, explicit dJ/dpsi) of w |P(m) - T| (derivative 0 at P = T)."""
        p, psi = self.p, self.psi
        P = self.curve_point(m)
        W = w * np.sign(P - T)
        S = psi.sum()
        g = np.zeros_like(m)
        g[p.comp] = W * psi / S
        return g, W * (m[p.comp] - P) / S

    def centre(self):
        """psi-weighted mean node index (x_c, y_c)."""
        psi = self.psi
        iy, ix = np.meshgrid(np.arange(self.p.ny), np.arange(self.p.nx), indexing="ij")
        S = psi.sum()
        return float((psi * ix).sum() / S), float((psi * iy).sum() / S)

    def penalties(self):
        """Size and centre terms of Eq. 9 (J_CURVE)."""
        p = self.p
        xc, yc = self.centre()
        size = p.penalty_w * (self.psi.mean() - p.area_target) ** 2
        return size + p.centre_w * (abs(xc - p.centre_target[0]) + abs(yc - p.centre_target[1]))

    def penalties_grad(self):
        p, psi = self.p, self.psi
        xc, yc = self.centre()
        iy, ix = np.meshgrid(np.arange(p.ny), np.arange(p.nx), indexing="ij")
        S = psi.sum()
        g = 2.0 * p.penalty_w * (psi.mean() - p.area_target) / psi.size * np.ones(self.shape)
        g += p.centre_w * (np.sign(xc - p.centre_target[0]) * (ix - xc)
                           + np.sign(yc - p.centre_target[1]) * (iy - yc)) / S
        return g

    def energy_terms(self, m):
        """(E_demag, E_exchange) in joules."""
        p, psi, V = self.p, self.psi, self.V
        Bd = self.demag(m)
        Ed = -0.5 * V * (p.Ms * psi * dot(m, Bd)).sum()
        Ee = 0.0
        for I, Jn, ax in _edges(self.shape):
            if Jn[ax].start != 1:      # count each undirected edge once
                continue
            Aij = 2.0 * p.A * psi[I] * psi[Jn] / (psi[I] + psi[Jn])
            d = m[(slice(None),) + Jn] - m[(slice(None),) + I]
            Ee += (Aij * V * dot(d, d) / self.h[ax] ** 2).sum()
        return Ed, Ee

    def _energy_scale(self):
        p = self.p
        Kd = 0.5 * MU0 * p.Ms * p.Ms
        return 1.0 / (Kd * self.V * p.nx * p.ny * p.nz)

    def terminal(self, m):
        p = self.p
        if p.objective == J_CURVE:
            return self.penalties()
        if p.objective != J_ENERGY_AREA:
            return 0.0
        Ed, Ee = self.energy_terms(m)
        frac = self.psi.mean()
        return (Ed + Ee) * self._energy_scale() + p.penalty_w * (frac - p.area_target) ** 2

    def terminal_grads(self, m):
        """(dJ_term/dm_N, explicit dJ/dpsi)."""
        p, psi, V = self.p, self.psi, self.V
        gm = np.zeros_like(m)
        gpsi = np.zeros(self.shape)
        if p.objective == J_CURVE:
            return gm, self.penalties_grad()
        if p.objective != J_ENERGY_AREA:
            return gm, gpsi
        s = self._energy_scale()
        Bd = self.demag(m)
        Be = self.exchange(m)
        gm = -V * p.Ms * psi * (Bd + Be) * s
        gpsi += -V * p.Ms * dot(m, Bd) * s
        for I, Jn, ax in _edges(self.shape):
            d = m[(slice(None),) + Jn] - m[(slice(None),) + I]
            dA = 2.0 * p.A * psi[Jn] ** 2 / (psi[I] + psi[Jn]) ** 2     # dA_ij/dpsi_i
            gpsi[I] += dA * V * dot(d, d) / self.h[ax] ** 2 * s
        gpsi += 2.0 * p.penalty_w * (psi.mean() - p.area_target) / psi.size
        return gm, gpsi

    # ---- forward -----------------------------------------------------------
    def forward(self, m0, keep=True):
        """Returns (J, m_N, trajectory [m_0..m_N] or None)."""
        p = self.p
        m = np.array(m0, float).reshape((3,) + self.shape)
        traj = [m] if keep else None
        J = 0.0
        if p.objective == J_SPECTRAL and p.n_from < 1:
            raise ValueError("the spectral objective needs n_from >= 1")
        series = []
        samples = self.curve_samples() if p.objective == J_CURVE else {}
        self.curve = []
        if p.objective == J_PORT and p.n_from <= 0:
            J += self.port_term(m)
        for n in range(p.nsteps):
            m = self.step(m, n)
            if keep:
                traj.append(m)
            if p.objective == J_PORT and n + 1 >= p.n_from:
                J += self.port_term(m)
            if p.objective == J_SPECTRAL and n + 1 >= p.n_from:
                series.append(self.port_means(m))
            if n + 1 in samples:
                T, w = samples[n + 1]
                P = self.curve_point(m)
                self.curve.append(P)
                J += w * abs(P - T)
        if p.objective == J_SPECTRAL:
            self.series = np.array(series).reshape(-1, 2)
            J += self.spectral_value(self.series)
        J += self.terminal(m)
        return J, m, traj

    # ---- adjoint -----------------------------------------------------------
    def stage_vjp(self, u, Y, B):
        """Given the cotangent u of a slope k = f(Y, B(Y)), return
        (dJ/dY contribution g, dJ/dpsi contribution)."""
        p, psi = self.p, self.psi
        a = self.alpha
        gp = GAMMA / (1.0 + a * a)
        # k = -gp [Y x B + a (Y (Y.B) - B (Y.Y))]
        Bbar = -gp * (cross(u, Y) + a * (dot(u, Y) * Y - dot(Y, Y) * u))
        g = -gp * (cross(B, u) + a * (dot(Y, B) * u + dot(u, Y) * B - 2.0 * dot(u, B) * Y))
        ge, qe = self.exchange_T(Bbar, Y)
        gd, qd = self.demag_T(Bbar, Y)
        return g + ge + gd + self.anisotropy_T(Bbar), qe + qd

    def exchange_T(self, Bbar, Y):
        """Transpose of the exchange field map m -> B_ex at fixed psi, applied
        to Bbar, and the derivative of <Bbar, B_ex(Y)> with respect to psi.
        Written as a scatter over directed edges (i receives c w_ij (Y_j - Y_i))."""
        p, psi = self.p, self.psi
        g = np.zeros_like(Bbar)
        gpsi = np.zeros(self.shape)
        for I, Jn, ax in _edges(self.shape):
            c = 2.0 * p.A / (p.Ms * self.h[ax] ** 2)
            pi, pj = psi[I], psi[Jn]
            w = 2.0 * pj / (pi + pj)
            bi = Bbar[(slice(None),) + I]
            g[(slice(None),) + Jn] += c * w * bi
            g[(slice(None),) + I] -= c * w * bi
            e = c * dot(bi, Y[(slice(None),) + Jn] - Y[(slice(None),) + I])
            gpsi[Jn] += e * 2.0 * pi / (pi + pj) ** 2
            gpsi[I] += e * (-2.0 * pj / (pi + pj) ** 2)
        return g, gpsi

    def demag_T(self, Bbar, Y):
        """Transpose of m -> B_d = -mu0 N * (Ms psi m) applied to Bbar, and the
        derivative of <Bbar, B_d(Y)> with respect to psi.  N is even and each
        N(r) symmetric, so the transpose is the same convolution of Bbar."""
        p, psi = self.p, self.psi
        D = dm.demag_field_fft(Bbar, p.dx, p.dy, p.dz, self.spectrum)
        return p.Ms * psi * D, p.Ms * dot(Y, D)

    def anisotropy_T(self, Bbar):
        if self.p.Ku == 0.0:
            return np.zeros_like(Bbar)
        u = self.ku.reshape(3, 1, 1, 1)
        return (2.0 * self.p.Ku / self.p.Ms) * dot(Bbar, u) * u

    def adjoint(self, m0, traj=None):
        """Store-all discrete adjoint.  Returns (dJ/dPhi, dJ/dm0, J)."""
        p = self.p
        dt = p.dt
        if traj is None:
            J, _, traj = self.forward(m0, keep=True)
        else:
            J = None
        N = p.nsteps
        lam, gpsi = self.terminal_grads(traj[N])
        if p.objective == J_PORT and N >= p.n_from:
            lam = lam + self.port_term_grad(traj[N])
        if p.objective == J_SPECTRAL:
            series = np.array([self.port_means(traj[k]) for k in range(p.n_from, N + 1)]).reshape(-1, 2)
            SW = self.spectral_weights(series)             # row k - n_from: step k
            if N >= p.n_from:
                lam = lam + self.spectral_source(SW[N - p.n_from])
        samples = self.curve_samples() if p.objective == J_CURVE else {}
        if N in samples:
            g, q = self.curve_source(traj[N], *samples[N])
            lam, gpsi = lam + g, gpsi + q
        for n in range(N - 1, -1, -1):
            Y, B, _ = self.stages(traj[n], n)
            u4 = dt / 6.0 * lam
            g4, q4 = self.stage_vjp(u4, Y[3], B[3])
            u3 = dt / 3.0 * lam + dt * g4
            g3, q3 = self.stage_vjp(u3, Y[2], B[2])
            u2 = dt / 3.0 * lam + 0.5 * dt * g3
            g2, q2 = self.stage_vjp(u2, Y[1], B[1])
            u1 = dt / 6.0 * lam + 0.5 * dt * g2
            g1, q1 = self.stage_vjp(u1, Y[0], B[0])
            gpsi = gpsi + q1 + q2 + q3 + q4
            lam = lam + g1 + g2 + g3 + g4
            if p.objective == J_PORT and n >= p.n_from:
                lam = lam + self.port_term_grad(traj[n])
            if p.objective == J_SPECTRAL and n >= p.n_from:
                lam = lam + self.spectral_source(SW[n - p.n_from])
            if n in samples:
                g, q = self.curve_source(traj[n], *samples[n])
                lam, gpsi = lam + g, gpsi + q
        dphi = p.sigmoid_a * self.psi * (1.0 - self.psi) * gpsi
        return dphi, lam, J


def forward(inst_or_problem, phi=None, m0=None, keep=False):
    """J, m_N for a workloads.Instance (or problem, phi, m0)."""
    if phi is None:
        inst = inst_or_problem
        p, phi, m0 = inst.problem, inst.phi, inst.m0
    else:
        p = inst_or_problem
    model = Model(p, phi)
    J, mN, traj = model.forward(m0, keep=keep)
    return J, mN


def gradient(inst_or_problem, phi=None, m0=None):
    """(J, dJ/dPhi, dJ/dm0)."""
    if phi is None:
        inst = inst_or_problem
        p, phi, m0 = inst.problem, inst.phi, inst.m0
    else:
        p = inst_or_problem
    model = Model(p, phi)
    J, _, traj = model.forward(m0, keep=True)
    dphi, dm0, _ = model.adjoint(m0, traj)
    return J, dphi, dm0


def levelset_step(phi, grad, mask, lr):
    """Eq. 5 on the design region, then renormalisation of Phi to [-1, 1]."""
    out = np.array(phi, float)
    sel = np.asarray(mask).astype(bool)
    out[sel] = out[sel] - lr * np.asarray(grad)[sel]
    mx = np.abs(out[sel]).max() if sel.any() else 0.0
    if mx > 0.0:
        out[sel] = out[sel] / mx
    return out
