"""RBF parameterisation of the level-set function and the Adam update, FP64
(test infrastructure only: the tests, smoke() and bench.py's CPU leg use it).

The paper builds Phi on the design region from n radial basis functions
(multiquadric cones, Eq. 2)

    g_k(x, y) = s_k - sqrt((x - x_k)^2 + (y - y_k)^2 + c^2),

combines them by a p-norm that approximates their maximum (Eq. 3)

    F(x, y) = [ sum_k (g_k + dphi)^p ]^(1/p) - dphi,

with the shift dphi = |smallest g_k over the design region| (so that every
g_k + dphi >= 0) and p = 90, and keeps Phi in [-1, 1] by renormalisation
after each step (Results, "Level-set method").  The amplitudes s are what the
optimiser (Adam, Methods) updates, through dJ/ds = sum_j dJ/dPhi_j dPhi_j/ds.

Readings (the paper leaves these open):
* the RBF centres form an nrx x nry grid at the centres of equal cells of the
  design box; c is the centre spacing (the smaller of the two);
* the p-norm is evaluated as U (sum_k (u_k/U)^p)^(1/p), U = max_k u_k, which
  equals Eq. 3 and cannot overflow;
* the renormalisation is part of the map: Phi = F / max_design |F|;
* the gradient is the exact derivative of that map, dphi and the max
  included, taken at the minimising (RBF, node) pair and the maximising node
  (the first in index order on ties), as automatic differentiation would;
  at a node where every g_k + dphi is 0 the p-norm is 0 and its weights are
  taken as 0 (the norm has no derivative there).
"""
from __future__ import annotations

import numpy as np


def centres(nx, ny, dx, dy, box, nrx, nry):
    """Centre coordinates (metres) of an nrx x nry grid over the design box
    x0 <= ix < x1, y0 <= iy < y1 (node indices), and the spacing c."""
    x0, x1, y0, y1 = box
    wx, wy = (x1 - x0) * dx, (y1 - y0) * dy
    hx, hy = wx / nrx, wy / nry
    cx = x0 * dx + (np.arange(nrx) + 0.5) * hx
    cy = y0 * dy + (np.arange(nry) + 0.5) * hy
    X, Y = np.meshgrid(cx, cy, indexing="xy")        # k = iy * nrx + ix
    return X.ravel(), Y.ravel(), min(hx, hy)


def design_nodes(nx, ny, dx, dy, box):
    """Node coordinates of the design box in [y][x] order (flattened)."""
    x0, x1, y0, y1 = box
    ix, iy = np.meshgrid(np.arange(x0, x1), np.arange(y0, y1), indexing="xy")
    return ix.ravel() * dx, iy.ravel() * dy


def rbf_values(s, xk, yk, c, xj, yj):
    """G[j, k] = g_k(x_j) (Eq. 2)."""
    d = np.sqrt((xj[:, None] - xk[None, :]) ** 2 + (yj[:, None] - yk[None, :]) ** 2 + c * c)
    return np.asarray(s, float)[None, :] - d


def phi_map(s, xk, yk, c, xj, yj, p):
    """Phi on the design nodes (Eq. 3 and the renormalisation), with the
    intermediate quantities the gradient needs."""
    G = rbf_values(s, xk, yk, c, xj, yj)
    jm, km = np.unravel_index(np.argmin(G), G.shape)
    m = G[jm, km]
    dphi = abs(m)
    u = G + dphi                                    # >= 0
    U = u.max(axis=1)
    Us = np.where(U > 0, U, 1.0)
    norm = np.where(U > 0, U * ((u / Us[:, None]) ** p).sum(axis=1) ** (1.0 / p), 0.0)   # 0 where all u are 0
    F = norm - dphi
    jM = int(np.argmax(np.abs(F)))
    M = abs(F[jM])
    return F / M, dict(G=G, u=u, norm=norm, F=F, M=M, jM=jM, km=km, m=m, dphi=dphi)


def phi_grad(s, xk, yk, c, xj, yj, p, dJdphi):
    """dJ/ds for dJ/dPhi given on the design nodes: the chain rule through the
    renormalisation, the p-norm and the shift."""
    phi, q = phi_map(s, xk, yk, c, xj, yj, p)
    g = np.asarray(dJdphi, float)
    F, M, jM = q["F"], q["M"], q["jM"]
    H = g / M                                       # dJ/dF_j through Phi_j = F_j / M
    H[jM] += np.sign(F[jM]) * (-(g * F).sum() / (M * M))
    nz = q["norm"] > 0
    W = np.where(nz[:, None], (q["u"] / np.where(nz, q["norm"], 1.0)[:, None]) ** (p - 1), 0.0)   # dF_j / du_jk
    dJds = H @ W
    dJ_ddphi = (H * (W.sum(axis=1) - 1.0)).sum()    # u_jk and F_j both shift with dphi
    dJds[q["km"]] += dJ_ddphi * np.sign(q["m"])     # dphi = |G[jm, km]|
    return dJds


def adam(s, grad, mom, vel, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba's algorithm, step number t >= 1); returns
    the new (s, m, v)."""
    mom = b1 * mom + (1.0 - b1) * grad
    vel = b2 * vel + (1.0 - b2) * grad * grad
    mh = mom / (1.0 - b1 ** t)
    vh = vel / (1.0 - b2 ** t)
    return s - lr * mh / (np.sqrt(vh) + eps), mom, vel
