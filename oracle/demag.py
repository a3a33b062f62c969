"""Demagnetising tensor and demag field, FP64 (test infrastructure only).

The demag field of the Methods section (effective field: Zeeman, demag,
exchange) is computed on the node-as-cell grid: node i owns the cuboid
dx x dy x dz centred on it, and

    B_d,i = -mu0 * sum_j N(r_i - r_j) M_j,      M_j = Ms psi_j m_j,

with N the cell-averaged demagnetising tensor of two cuboids at offset r.

N is evaluated two ways:
  * near the origin by the closed form of Newell, Williams and Dunlop (1993):
    a 27-point second difference of the functions f (diagonal) and g
    (off-diagonal);
  * far from it (|r| >= NEAR_RADIUS * max(dx,dy,dz)) by Gauss-Legendre
    quadrature of the point-dipole kernel K(u) = (I - 3 u u^T/|u|^2)/(4 pi |u|^3)
    against the tent-shaped overlap density of two cells, which is the
    definition N(r) = V * E_s[K(r + s)], s ~ prod_k (h_k - |s_k|)/h_k^2.
The closed form loses about (R/h)^6 * eps to cancellation; the quadrature
converges geometrically once the cells are a few widths apart.  Both agree
to ~1e-11 relative at the switch radius.

Parity status: pinned (self term 1/3, trace identity, symmetry, far-field
dipole limit, Aharoni prism factors, FFT convolution == direct sum).
"""
from __future__ import annotations

import numpy as np
from numpy.polynomial.legendre import leggauss

MU0 = 4e-7 * np.pi
NEAR_RADIUS = 6.0      # switch radius, in units of max(dx, dy, dz)
QUAD_POINTS = 6        # Gauss points per half of each tent


def _asinh_ratio(num, den):
    """asinh(num/den) with 0 where den == 0 (every caller multiplies the
    result by a factor that vanishes there)."""
    out = np.zeros(np.broadcast(num, den).shape)
    ok = den > 0
    out[ok] = np.arcsinh((num * np.ones_like(den))[ok] / den[ok])
    return out


def _atan_ratio(num, den):
    out = np.zeros(np.broadcast(num, den).shape)
    ok = den > 0
    out[ok] = np.arctan((num * np.ones_like(den))[ok] / den[ok])
    return out


def newell_f(x, y, z):
    """Newell's f(x, y, z); even in every argument."""
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t = 0.5 * y * (z2 - x2) * _asinh_ratio(y, np.sqrt(x2 + z2))
    t = t + 0.5 * z * (y2 - x2) * _asinh_ratio(z, np.sqrt(x2 + y2))
    t = t - x * y * z * _atan_ratio(y * z, x * R)
    t = t + (2 * x2 - y2 - z2) * R / 6.0
    return t


def newell_g(x, y, z):
    """Newell's g(x, y, z); odd in x and in y, even in z."""
    sgn = np.sign(x) * np.sign(y)
    x, y, z = np.abs(x), np.abs(y), np.abs(z)
    x2, y2, z2 = x * x, y * y, z * z
    R = np.sqrt(x2 + y2 + z2)
    t = x * y * z * _asinh_ratio(z, np.sqrt(x2 + y2))
    t = t + y / 6.0 * (3 * z2 - y2) * _asinh_ratio(x, np.sqrt(y2 + z2))
    t = t + x / 6.0 * (3 * z2 - x2) * _asinh_ratio(y, np.sqrt(x2 + z2))
    t = t - z2 * z / 6.0 * _atan_ratio(x * y, z * R)
    t = t - z * y2 / 2.0 * _atan_ratio(x * z, y * R)
    t = t - z * x2 / 2.0 * _atan_ratio(y * z, x * R)
    t = t - x * y * R / 3.0
    return sgn * t


_W = {-1: -1.0, 0: 2.0, 1: -1.0}


def _second_difference(fun, X, Y, Z, dx, dy, dz):
    """(1/(4 pi V)) sum_{i,j,k in {-1,0,1}} w_i w_j w_k fun(X+i dx, Y+j dy, Z+k dz)
    with w_0 = 2, w_{+-1} = -1 (Newell's 27-point combination)."""
    s = 0.0
    for i in (-1, 0, 1):
        for j in (-1, 0, 1):
            for k in (-1, 0, 1):
                s = s + _W[i] * _W[j] * _W[k] * fun(X + i * dx, Y + j * dy, Z + k * dz)
    return s / (4.0 * np.pi * dx * dy * dz)


def tensor_newell(X, Y, Z, dx, dy, dz):
    """Closed-form cell-averaged tensor at offsets (X, Y, Z) in metres.
    Returns (xx, yy, zz, xy, xz, yz)."""
    xx = _second_difference(newell_f, X, Y, Z, dx, dy, dz)
    yy = _second_difference(newell_f, Y, X, Z, dy, dx, dz)
    zz = _second_difference(newell_f, Z, Y, X, dz, dy, dx)
    xy = _second_difference(newell_g, X, Y, Z, dx, dy, dz)
    xz = _second_difference(newell_g, X, Z, Y, dx, dz, dy)
    yz = _second_difference(newell_g, Y, Z, X, dy, dz, dx)
    return xx, yy, zz, xy, xz, yz


def _tent_rule(h, n):
    """Nodes and weights on [-h, h] for the density (h - |s|)/h^2."""
    t, w = leggauss(n)
    s = 0.5 * h * (t + 1.0)
    wt = (h - s) / (h * h) * 0.5 * h * w
    return np.concatenate([-s[::-1], s]), np.concatenate([wt[::-1], wt])


def tensor_quadrature(X, Y, Z, dx, dy, dz, n=QUAD_POINTS):
    """Cell-averaged tensor by quadrature of the dipole kernel (valid when
    the two cells are well separated).  Returns (xx, yy, zz, xy, xz, yz)."""
    X = np.asarray(X, float)
    Y = np.asarray(Y, float)
    Z = np.asarray(Z, float)
    sx, wx = _tent_rule(dx, n)
    sy, wy = _tent_rule(dy, n)
    sz, wz = _tent_rule(dz, n)
    acc = [np.zeros(np.broadcast(X, Y, Z).shape) for _ in range(6)]
    for a, wa in zip(sx, wx):
        for b, wb in zip(sy, wy):
            for c, wc in zip(sz, wz):
                u, v, w = X + a, Y + b, Z + c
                r2 = u * u + v * v + w * w
                k = wa * wb * wc / (4.0 * np.pi * r2 * np.sqrt(r2))
                acc[0] += k * (1.0 - 3.0 * u * u / r2)
                acc[1] += k * (1.0 - 3.0 * v * v / r2)
                acc[2] += k * (1.0 - 3.0 * w * w / r2)
                acc[3] += k * (-3.0 * u * v / r2)
                acc[4] += k * (-3.0 * u * w / r2)
                acc[5] += k * (-3.0 * v * w / r2)
    V = dx * dy * dz
    return tuple(V * a for a in acc)


def demag_tensor(ix, iy, iz, dx, dy, dz):
    """Cell-averaged tensor at integer offsets (ix, iy, iz) (arrays of equal
    shape).  Closed form inside NEAR_RADIUS * max(dx,dy,dz), quadrature
    outside.  Returns a [6, ...] array (xx, yy, zz, xy, xz, yz)."""
    ix, iy, iz = np.broadcast_arrays(np.asarray(ix), np.asarray(iy), np.asarray(iz))
    shape = ix.shape
    X, Y, Z = (np.ravel(ix) * dx, np.ravel(iy) * dy, np.ravel(iz) * dz)
    hmax = max(dx, dy, dz)
    near = (X * X + Y * Y + Z * Z) < (NEAR_RADIUS * hmax) ** 2
    out = np.zeros((6,) + X.shape)
    if near.any():
        comps = tensor_newell(X[near], Y[near], Z[near], dx, dy, dz)
        for c in range(6):
            out[c][near] = comps[c]
    far = ~near
    if far.any():
        comps = tensor_quadrature(X[far], Y[far], Z[far], dx, dy, dz)
        for c in range(6):
            out[c][far] = comps[c]
    return out.reshape((6,) + shape)


def _full3x3(t6):
    xx, yy, zz, xy, xz, yz = t6
    return np.array([[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]])


def demag_field_direct(M, dx, dy, dz):
    """Direct O(N^2) sum B_d,i = -mu0 sum_j N(r_i - r_j) M_j.
    M is [3][nz][ny][nx] (A/m); returns B_d in tesla, same layout."""
    _, nz, ny, nx = M.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    z, y, x = z.ravel(), y.ravel(), x.ravel()
    Mf = M.reshape(3, -1)
    out = np.zeros_like(Mf)
    for i in range(x.size):
        t = _full3x3(demag_tensor(x[i] - x, y[i] - y, z[i] - z, dx, dy, dz))  # [3][3][nodes]
        out[:, i] = -MU0 * np.einsum("abj,bj->a", t, Mf)
    return out.reshape(M.shape)


def padded_shape(nx, ny, nz):
    """Zero-padded FFT grid: twice each extent (1 layer stays 1)."""
    return (2 * nz if nz > 1 else 1, 2 * ny, 2 * nx)


def tensor_spectrum(nx, ny, nz, dx, dy, dz):
    """Real FFT of the tensor placed at offsets modulo the padded grid.
    Returns a [6][Pz][Py][Px//2+1] complex array."""
    Pz, Py, Px = padded_shape(nx, ny, nz)
    oz = np.arange(-(nz - 1), nz)
    oy = np.arange(-(ny - 1), ny)
    ox = np.arange(-(nx - 1), nx)
    Z, Y, X = np.meshgrid(oz, oy, ox, indexing="ij")
    t = demag_tensor(X, Y, Z, dx, dy, dz)
    grid = np.zeros((6, Pz, Py, Px))
    grid[:, Z % Pz, Y % Py, X % Px] = t
    return np.fft.rfftn(grid, axes=(1, 2, 3))


def demag_field_fft(M, dx, dy, dz, spectrum=None):
    """Zero-padded FFT convolution; same result as demag_field_direct."""
    _, nz, ny, nx = M.shape
    Pz, Py, Px = padded_shape(nx, ny, nz)
    if spectrum is None:
        spectrum = tensor_spectrum(nx, ny, nz, dx, dy, dz)
    Mp = np.zeros((3, Pz, Py, Px))
    Mp[:, :nz, :ny, :nx] = M
    Mh = np.fft.rfftn(Mp, axes=(1, 2, 3))
    xx, yy, zz, xy, xz, yz = spectrum
    Hh = np.array([xx * Mh[0] + xy * Mh[1] + xz * Mh[2],
                   xy * Mh[0] + yy * Mh[1] + yz * Mh[2],
                   xz * Mh[0] + yz * Mh[1] + zz * Mh[2]])
    H = np.fft.irfftn(Hh, s=(Pz, Py, Px), axes=(1, 2, 3))[:, :nz, :ny, :nx]
    return -MU0 * H
