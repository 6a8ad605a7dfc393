"""FP64 oracle of the Smagorinsky eddy viscosity with van Driest damping.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Eq. 4 (Sec. 2.1): nu_t = (C_s Delta D)^2 |S|, |S| = sqrt(2 S_ij S_ij), with
the van Driest damping D = 1 - exp(-y*/25), y* the wall distance in wall
units.  Sec. 2.2 places the model at cell centres: the diagonal strain-rate
components are computed there, the off-diagonal ones on the cell edges and
averaged to the centres.  The paper leaves open, read here as:

S1  filter width Delta_k = (dx dy dzf_k)^(1/3) (cube root of the cell volume);
S2  y* = d u_tau / nu with d the distance from the cell centre to the nearer
    z wall (channel walls at z = 0 and z = sum dzf), u_tau and nu inputs;
S3  no-slip walls: the ghost of u and v below/above a wall is minus the first
    interior value at the mirror distance dzc[0] = dzf[0] (dzc[nz] = dzf[nz-1]),
    w = 0 on the wall faces; x and y periodic.

Layout: u on x-faces (i + 1/2) and v on y-faces (j + 1/2), [nz][ny][nx];
w on z-faces, [nz+1][ny][nx]; nu_t at cell centres [nz][ny][nx].
"""
from __future__ import annotations

import numpy as np

from .cales_oracle import Grid

__all__ = ["strain_rate", "van_driest", "eddy_viscosity"]


def _dz_wall(c: np.ndarray, g: Grid) -> np.ndarray:
    """d c / d z on the z-faces 0..nz of a cell-centred (in z) component with
    the S3 no-slip ghosts: (c[k] - c[k-1]) / dzc[k]."""
    nz = g.nz
    out = np.empty((nz + 1,) + c.shape[1:])
    out[1:nz] = (c[1:] - c[:-1]) / g.dzc[1:nz].reshape(-1, 1, 1)
    out[0] = (c[0] - (-c[0])) / g.dzc[0]
    out[nz] = (-c[nz - 1] - c[nz - 1]) / g.dzc[nz]
    return out


def strain_rate(u, v, w, g: Grid):
    """The six components (S11, S22, S33, S12, S13, S23) at the cell centres."""
    s11 = (u - np.roll(u, 1, axis=2)) / g.dx
    s22 = (v - np.roll(v, 1, axis=1)) / g.dy
    s33 = (w[1:] - w[:-1]) / g.dzf.reshape(-1, 1, 1)
    # edges (i+1/2, j+1/2) of each plane, averaged over the four around a centre
    e12 = 0.5 * ((np.roll(u, -1, axis=1) - u) / g.dy + (np.roll(v, -1, axis=2) - v) / g.dx)
    s12 = 0.25 * (e12 + np.roll(e12, 1, axis=1) + np.roll(e12, 1, axis=2) + np.roll(np.roll(e12, 1, axis=1), 1, axis=2))
    # edges (i+1/2, z-face k), k = 0..nz
    e13 = 0.5 * (_dz_wall(u, g) + (np.roll(w, -1, axis=2) - w) / g.dx)
    s13 = 0.25 * (e13[:-1] + e13[1:] + np.roll(e13[:-1], 1, axis=2) + np.roll(e13[1:], 1, axis=2))
    # edges (j+1/2, z-face k)
    e23 = 0.5 * (_dz_wall(v, g) + (np.roll(w, -1, axis=1) - w) / g.dy)
    s23 = 0.25 * (e23[:-1] + e23[1:] + np.roll(e23[:-1], 1, axis=1) + np.roll(e23[1:], 1, axis=1))
    return s11, s22, s33, s12, s13, s23


def van_driest(g: Grid, nu: float, utau: float) -> np.ndarray:
    """D_k = 1 - exp(-y*_k / 25) per cell plane (S2)."""
    zf = np.concatenate([[0.0], np.cumsum(g.dzf)])
    zc = 0.5 * (zf[:-1] + zf[1:])
    d = np.minimum(zc, zf[-1] - zc)
    return 1.0 - np.exp(-d * utau / nu / 25.0)


def eddy_viscosity(u, v, w, g: Grid, cs: float, nu: float, utau: float) -> np.ndarray:
    """nu_t = (cs Delta D)^2 |S| at the cell centres (Eq. 4, readings S1-S3)."""
    s11, s22, s33, s12, s13, s23 = strain_rate(u, v, w, g)
    smag = np.sqrt(2.0 * (s11 ** 2 + s22 ** 2 + s33 ** 2 + 2.0 * (s12 ** 2 + s13 ** 2 + s23 ** 2)))
    delta = np.cbrt(g.dx * g.dy * g.dzf)
    coef = (cs * delta * van_driest(g, nu, utau)) ** 2
    return coef.reshape(-1, 1, 1) * smag
