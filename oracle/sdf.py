"""Oracle: bodies given by a discrete signed distance function (FP64).

TEST INFRASTRUCTURE (see the package header): only tests, smoke() and the
bench's CPU-baseline leg may use it.

Restates Sec. 2.5 of arXiv 2404.17542: a body is described by SDF samples
psi_ij (> 0 in the fluid) on a uniform Cartesian grid attached to the body;
psi and grad psi at any point x_c come from the MLS fit of Sec. 3.2 over the
3x3 compact support D^SDF centred at the grid point nearest x_c; the body's
local frame is rotated by its posture angle theta.

Readings (the paper leaves them open):
  * the fit is the chi = 1 quadratic fit (the only one the paper uses, end of
    Sec. 3.2) centred at the nearest grid point x_s (g = psi_s), weight
    cos^2 with r_e = 2.5 h and r_s = h (h the grid spacing, Eq. (17)); the
    reconstruction psi_s + p(X) . Phi_s is then evaluated at x_c, and its
    gradient gives grad psi (as in Appendix A, where a fit is evaluated at
    a point other than its centre);
  * the nearest grid point is clamped so that its 3x3 support lies inside
    the grid; a point outside the box spanned by the grid points
    1 .. n - 2 of each axis has psi = +inf (no boundary near it): the grid
    has to cover the DP band around the body;
  * local coordinates x_l = R(-theta) (x - c), gradients back to the world
    frame by R(theta); the grid's point (i, j) is at origin + (i, j) h in
    the local frame.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg


def lattice_fit_weights(r_e_over_h=2.5):
    """(5, 9) weights Z with Phi = Z @ (psi_j - psi_s) over the 3x3 lattice
    (slot s = (di+1) + 3 (dj+1), centre slot unused), the chi = 1 quadratic
    MLS fit of Eqs. (12)-(17) in units of the grid spacing (X = offset / h):
    Phi = (psi_X, psi_Y, psi_XX, psi_XY, psi_YY), derivatives per unit X."""
    M = np.zeros((5, 5))
    P = np.zeros((5, 9))
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            if di == 0 and dj == 0:
                continue
            r = math.hypot(di, dj)
            w = math.cos(math.pi * r / (2.0 * r_e_over_h)) ** 2 if r <= r_e_over_h else 0.0
            p = np.array([di, dj, 0.5 * di * di, di * dj, 0.5 * dj * dj], dtype=float)
            M += w * np.outer(p, p)
            P[:, (di + 1) + 3 * (dj + 1)] = w * p
    return scipy.linalg.cho_solve(scipy.linalg.cho_factor(M), P)


class SdfBody:
    """A rigid body given by SDF samples grid[j, i] at origin + (i, j) h in
    its local frame, placed at `centre` with posture angle `theta`."""

    def __init__(self, body_id, centre, theta, grid, origin, h, vel=(0.0, 0.0), omega=0.0):
        self.id = body_id
        self.centre = (float(centre[0]), float(centre[1]))
        self.theta = float(theta)
        self.grid = np.asarray(grid, dtype=np.float64)
        self.origin = (float(origin[0]), float(origin[1]))
        self.h = float(h)
        self.vel = (float(vel[0]), float(vel[1]))
        self.omega = float(omega)
        self.Z = lattice_fit_weights()

    def local(self, x, y):
        c, s = math.cos(self.theta), math.sin(self.theta)
        dx, dy = x - self.centre[0], y - self.centre[1]
        return c * dx + s * dy, -s * dx + c * dy

    def eval(self, x, y):
        """(psi, grad psi (world frame)) at (x, y); (inf, (0, 0)) outside the
        grid's interior box."""
        ny, nx = self.grid.shape
        xl, yl = self.local(x, y)
        fx = (xl - self.origin[0]) / self.h
        fy = (yl - self.origin[1]) / self.h
        if not (1.0 <= fx <= nx - 2 and 1.0 <= fy <= ny - 2):
            return math.inf, (0.0, 0.0)
        i = min(max(int(math.floor(fx + 0.5)), 1), nx - 2)
        j = min(max(int(math.floor(fy + 0.5)), 1), ny - 2)
        ps = self.grid[j, i]
        d = np.array([self.grid[j + dj, i + di] - ps for dj in (-1, 0, 1) for di in (-1, 0, 1)])
        Phi = self.Z @ d
        X, Y = fx - i, fy - j
        psi = ps + Phi[0] * X + Phi[1] * Y + 0.5 * Phi[2] * X * X + Phi[3] * X * Y + 0.5 * Phi[4] * Y * Y
        gxl = (Phi[0] + Phi[2] * X + Phi[3] * Y) / self.h
        gyl = (Phi[1] + Phi[3] * X + Phi[4] * Y) / self.h
        c, s = math.cos(self.theta), math.sin(self.theta)
        return psi, (c * gxl - s * gyl, s * gxl + c * gyl)

