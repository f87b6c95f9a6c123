"""Oracle: DP masking, arrangement and moving-boundary role reassignment.

TEST INFRASTRUCTURE (see the package header): only tests, smoke() and the
bench's CPU-baseline leg may use it.

Restates Sec. 2 of arXiv 2404.17542 for circular bodies in 2D:
  * mask from the count of cell vertices with SDF >= 0: 0/1 -> void (0),
    2/3 -> boundary id (>= 1), 4 -> inner (-1)                    (Sec. 2.2, Eq. (1))
  * arrangement: (ii) spring relaxation x^ * = x^ - kappa F^ with
    F^_i = sum_j (1 - r'_ij) x~_ij, r' = |x_ij| / l0^SPG, l0^SPG = sqrt(2) l0
    for diagonal neighbours and l0 otherwise, over the non-void neighbours
    of the 3x3 local mesh                                       (Eqs. (2)-(8))
    (iii) boundary DPs relocated x** = x* + psi d^, d^ = -grad psi / |grad psi|
                                                                  (Eq. (9))
    optional boundary-fitted inner move beta psi d^              (Sec. 4.7, Eqs. (45)-(46))
    (iv) clamp to the DP's own cell (nearest edge or vertex)      (Sec. 2.3, Fig. 2)
  * SDF of a circle psi = |x - c| - R, > 0 in the fluid          (Sec. 2.5)
  * only DPs whose cell lies within `band` of the boundary are re-masked
    and rearranged                                               (Sec. 2.4)

Readings (the paper leaves them open):
  * the vertex test psi >= 0 is evaluated as dx*dx + dy*dy >= R*R with each
    operation rounded on its own (no fused multiply-add), vertex coordinate
    origin + i*l0; both sides of the parity test use exactly this sequence;
  * band membership: |psi(cell centroid)| < band with centroid
    origin + (i + 0.5) l0; band <= 0 re-masks every cell (initial call);
  * cells with a face on the domain wall keep the wall id and never move;
  * a fixed number n_relax of Jacobi sweeps (all DPs read iterate k);
  * a DP whose cell becomes void is reset to its centroid;
  * relocation and the boundary-fitted move use the analytic circle SDF.
"""
from __future__ import annotations

import math

import numpy as np

INNER, VOID = -1, 0


def vertex_fluid(mesh, centre, radius):
    """Boolean (n_x+1, n_y+1): vertex (i, j) has psi >= 0 (Sec. 2.2)."""
    nx, ny = mesh.n[0], mesh.n[1]
    ox, oy = mesh.origin[0], mesh.origin[1]
    l0 = mesh.l0
    out = np.zeros((nx + 1, ny + 1), dtype=bool)
    R2 = radius * radius
    for i in range(nx + 1):
        vx = ox + float(i) * l0
        dx = vx - centre[0]
        for j in range(ny + 1):
            vy = oy + float(j) * l0
            dy = vy - centre[1]
            out[i, j] = (dx * dx + dy * dy) >= R2
    return out


def cell_mask_from_count(count, body_id):
    """Eq. (1): number of fluid vertices -> mask value."""
    if count <= 1:
        return VOID
    if count <= 3:
        return body_id
    return INNER


def centroid(mesh, i, j):
    return (mesh.origin[0] + (float(i) + 0.5) * mesh.l0,
            mesh.origin[1] + (float(j) + 0.5) * mesh.l0)


def in_band(mesh, i, j, centre, radius, band):
    if band <= 0.0:
        return True
    cx, cy = centroid(mesh, i, j)
    dx = cx - centre[0]
    dy = cy - centre[1]
    psi = math.sqrt(dx * dx + dy * dy) - radius
    return abs(psi) < band


def is_wall_cell(mesh, i, j):
    return i == 0 or j == 0 or i == mesh.n[0] - 1 or j == mesh.n[1] - 1


def remask(mesh, mask, centre, radius, body_id, band):
    """Role reassignment of Sec. 2.4: new masks inside the band."""
    nx, ny = mesh.n[0], mesh.n[1]
    fl = vertex_fluid(mesh, centre, radius)
    new = mask.copy()
    for j in range(ny):
        for i in range(nx):
            if is_wall_cell(mesh, i, j):
                continue
            if not in_band(mesh, i, j, centre, radius, band):
                continue
            cnt = int(fl[i, j]) + int(fl[i + 1, j]) + int(fl[i, j + 1]) + int(fl[i + 1, j + 1])
            new[i + nx * j] = cell_mask_from_count(cnt, body_id)
    return new


def relax_sweep(mesh, pos, mask, movable, centre, radius, body_id, kappa,
                alpha=0.0, r_e_fit=None):
    """One Jacobi sweep of steps (ii)-(iv) of Sec. 2.3 on the movable DPs."""
    nx, ny = mesh.n[0], mesh.n[1]
    l0 = mesh.l0
    r_e_fit = 5.0 * l0 if r_e_fit is None else r_e_fit
    new = pos.copy()
    for k in np.nonzero(movable)[0]:
        i, j = k % nx, k // nx
        xi = pos[:, k]
        F = np.zeros(2)
        for dj in (-1, 0, 1):
            for di in (-1, 0, 1):
                if di == 0 and dj == 0:
                    continue
                ii, jj = i + di, j + dj
                if ii < 0 or jj < 0 or ii >= nx or jj >= ny:
                    continue
                kk = ii + nx * jj
                if mask[kk] == VOID:
                    continue
                xij = pos[:, kk] - xi                     # x_ij = x_j - x_i
                r = math.sqrt(xij[0] * xij[0] + xij[1] * xij[1])
                if r == 0.0:
                    continue
                lspg = math.sqrt(2.0) * l0 if (di != 0 and dj != 0) else l0   # Eq. (7)
                G = 1.0 - r / lspg                         # Eq. (6)
                F += G * (xij / r)                         # Eq. (5)
        xs = xi - kappa * l0 * F                           # Eq. (8), dimensional
        dxc = xs[0] - centre[0]
        dyc = xs[1] - centre[1]
        dist = math.sqrt(dxc * dxc + dyc * dyc)
        if dist > 0.0:
            psi = dist - radius
            dhat = np.array([-dxc / dist, -dyc / dist])   # -grad psi / |grad psi|
            if mask[k] == body_id:
                xs = xs + psi * dhat                       # Eq. (9)
            elif mask[k] == INNER and alpha > 0.0 and psi < r_e_fit:
                beta = 0.5 * alpha * (1.0 + math.cos(math.pi * psi / r_e_fit))  # Eq. (46)
                xs = xs + beta * psi * dhat                # Eq. (45)
        lo = (mesh.origin[0] + i * l0, mesh.origin[1] + j * l0)
        hi = (mesh.origin[0] + (i + 1) * l0, mesh.origin[1] + (j + 1) * l0)
        new[0, k] = min(max(xs[0], lo[0]), hi[0])          # step (iv)
        new[1, k] = min(max(xs[1], lo[1]), hi[1])
    return new


def update_dps(mesh, pos, mask, centre, radius, body_id=2, kappa=0.2,
               n_relax=10, band=None, alpha=0.0):
    """One moving-boundary DP update (Sec. 2.3-2.4) for one circular body.

    Returns (pos_new, mask_new, mask_prev).
    """
    nx, ny = mesh.n[0], mesh.n[1]
    band = 5.0 * mesh.l0 if band is None else band
    mask_prev = mask.copy()
    mask_new = remask(mesh, mask, centre, radius, body_id, band)
    pos = pos.copy()
    movable = np.zeros(mesh.N, dtype=bool)
    for j in range(ny):
        for i in range(nx):
            k = i + nx * j
            if is_wall_cell(mesh, i, j) or not in_band(mesh, i, j, centre, radius, band):
                continue
            if mask_new[k] == VOID:
                if mask_prev[k] != VOID:
                    c = centroid(mesh, i, j)
                    pos[0, k], pos[1, k] = c
                continue
            movable[k] = True
    for _ in range(n_relax):
        pos = relax_sweep(mesh, pos, mask_new, movable, centre, radius,
                          body_id, kappa, alpha)
    return pos, mask_new, mask_prev


def circle_normals(pos, mask, centre, body_id):
    """Unit normal (x - c)/|x - c| at body DPs, zero elsewhere (dim 2)."""
    n = np.zeros_like(pos)
    sel = mask == body_id
    d = pos[:, sel] - np.array(centre)[:, None]
    n[:, sel] = d / np.sqrt((d * d).sum(axis=0))
    return n
