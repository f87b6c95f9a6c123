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
  * several bodies: at each point the SDF of smallest magnitude is taken
    (Sec. 2.5, last paragraph), and boundary cells carry the id of their
    body (Sec. 2.2)
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
  * relocation and the boundary-fitted move use the analytic circle SDF, or
    for a body given by a discrete SDF (oracle.sdf.SdfBody, Sec. 2.5) its
    interpolated psi and grad psi: d^ = -grad psi / |grad psi|; its vertex
    test is psi >= 0 of the interpolated psi;
  * with several bodies: a vertex is classified by the SDF of its nearest
    body (smallest |psi|, the first body in list order on a tie, psi
    evaluated as sqrt(dx*dx + dy*dy) - R with each operation rounded on its
    own), then by the test above for that body; a cell's band test and its
    boundary id use the body nearest its centroid; a boundary DP is
    relocated onto the body whose id it carries, an inner DP's
    boundary-fitted move follows the body nearest its spring-relaxed
    position.  For disjoint circles the nearest-SDF rule classifies every
    point as the union SDF min_b psi_b does: a point at depth d inside one
    circle lies at least d + (gap) from every other circle.
"""
from __future__ import annotations

import math

import numpy as np

INNER, VOID = -1, 0


def is_sdf(b):
    return hasattr(b, "eval")


def body_id_of(b):
    return b.id if is_sdf(b) else b[0]


def as_bodies(centre, radius, body_id):
    """The body list [(id, centre, radius)] of one circular body."""
    return [(body_id, (float(centre[0]), float(centre[1])), float(radius))]


def nearest_body(bodies, x, y):
    """(index, psi): the body whose circle SDF has the smallest magnitude at
    (x, y), the first in list order on a tie (Sec. 2.5)."""
    best, best_psi = 0, None
    for b, body in enumerate(bodies):
        if is_sdf(body):
            psi = body.eval(x, y)[0]
        else:
            _bid, c, R = body
            dx = x - c[0]
            dy = y - c[1]
            psi = math.sqrt(dx * dx + dy * dy) - R
        if best_psi is None or abs(psi) < abs(best_psi):
            best, best_psi = b, psi
    return best, best_psi


def psi_grad(body, x, y):
    """(psi, unit direction of grad psi or None) of one body at (x, y)."""
    if is_sdf(body):
        psi, g = body.eval(x, y)
        n = math.sqrt(g[0] * g[0] + g[1] * g[1])
        return psi, ((g[0] / n, g[1] / n) if n > 0.0 and math.isfinite(psi) else None)
    _bid, c, R = body
    dx, dy = x - c[0], y - c[1]
    d = math.sqrt(dx * dx + dy * dy)
    return d - R, ((dx / d, dy / d) if d > 0.0 else None)


def body_index(bodies, body_id):
    for b, body in enumerate(bodies):
        if body_id_of(body) == body_id:
            return b
    return None


def vertex_fluid_bodies(mesh, bodies):
    """Boolean (n_x+1, n_y+1): vertex (i, j) has psi >= 0 for its nearest
    body (Sec. 2.2, Sec. 2.5)."""
    nx, ny = mesh.n[0], mesh.n[1]
    ox, oy = mesh.origin[0], mesh.origin[1]
    l0 = mesh.l0
    out = np.zeros((nx + 1, ny + 1), dtype=bool)
    for i in range(nx + 1):
        vx = ox + float(i) * l0
        for j in range(ny + 1):
            vy = oy + float(j) * l0
            b = nearest_body(bodies, vx, vy)[0] if len(bodies) > 1 else 0
            if is_sdf(bodies[b]):
                out[i, j] = bodies[b].eval(vx, vy)[0] >= 0.0
                continue
            _bid, c, R = bodies[b]
            dx = vx - c[0]
            dy = vy - c[1]
            out[i, j] = (dx * dx + dy * dy) >= R * R
    return out


def vertex_fluid(mesh, centre, radius):
    """Boolean (n_x+1, n_y+1): vertex (i, j) has psi >= 0 (Sec. 2.2)."""
    return vertex_fluid_bodies(mesh, as_bodies(centre, radius, 2))


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


def in_band_bodies(mesh, i, j, bodies, band):
    if band <= 0.0:
        return True
    cx, cy = centroid(mesh, i, j)
    return abs(nearest_body(bodies, cx, cy)[1]) < band


def in_band(mesh, i, j, centre, radius, band):
    return in_band_bodies(mesh, i, j, as_bodies(centre, radius, 2), band)


def is_wall_cell(mesh, i, j):
    return i == 0 or j == 0 or i == mesh.n[0] - 1 or j == mesh.n[1] - 1


def remask_bodies(mesh, mask, bodies, band):
    """Role reassignment of Sec. 2.4: new masks inside the band; a boundary
    cell takes the id of the body nearest its centroid."""
    nx, ny = mesh.n[0], mesh.n[1]
    fl = vertex_fluid_bodies(mesh, bodies)
    new = mask.copy()
    for j in range(ny):
        for i in range(nx):
            if is_wall_cell(mesh, i, j):
                continue
            if not in_band_bodies(mesh, i, j, bodies, band):
                continue
            cnt = int(fl[i, j]) + int(fl[i + 1, j]) + int(fl[i, j + 1]) + int(fl[i + 1, j + 1])
            cx, cy = centroid(mesh, i, j)
            bid = body_id_of(bodies[nearest_body(bodies, cx, cy)[0]])
            new[i + nx * j] = cell_mask_from_count(cnt, bid)
    return new


def remask(mesh, mask, centre, radius, body_id, band):
    """Role reassignment of Sec. 2.4 for one body."""
    return remask_bodies(mesh, mask, as_bodies(centre, radius, body_id), band)


def relax_sweep(mesh, pos, mask, movable, centre, radius, body_id, kappa,
                alpha=0.0, r_e_fit=None):
    """One Jacobi sweep of steps (ii)-(iv) of Sec. 2.3 for one body."""
    return relax_sweep_bodies(mesh, pos, mask, movable, as_bodies(centre, radius, body_id),
                              kappa, alpha, r_e_fit)


def relax_sweep_bodies(mesh, pos, mask, movable, bodies, kappa, alpha=0.0,
                       r_e_fit=None):
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
        if mask[k] >= 1:
            b = body_index(bodies, int(mask[k]))           # the DP's own body
        elif mask[k] == INNER and alpha > 0.0:
            b = nearest_body(bodies, xs[0], xs[1])[0] if len(bodies) > 1 else 0
        else:
            b = None
        psi, unit = psi_grad(bodies[b], xs[0], xs[1]) if b is not None else (0.0, None)
        if unit is not None:
            dhat = np.array([-unit[0], -unit[1]])          # -grad psi / |grad psi|
            if mask[k] >= 1:
                xs = xs + psi * dhat                       # Eq. (9)
            elif psi < r_e_fit:
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
    return update_dps_bodies(mesh, pos, mask, as_bodies(centre, radius, body_id),
                             kappa, n_relax, band, alpha)


def update_dps_bodies(mesh, pos, mask, bodies, kappa=0.2, n_relax=10,
                      band=None, alpha=0.0):
    """One moving-boundary DP update (Sec. 2.3-2.4) for the circular bodies
    [(id, centre, radius)] (ids >= 2, disjoint circles).

    Returns (pos_new, mask_new, mask_prev).
    """
    nx, ny = mesh.n[0], mesh.n[1]
    band = 5.0 * mesh.l0 if band is None else band
    mask_prev = mask.copy()
    mask_new = remask_bodies(mesh, mask, bodies, band)
    pos = pos.copy()
    movable = np.zeros(mesh.N, dtype=bool)
    for j in range(ny):
        for i in range(nx):
            k = i + nx * j
            if is_wall_cell(mesh, i, j) or not in_band_bodies(mesh, i, j, bodies, band):
                continue
            if mask_new[k] == VOID:
                if mask_prev[k] != VOID:
                    c = centroid(mesh, i, j)
                    pos[0, k], pos[1, k] = c
                continue
            movable[k] = True
    for _ in range(n_relax):
        pos = relax_sweep_bodies(mesh, pos, mask_new, movable, bodies, kappa, alpha)
    return pos, mask_new, mask_prev


def circle_normals(pos, mask, centre, body_id):
    """Unit normal (x - c)/|x - c| at body DPs, zero elsewhere (dim 2)."""
    n = np.zeros_like(pos)
    sel = mask == body_id
    d = pos[:, sel] - np.array(centre)[:, None]
    n[:, sel] = d / np.sqrt((d * d).sum(axis=0))
    return n


def bodies_normals(pos, mask, bodies):
    """Unit normal grad psi / |grad psi| of every body on the DPs carrying its
    id (for a circle (x - c)/|x - c|); zero elsewhere."""
    n = np.zeros_like(pos)
    for body in bodies:
        if is_sdf(body):
            for k in np.nonzero(mask == body.id)[0]:
                _psi, unit = psi_grad(body, pos[0, k], pos[1, k])
                if unit is not None:
                    n[:, k] = unit
            continue
        bid, c, _R = body
        sel = mask == bid
        d = pos[:, sel] - np.array(c)[:, None]
        n[:, sel] = d / np.sqrt((d * d).sum(axis=0))
    return n
