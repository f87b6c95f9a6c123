"""Oracle: the ALE velocity interpolation and the fluid force on a body (FP64).

TEST INFRASTRUCTURE (see the package header): only tests, smoke() and the
bench's CPU-baseline leg may use it.

Restates arXiv 2404.17542 for 2D circular bodies and 3x3 stencils:
  * ALE interpolation (Sec. 3.3, Eq. (19) with p = 2): the step-k velocity
    at the new position x^{k+1},
        u~ = u + dx u_x + dy u_y + 1/2 (dx^2 u_xx + 2 dx dy u_xy + dy^2 u_yy),
    (dx, dy) = x^{k+1} - x_c^k, derivatives of the chi=1 quadratic MLS fit
    of the step-k cloud (Eq. (14)): the fit's own reconstruction at x^{k+1}
    (Appendix A, Eq. (A.1));
  * a DP whose mask changed into the fluid has no step-k fit of its own: the
    support is shifted by one cell along the signs of the boundary normal
    and the fit of the DP at the centre of the shifted support, c, is
    evaluated at x^{k+1} (Appendix A, Eq. (A.2); Sec. 3.4);
  * fluid force F = sum_i t_i dGamma_i over the DPs of the body (Eq. (30)),
    t = (-P I + mu (grad u + grad u^T)) . n, dGamma_i the mean distance to
    the two neighbouring boundary DPs (Eq. (31)); P and grad u at a
    boundary DP from the fit of the DP at the centre of its shifted support
    (Sec. 3.4), the pressure fit including the Neumann data of Eq. (15).

Readings (the paper leaves them open):
  * the shift is sign(n_x), sign(n_y) cells (0 for an exactly zero
    component), with n the outward normal of the body nearest the DP at its
    step-k position (for a boundary DP, its own boundary normal);
  * a DP that is inner at k+1 but whose shifted-centre DP is not inner at
    step k keeps its step-k velocity (counted as a fallback); DPs that are
    not inner at k+1 keep their step-k value (the driver imposes boundary
    values on them);
  * the two neighbouring boundary DPs of Eq. (31) are, among the DPs with
    the same boundary id in the 5x5 cells around the DP, the nearest one on
    each side of the tangent t = (-n_y, n_x); a side without one adds 0;
  * a boundary DP whose shifted-centre DP is not inner adds no traction
    (counted as skipped);
  * n is the outward normal of the body (pointing into the fluid); F is the
    force the fluid exerts on the body.
"""
from __future__ import annotations

import math

import numpy as np

from .flow import derivatives, neighbour_table, neumann_terms
from .mask import nearest_body, psi_grad

INNER = -1


def taylor2(phi, d, dx, dy):
    """Second-order Taylor value phi(x + (dx, dy)) from the derivatives
    d = (phi_x, phi_y, phi_xx, phi_xy, phi_yy) at x (Eq. (19), p = 2)."""
    return (phi + dx * d[0] + dy * d[1]
            + 0.5 * (dx * dx * d[2] + 2.0 * dx * dy * d[3] + dy * dy * d[4]))


def sgn(v):
    return 1 if v > 0.0 else (-1 if v < 0.0 else 0)


def shifted_centre(mesh, k, nx_, ny_):
    """Cell of the centre of the support of DP k shifted by one cell along
    the signs of (n_x, n_y) (Sec. 3.4), clamped into the mesh."""
    nx, ny = mesh.n[0], mesh.n[1]
    i, j = k % nx, k // nx
    i = min(max(i + sgn(nx_), 0), nx - 1)
    j = min(max(j + sgn(ny_), 0), ny - 1)
    return i + nx * j


def body_normal(bodies, x, y):
    """Outward unit normal grad psi / |grad psi| of the body nearest (x, y)."""
    b = nearest_body(bodies, x, y)[0]
    _psi, unit = psi_grad(bodies[b], x, y)
    return unit if unit is not None else (0.0, 0.0)


def ale_interpolate(mesh, pos_k, pos_k1, mask_k, mask_k1, u_k, Wv_k, bodies_k, nbr=None):
    """u~^k at the step-(k+1) positions for one velocity component.

    Wv_k: the step-k velocity weights (oracle.mls.build_weights of pos_k,
    mask_k, every boundary a Dirichlet boundary).  bodies_k: the bodies at
    step k [(id, centre, radius)].  Returns (u~, number of fallbacks).
    """
    nbr = neighbour_table(mesh) if nbr is None else nbr
    D = derivatives(Wv_k, u_k, nbr)
    out = u_k.astype(np.float64).copy()
    fallbacks = 0
    for c in np.nonzero(mask_k1 == INNER)[0]:
        if mask_k[c] == INNER:
            src = c                                            # Eq. (A.1)
        else:
            n = body_normal(bodies_k, pos_k[0, c], pos_k[1, c])
            src = shifted_centre(mesh, c, n[0], n[1])          # Eq. (A.2)
            if mask_k[src] != INNER:
                fallbacks += 1
                continue
        dx = pos_k1[0, c] - pos_k[0, src]
        dy = pos_k1[1, c] - pos_k[1, src]
        out[c] = taylor2(u_k[src], D[:, src], dx, dy)
    return out, fallbacks


def boundary_neighbours(mesh, pos, mask, k, n):
    """(j1, j2): the nearest DP with the id of DP k in the 5x5 cells around
    it on each side of the tangent (-n_y, n_x); None where a side has none."""
    nx, ny = mesh.n[0], mesh.n[1]
    i, j = k % nx, k // nx
    t = (-n[1], n[0])
    best = {1: (None, math.inf), -1: (None, math.inf)}
    for dj in range(-2, 3):
        for di in range(-2, 3):
            ii, jj = i + di, j + dj
            if (di == 0 and dj == 0) or not (0 <= ii < nx and 0 <= jj < ny):
                continue
            q = ii + nx * jj
            if mask[q] != mask[k]:
                continue
            ex, ey = pos[0, q] - pos[0, k], pos[1, q] - pos[1, k]
            side = ex * t[0] + ey * t[1]
            if side == 0.0:
                continue
            s = 1 if side > 0.0 else -1
            d = math.sqrt(ex * ex + ey * ey)
            if d < best[s][1]:
                best[s] = (q, d)
    return best[1], best[-1]


def fluid_force(mesh, pos, mask, body_id, normal, P, bnd_p, u, v, mu, Wp, Wv, nbr=None):
    """Force of the fluid on body `body_id` (Eqs. (30)-(31)).

    Wp: pressure weights (with Neumann data weights QD), bnd_p: their
    boundary data; Wv: velocity weights.  Returns (F (2,), perimeter
    sum dGamma, number of skipped DPs).
    """
    nbr = neighbour_table(mesh) if nbr is None else nbr
    dP = derivatives(Wp, P, nbr) + neumann_terms(Wp, bnd_p, nbr)
    du = derivatives(Wv, u, nbr)
    dv = derivatives(Wv, v, nbr)
    F = np.zeros(2)
    perim = 0.0
    skipped = 0
    for k in np.nonzero(mask == body_id)[0]:
        n = normal[:, k]
        (j1, d1), (j2, d2) = boundary_neighbours(mesh, pos, mask, k, n)
        dG = 0.5 * ((d1 if j1 is not None else 0.0) + (d2 if j2 is not None else 0.0))   # Eq. (31)
        perim += dG
        c = shifted_centre(mesh, k, n[0], n[1])
        if mask[c] != INNER:
            skipped += 1
            continue
        dx = pos[0, k] - pos[0, c]
        dy = pos[1, k] - pos[1, c]
        Pk = taylor2(P[c], dP[:, c], dx, dy)
        ux = du[0, c] + du[2, c] * dx + du[3, c] * dy
        uy = du[1, c] + du[3, c] * dx + du[4, c] * dy
        vx = dv[0, c] + dv[2, c] * dx + dv[3, c] * dy
        vy = dv[1, c] + dv[3, c] * dx + dv[4, c] * dy
        tx = -Pk * n[0] + mu * (2.0 * ux * n[0] + (uy + vx) * n[1])
        ty = -Pk * n[1] + mu * ((uy + vx) * n[0] + 2.0 * vy * n[1])
        F[0] += tx * dG                                        # Eq. (30)
        F[1] += ty * dG
    return F, perim, skipped


def body_frame(body):
    """(id, centre, angular velocity) of a circle tuple or an SDF body."""
    if hasattr(body, "eval"):
        return body.id, body.centre, body.omega
    return body[0], body[1], 0.0


def boundary_velocity(mask, bodies_vel, pos=None):
    """(ubc, vbc): the rigid-body velocity V + omega x (x - c) (Eqs.
    (24)-(25)) of the body whose id a DP carries, 0 at every other DP;
    bodies_vel = [(id, (vx, vy))] or [(id, (vx, vy), omega, centre)]."""
    ubc = np.zeros(mask.shape[0])
    vbc = np.zeros(mask.shape[0])
    for entry in bodies_vel:
        bid, V = entry[0], entry[1]
        sel = mask == bid
        ubc[sel] = V[0]
        vbc[sel] = V[1]
        if len(entry) > 2 and entry[2] != 0.0:
            om, c = entry[2], entry[3]
            ubc[sel] -= om * (pos[1, sel] - c[1])
            vbc[sel] += om * (pos[0, sel] - c[0])
    return ubc, vbc


def rigid_acceleration(pos, centre, V0, V1, om0, om1, dt):
    """dV/dt of a rigid body at the points pos (2, m) at t_{k+1} (Eqs.
    (26)-(29)): the finite differences over the step of the translational
    velocity (V0 -> V1) and of the angular velocity (om0 -> om1), with the
    angular acceleration acting on r = x - centre, plus the centripetal
    term omega x (omega x r) = -omega^2 r."""
    rx, ry = pos[0] - centre[0], pos[1] - centre[1]
    omd = (om1 - om0) / dt
    ax = (V1[0] - V0[0]) / dt - omd * ry - om1 * om1 * rx
    ay = (V1[1] - V0[1]) / dt + omd * rx - om1 * om1 * ry
    return ax, ay


def moving_step(mesh, pos_k, mask_k, u_k, v_k, Wv_k, bodies_k, bodies_k1, V_k, V_k1, dt, nu,
                weight_kind=0, r_e=None, kappa=0.2, n_relax=10, band=None):
    """One moving-boundary fractional step in the order of Sec. 3.3.

    bodies_k, bodies_k1: the bodies at t_k and t_{k+1}, circles
    (id, centre, radius) or SDF bodies (oracle.sdf.SdfBody, with their
    angular velocity omega); V_k, V_k1: their translational velocities
    [(vx, vy)]; Wv_k: the step-k velocity weights.
      1. DP update to the bodies at t_{k+1} (Sec. 2.3-2.4);
      2. u~ = u^k(x^{k+1}) (Eq. (19), Appendix A);
      3. MLS weights of the step-(k+1) cloud: velocity (every boundary a
         Dirichlet boundary) and pressure (bodies Neumann, walls Dirichlet);
      4. u* and the PPE source (Eqs. (20)-(21)) with the bodies' velocities
         on their DPs and 0 on the walls;
      5. the PPE (direct solve) with dP/dn = -dV/dt . n on the bodies,
         dV/dt = (V^{k+1} - V^k) / dt (Eqs. (23), (29)), P = 0 on the walls;
      6. u^{k+1} = u* - dt grad P (Eq. (22));
      7. the force on each body (Eqs. (30)-(31)), mu = nu (unit density).
    Returns a dict with pos, mask, u, v, P, F {id: (F, perimeter, skipped)},
    Wv (the step-(k+1) velocity weights), normal, fallbacks.
    """
    from . import flow, mls, solve
    from . import mask as omask
    pos1, mask1, _prev = omask.update_dps_bodies(mesh, pos_k, mask_k, bodies_k1, kappa, n_relax, band)
    ut, fb = ale_interpolate(mesh, pos_k, pos1, mask_k, mask1, u_k, Wv_k, bodies_k)
    vt, _ = ale_interpolate(mesh, pos_k, pos1, mask_k, mask1, v_k, Wv_k, bodies_k)
    normal = omask.bodies_normals(pos1, mask1, bodies_k1)
    frames_k = [body_frame(b) for b in bodies_k]
    frames_1 = [body_frame(b) for b in bodies_k1]
    bc_p = np.zeros(128, dtype=np.uint8)
    for bid, _c, _om in frames_1:
        bc_p[bid] = 1
    Wv = mls.build_weights(mesh, pos1, mask1, weight_kind=weight_kind, r_e=r_e)
    Wp = mls.build_weights(mesh, pos1, mask1, normal, bc_p, weight_kind, r_e)
    ubc, vbc = boundary_velocity(mask1, [(f[0], V, f[2], f[1]) for f, V in zip(frames_1, V_k1)], pos1)
    us, vs, src = flow.predict(mesh, Wv, ut, vt, ubc, vbc, nu, dt, mask1)
    bnd = np.zeros(mesh.N)
    for (bid, c, om1), (_b0, _c0, om0), V0, V1 in zip(frames_1, frames_k, V_k, V_k1):
        sel = mask1 == bid
        ax, ay = rigid_acceleration(pos1[:, sel], c, V0, V1, om0, om1, dt)
        bnd[sel] = -(ax * normal[0, sel] + ay * normal[1, sel])
    A = solve.assemble(mesh, Wp["row"])
    b = solve.form_rhs(mesh, Wp["kind"], Wp["QL"], src, bnd, Wp["rscale"])
    P = solve.direct_solve(A, b)
    u1, v1 = flow.project(mesh, Wp, P, bnd, us, vs, ubc, vbc, dt, mask1)
    F = {bid: fluid_force(mesh, pos1, mask1, bid, normal, P, bnd, u1, v1, nu, Wp, Wv)
         for bid, _c, _om in frames_1}
    return dict(pos=pos1, mask=mask1, u=u1, v=v1, P=P, F=F, Wv=Wv, normal=normal, fallbacks=fb)
