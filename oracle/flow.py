"""Oracle: the fractional-step driver around the pressure solve (FP64).

TEST INFRASTRUCTURE (see the package header): only tests, smoke() and the
bench's CPU-baseline leg may use it.

Restates Sec. 3.3 of arXiv 2404.17542 for DPs that do not move between the
two evaluations (the ALE interpolation of Eq. (19) is not part of it):
  * u* = F_MOC + nu dt lap u                                      (Eq. (20))
    F_MOC is the velocity at the departure point x - u dt, evaluated, like
    Eq. (19), by the second-order Taylor expansion about the DP:
        F = u + d . grad u + 1/2 d^T H u d,   d = -u_i dt
    with grad and Hessian from the chi=1 quadratic MLS weights (Eq. (14));
  * PPE right-hand side (1/dt) div u*                             (Eq. (21))
  * u^{k+1} = u* - dt grad P                                      (Eq. (22))
    where grad P at an inner DP includes the Neumann-data terms of Eq. (15).
Boundary DPs (any non-void, non-inner DP) take their prescribed velocity;
void DPs carry zero.

Readings: the MOC value uses the DP's own Taylor expansion (the paper says
"evaluated using a similar approach to that in Eq. (19)"); the velocity
stencils treat every boundary id as a Dirichlet (value) boundary.
"""
from __future__ import annotations

import numpy as np

from .mls import stencil_slots


def neighbour_table(mesh):
    """nbr[s, i] = DP in slot s of DP i, or i itself where the slot is empty."""
    S = 3 ** mesh.dim
    nbr = np.zeros((S, mesh.N), dtype=np.int64)
    for i in range(mesh.N):
        for s, j, _off in stencil_slots(mesh, i):
            nbr[s, i] = i if j is None else j
    return nbr


def apply_weights(Wk, phi, nbr):
    """sum_s Wk[s, i] phi[nbr[s, i]] for every DP (Wk: (S, N))."""
    return (Wk * phi[nbr]).sum(axis=0)


def derivatives(W, phi, nbr):
    """Physical derivatives (nb, N) of a field from the value weights D."""
    nb = W["D"].shape[0]
    return np.stack([apply_weights(W["D"][c], phi, nbr) for c in range(nb)])


def neumann_terms(W, f, nbr):
    """(nb, N) Neumann-data contributions sum_s QD[c, s] f_{j_s}."""
    nb = W["QD"].shape[0]
    return np.stack([apply_weights(W["QD"][c], f, nbr) for c in range(nb)])


def predict(mesh, Wv, u, v, ubc, vbc, nu, dt, mask, nbr=None):
    """u*, v* (Eq. (20)) and the PPE source (1/dt) div u* (Eq. (21)) in 2D."""
    nbr = neighbour_table(mesh) if nbr is None else nbr
    inner = mask == -1
    du = derivatives(Wv, u, nbr)     # (ux, uy, uxx, uxy, uyy)
    dv = derivatives(Wv, v, nbr)
    dx = -u * dt
    dy = -v * dt

    def moc(phi, d):
        return (phi + dx * d[0] + dy * d[1]
                + 0.5 * (dx * dx * d[2] + 2.0 * dx * dy * d[3] + dy * dy * d[4]))

    us = moc(u, du) + nu * dt * (du[2] + du[4])
    vs = moc(v, dv) + nu * dt * (dv[2] + dv[4])
    us = np.where(inner, us, np.where(mask == 0, 0.0, ubc))
    vs = np.where(inner, vs, np.where(mask == 0, 0.0, vbc))
    dus = derivatives(Wv, us, nbr)
    dvs = derivatives(Wv, vs, nbr)
    src = np.where(inner, (dus[0] + dvs[1]) / dt, 0.0)
    return us, vs, src


def project(mesh, Wp, P, bnd, us, vs, ubc, vbc, dt, mask, nbr=None):
    """u^{k+1} = u* - dt grad P (Eq. (22)); grad P includes Neumann data."""
    nbr = neighbour_table(mesh) if nbr is None else nbr
    inner = mask == -1
    dP = derivatives(Wp, P, nbr) + neumann_terms(Wp, bnd, nbr)
    u = us - dt * dP[0]
    v = vs - dt * dP[1]
    u = np.where(inner, u, np.where(mask == 0, 0.0, ubc))
    v = np.where(inner, v, np.where(mask == 0, 0.0, vbc))
    return u, v


def step(mesh, pos, mask, u, v, ubc, vbc, P_bc, nu, dt, weight_kind=0, r_e=None,
         normal=None, bc_kind_p=None, neumann_f=None):
    """One fractional step (Eqs. (20)-(22)) with DPs held in place.

    Velocity stencils treat every boundary as Dirichlet; the pressure
    stencils use bc_kind_p (Dirichlet values P_bc, Neumann data neumann_f).
    Returns (u, v, P).
    """
    from . import mls, solve
    nbr = neighbour_table(mesh)
    Wv = mls.build_weights(mesh, pos, mask, weight_kind=weight_kind, r_e=r_e)
    Wp = Wv if bc_kind_p is None else mls.build_weights(mesh, pos, mask, normal, bc_kind_p,
                                                          weight_kind, r_e)
    us, vs, src = predict(mesh, Wv, u, v, ubc, vbc, nu, dt, mask, nbr)
    bnd = P_bc.copy() if neumann_f is None else np.where(Wp["kind"] == 3, neumann_f, P_bc)
    A = solve.assemble(mesh, Wp["row"])
    b = solve.form_rhs(mesh, Wp["kind"], Wp["QL"], src, bnd, Wp["rscale"])
    P = solve.direct_solve(A, b)
    un, vn = project(mesh, Wp, P, bnd, us, vs, ubc, vbc, dt, mask, nbr)
    return un, vn, P
