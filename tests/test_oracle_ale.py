"""Pins of the oracle's ALE interpolation and fluid force (Sec. 3.3, Eq. (19),
Appendix A; Sec. 3.4, Eqs. (30)-(31)).

  * ALE interpolation across a real moving-boundary step reproduces a
    quadratic velocity field exactly at every DP inside the fluid at k+1,
    also at DPs whose role changed (the shifted-support fit, Eq. (A.2));
  * the force of a linear pressure on a circle is -grad P times its area,
    the viscous force of u = (alpha x^2, beta x^2) is mu pi R^2
    (4 alpha, 2 beta), and the surface elements add up to 2 pi R: closed
    forms by the divergence theorem.  The tractions are exact for these
    fields, so what remains is the quadrature of Eqs. (30)-(31) over the
    ring of boundary DPs; their spacing is irregular (and a few are clamped
    off the circle), which leaves a relative error of about 1e-3 that does
    not shrink with the mesh (6.5e-4 at 48^2, 6.3e-4 at 96^2, 7.2e-4 at
    192^2 for the pressure force), so the bound is 2e-3 at every size;
  * planted mistakes (a dropped 1/2, a shift into the body, a dropped 1/2 in
    dGamma) break a pin.
"""
import math

import numpy as np
import pytest

from oracle import ale
from oracle import mask as omask
from oracle import mls
from paper_2404_17542_gb300 import inputs


def quad(x, y, c):
    return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y


def moving_step(n=64, shift_cells=0.6):
    """Two DP updates of the oscillating cylinder, dt chosen so that the body
    moves about shift_cells l0: returns (pb, pos_k, mask_k, pos_k1, mask_k1,
    bodies_k)."""
    pb = inputs.cylinder_box(n)
    cyl = pb.meta["cylinder"]
    l0 = pb.mesh.l0
    t0 = 0.0
    dt = shift_cells * l0 / abs(cyl.velocity(t0)[0])
    ck, ck1 = cyl.centre(t0), cyl.centre(t0 + dt)
    pos_k, mask_k, _ = omask.update_dps(pb.mesh, pb.pos, pb.mask, ck, cyl.radius, band=0.0, n_relax=6)
    pos_k1, mask_k1, _ = omask.update_dps(pb.mesh, pos_k, mask_k, ck1, cyl.radius, n_relax=6)
    return pb, pos_k, mask_k, pos_k1, mask_k1, [(cyl.body_id, ck, cyl.radius)]


@pytest.mark.parametrize("weight_kind,r_e", [(0, 1.0), (1, 2.5)])
def test_ale_reproduces_quadratics(weight_kind, r_e):
    pb, pos_k, mask_k, pos_k1, mask_k1, bodies = moving_step()
    W = mls.build_weights(pb.mesh, pos_k, mask_k, weight_kind=weight_kind, r_e=r_e * pb.mesh.l0)
    c = (0.3, -0.7, 0.4, 1.3, -0.9, 0.6)
    u_k = quad(pos_k[0], pos_k[1], c)
    got, fallbacks = ale.ale_interpolate(pb.mesh, pos_k, pos_k1, mask_k, mask_k1, u_k, W, bodies)
    inner1 = mask_k1 == -1
    want = quad(pos_k1[0], pos_k1[1], c)
    assert fallbacks == 0
    assert np.abs(got[inner1] - want[inner1]).max() <= 1e-11
    changed = inner1 & (mask_k != -1)
    assert changed.sum() >= 5          # role-changed DPs take the shifted fit
    assert np.abs(pos_k1[:, inner1] - pos_k[:, inner1]).max() > 0.05 * pb.mesh.l0
    # DPs outside the fluid at k+1 keep their step-k value
    assert np.array_equal(got[~inner1], u_k[~inner1])


def test_planted_mistake_taylor_half(monkeypatch):
    def bad(phi, d, dx, dy):
        return phi + dx * d[0] + dy * d[1] + (dx * dx * d[2] + 2.0 * dx * dy * d[3] + dy * dy * d[4])

    monkeypatch.setattr(ale, "taylor2", bad)
    pb, pos_k, mask_k, pos_k1, mask_k1, bodies = moving_step()
    W = mls.build_weights(pb.mesh, pos_k, mask_k)
    c = (0.3, -0.7, 0.4, 1.3, -0.9, 0.6)
    got, _f = ale.ale_interpolate(pb.mesh, pos_k, pos_k1, mask_k, mask_k1,
                                  quad(pos_k[0], pos_k[1], c), W, bodies)
    inner1 = mask_k1 == -1
    assert np.abs(got[inner1] - quad(pos_k1[0], pos_k1[1], c)[inner1]).max() > 1e-6


def test_planted_mistake_shift_into_body(monkeypatch):
    orig = ale.shifted_centre
    monkeypatch.setattr(ale, "shifted_centre", lambda mesh, k, nx, ny: orig(mesh, k, -nx, -ny))
    pb, pos_k, mask_k, pos_k1, mask_k1, bodies = moving_step()
    W = mls.build_weights(pb.mesh, pos_k, mask_k)
    c = (0.3, -0.7, 0.4, 1.3, -0.9, 0.6)
    got, fallbacks = ale.ale_interpolate(pb.mesh, pos_k, pos_k1, mask_k, mask_k1,
                                         quad(pos_k[0], pos_k[1], c), W, bodies)
    inner1 = mask_k1 == -1
    assert fallbacks > 0
    assert np.abs(got[inner1] - quad(pos_k1[0], pos_k1[1], c)[inner1]).max() > 1e-6


def body_state(n):
    """Disc of Neumann boundary DPs (id 2), R = 0.2, in the unit box."""
    pb = inputs.jittered_box(n, 2, 5)
    c, R = (0.5 + 0.013, 0.5 - 0.007), 0.2
    pos, mask, _ = omask.update_dps(pb.mesh, pb.pos, pb.mask, c, R, band=0.0, n_relax=6)
    normal = omask.circle_normals(pos, mask, c, 2)
    return pb.mesh, pos, mask, normal, R


def force(n, P_fn, gradP, u_fn, v_fn, mu):
    mesh, pos, mask, normal, R = body_state(n)
    bc = inputs.default_bc_kind(neumann_ids=(2,))
    Wp = mls.build_weights(mesh, pos, mask, normal, bc)
    Wv = mls.build_weights(mesh, pos, mask)
    x, y = pos
    P = P_fn(x, y)
    dPn = gradP[0] * normal[0] + gradP[1] * normal[1]
    bnd_p = np.where(mask == 2, dPn, np.where(mask == 1, P, 0.0))
    F, perim, skipped = ale.fluid_force(mesh, pos, mask, 2, normal, P, bnd_p, u_fn(x, y), v_fn(x, y), mu,
                                        Wp, Wv)
    return F, perim, skipped, R


def test_pressure_force_and_perimeter_closed_forms():
    a = (0.7, -0.4)
    for n in (48, 96):
        F, perim, skipped, R = force(n, lambda x, y: 0.3 + a[0] * x + a[1] * y, a,
                                     lambda x, y: 0 * x, lambda x, y: 0 * x, 0.0)
        assert skipped == 0
        want = -np.array(a) * math.pi * R * R
        assert np.abs(F - want).max() <= 2e-3 * np.abs(want).max()
        assert abs(perim - 2 * math.pi * R) <= 2e-3 * 2 * math.pi * R


def test_viscous_force_closed_form():
    mu, al, be = 0.03, 1.3, -0.8
    for n in (48, 96):
        F, _perim, skipped, R = force(n, lambda x, y: 0 * x, (0.0, 0.0),
                                      lambda x, y: al * x * x, lambda x, y: be * x * x, mu)
        assert skipped == 0
        want = mu * math.pi * R * R * np.array([4 * al, 2 * be])
        assert np.abs(F - want).max() <= 2e-3 * np.abs(want).max()


def test_planted_mistake_surface_element(monkeypatch):
    orig = ale.boundary_neighbours

    def doubled(mesh, pos, mask, k, n):
        (j1, d1), (j2, d2) = orig(mesh, pos, mask, k, n)
        return (j1, 2 * d1), (j2, 2 * d2)

    monkeypatch.setattr(ale, "boundary_neighbours", doubled)
    _F, perim, _s, R = force(48, lambda x, y: 0 * x, (0.0, 0.0), lambda x, y: 0 * x, lambda x, y: 0 * x, 0.0)
    assert abs(perim - 2 * math.pi * R) / (2 * math.pi * R) > 0.5
