"""Pins of the oracle's fractional-step driver (Sec. 3.3, Eqs. (20)-(22)).

  * MOC departure value: for a quadratic field the second-order Taylor
    expansion is exact, so F equals the field at x - u dt;
  * linear velocity: u* and div u* are known in closed form;
  * projection: the pressure gradient (with Neumann data) is exact for a
    quadratic pressure;
  * Taylor-Green vortex: the error against the closed form falls with
    refinement.
"""
import math
import os
import sys

import numpy as np
import pytest

from oracle import flow, mls
from paper_2404_17542_gb300 import inputs

sys.path.insert(0, os.path.dirname(__file__))
from test_oracle_mls import cylinder_fixture  # noqa: E402


def quad(c, x, y):
    return c[0] + c[1] * x + c[2] * y + c[3] * x * x + c[4] * x * y + c[5] * y * y


def lap_quad(c):
    return 2 * c[3] + 2 * c[5]


def test_moc_is_exact_for_quadratic_fields():
    pb = inputs.jittered_box(12, 2, seed=7)
    x, y = pb.pos
    rng = np.random.default_rng(1)
    cu, cv = rng.uniform(-1, 1, 6), rng.uniform(-1, 1, 6)
    u, v = quad(cu, x, y), quad(cv, x, y)
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    dt, nu = 0.013, 0.02
    us, vs, _src = flow.predict(pb.mesh, W, u, v, u, v, nu, dt, pb.mask)
    inner = pb.mask == -1
    xd, yd = x - u * dt, y - v * dt
    want_u = quad(cu, xd, yd) + nu * dt * lap_quad(cu)
    want_v = quad(cv, xd, yd) + nu * dt * lap_quad(cv)
    assert np.abs(us[inner] - want_u[inner]).max() <= 1e-10
    assert np.abs(vs[inner] - want_v[inner]).max() <= 1e-10
    assert np.array_equal(us[~inner], u[~inner])


def test_linear_velocity_divergence_closed_form():
    pb = inputs.jittered_box(12, 2, seed=8)
    x, y = pb.pos
    a, b, c, d, e, f = 0.3, 0.7, -0.2, -0.1, 0.4, 0.25
    u = a + b * x + c * y
    v = d + e * x + f * y
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    dt = 0.01
    us, vs, src = flow.predict(pb.mesh, W, u, v, u, v, 0.0, dt, pb.mask)
    # u* = u - dt (u u_x + v u_y) is linear: its divergence is closed form
    inner = pb.mask == -1
    want_us = u - dt * (u * b + v * c)
    want_vs = v - dt * (u * e + v * f)
    assert np.abs(us[inner] - want_us[inner]).max() <= 1e-12
    assert np.abs(vs[inner] - want_vs[inner]).max() <= 1e-12
    # only inner DPs whose whole stencil is inner see a linear u* field
    nbr = flow.neighbour_table(pb.mesh)
    deep = inner & np.all(inner[nbr], axis=0)
    # div u* = d/dx[u - dt(u b + v c)] + d/dy[v - dt(u e + v f)]
    dux = b - dt * (b * b + e * c)
    dvy = f - dt * (c * e + f * f)
    assert np.abs(src[deep] - (dux + dvy) / dt).max() <= 1e-9


def test_projection_gradient_with_neumann_data_is_exact():
    pb, mask, normal, bc = cylinder_fixture(n=24, jitter_seed=8)
    x, y = pb.pos
    cp = np.array([0.1, -0.3, 0.5, 0.2, -0.4, 0.3])
    P = quad(cp, x, y)
    gx = cp[1] + 2 * cp[3] * x + cp[4] * y
    gy = cp[2] + cp[4] * x + 2 * cp[5] * y
    f = normal[0] * gx + normal[1] * gy
    bnd = np.where(mask == 2, f, np.where(mask == 1, P, 0.0))
    W = mls.build_weights(pb.mesh, pb.pos, mask, normal, bc)
    us = np.full(pb.mesh.N, 0.7)
    vs = np.full(pb.mesh.N, -0.2)
    dt = 0.05
    un, vn = flow.project(pb.mesh, W, P, bnd, us, vs, us, vs, dt, mask)
    inner = mask == -1
    assert np.abs(un[inner] - (0.7 - dt * gx[inner])).max() <= 1e-9
    assert np.abs(vn[inner] - (-0.2 - dt * gy[inner])).max() <= 1e-9


def tgv_error(n, steps):
    pb = inputs.tgv_box(n, seed=1)
    nu = pb.meta["nu"]
    u, v = pb.meta["u"].copy(), pb.meta["v"].copy()
    dt = 0.2 * pb.mesh.l0
    t = 0.0
    for _ in range(steps):
        t += dt
        ue, ve, pe = inputs.tgv_fields(pb.pos, t, nu)
        u, v, P = flow.step(pb.mesh, pb.pos, pb.mask, u, v, ue, ve, pe, nu, dt)
    ue, ve, pe = inputs.tgv_fields(pb.pos, t, nu)
    eu = np.sqrt(np.mean((u - ue) ** 2 + (v - ve) ** 2)) / np.sqrt(np.mean(ue ** 2 + ve ** 2))
    return eu


@pytest.mark.slow
def test_taylor_green_error_falls_with_refinement():
    e16 = tgv_error(16, 4)
    e32 = tgv_error(32, 8)
    assert e32 < 0.7 * e16, (e16, e32)
    assert e32 < 0.05
