"""Pin of the oracle's moving-boundary step (oracle.ale.moving_step, the
composition of Sec. 3.3) against a closed form: a cylinder that starts to
accelerate in fluid at rest.

Set-up: u = 0 everywhere, the body's velocity is 0 at t_{k+1} and -a dt at
t_k, so dV/dt = a (Eq. (29)).  ALE, predict and the PPE source then vanish
(u* = 0), and the step's pressure solves Laplace's equation with
dP/dn = -a . n on the body (Eq. (23)) and P = 0 on the box walls.

Closed form (potential flow, unit density): a cylinder of radius R
accelerating at a along x through fluid at rest has the potential
phi = -U R^2 cos(theta) / r, and the linearised unsteady Bernoulli equation
gives P_inf = -d phi/dt = a R^2 cos(theta) / r.  It meets the Neumann datum
(dP_inf/dr = -a cos(theta) at r = R) and gives the added-mass force
F_x = -pi R^2 a.

Walls: the unit box centred on the body holds P = 0 instead of P_inf.  The
correction h is harmonic, h = -P_inf on the walls and dh/dn = 0 on the body.
Near the body h = c1 (r + R^2 / r) cos(theta) + O((R/L)^4), where c1 is the
x-gradient at the centre of the harmonic function of the square with wall
values -P_inf (a sine series of the square's Dirichlet problem, below).  So
    P = (a + c1) R^2 cos(theta) / r + c1 r cos(theta),
    F_x = -pi R^2 (a + 2 c1).
At R = 0.1, 2 c1 / a = -0.069: the wall term is far above the quadrature's
own error, and the test needs it.

Planted mistakes (in the oracle, on the CPU) that must fail: the datum's
sign, and normals taken from the step-k bodies of a translating body.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import ale, mls
from oracle import mask as omask
from paper_2404_17542_gb300 import inputs

R = 0.1        # cylinder radius (the box is the unit square)
A = 1.0        # body acceleration along x
DT = 1e-3
NU = 1e-3      # viscous traction ~ mu dt |lap P|: negligible here


def box_gradient(a, radius, terms=40):
    """c1 = dh0/dx at the centre of [-1/2, 1/2]^2, h0 harmonic with
    h0 = -a radius^2 x / r^2 on the walls: separation of variables, the left
    and right walls by sinh(k x) modes, top and bottom by cosh(k y) modes,
    k = n pi, sine coefficients by quadrature."""
    fr = lambda y: -a * radius * radius * 0.5 / (0.25 + y * y)     # wall x = +1/2  # noqa: E731
    ft = lambda x: -a * radius * radius * x / (x * x + 0.25)       # walls y = +-1/2  # noqa: E731
    c1 = 0.0
    for n in range(1, terms + 1):
        k = n * math.pi
        b = 2.0 * integrate.quad(lambda y: fr(y) * math.sin(k * (y + 0.5)), -0.5, 0.5, limit=200)[0]
        c = 2.0 * integrate.quad(lambda x: ft(x) * math.sin(k * (x + 0.5)), -0.5, 0.5, limit=200)[0]
        c1 += b * k / math.sinh(0.5 * k) * math.sin(0.5 * k)
        c1 += c * k / math.cosh(0.5 * k) * math.cos(0.5 * k)
    return c1


C1 = box_gradient(A, R)


def accelerating_step(n, shift_cells=0.0):
    """moving_step of the body accelerating from rest; at t_{k+1} its centre
    is the box centre, at t_k `shift_cells` cells to the left."""
    cyl = inputs.Cylinder(radius=R)
    pb = inputs.cylinder_box(n, cyl)
    mesh = pb.mesh
    bid = cyl.body_id
    bodies_k = [(bid, (0.5 - shift_cells * mesh.l0, 0.5), R)]
    bodies_k1 = [(bid, (0.5, 0.5), R)]
    pos, m, _ = omask.update_dps_bodies(mesh, pb.pos, pb.mask, bodies_k, 0.2, 30, 0.0)
    Wv = mls.build_weights(mesh, pos, m)
    z = np.zeros(mesh.N)
    return ale.moving_step(mesh, pos, m, z, z, Wv, bodies_k, bodies_k1, [(-A * DT, 0.0)], [(0.0, 0.0)],
                           DT, NU)


def errors(out):
    """(relative L2 error of P over the fluid DPs within 3R of the centre,
    relative error of F_x, |F_y| / |F_x|) against the closed form."""
    pos, m, P = out["pos"], out["mask"], out["P"]
    x, y = pos[0] - 0.5, pos[1] - 0.5
    r = np.hypot(x, y)
    cos_t = x / r
    want = (A + C1) * R * R * cos_t / r + C1 * r * cos_t
    sel = (m != 0) & (r < 3 * R)
    e_p = np.linalg.norm(P[sel] - want[sel]) / np.linalg.norm(want[sel])
    F = out["F"][2][0]
    F_want = -math.pi * R * R * (A + 2 * C1)
    return e_p, abs(F[0] - F_want) / abs(F_want), abs(F[1]) / abs(F[0])


@pytest.fixture(scope="module")
def coarse():
    return errors(accelerating_step(64, shift_cells=2.0))


def test_box_gradient_series_converged():
    # the series' terms decay like exp(-k/2): 20 more terms change nothing
    assert abs(box_gradient(A, R, 60) - C1) <= 1e-12 * abs(C1)
    assert -0.075 < 2 * C1 / A < -0.065   # the 6.9 % wall term quoted above


def test_moving_step_matches_added_mass_closed_form(coarse):
    e_p, e_f, e_fy = coarse
    assert e_p < 0.08, e_p
    assert e_f < 0.06, e_f
    assert e_fy < 1e-6, e_fy


@pytest.mark.slow
def test_moving_step_converges_to_closed_form(coarse):
    # at 128^2 the errors fall to about 2.0e-2 (pressure) and 1.4e-2
    # (force) from 5.4e-2 and 4.3e-2 at 64^2; without the wall term the
    # force would stay 5-6 % off at both sizes
    e_p, e_f, _ = errors(accelerating_step(128, shift_cells=2.0))
    assert e_p < 0.03 and e_f < 0.02, (e_p, e_f)
    assert e_p < 0.5 * coarse[0] and e_f < 0.5 * coarse[1]


def test_planted_datum_sign_is_caught(monkeypatch):
    exact = ale.rigid_acceleration
    monkeypatch.setattr(ale, "rigid_acceleration", lambda *a: tuple(-v for v in exact(*a)))
    e_p, e_f, _ = errors(accelerating_step(64, shift_cells=2.0))
    assert e_p > 0.5 and e_f > 0.5


def test_planted_step_k_normals_are_caught(monkeypatch):
    exact = omask.bodies_normals
    l0 = 1.0 / 64

    def step_k_normals(pos, mask, bodies):
        bid, (cx, cy), rad = bodies[0]
        return exact(pos, mask, [(bid, (cx - 2.0 * l0, cy), rad)])
    monkeypatch.setattr(omask, "bodies_normals", step_k_normals)
    e_p, _e_f, _ = errors(accelerating_step(64, shift_cells=2.0))
    assert e_p > 0.5
