"""Pins of the oracle's rigid-body kinematics (Sec. 2.5, Eqs. (24)-(29)):
the velocity and acceleration it gives a body's boundary DPs, against the
trajectory of material points of a moving, rotating body.

  * boundary_velocity, V + omega x (x - c), equals the time derivative of a
    material point x(t) = c(t) + R(theta(t)) r0, taken by central
    differences of the trajectory itself;
  * rigid_acceleration, from the finite differences of V and omega over a
    step (Eq. (29)) plus -omega^2 r, converges at first order in the step
    to the second time derivative of the trajectory;
  * a planted mistake (the centripetal term with the wrong sign, or the
    angular acceleration dropped) does not converge.
"""
import math

import numpy as np

from oracle import ale


def centre(t):
    return np.array([0.5 + 0.1 * math.sin(3.0 * t), 0.4 + 0.05 * math.cos(2.0 * t)])


def centre_dot(t):
    return np.array([0.3 * math.cos(3.0 * t), -0.1 * math.sin(2.0 * t)])


def theta(t):
    return 0.3 + 0.7 * math.sin(1.7 * t)


def theta_dot(t):
    return 1.19 * math.cos(1.7 * t)


R0 = np.array([[0.12, -0.05, 0.0, 0.08, -0.11],
               [0.02, 0.09, -0.13, -0.07, -0.01]])   # material points in the body frame


def material(t):
    c, s = math.cos(theta(t)), math.sin(theta(t))
    return centre(t)[:, None] + np.array([[c, -s], [s, c]]) @ R0


def test_boundary_velocity_is_the_material_derivative():
    t, h = 0.37, 1e-6
    x = material(t)
    fd = (material(t + h) - material(t - h)) / (2.0 * h)
    mask = np.full(x.shape[1], 2, dtype=np.int8)
    ubc, vbc = ale.boundary_velocity(mask, [(2, tuple(centre_dot(t)), theta_dot(t), tuple(centre(t)))], x)
    assert np.abs(ubc - fd[0]).max() <= 1e-8 and np.abs(vbc - fd[1]).max() <= 1e-8
    # without rotation terms the same DPs move with the centre only
    ubc0, vbc0 = ale.boundary_velocity(mask, [(2, tuple(centre_dot(t)))], x)
    assert np.allclose(ubc0, centre_dot(t)[0]) and np.allclose(vbc0, centre_dot(t)[1])


def acceleration_errors(accel):
    t1 = 0.61
    h = 1e-4
    exact = (material(t1 + h) - 2.0 * material(t1) + material(t1 - h)) / (h * h)
    errs = []
    for dt in (1e-2, 5e-3, 2.5e-3):
        t0 = t1 - dt
        ax, ay = accel(material(t1), centre(t1), centre_dot(t0), centre_dot(t1), theta_dot(t0),
                       theta_dot(t1), dt)
        errs.append(max(np.abs(ax - exact[0]).max(), np.abs(ay - exact[1]).max()))
    return errs, np.abs(exact).max()


def converges_first_order(accel):
    errs, scale = acceleration_errors(accel)
    ratios = [errs[0] / errs[1], errs[1] / errs[2]]
    return all(1.6 <= r <= 2.4 for r in ratios) and errs[-1] <= 0.02 * scale


def test_rigid_acceleration_converges_to_the_material_acceleration():
    assert converges_first_order(ale.rigid_acceleration)


def test_planted_mistakes_do_not_converge():
    def wrong_centripetal(pos, c, V0, V1, om0, om1, dt):
        ax, ay = ale.rigid_acceleration(pos, c, V0, V1, om0, om1, dt)
        return ax + 2.0 * om1 * om1 * (pos[0] - c[0]), ay + 2.0 * om1 * om1 * (pos[1] - c[1])

    def no_angular_acceleration(pos, c, V0, V1, om0, om1, dt):
        return ale.rigid_acceleration(pos, c, V0, V1, om1, om1, dt)

    assert not converges_first_order(wrong_centripetal)
    assert not converges_first_order(no_angular_acceleration)
