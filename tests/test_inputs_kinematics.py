"""The prescribed motions of the moving-body workloads are self-consistent:
each velocity is the time derivative of its position, each angular
velocity that of its posture angle, and the cylinder's acceleration that
of its velocity.  Derivatives are taken by central differences.  The
device driver and the oracle both take these motions as inputs, so a
sign slip here would go unnoticed by the parity tests.
"""
import math

import numpy as np
import pytest

from paper_2404_17542_gb300 import inputs

H = 1e-6
TIMES = (0.0, 0.37, 1.9, 4.2, 7.7)


def central(f, t):
    return (np.asarray(f(t + H)) - np.asarray(f(t - H))) / (2.0 * H)


@pytest.mark.parametrize("t", TIMES)
def test_oscillating_cylinder(t):
    cyl = inputs.Cylinder()
    assert np.allclose(cyl.velocity(t), central(cyl.centre, t), atol=1e-8)
    assert np.allclose(cyl.acceleration(t), central(cyl.velocity, t), atol=1e-6)


@pytest.mark.parametrize("t", TIMES + (15.9, 16.1, 23.5))
def test_passing_cylinders(t):
    cfg = inputs.PassingCylinders()
    if abs(t - 2 * cfg.T) < 10 * H:
        pytest.skip("the switch to constant speed")
    centres = lambda s: np.array([b[1] for b in cfg.bodies(s)[0]])   # noqa: E731
    vel = np.array(cfg.bodies(t)[1])
    assert np.allclose(vel, central(centres, t), atol=1e-8)
    # the two motions are opposite and the speed is continuous at 2 T
    assert np.allclose(vel[0], -vel[1])
    assert abs(cfg.x_offset(2 * cfg.T - 1e-9)[1] - cfg.x_offset(2 * cfg.T + 1e-9)[1]) < 1e-6


@pytest.mark.parametrize("t", TIMES)
def test_flapping_wing(t):
    w = inputs.FlappingWing()
    assert np.allclose(w.velocity(t), central(w.centre, t), atol=1e-8)
    assert abs(w.omega(t) - central(w.posture, t)) < 1e-8
    # the stroke runs along the plane at beta, between a = 0 and a = a0
    c = np.array(w.centre(t))
    assert abs(c[1] * math.cos(w.beta) - c[0] * math.sin(w.beta)) < 1e-12
    assert -1e-12 <= w.a(t) <= w.a0 + 1e-12
