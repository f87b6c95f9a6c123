"""Pins of the oracle's bodies given by a discrete SDF (Sec. 2.5).

  * the lattice fit weights equal their closed form (on the symmetric 3x3
    lattice the fit decouples: psi_X = sum w X dpsi / sum w X^2, psi_XY =
    sum w X Y dpsi / sum w X^2 Y^2, and a 2x2 system for psi_XX, psi_YY);
  * a quadratic sampled on the grid is reproduced exactly, with its
    gradient, at any point, for a translated and rotated body;
  * the circle's SDF is interpolated to third order in the grid spacing;
  * masks from the SDF grid of a circle, and of a rotated ellipse, equal the
    masks of the exact shape except at vertices within rounding of the
    boundary; relocated boundary DPs sit on psi = 0 to within the one
    projection step of Eq. (9);
  * a planted mistake (rotation by -theta instead of theta) fails a pin.
"""
import math

import numpy as np
import pytest

from oracle import mask as omask
from oracle import sdf
from paper_2404_17542_gb300 import inputs


def closed_form_weights(r_e=2.5):
    wa = math.cos(math.pi * 1.0 / (2 * r_e)) ** 2
    wd = math.cos(math.pi * math.sqrt(2.0) / (2 * r_e)) ** 2
    a = (2 * wa + 4 * wd) / 4.0
    b = wd
    Z = np.zeros((5, 9))
    for dj in (-1, 0, 1):
        for di in (-1, 0, 1):
            if di == 0 and dj == 0:
                continue
            s = (di + 1) + 3 * (dj + 1)
            w = wa if di == 0 or dj == 0 else wd
            Z[0, s] = w * di / (2 * wa + 4 * wd)
            Z[1, s] = w * dj / (2 * wa + 4 * wd)
            Z[3, s] = w * di * dj / (4 * wd)
            r1, r3 = w * di * di / 2.0, w * dj * dj / 2.0
            Z[2, s] = (a * r1 - b * r3) / (a * a - b * b)
            Z[4, s] = (a * r3 - b * r1) / (a * a - b * b)
    return Z


def test_lattice_weights_closed_form():
    assert np.allclose(sdf.lattice_fit_weights(), closed_form_weights(), rtol=1e-13, atol=1e-14)


def quad_local(x, y):
    return 0.2 - 0.5 * x + 0.3 * y + 0.9 * x * x - 0.6 * x * y + 0.4 * y * y


@pytest.mark.parametrize("theta", [0.0, 0.37, -2.1])
def test_quadratic_reproduced_anywhere(theta):
    h = 0.05
    grid = inputs.sample_sdf_grid(quad_local, (-1.0, -1.0), h, (41, 41))
    c = (0.31, -0.12)
    body = sdf.SdfBody(2, c, theta, grid, (-1.0, -1.0), h)
    rng = np.random.default_rng(1)
    ct, st = math.cos(theta), math.sin(theta)
    for _ in range(200):
        xl, yl = rng.uniform(-0.9, 0.9, size=2)
        x, y = c[0] + ct * xl - st * yl, c[1] + st * xl + ct * yl     # world point
        psi, g = body.eval(x, y)
        assert psi == pytest.approx(quad_local(xl, yl), abs=1e-12)
        gxl, gyl = -0.5 + 1.8 * xl - 0.6 * yl, 0.3 - 0.6 * xl + 0.8 * yl
        assert g[0] == pytest.approx(ct * gxl - st * gyl, abs=1e-11)
        assert g[1] == pytest.approx(st * gxl + ct * gyl, abs=1e-11)
    assert body.eval(c[0] + 2.0, c[1])[0] == math.inf   # outside the grid


def test_circle_sdf_third_order():
    R = 0.3
    rng = np.random.default_rng(2)
    pts = [(r * math.cos(a), r * math.sin(a)) for r, a in zip(rng.uniform(0.2, 0.5, 100),
                                                            rng.uniform(0, 2 * math.pi, 100))]
    errs = []
    for h in (0.04, 0.02):
        n = int(round(1.6 / h)) + 1
        body = sdf.SdfBody(2, (0.0, 0.0), 0.0, inputs.sample_sdf_grid(inputs.circle_sdf(R), (-0.8, -0.8), h, (n, n)),
                           (-0.8, -0.8), h)
        errs.append(max(abs(body.eval(x, y)[0] - (math.hypot(x, y) - R)) for x, y in pts))
    assert errs[1] < errs[0] / 6.0        # third order: a factor of 8
    assert errs[1] < 1e-4


def exact_vertex_psi(mesh, psi_world):
    nx, ny = mesh.n[0], mesh.n[1]
    return np.array([[psi_world(i * mesh.l0, j * mesh.l0) for j in range(ny + 1)] for i in range(nx + 1)])


def mask_vs_exact(mesh, bodies, psi_world, tol):
    new = omask.remask_bodies(mesh, np.full(mesh.N, -1, dtype=np.int8), bodies, band=0.0)
    ex = exact_vertex_psi(mesh, psi_world)
    nx = mesh.n[0]
    bad = 0
    for j in range(1, mesh.n[1] - 1):
        for i in range(1, nx - 1):
            v = [ex[i, j], ex[i + 1, j], ex[i, j + 1], ex[i + 1, j + 1]]
            cnt = sum(x >= 0 for x in v)
            want = 0 if cnt <= 1 else (2 if cnt <= 3 else -1)
            if new[i + nx * j] != want:
                assert min(abs(x) for x in v) < tol    # only at near-ties
                bad += 1
    return new, bad


def test_sdf_circle_masks_match_exact_circle():
    mesh = inputs.Mesh(dim=2, n=(64, 64, 1), l0=1.0 / 64)
    c, R = (0.503, 0.488), 0.21
    h = mesh.l0 / 4
    n = int(round(0.6 / h)) + 1
    body = sdf.SdfBody(2, c, 0.0, inputs.sample_sdf_grid(inputs.circle_sdf(R), (-0.3, -0.3), h, (n, n)),
                       (-0.3, -0.3), h)
    new, bad = mask_vs_exact(mesh, [body], lambda x, y: math.hypot(x - c[0], y - c[1]) - R, 1e-6)
    assert bad <= 2 and (new == 2).sum() > 40


def ellipse_body(theta, h=None, flip=False):
    a, b = 0.25, 0.12
    mesh = inputs.Mesh(dim=2, n=(64, 64, 1), l0=1.0 / 64)
    h = mesh.l0 / 4 if h is None else h
    n = int(round(0.8 / h)) + 1
    grid = inputs.sample_sdf_grid(inputs.ellipse_sdf(a, b), (-0.4, -0.4), h, (n, n))
    c = (0.51, 0.47)
    body = sdf.SdfBody(2, c, -theta if flip else theta, grid, (-0.4, -0.4), h)
    f = inputs.ellipse_sdf(a, b)
    ct, st = math.cos(theta), math.sin(theta)

    def psi_world(x, y):
        dx, dy = x - c[0], y - c[1]
        return float(f(ct * dx + st * dy, -st * dx + ct * dy))
    return mesh, body, psi_world


def test_rotated_ellipse_masks_and_relocation():
    mesh, body, psi_world = ellipse_body(0.6)
    new, bad = mask_vs_exact(mesh, [body], psi_world, 1e-5)
    assert bad <= 2
    pb = inputs.jittered_box(64, 2, seed=3)
    pos, m, _ = omask.update_dps_bodies(mesh, pb.pos, pb.mask, [body], n_relax=4, band=0.0)
    nx = mesh.n[0]
    onb = 0
    for k in np.nonzero(m == 2)[0]:
        i, j = k % nx, k // nx
        x, y = pos[:, k]
        inside = (i * mesh.l0 < x < (i + 1) * mesh.l0) and (j * mesh.l0 < y < (j + 1) * mesh.l0)
        if inside:
            # not clamped: relocated onto psi = 0 by Eq. (9), one step
            # x + psi d^; exact for a distance function, here within
            # 5e-4 l0 because the ellipse function's |grad psi| is 1 only
            # on the boundary
            assert abs(psi_world(x, y)) < 2e-3 * mesh.l0
            onb += 1
    assert onb > 20


def test_planted_mistake_rotation_sign():
    mesh, body, psi_world = ellipse_body(0.6, flip=True)
    new = omask.remask_bodies(mesh, np.full(mesh.N, -1, dtype=np.int8), [body], band=0.0)
    bad = 0
    ex = exact_vertex_psi(mesh, psi_world)
    nx = mesh.n[0]
    for j in range(1, mesh.n[1] - 1):
        for i in range(1, nx - 1):
            v = [ex[i, j], ex[i + 1, j], ex[i, j + 1], ex[i + 1, j + 1]]
            cnt = sum(x >= 0 for x in v)
            want = 0 if cnt <= 1 else (2 if cnt <= 3 else -1)
            bad += new[i + nx * j] != want
    assert bad > 20
