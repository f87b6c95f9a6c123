"""Pins of the oracle's DP masking and arrangement (Sec. 2.2-2.4).

  * vertex classification checked in exact rational arithmetic;
  * mask invariants of Eq. (1) and of the band rule of Sec. 2.4;
  * spring relaxation: regular-lattice fixed point and the closed-form
    linear response of Eqs. (5)-(8);
  * boundary DPs on the circle after relocation (Eq. (9)) unless clamped.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import mask as omask
from paper_2404_17542_gb300 import inputs


def exact_fluid(mesh, centre, radius):
    """psi >= 0 at every vertex, decided in exact rational arithmetic."""
    nx, ny = mesh.n[0], mesh.n[1]
    l0 = Fraction(mesh.l0)
    cx, cy, R = Fraction(centre[0]), Fraction(centre[1]), Fraction(radius)
    out = np.zeros((nx + 1, ny + 1), dtype=bool)
    for i in range(nx + 1):
        for j in range(ny + 1):
            dx = i * l0 - cx
            dy = j * l0 - cy
            out[i, j] = dx * dx + dy * dy >= R * R
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_vertex_classification_matches_exact_arithmetic(seed):
    rng = np.random.default_rng(seed)
    mesh = inputs.Mesh(dim=2, n=(40, 40, 1), l0=1.0 / 40)
    c = (0.5 + rng.uniform(-0.05, 0.05), 0.5 + rng.uniform(-0.05, 0.05))
    R = rng.uniform(0.1, 0.3)
    fl = omask.vertex_fluid(mesh, c, R)
    ex = exact_fluid(mesh, c, R)
    # FP64 and exact decisions may differ only at near-ties
    diff = np.argwhere(fl != ex)
    for i, j in diff:
        d2 = (i * mesh.l0 - c[0]) ** 2 + (j * mesh.l0 - c[1]) ** 2
        assert abs(d2 - R * R) < 1e-14
    assert len(diff) <= 1


def test_mask_rule_of_eq1():
    mesh = inputs.Mesh(dim=2, n=(32, 32, 1), l0=1.0 / 32)
    c, R = (0.47, 0.52), 0.23
    m = np.full(mesh.N, -1, dtype=np.int8)
    new = omask.remask(mesh, m, c, R, 2, band=0.0)
    ex = exact_fluid(mesh, c, R)
    for j in range(1, 31):
        for i in range(1, 31):
            cnt = int(ex[i, j]) + int(ex[i + 1, j]) + int(ex[i, j + 1]) + int(ex[i + 1, j + 1])
            want = 0 if cnt <= 1 else (2 if cnt <= 3 else -1)
            assert new[i + 32 * j] == want
    # the boundary ring is closed around the body: every void cell has no
    # inner neighbour (4-neighbourhood)
    for j in range(1, 31):
        for i in range(1, 31):
            if new[i + 32 * j] == 0:
                for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                    assert new[(i + di) + 32 * (j + dj)] != -1


def test_band_limits_changes():
    pb = inputs.cylinder_box(48)
    cyl = pb.meta["cylinder"]
    c0 = cyl.centre(0.0)
    pos, m, _ = omask.update_dps(pb.mesh, pb.pos, pb.mask, c0, cyl.radius,
                                 band=0.0, n_relax=2)
    c1 = cyl.centre(0.02)
    band = 5 * pb.mesh.l0
    pos2, m2, prev = omask.update_dps(pb.mesh, pos, m, c1, cyl.radius,
                                      band=band, n_relax=2)
    assert (prev == m).all()
    changed = np.nonzero(m2 != m)[0]
    assert len(changed) > 0
    moved = np.nonzero(np.any(pos2 != pos, axis=0))[0]
    cent = pb.mesh.centroids()
    for k in np.concatenate([changed, moved]):
        d = math.hypot(cent[0, k] - c1[0], cent[1, k] - c1[1]) - cyl.radius
        assert abs(d) < band


def test_every_dp_inside_its_cell_and_on_boundary():
    pb = inputs.cylinder_box(40)
    cyl = pb.meta["cylinder"]
    c = cyl.centre(0.013)
    pos, m, _ = omask.update_dps(pb.mesh, pb.pos, pb.mask, c, cyl.radius,
                                 band=0.0, n_relax=6)
    ijk = pb.mesh.cell_ijk()
    l0 = pb.mesh.l0
    lo = ijk * l0
    assert np.all(pos >= lo - 1e-15) and np.all(pos <= lo + l0 + 1e-15)
    on = 0
    for k in np.nonzero(m == 2)[0]:
        d = math.hypot(pos[0, k] - c[0], pos[1, k] - c[1])
        on_edge = np.any(np.isclose(pos[:, k], lo[:, k], atol=1e-15, rtol=0) |
                         np.isclose(pos[:, k], lo[:, k] + l0, atol=1e-15, rtol=0))
        if abs(d - cyl.radius) < 1e-12:
            on += 1
        else:
            assert on_edge
    assert on > 0.5 * (m == 2).sum()


def test_regular_lattice_is_a_fixed_point():
    """Far from any boundary F = 0 exactly on the lattice (Eqs. (6)-(7))."""
    mesh = inputs.Mesh(dim=2, n=(12, 12, 1), l0=1.0 / 12)
    pos = mesh.centroids()
    m = np.full(mesh.N, -1, dtype=np.int8)
    movable = np.ones(mesh.N, dtype=bool)
    new = omask.relax_sweep(mesh, pos, m, movable, (5.0, 5.0), 0.1, 2, 0.2)
    assert np.abs(new - pos).max() <= 1e-15


def test_linear_response_closed_form():
    """A DP displaced by delta along x on the lattice moves back to
    delta (1 - kappa (2 + sqrt 2)): axis springs give 2 delta / l0 and the
    four diagonal springs (natural length sqrt(2) l0) give sqrt(2) delta / l0.
    """
    mesh = inputs.Mesh(dim=2, n=(5, 5, 1), l0=0.1)
    pos = mesh.centroids()
    k = 2 + 5 * 2
    delta = 1e-7 * mesh.l0
    pos[0, k] += delta
    m = np.full(mesh.N, -1, dtype=np.int8)
    movable = np.zeros(mesh.N, dtype=bool)
    movable[k] = True
    kappa = 0.2
    new = omask.relax_sweep(mesh, pos, m, movable, (50.0, 50.0), 0.1, 2, kappa)
    ratio = (new[0, k] - mesh.centroids()[0, k]) / delta
    assert ratio == pytest.approx(1 - kappa * (2 + math.sqrt(2)), rel=1e-5)
    assert abs(new[1, k] - pos[1, k]) < 1e-12 * mesh.l0


def test_planted_mistake_natural_length(monkeypatch):
    """Using l0 instead of sqrt(2) l0 for diagonal springs breaks the pin."""
    mesh = inputs.Mesh(dim=2, n=(12, 12, 1), l0=1.0 / 12)
    pos = mesh.centroids()
    m = np.full(mesh.N, -1, dtype=np.int8)
    movable = np.ones(mesh.N, dtype=bool)
    real_sqrt = math.sqrt

    class FakeMath:
        def __getattr__(self, name):
            return getattr(math, name)

        @staticmethod
        def sqrt(x):
            return 1.0 if x == 2.0 else real_sqrt(x)

    monkeypatch.setattr(omask, "math", FakeMath())
    new = omask.relax_sweep(mesh, pos, m, movable, (5.0, 5.0), 0.1, 2, 0.2)
    assert np.abs(new - pos).max() > 1e-6


def test_boundary_fitted_move_shape():
    """Sec. 4.7 (Eqs. (45)-(46)) with the spring forces off (kappa = 0):
    an inner DP within r_e of the body moves along the ray to the centre,
    towards the body, by at most alpha psi; the relative pull is close to
    alpha next to the surface, falls with the distance and is nearly 0 at
    r_e; DPs at psi >= r_e stay put."""
    from oracle import mask as om
    n = 64
    pb = inputs.jittered_box(n, 2, seed=11, jitter=0.0)
    mesh = pb.mesh
    c, R = (0.5, 0.5), 0.1
    mask = om.remask(mesh, pb.mask, c, R, 2, 0.0)
    movable = mask == -1
    alpha, r_e = 0.03, 5.0 * mesh.l0
    new = om.relax_sweep(mesh, pb.pos, mask, movable, c, R, 2, 0.0, alpha=alpha)
    d0 = pb.pos - np.array(c)[:, None]
    d1 = new - np.array(c)[:, None]
    psi0 = np.hypot(*d0) - R
    psi1 = np.hypot(*d1) - R
    near = movable & (psi0 < r_e) & (psi0 > 0)
    far = movable & (psi0 >= r_e)
    assert near.sum() > 100 and far.sum() > 100
    assert np.array_equal(new[:, far], pb.pos[:, far])
    cross = d0[0] * d1[1] - d0[1] * d1[0]
    assert np.abs(cross[near]).max() <= 1e-15                 # radial
    assert np.all(psi1[near] <= psi0[near])                   # towards the body
    assert np.all(psi0[near] - psi1[near] <= alpha * psi0[near] * (1 + 1e-12))
    pull = (psi0[near] - psi1[near]) / (alpha * psi0[near])
    order = np.argsort(psi0[near])
    assert pull[order[0]] > 0.9 and pull[order[-1]] < 0.05   # ~alpha near the surface, 0 at r_e
    assert np.all(np.diff(pull[order]) <= 1e-12)             # decreasing with distance
