"""Pins of the oracle's masking and arrangement with several bodies.

Sec. 2.5 of arXiv 2404.17542 takes, at each point, the SDF of the body with
the smallest magnitude; Sec. 2.2 gives each boundary its own mask id.
  * vertex classification of the 25-cylinder array against the union of
    discs decided in exact rational arithmetic (a different definition that
    coincides for disjoint circles);
  * every boundary cell carries the id of a circle that passes through it;
  * bodies whose bands are far apart: the joint update equals the
    single-body updates applied one after the other (reduces to the
    single-body oracle);
  * a planted mistake (largest instead of smallest |psi|) fails the first pin.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import mask as omask
from paper_2404_17542_gb300 import inputs


def exact_union_fluid(mesh, bodies):
    """Vertex (i, j) lies outside every disc, in exact rational arithmetic."""
    nx, ny = mesh.n[0], mesh.n[1]
    l0 = Fraction(mesh.l0)
    discs = [(Fraction(c[0]), Fraction(c[1]), Fraction(R)) for _bid, c, R in bodies]
    out = np.ones((nx + 1, ny + 1), dtype=bool)
    for i in range(nx + 1):
        for j in range(ny + 1):
            x, y = i * l0, j * l0
            for cx, cy, R in discs:
                if (x - cx) ** 2 + (y - cy) ** 2 < R * R:
                    out[i, j] = False
                    break
    return out


def near_tie(mesh, bodies, i, j):
    x, y = i * mesh.l0, j * mesh.l0
    return any(abs((x - c[0]) ** 2 + (y - c[1]) ** 2 - R * R) < 1e-13 for _b, c, R in bodies)


@pytest.mark.parametrize("gap_cells", [12, 2])
def test_array_vertices_match_exact_union(gap_cells):
    pb = inputs.cylinder_array_box(64, gap_cells)
    bodies = pb.meta["bodies"]
    fl = omask.vertex_fluid_bodies(pb.mesh, bodies)
    ex = exact_union_fluid(pb.mesh, bodies)
    for i, j in np.argwhere(fl != ex):
        assert near_tie(pb.mesh, bodies, i, j)
    assert (fl != ex).sum() <= 2
    assert (~ex).sum() > 100   # the discs cover vertices


@pytest.mark.parametrize("gap_cells", [12, 2])
def test_array_masks_and_boundary_ids(gap_cells):
    pb = inputs.cylinder_array_box(64, gap_cells)
    bodies = pb.meta["bodies"]
    new = omask.remask_bodies(pb.mesh, pb.mask, bodies, band=0.0)
    ex = exact_union_fluid(pb.mesh, bodies)
    nx = pb.mesh.n[0]
    l0 = Fraction(pb.mesh.l0)
    seen = set()
    for j in range(1, nx - 1):
        for i in range(1, nx - 1):
            cnt = int(ex[i, j]) + int(ex[i + 1, j]) + int(ex[i, j + 1]) + int(ex[i + 1, j + 1])
            m = int(new[i + nx * j])
            if cnt <= 1:
                assert m == 0
            elif cnt == 4:
                assert m == -1
            else:
                # a vertex of the cell lies inside the circle whose id the cell carries
                bid, c, R = next(b for b in bodies if b[0] == m)
                cx, cy, RR = Fraction(c[0]), Fraction(c[1]), Fraction(R)
                inside = [(ii * l0 - cx) ** 2 + (jj * l0 - cy) ** 2 < RR * RR
                          for ii in (i, i + 1) for jj in (j, j + 1)]
                assert any(inside)
                seen.add(m)
    assert seen == {b[0] for b in bodies}   # every cylinder has a boundary ring


def test_far_bodies_equal_sequential_single_body_updates():
    mesh_pb = inputs.jittered_box(48, 2, seed=6)
    mesh = mesh_pb.mesh
    # two discs whose 5 l0 bands are far apart
    A = (2, (0.27, 0.29), 0.09)
    B = (3, (0.71, 0.68), 0.11)
    pos0, mask0 = mesh_pb.pos, mesh_pb.mask
    pj, mj, mpj = omask.update_dps_bodies(mesh, pos0, mask0, [A, B], n_relax=4, alpha=0.03)
    p1, m1, _ = omask.update_dps(mesh, pos0, mask0, A[1], A[2], body_id=A[0], n_relax=4, alpha=0.03)
    p2, m2, _ = omask.update_dps(mesh, p1, m1, B[1], B[2], body_id=B[0], n_relax=4, alpha=0.03)
    assert np.array_equal(mj, m2)
    assert np.array_equal(pj, p2)
    assert np.array_equal(mpj, mask0)
    assert (mj == 2).sum() > 10 and (mj == 3).sum() > 10


def test_planted_mistake_farthest_body(monkeypatch):
    def farthest(bodies, x, y):
        best, best_psi = 0, None
        for b, (_bid, c, R) in enumerate(bodies):
            psi = ((x - c[0]) ** 2 + (y - c[1]) ** 2) ** 0.5 - R
            if best_psi is None or abs(psi) > abs(best_psi):
                best, best_psi = b, psi
        return best, best_psi

    monkeypatch.setattr(omask, "nearest_body", farthest)
    pb = inputs.cylinder_array_box(64, 12)
    fl = omask.vertex_fluid_bodies(pb.mesh, pb.meta["bodies"])
    ex = exact_union_fluid(pb.mesh, pb.meta["bodies"])
    assert (fl != ex).sum() > 100
