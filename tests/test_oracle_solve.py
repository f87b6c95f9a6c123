"""Pins of the oracle's PPE assembly and Bi-CGSTAB (Sec. 3.3).

  * Bi-CGSTAB and the sparse direct solve agree with dense LU (numpy);
  * the discrete solution is exact where the MLS fit is exact (quadratic
    data in a Dirichlet box; linear data with Neumann bodies);
  * manufactured u = sin(pi x) sin(pi y): the error decays at order >= 1.5.
"""
import math
import sys
import os

import numpy as np
import pytest

from oracle import mls, solve
from paper_2404_17542_gb300 import inputs

sys.path.insert(0, os.path.dirname(__file__))
from test_oracle_mls import cylinder_fixture  # noqa: E402


def system(pb, mask=None, normal=None, bc=None, rhs=None, bnd=None):
    mask = pb.mask if mask is None else mask
    W = mls.build_weights(pb.mesh, pb.pos, mask, normal, bc)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"],
                       pb.rhs if rhs is None else rhs,
                       pb.bnd if bnd is None else bnd, W["rscale"])
    return W, A, b


@pytest.mark.parametrize("n", [8, 16])
def test_bicgstab_matches_dense_lu(n):
    pb = inputs.manufactured_box(n, 2, seed=n)
    _W, A, b = system(pb)
    xd = np.linalg.solve(A.toarray(), b)
    x, it, rel = solve.bicgstab(A, b, tol=1e-12)
    assert rel <= 1e-12
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    xs = solve.direct_solve(A, b)
    assert np.linalg.norm(xs - xd) <= 1e-12 * np.linalg.norm(xd)


def test_bicgstab_matches_dense_lu_with_neumann_body():
    pb, mask, normal, bc = cylinder_fixture(n=20, jitter_seed=3)
    rng = np.random.default_rng(0)
    rhs = np.where(mask == -1, rng.normal(size=pb.mesh.N), 0.0)
    bnd = np.where(mask == 2, rng.normal(size=pb.mesh.N), 0.0)
    _W, A, b = system(pb, mask, normal, bc, rhs, bnd)
    xd = np.linalg.solve(A.toarray(), b)
    x, it, rel = solve.bicgstab(A, b, tol=1e-12)
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_quadratic_solution_is_exact_in_dirichlet_box():
    pb = inputs.jittered_box(12, 2, seed=4)
    x, y = pb.pos
    u = 0.3 + 0.5 * x - 0.2 * y + 0.7 * x * x - 0.4 * x * y + 0.9 * y * y
    f = np.full(pb.mesh.N, 2 * 0.7 + 2 * 0.9)
    _W, A, b = system(pb, rhs=f, bnd=np.where(pb.mask >= 1, u, 0.0))
    xs = solve.direct_solve(A, b)
    assert np.abs(xs - u).max() <= 1e-11


def test_linear_solution_is_exact_with_neumann_body():
    pb, mask, normal, bc = cylinder_fixture(n=24, jitter_seed=8)
    x, y = pb.pos
    g = np.array([0.8, -0.35])
    u = 0.1 + g[0] * x + g[1] * y
    bnd = np.where(mask == 1, u, 0.0) + np.where(mask == 2, normal[0] * g[0] + normal[1] * g[1], 0.0)
    W, A, b = system(pb, mask, normal, bc, np.zeros(pb.mesh.N), bnd)
    xs = solve.direct_solve(A, b)
    fluid = mask != 0
    assert np.abs(xs[fluid] - u[fluid]).max() <= 1e-10
    assert np.all(xs[~fluid] == 0.0)


def test_planted_mistake_in_rhs_sign():
    """Adding instead of subtracting the moved Neumann terms breaks exactness."""
    pb, mask, normal, bc = cylinder_fixture(n=24, jitter_seed=8)
    x, y = pb.pos
    g = np.array([0.8, -0.35])
    u = 0.1 + g[0] * x + g[1] * y
    bnd = np.where(mask == 1, u, 0.0) + np.where(mask == 2, normal[0] * g[0] + normal[1] * g[1], 0.0)
    W = mls.build_weights(pb.mesh, pb.pos, mask, normal, bc)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], -W["QL"], np.zeros(pb.mesh.N), bnd, W["rscale"])
    xs = solve.direct_solve(A, b)
    assert np.abs(xs[mask != 0] - u[mask != 0]).max() > 1e-3


def test_manufactured_convergence_order():
    errs = []
    ns = [16, 32, 64]
    for n in ns:
        pb = inputs.manufactured_box(n, 2, seed=0)
        _W, A, b = system(pb)
        xs = solve.direct_solve(A, b)
        errs.append(np.linalg.norm(xs - pb.exact) / np.linalg.norm(pb.exact))
    orders = [math.log(errs[k] / errs[k + 1], 2) for k in range(len(ns) - 1)]
    assert min(orders) >= 1.5, orders
