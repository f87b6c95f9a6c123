"""Pins of the oracle's expanded 9x9 stencil (Sec. 4.1 of arXiv 2404.17542).

The multiple-cylinder experiment compares the chi=1 quadratic MLS fit on the
compact 3x3 support with the same fit on a 9x9 support, influence radius
r_e = 3.5 l0, least-squares MPS weight (1 - r/r_e)^2.
  * closed-form lattice weights of the Laplacian row over all 81 slots;
  * exact reproduction of quadratics, with and without Neumann data;
  * dense weighted least squares by QR on single stencils;
  * the discrete solution converges at order >= 1.5 and Bi-CGSTAB agrees
    with dense LU;
  * planted mistakes (weight, support range) make a pin fail.
"""
import math
import os
import sys

import numpy as np
import pytest

from oracle import mls, solve
from paper_2404_17542_gb300 import inputs

sys.path.insert(0, os.path.dirname(__file__))
from test_oracle_mls import (cylinder_fixture, phi_components, quad_eval,  # noqa: E402
                             quad_grad, random_quadratic)

R9 = 4            # support radius of the 9x9 stencil
RE9 = 3.5         # influence radius in units of l0 (Sec. 4.1)
TYPE_A = 2        # weight kind: (1 - r/r_e)^2 below r_e


def lattice_closed_form(r_e):
    """Laplacian weights (times l0^2) of the chi=1 quadratic fit on a regular
    2D lattice over the 9x9 support.  On a lattice with the square's
    symmetry all odd moments vanish, (1, 0, 1) is an eigenvector of the
    second-order moment block with eigenvalue sum_k w_k |X_k|^4 / 8, so the
    Laplacian weight of neighbour j is c_j = 4 w_j |X_j|^2 / sum_k w_k |X_k|^4
    and the centre weight is -sum_j c_j.  Slot s = (di + 4) + 9 (dj + 4)."""
    w = {}
    for dj in range(-R9, R9 + 1):
        for di in range(-R9, R9 + 1):
            r = math.hypot(di, dj)
            w[(di, dj)] = (1.0 - r / r_e) ** 2 if 0.0 < r < r_e else 0.0
    tot = sum(wk * (di * di + dj * dj) ** 2 for (di, dj), wk in w.items())
    row = np.zeros(81)
    for (di, dj), wk in w.items():
        row[(di + R9) + 9 * (dj + R9)] = 4.0 * wk * (di * di + dj * dj) / tot
    row[40] = -row.sum()
    return row


def lattice_row():
    pb = inputs.jittered_box(11, 2, 0, jitter=0.0, periodic=True)
    i = 5 + 11 * 5
    f = mls.dp_fit(pb.mesh, pb.pos, pb.mask, np.zeros((2, pb.mesh.N)),
                   inputs.default_bc_kind(), i, TYPE_A, RE9 * pb.mesh.l0, support=R9)
    return f["row"] * pb.mesh.l0 ** 2


def test_lattice_closed_form_all_slots():
    got = lattice_row()
    want = lattice_closed_form(RE9)
    assert np.abs(got - want).max() <= 1e-12 * np.abs(want).max()
    # slots beyond r_e carry no weight: (4, 3), (3, 4), (4, 4) and mirrors
    for di, dj in ((4, 3), (3, 4), (4, 4), (-4, 3), (4, -4)):
        assert got[(di + 4) + 9 * (dj + 4)] == 0.0
    # 3 l0 (axis) and (3, 1) are inside, with positive weight
    assert got[(3 + 4) + 9 * 4] > 0.0 and got[(3 + 4) + 9 * (1 + 4)] > 0.0


def test_type_a_weight_values():
    """w = (1 - r/r_e)^2 below r_e, 0 at and beyond it."""
    assert mls.weight(0.0, TYPE_A, 3.5) == 1.0
    assert mls.weight(1.75, TYPE_A, 3.5) == 0.25
    assert mls.weight(3.5, TYPE_A, 3.5) == 0.0
    assert mls.weight(4.0, TYPE_A, 3.5) == 0.0


def test_expanded_quadratic_reproduction():
    """The chi=1 quadratic fit is exact on quadratics on any support, also
    where walls truncate the 9x9 window."""
    pb = inputs.jittered_box(14, 2, seed=3)
    l0 = pb.mesh.l0
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask, weight_kind=TYPE_A, r_e=RE9 * l0, support=R9)
    assert W["row"].shape == (81, pb.mesh.N)
    rng = np.random.default_rng(11)
    for _ in range(2):
        q = random_quadratic(rng, 2)
        vals = np.array([quad_eval(q, pb.pos[:, k]) for k in range(pb.mesh.N)])
        for i in np.nonzero(W["kind"] == 1)[0]:
            nb = [j for _s, j, _o in mls.stencil_slots(pb.mesh, i, R9)]
            phi = np.array([vals[j] if j is not None else 0.0 for j in nb])
            want = phi_components(q, pb.pos[:, i], 2)
            assert np.abs(W["D"][:, :, i] @ phi - want).max() <= 1e-9 / l0 ** 2
            assert W["row"][:, i] @ phi == pytest.approx(np.trace(q[2]), abs=1e-9 / l0 ** 2)


def test_expanded_neumann_terms():
    """Consistent Neumann data keep the 9x9 fit exact (Eq. (15)); Neumann
    rows are exact on linear data with diagonal -1/l0^2."""
    pb, mask, normal, bc = cylinder_fixture()
    l0 = pb.mesh.l0
    W = mls.build_weights(pb.mesh, pb.pos, mask, normal, bc, TYPE_A, RE9 * l0, support=R9)
    rng = np.random.default_rng(2)
    q = random_quadratic(rng, 2)
    vals = np.array([quad_eval(q, pb.pos[:, k]) for k in range(pb.mesh.N)])
    fN = np.array([normal[:, k] @ quad_grad(q, pb.pos[:, k]) for k in range(pb.mesh.N)])
    tested = 0
    for i in np.nonzero(W["kind"] == 1)[0]:
        nb = [j for _s, j, _o in mls.stencil_slots(pb.mesh, i, R9)]
        if not any(j is not None and mask[j] == 2 for j in nb):
            continue
        phi = np.array([vals[j] if j is not None else 0.0 for j in nb])
        f = np.array([fN[j] if j is not None else 0.0 for j in nb])
        got = W["D"][:, :, i] @ phi + W["QD"][:, :, i] @ f
        assert np.abs(got - phi_components(q, pb.pos[:, i], 2)).max() <= 1e-8 / l0 ** 2
        lap = W["row"][:, i] @ phi + W["QL"][:, i] @ f
        assert lap == pytest.approx(np.trace(q[2]), abs=1e-8 / l0 ** 2)
        tested += 1
    assert tested > 50
    ql = (q[0], q[1], np.zeros((2, 2)))
    lvals = np.array([quad_eval(ql, pb.pos[:, k]) for k in range(pb.mesh.N)])
    for i in np.nonzero(W["kind"] == 3)[0]:
        nb = [j for _s, j, _o in mls.stencil_slots(pb.mesh, i, R9)]
        phi = np.array([lvals[j] if j is not None else 0.0 for j in nb])
        want = W["rscale"][i] * (normal[:, i] @ q[1])
        assert W["row"][:, i] @ phi == pytest.approx(want, abs=1e-8 / l0 ** 2)
        assert W["row"][40, i] == pytest.approx(-1.0 / l0 ** 2, rel=1e-12)


def brute_force_fit9(pb, mask, normal, bc, i, phi_all, fN_all):
    """Dense weighted least squares by QR of the MLS objective over the 9x9
    window, weights (1 - r/r_e)^2 with r_e = 3.5 l0."""
    l0 = pb.mesh.l0
    nx = pb.mesh.n[0]
    ci, cj = i % nx, i // nx
    rows, rhs = [], []
    for dj in range(-4, 5):
        for di in range(-4, 5):
            ii, jj = ci + di, cj + dj
            if (di == 0 and dj == 0) or not (0 <= ii < nx and 0 <= jj < pb.mesh.n[1]):
                continue
            j = ii + nx * jj
            if mask[j] == 0:
                continue
            X = (pb.pos[:, j] - pb.pos[:, i]) / l0
            r = math.hypot(*X)
            w = (1.0 - r / RE9) ** 2 if r < RE9 else 0.0
            sw = math.sqrt(w)
            x, y = X
            if mask[j] >= 1 and bc[mask[j]] == 1 and mask[i] == -1:
                n = normal[:, j]
                rows.append(sw * np.array([n[0], n[1], n[0] * x, n[0] * y + n[1] * x, n[1] * y]))
                rhs.append(sw * l0 * fN_all[j])
            else:
                rows.append(sw * np.array([x, y, 0.5 * x * x, x * y, 0.5 * y * y]))
                rhs.append(sw * (phi_all[j] - phi_all[i]))
    A = np.array(rows)
    if mask[i] >= 1:
        A = A[:, :2]
    Phi, *_ = np.linalg.lstsq(A, np.array(rhs), rcond=None)
    out = np.zeros(5)
    out[:len(Phi)] = Phi
    return out / np.array([l0, l0, l0 * l0, l0 * l0, l0 * l0])


def wide_jitter_fixture():
    """Dirichlet box whose DPs sit up to 0.45 l0 off their centroids, so that
    DPs four cells apart come within r_e = 3.5 l0 of each other."""
    pb = inputs.jittered_box(16, 2, seed=21, jitter=0.45)
    return pb, pb.mask, np.zeros((2, pb.mesh.N)), inputs.default_bc_kind()


def ring_pairs_within_re(pb, mask):
    nx, ny = pb.mesh.n[0], pb.mesh.n[1]
    cnt = 0
    for i in range(pb.mesh.N):
        ci, cj = i % nx, i // nx
        for dj in range(-4, 5):
            ii, jj = ci + 4, cj + dj
            if ii < nx and 0 <= jj < ny and mask[i] != 0 and mask[ii + nx * jj] != 0:
                d = np.linalg.norm(pb.pos[:, ii + nx * jj] - pb.pos[:, i])
                cnt += d < RE9 * pb.mesh.l0
    return cnt


@pytest.mark.parametrize("fixture", ["cylinder", "wide_jitter"])
def test_expanded_brute_force_least_squares(fixture):
    if fixture == "cylinder":
        pb, mask, normal, bc = cylinder_fixture(n=16, jitter_seed=9)
    else:
        pb, mask, normal, bc = wide_jitter_fixture()
        assert ring_pairs_within_re(pb, mask) > 10   # the outer ring is exercised
    W = mls.build_weights(pb.mesh, pb.pos, mask, normal, bc, TYPE_A, RE9 * pb.mesh.l0, support=R9)
    rng = np.random.default_rng(4)
    phi = rng.normal(size=pb.mesh.N)
    fN = rng.normal(size=pb.mesh.N)
    for i in range(pb.mesh.N):
        if W["kind"][i] not in (1, 3):
            continue
        nb = [j for _s, j, _o in mls.stencil_slots(pb.mesh, i, R9)]
        ph = np.array([phi[j] if j is not None else 0.0 for j in nb])
        ff = np.array([fN[j] if j is not None else 0.0 for j in nb])
        want = brute_force_fit9(pb, mask, normal, bc, i, phi, fN)
        got = W["D"][:, :, i] @ ph + W["QD"][:, :, i] @ ff
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def system9(pb, mask=None, normal=None, bc=None, rhs=None, bnd=None):
    mask = pb.mask if mask is None else mask
    W = mls.build_weights(pb.mesh, pb.pos, mask, normal, bc, TYPE_A, RE9 * pb.mesh.l0, support=R9)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], pb.rhs if rhs is None else rhs,
                       pb.bnd if bnd is None else bnd, W["rscale"])
    return W, A, b


def test_expanded_manufactured_convergence_order():
    errs = []
    ns = [12, 24, 48]
    for n in ns:
        pb = inputs.manufactured_box(n, 2, seed=0)
        _W, A, b = system9(pb)
        xs = solve.direct_solve(A, b)
        errs.append(np.linalg.norm(xs - pb.exact) / np.linalg.norm(pb.exact))
    orders = [math.log(errs[k] / errs[k + 1], 2) for k in range(len(ns) - 1)]
    assert min(orders) >= 1.5, orders


def test_expanded_bicgstab_matches_dense_lu_with_neumann_body():
    pb, mask, normal, bc = cylinder_fixture(n=20, jitter_seed=3)
    rng = np.random.default_rng(0)
    rhs = np.where(mask == -1, rng.normal(size=pb.mesh.N), 0.0)
    bnd = np.where(mask == 2, rng.normal(size=pb.mesh.N), 0.0)
    _W, A, b = system9(pb, mask, normal, bc, rhs, bnd)
    xd = np.linalg.solve(A.toarray(), b)
    x, _it, rel = solve.bicgstab(A, b, tol=1e-12)
    assert rel <= 1e-11
    assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)


def test_planted_mistake_weight_without_square(monkeypatch):
    orig = mls.weight

    def bad(r, kind, r_e):
        if kind == TYPE_A:
            return (1.0 - r / r_e) if r < r_e else 0.0
        return orig(r, kind, r_e)

    monkeypatch.setattr(mls, "weight", bad)
    got = lattice_row()
    assert np.abs(got - lattice_closed_form(RE9)).max() > 1e-3


def test_planted_mistake_support_range(monkeypatch):
    """A support loop that stops one offset short drops DPs of the outer
    ring.  On a lattice they lie beyond r_e, but DPs far off their centroids
    (here up to 0.45 l0) come within r_e of a DP four cells away: the
    brute-force pin must see the difference."""
    orig = mls.stencil_slots

    def short(mesh, k, support=1):
        out = orig(mesh, k, support)
        return [(s, (None if off[0] == support else j), off) for s, j, off in out]

    monkeypatch.setattr(mls, "stencil_slots", short)
    pb, mask, normal, bc = wide_jitter_fixture()
    W = mls.build_weights(pb.mesh, pb.pos, mask, normal, bc, TYPE_A, RE9 * pb.mesh.l0, support=R9)
    rng = np.random.default_rng(4)
    phi = rng.normal(size=pb.mesh.N)
    fN = rng.normal(size=pb.mesh.N)
    worst = 0.0
    for i in range(pb.mesh.N):
        if W["kind"][i] not in (1, 3):
            continue
        nb = [j for _s, j, _o in short(pb.mesh, i, R9)]
        ph = np.array([phi[j] if j is not None else 0.0 for j in nb])
        ff = np.array([fN[j] if j is not None else 0.0 for j in nb])
        want = brute_force_fit9(pb, mask, normal, bc, i, phi, fN)
        got = W["D"][:, :, i] @ ph + W["QD"][:, :, i] @ ff
        worst = max(worst, np.abs(got - want).max() / np.abs(want).max())
    assert worst > 1e-6
