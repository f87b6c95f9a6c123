"""Pins of the oracle's MLS weights against what the paper and mathematics fix.

Sec. 3.2 of arXiv 2404.17542: the chi=1 quadratic MLS fit (Eqs. (12)-(17)).
  * closed-form lattice weights (tests/golden/lattice_weights.txt);
  * exact reproduction of quadratics (values and Neumann data);
  * brute-force dense weighted least squares (QR) on single stencils;
  * scaling: Laplacian weights scale as l0^-2;
  * planted mistakes in the oracle must make a pin fail.
"""
import math
import os

import numpy as np
import pytest

from oracle import mls
from paper_2404_17542_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lattice_weights.txt")


def load_golden():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        kind, r_e, where, val = line.split()
        rows.append((kind, float(r_e), where, float(val)))
    return rows


def lattice_fit(dim, weight_kind, r_e_cells):
    n = 5
    pb = inputs.jittered_box(n, dim, 0, jitter=0.0, periodic=True)
    i = pb.mesh.N // 2
    f = mls.dp_fit(pb.mesh, pb.pos, pb.mask, np.zeros((dim, pb.mesh.N)),
                   inputs.default_bc_kind(), i, weight_kind,
                   r_e_cells * pb.mesh.l0)
    return f["row"] * pb.mesh.l0 ** 2


@pytest.mark.parametrize("entry", load_golden(), ids=lambda e: f"{e[0]}-{e[2]}")
def test_lattice_closed_form(entry):
    kind, r_e, where, val = entry
    if kind == "gauss3d":
        row = lattice_fit(3, 0, r_e)
        slot = {"face": 13 + 1, "edge": 13 + 1 + 3, "corner": 13 + 1 + 3 + 9}[where]
    else:
        row = lattice_fit(2, 0 if kind == "gauss" else 1, r_e)
        slot = {"axis": 5, "diagonal": 8}[where]
    assert row[slot] == pytest.approx(val, rel=1e-12, abs=1e-13)


def test_lattice_symmetry_and_row_sum():
    row = lattice_fit(2, 0, 1.0)
    assert row.sum() == pytest.approx(0.0, abs=1e-12)
    for s in (1, 3, 5, 7):
        assert row[s] == pytest.approx(row[5], rel=1e-13)


def random_quadratic(rng, dim):
    c0 = rng.uniform(-1, 1)
    g = rng.uniform(-1, 1, size=dim)
    H = rng.uniform(-1, 1, size=(dim, dim))
    H = 0.5 * (H + H.T)
    return c0, g, H


def quad_eval(q, x):
    c0, g, H = q
    return c0 + g @ x + 0.5 * x @ H @ x


def quad_grad(q, x):
    _c0, g, H = q
    return g + H @ x


def phi_components(q, x, dim):
    gr = quad_grad(q, x)
    H = q[2]
    if dim == 2:
        return np.array([gr[0], gr[1], H[0, 0], H[0, 1], H[1, 1]])
    return np.array([gr[0], gr[1], gr[2], H[0, 0], H[1, 1], H[2, 2],
                     H[0, 1], H[1, 2], H[0, 2]])


@pytest.mark.parametrize("dim,weight_kind", [(2, 0), (2, 1), (3, 0)])
def test_quadratic_reproduction(dim, weight_kind):
    """chi=1 quadratic MLS is exact on quadratics (Sec. 3.2, Eq. (12))."""
    n = 6 if dim == 2 else 4
    pb = inputs.jittered_box(n, dim, seed=3)
    rng = np.random.default_rng(11)
    r_e = (2.5 if weight_kind == 1 else 1.0) * pb.mesh.l0
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask, weight_kind=weight_kind, r_e=r_e)
    S = 3 ** dim
    for _ in range(3):
        q = random_quadratic(rng, dim)
        vals = np.array([quad_eval(q, pb.pos[:, k]) for k in range(pb.mesh.N)])
        for i in np.nonzero(W["kind"] == 1)[0]:
            nb = [j for _s, j, _o in mls.stencil_slots(pb.mesh, i)]
            phi = np.array([vals[j] if j is not None else 0.0 for j in nb])
            want = phi_components(q, pb.pos[:, i], dim)
            got = W["D"][:, :, i] @ phi
            scale = 1.0 / pb.mesh.l0 ** 2
            assert np.abs(got - want).max() <= 1e-9 * scale
            lap = W["row"][:, i] @ phi
            assert lap == pytest.approx(np.trace(q[2]), abs=1e-9 * scale)
            assert S == len(nb)


def cylinder_fixture(n=24, jitter_seed=5):
    """Jittered 2D box with a disc of Neumann boundary DPs (id 2).

    Masks and DP positions come from the oracle's own DP update (Sec. 2.2-2.3)
    so that the boundary ring has the structure the method produces.
    """
    from oracle import mask as omask
    pb = inputs.jittered_box(n, 2, jitter_seed)
    c = (0.5 + 0.013, 0.5 - 0.007)
    R = 0.2
    pos, mask, _prev = omask.update_dps(pb.mesh, pb.pos, pb.mask, c, R,
                                        body_id=2, band=0.0, n_relax=3)
    normal = omask.circle_normals(pos, mask, c, 2)
    pb.pos = pos
    bc = inputs.default_bc_kind(neumann_ids=(2,))
    return pb, mask, normal, bc


def test_quadratic_reproduction_with_neumann_terms():
    """Consistent Neumann data f = n . grad q keep the fit exact (Eq. (15))."""
    pb, mask, normal, bc = cylinder_fixture()
    W = mls.build_weights(pb.mesh, pb.pos, mask, normal, bc)
    rng = np.random.default_rng(2)
    q = random_quadratic(rng, 2)
    vals = np.array([quad_eval(q, pb.pos[:, k]) for k in range(pb.mesh.N)])
    fN = np.array([normal[:, k] @ quad_grad(q, pb.pos[:, k]) for k in range(pb.mesh.N)])
    tested = 0
    for i in np.nonzero(W["kind"] == 1)[0]:
        nb = [j for _s, j, _o in mls.stencil_slots(pb.mesh, i)]
        if not any(j is not None and mask[j] == 2 for j in nb):
            continue
        phi = np.array([vals[j] if j is not None else 0.0 for j in nb])
        f = np.array([fN[j] if j is not None else 0.0 for j in nb])
        got = W["D"][:, :, i] @ phi + W["QD"][:, :, i] @ f
        want = phi_components(q, pb.pos[:, i], 2)
        assert np.abs(got - want).max() <= 1e-8 / pb.mesh.l0 ** 2
        # the PPE row plus its moved Neumann terms gives the Laplacian
        lap = W["row"][:, i] @ phi + W["QL"][:, i] @ f
        assert lap == pytest.approx(np.trace(q[2]), abs=1e-8 / pb.mesh.l0 ** 2)
        tested += 1
    assert tested > 10
    # Neumann DP rows (linear fit): sigma * n . grad q exactly for linear q
    ql = (q[0], q[1], np.zeros((2, 2)))
    lvals = np.array([quad_eval(ql, pb.pos[:, k]) for k in range(pb.mesh.N)])
    nrows = np.nonzero(W["kind"] == 3)[0]
    assert len(nrows) > 10
    for i in nrows:
        nb = [j for _s, j, _o in mls.stencil_slots(pb.mesh, i)]
        phi = np.array([lvals[j] if j is not None else 0.0 for j in nb])
        got = W["row"][:, i] @ phi
        want = W["rscale"][i] * (normal[:, i] @ q[1])
        assert got == pytest.approx(want, abs=1e-8 / pb.mesh.l0 ** 2)
        assert W["row"][4, i] == pytest.approx(-1.0 / pb.mesh.l0 ** 2, rel=1e-12)


def brute_force_fit(pb, mask, normal, bc, i, phi_all, fN_all, weight_kind=0):
    """Dense weighted least squares by QR (numpy lstsq) of the MLS objective."""
    dim = pb.mesh.dim
    l0 = pb.mesh.l0
    rows, rhs = [], []
    for _s, j, _o in mls.stencil_slots(pb.mesh, i):
        if j is None or j == i or mask[j] == 0:
            continue
        X = (pb.pos[:, j] - pb.pos[:, i]) / l0
        r = np.linalg.norm(pb.pos[:, j] - pb.pos[:, i])
        w = math.exp(-(r / l0) ** 2) if weight_kind == 0 else math.cos(math.pi * r / (5 * l0)) ** 2
        sw = math.sqrt(w)
        if mask[j] >= 1 and bc[mask[j]] == 1 and mask[i] == -1:
            n = normal[:, j]
            x, y = X
            pn = np.array([n[0], n[1], n[0] * x, n[0] * y + n[1] * x, n[1] * y])
            rows.append(sw * pn)
            rhs.append(sw * l0 * fN_all[j])
        else:
            x, y = X
            rows.append(sw * np.array([x, y, 0.5 * x * x, x * y, 0.5 * y * y]))
            rhs.append(sw * (phi_all[j] - phi_all[i]))
    A = np.array(rows)
    if mask[i] >= 1:          # Neumann DP's own fit: linear basis
        A = A[:, :2]
    Phi, *_ = np.linalg.lstsq(A, np.array(rhs), rcond=None)
    out = np.zeros(5)
    out[:len(Phi)] = Phi
    return out / np.array([l0, l0, l0 * l0, l0 * l0, l0 * l0])


@pytest.mark.parametrize("weight_kind", [0, 1])
def test_brute_force_least_squares(weight_kind):
    pb, mask, normal, bc = cylinder_fixture(n=16, jitter_seed=9)
    r_e = (1.0 if weight_kind == 0 else 2.5) * pb.mesh.l0
    W = mls.build_weights(pb.mesh, pb.pos, mask, normal, bc, weight_kind, r_e)
    rng = np.random.default_rng(4)
    phi = rng.normal(size=pb.mesh.N)
    fN = rng.normal(size=pb.mesh.N)
    for i in range(pb.mesh.N):
        if W["kind"][i] not in (1, 3):
            continue
        nb = [j for _s, j, _o in mls.stencil_slots(pb.mesh, i)]
        ph = np.array([phi[j] if j is not None else 0.0 for j in nb])
        ff = np.array([fN[j] if j is not None else 0.0 for j in nb])
        want = brute_force_fit(pb, mask, normal, bc, i, phi, fN, weight_kind)
        got = W["D"][:, :, i] @ ph + W["QD"][:, :, i] @ ff
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9 * np.abs(want).max())


def test_laplacian_scales_as_inverse_square():
    a = inputs.jittered_box(6, 2, seed=1)
    b = inputs.jittered_box(6, 2, seed=1, length=3.0)
    Wa = mls.build_weights(a.mesh, a.pos, a.mask)
    Wb = mls.build_weights(b.mesh, b.pos, b.mask)
    inner = Wa["kind"] == 1
    assert np.allclose(Wb["row"][:, inner] * 9.0, Wa["row"][:, inner], rtol=1e-11)


def test_singular_stencil_raises():
    pb = inputs.jittered_box(6, 2, seed=1)
    mask = pb.mask.copy()
    mask[:] = 0
    mask[14] = -1
    mask[15] = -1
    mask[20] = -1
    with pytest.raises(mls.SingularStencil):
        mls.build_weights(pb.mesh, pb.pos, mask)


def test_planted_mistake_is_caught(monkeypatch):
    """A dropped basis term (XY -> 0) must break quadratic reproduction."""
    orig = mls.basis

    def bad_basis(X):
        p = orig(X)
        if len(X) == 2:
            p[3] = p[3] * -1.0   # sign error on the mixed term
        return p

    monkeypatch.setattr(mls, "basis", bad_basis)
    pb = inputs.jittered_box(6, 2, seed=3)
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    q = (0.3, np.array([0.2, -0.1]), np.array([[0.5, 0.7], [0.7, -0.3]]))
    vals = np.array([quad_eval(q, pb.pos[:, k]) for k in range(pb.mesh.N)])
    i = int(np.nonzero(W["kind"] == 1)[0][5])
    nb = [j for _s, j, _o in mls.stencil_slots(pb.mesh, i)]
    phi = np.array([vals[j] if j is not None else 0.0 for j in nb])
    got = W["D"][:, :, i] @ phi
    want = phi_components(q, pb.pos[:, i], 2)
    assert np.abs(got - want).max() > 1e-3
