"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (FP64 arithmetic on both sides, different summation orders and
libm): stencil rows and derivative weights 1e-10 relative to the row scale;
FP64 solves 1e-8 relative L2 at tol 1e-11; mixed FP32/FP64 solves 1e-6
relative L2; masks bit-exact; positions 1e-12 l0.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mask as omask  # noqa: E402
from oracle import mls, solve  # noqa: E402
from paper_2404_17542_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

WEIGHT_TOL = 1e-10


@pytest.fixture(scope="module")
def mcd():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_17542_gb300 import build
    build.build()
    from paper_2404_17542_gb300 import mcd as m
    m.lib()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def gpu_stencils(mcd, pb, mask=None, normal=None, bc=None, weight_kind=0, r_e=None,
                 precision=1, want_derivs=True):
    mask = pb.mask if mask is None else mask
    st = mcd.Stencils(pb.mesh, dev(pb.pos.ravel()), dev(mask),
                      None if normal is None else dev(normal.ravel()),
                      bc_kind=bc, weight_kind=weight_kind, r_e=r_e, precision=precision,
                      want_derivs=want_derivs)
    return st


def compare_weights(mcd, st, W, N, S, nb, kinds=True):
    row = st.array(mcd.ARR_ROW64).cpu().numpy().reshape(S, N)
    scale = np.abs(W["row"]).max(axis=0, keepdims=True) + 1e-300
    assert np.abs(row - W["row"]).max(axis=0).max() <= WEIGHT_TOL * scale.max()
    assert (np.abs(row - W["row"]) <= WEIGHT_TOL * scale).all()
    r32 = st.array(mcd.ARR_ROW32)
    if r32 is not None:
        # FP32 rows: difference form (off-centre = rounded FP64 weights,
        # centre = row sum: 0 for MLS rows, 1 for identity rows)
        r32 = r32.cpu().numpy().reshape(S, N)
        C = S // 2
        off = [s for s in range(S) if s != C]
        assert np.array_equal(r32[off], row[off].astype(np.float32))
        ident = np.isin(W["kind"], (0, 2))
        assert np.array_equal(r32[C], np.where(ident, 1.0, 0.0).astype(np.float32))
        assert np.abs(W["row"][:, ~ident].sum(axis=0)).max() <= 1e-9 * scale.max()
    if kinds:
        kind = st.array(mcd.ARR_KIND).cpu().numpy()
        assert np.array_equal(kind, W["kind"])
    d = st.array(mcd.ARR_D64)
    if d is not None:
        d = d.cpu().numpy().reshape(nb, S, N)
        ds = np.abs(W["D"]).max(axis=(0, 1)) + 1e-300
        assert (np.abs(d - W["D"]).max(axis=(0, 1)) <= WEIGHT_TOL * ds).all()
    rs = st.array(mcd.ARR_RSCALE).cpu().numpy()
    assert np.allclose(rs, W["rscale"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("shape,weight_kind,periodic", [
    ((70, 45), 0, False),     # several 32x8 tiles with ragged tails
    ((70, 45), 1, False),     # cos^2 weight, r_e = 2.5 l0 (Eq. (17))
    ((40, 33), 0, True),      # periodic minimum image
])
def test_weights_2d(mcd, shape, weight_kind, periodic):
    pb = inputs.jittered_box(shape, 2, seed=21, periodic=periodic)
    r_e = (2.5 if weight_kind == 1 else 1.0) * pb.mesh.l0
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask, weight_kind=weight_kind, r_e=r_e)
    st = gpu_stencils(mcd, pb, weight_kind=weight_kind, r_e=r_e)
    assert st.check()[0] == 0
    compare_weights(mcd, st, W, pb.mesh.N, 9, 5)


def test_weights_3d(mcd):
    pb = inputs.jittered_box((9, 7, 6), 3, seed=5)
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    st = gpu_stencils(mcd, pb)
    compare_weights(mcd, st, W, pb.mesh.N, 27, 9)


def cylinder_state(n, t=0.0, n_relax=8):
    pb = inputs.cylinder_box(n)
    cyl = pb.meta["cylinder"]
    c = cyl.centre(t)
    pos, m, _ = omask.update_dps(pb.mesh, pb.pos, pb.mask, c, cyl.radius, band=0.0, n_relax=n_relax)
    normal = omask.circle_normals(pos, m, c, cyl.body_id)
    return pb, pos, m, normal, cyl, c


def test_weights_with_neumann_body(mcd):
    pb, pos, m, normal, cyl, c = cylinder_state(48)
    pb.pos = pos
    W = mls.build_weights(pb.mesh, pos, m, normal, pb.bc_kind)
    st = gpu_stencils(mcd, pb, mask=m, normal=normal, bc=pb.bc_kind)
    assert st.check()[0] == 0
    compare_weights(mcd, st, W, pb.mesh.N, 9, 5)
    ql = st.array(mcd.ARR_QL64).cpu().numpy().reshape(9, -1)
    qs = np.abs(W["row"]).max(axis=0) + 1e-300
    assert (np.abs(ql - W["QL"]).max(axis=0) <= WEIGHT_TOL * qs).all()
    qd = st.array(mcd.ARR_QD64).cpu().numpy().reshape(5, 9, -1)
    assert np.abs(qd - W["QD"]).max() <= WEIGHT_TOL * np.abs(W["D"]).max()


def test_spmv_and_rhs(mcd):
    pb, pos, m, normal, cyl, c = cylinder_state(40)
    pb.pos = pos
    W = mls.build_weights(pb.mesh, pos, m, normal, pb.bc_kind)
    A = solve.assemble(pb.mesh, W["row"])
    st = gpu_stencils(mcd, pb, mask=m, normal=normal, bc=pb.bc_kind, want_derivs=False)
    rng = np.random.default_rng(3)
    x = rng.normal(size=pb.mesh.N)
    y64 = st.apply(dev(x)).cpu().numpy()
    want = A @ x
    assert np.abs(y64 - want).max() <= 1e-12 * np.abs(A).max() * np.abs(x).max() * 9
    y32 = st.apply(dev(x.astype(np.float32))).cpu().numpy()
    assert np.abs(y32 - want).max() <= 1e-5 * np.abs(A).max() * np.abs(x).max()
    rhs = rng.normal(size=pb.mesh.N)
    bnd = rng.normal(size=pb.mesh.N)
    b = st.assemble_rhs(dev(rhs), dev(bnd)).cpu().numpy()
    bw = solve.form_rhs(pb.mesh, W["kind"], W["QL"], rhs, bnd, W["rscale"])
    assert np.allclose(b, bw, rtol=1e-12, atol=1e-12 * np.abs(bw).max())


@pytest.mark.parametrize("mode", [0, 1])
def test_solve_manufactured(mcd, mode):
    pb = inputs.manufactured_box(64, 2, seed=0)
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], pb.rhs, pb.bnd, W["rscale"])
    x = solve.direct_solve(A, b)
    st = gpu_stencils(mcd, pb, want_derivs=False)
    tol = 1e-11 if mode == 0 else 1e-10
    p, info = st.solve(dev(pb.rhs), dev(pb.bnd), tol=tol, mode=mode)
    got = p.cpu().numpy()
    err = np.linalg.norm(got - x) / np.linalg.norm(x)
    assert info["rel_res"] <= tol
    assert err <= (1e-8 if mode == 0 else 1e-6), err
    # true residual of the returned field, judged by the oracle in FP64
    assert np.linalg.norm(b - A @ got) <= 1.01 * tol * np.linalg.norm(b)


@pytest.mark.parametrize("mode", [0, 1])
def test_solve_with_neumann_body(mcd, mode):
    pb, pos, m, normal, cyl, c = cylinder_state(64)
    pb.pos = pos
    W = mls.build_weights(pb.mesh, pos, m, normal, pb.bc_kind)
    A = solve.assemble(pb.mesh, W["row"])
    a = cyl.acceleration(0.05)
    bnd = np.where(m == cyl.body_id, -(a[0] * normal[0] + a[1] * normal[1]), 0.0)
    rhs = np.where(m == -1, np.sin(3 * pos[0]) * np.cos(2 * pos[1]), 0.0)
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], rhs, bnd, W["rscale"])
    x = solve.direct_solve(A, b)
    st = gpu_stencils(mcd, pb, mask=m, normal=normal, bc=pb.bc_kind, want_derivs=False)
    p, info = st.solve(dev(rhs), dev(bnd), tol=1e-10, mode=mode)
    got = p.cpu().numpy()
    assert np.linalg.norm(got - x) / np.linalg.norm(x) <= 1e-6


def test_update_dps_bit_exact_masks(mcd):
    n = 96
    pb = inputs.cylinder_box(n)
    cyl = pb.meta["cylinder"]
    pos_o, m_o = pb.pos.copy(), pb.mask.copy()
    pos_g, m_g = dev(pb.pos.ravel()), dev(pb.mask)
    prev_g = torch.empty_like(m_g)
    for step, t in enumerate([0.0, 0.004, 0.008, 0.05]):
        c = cyl.centre(t)
        band = 0.0 if step == 0 else 5 * pb.mesh.l0
        pos_o, m_new, prev_o = omask.update_dps(pb.mesh, pos_o, m_o, c, cyl.radius, band=band,
                                                n_relax=6)
        mcd.update_dps(pb.mesh, c, cyl.radius, cyl.body_id, pos_g, m_g, prev_g, kappa=0.2,
                       n_relax=6, band=band)
        assert np.array_equal(m_g.cpu().numpy(), m_new)
        assert np.array_equal(prev_g.cpu().numpy(), m_o)
        pg = pos_g.cpu().numpy().reshape(2, -1)
        assert np.abs(pg - pos_o).max() <= 1e-12 * pb.mesh.l0 * 1e2
        m_o = m_new
        # continue both from the oracle state so the comparison stays per-step
        pos_g.copy_(dev(pos_o.ravel()))


def test_body_boundary_data(mcd):
    pb, pos, m, normal, cyl, c = cylinder_state(40)
    acc = cyl.acceleration(0.031)
    ng, fg = mcd.body_boundary(pb.mesh, c, cyl.radius, cyl.body_id, dev(pos.ravel()), dev(m), acc=acc)
    assert np.allclose(ng.cpu().numpy().reshape(2, -1), normal, rtol=0, atol=1e-14)
    want = np.where(m == cyl.body_id, -(acc[0] * normal[0] + acc[1] * normal[1]), 0.0)
    assert np.allclose(fg.cpu().numpy(), want, rtol=0, atol=1e-13 * max(1.0, abs(acc[0])))


def test_singular_stencil_reports_esingular(mcd):
    pb = inputs.jittered_box(12, 2, seed=1)
    mask = np.zeros(pb.mesh.N, dtype=np.int8)
    mask[5 + 12 * 5] = -1
    mask[6 + 12 * 5] = -1
    mask[5 + 12 * 6] = -1
    st = gpu_stencils(mcd, pb, mask=mask, want_derivs=False)
    status, bad = st.check()
    assert status == mcd.ESINGULAR and bad == 5 + 12 * 5
    with pytest.raises(mcd.McdError):
        st.solve(dev(np.zeros(pb.mesh.N)), dev(np.zeros(pb.mesh.N)))


def test_nonfinite_rhs_and_max_iter(mcd):
    pb = inputs.manufactured_box(32, 2, seed=2)
    st = gpu_stencils(mcd, pb, want_derivs=False)
    rhs = pb.rhs.copy()
    rhs[100] = np.nan
    _p, info = st.solve(dev(rhs), dev(pb.bnd), raise_on_error=False)
    assert info["status"] == mcd.ENONFINITE
    _p, info = st.solve(dev(pb.rhs), dev(pb.bnd), tol=1e-12, max_iter=5, mode=0,
                        raise_on_error=False)
    assert info["status"] == mcd.ENOCONV
    assert info["iters"] <= 5 + 64


@pytest.mark.parametrize("mode", [0, 1])
def test_solve_manufactured_3d(mcd, mode):
    """27-point 3D system with ragged 32x4x4 tiles against the direct solve."""
    pb = inputs.manufactured_box((18, 14, 12), 3, seed=2)
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], pb.rhs, pb.bnd, W["rscale"])
    x = solve.direct_solve(A, b)
    st = gpu_stencils(mcd, pb, want_derivs=False)
    tol = 1e-11 if mode == 0 else 1e-10
    p, info = st.solve(dev(pb.rhs), dev(pb.bnd), tol=tol, mode=mode)
    got = p.cpu().numpy()
    assert info["rel_res"] <= tol
    assert np.linalg.norm(got - x) / np.linalg.norm(x) <= (1e-8 if mode == 0 else 1e-6)
    assert np.linalg.norm(b - A @ got) <= 1.01 * tol * np.linalg.norm(b)


def test_solve_3d_full_size(mcd):
    """The 128^3 Dirichlet sin^3 problem: rows of sampled DPs against the
    oracle's per-DP fit, the FP64 residual of the mixed solve, and the
    discretisation error against the closed form (second order in l0: the
    quadratic MLS Laplacian is exact on quadratics)."""
    n = 128
    pb = inputs.manufactured_box(n, 3, seed=2)
    N = pb.mesh.N
    st = gpu_stencils(mcd, pb, want_derivs=False)
    rows = st.array(mcd.ARR_ROW64).cpu().numpy().reshape(27, N)
    rng = np.random.default_rng(0)
    for i in rng.choice(N, 40, replace=False):
        f = mls.dp_fit(pb.mesh, pb.pos, pb.mask, None, pb.bc_kind, int(i))
        scale = np.abs(f["row"]).max()
        assert np.abs(rows[:, i] - f["row"]).max() <= WEIGHT_TOL * scale, i
    p, info = st.solve(dev(pb.rhs), dev(pb.bnd), tol=1e-8, mode=1)
    assert info["status"] == 0 and info["rel_res"] <= 1e-8
    # residual of the returned field with the FP64 SpMV (a separate kernel)
    b = st.assemble_rhs(dev(pb.rhs), dev(pb.bnd))
    r = b - st.apply(p)
    assert float(r.norm() / b.norm()) <= 1.01e-8
    err = np.linalg.norm(p.cpu().numpy() - pb.exact) / np.linalg.norm(pb.exact)
    assert err <= 20 * (1.0 / n) ** 2, err


def test_update_dps_boundary_fitted(mcd):
    """The DP update with the boundary-fitted move of Sec. 4.7 (alpha > 0)."""
    n = 96
    pb = inputs.cylinder_box(n)
    cyl = pb.meta["cylinder"]
    c = cyl.centre(0.0)
    pos_o, m_o, _ = omask.update_dps(pb.mesh, pb.pos, pb.mask, c, cyl.radius, band=0.0, n_relax=6,
                                     alpha=0.03)
    pos_g, m_g = dev(pb.pos.ravel()), dev(pb.mask)
    prev_g = torch.empty_like(m_g)
    mcd.update_dps(pb.mesh, c, cyl.radius, cyl.body_id, pos_g, m_g, prev_g, kappa=0.2, n_relax=6,
                   band=0.0, alpha=0.03)
    assert np.array_equal(m_g.cpu().numpy(), m_o)
    pg = pos_g.cpu().numpy().reshape(2, -1)
    assert np.abs(pg - pos_o).max() <= 1e-12 * pb.mesh.l0 * 1e2
    # the move is visible: DPs near the body differ from the alpha = 0 arrangement
    pos_0, _m, _ = omask.update_dps(pb.mesh, pb.pos, pb.mask, c, cyl.radius, band=0.0, n_relax=6)
    assert np.abs(pos_0 - pos_o).max() > 1e-3 * pb.mesh.l0
