"""GPU parity of the expanded 9x9 stencil (Sec. 4.1): the CUDA build, SpMV,
right-hand side and Bi-CGSTAB solves through the C ABI against the oracle.

Tolerances as for the 3x3 stencil: weights 1e-10 relative to the row scale,
FP32 rows bit-exact roundings of the FP64 rows, FP64 solves 1e-8 and mixed
solves 1e-6 relative L2 against the oracle's direct solve.
"""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mask as omask  # noqa: E402
from oracle import mls, solve  # noqa: E402
from paper_2404_17542_gb300 import inputs  # noqa: E402

sys.path.insert(0, os.path.dirname(__file__))
from test_gpu_parity import WEIGHT_TOL, compare_weights, cylinder_state  # noqa: E402

pytestmark = pytest.mark.gpu

R9, RE9, LSMPS = 4, 3.5, 2


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


def stencils9(mcd, pb, mask=None, normal=None, bc=None, precision=1, want_derivs=True):
    mask = pb.mask if mask is None else mask
    return mcd.Stencils(pb.mesh, dev(pb.pos.ravel()), dev(mask),
                        None if normal is None else dev(normal.ravel()), bc_kind=bc,
                        weight_kind=LSMPS, r_e=RE9 * pb.mesh.l0, precision=precision,
                        want_derivs=want_derivs, support=R9)


def oracle9(pb, mask, normal=None, bc=None):
    return mls.build_weights(pb.mesh, pb.pos, mask, normal, bc, LSMPS, RE9 * pb.mesh.l0, support=R9)


@pytest.mark.parametrize("shape,periodic,jitter", [
    ((70, 45), False, 0.45),   # ragged 32x16 tiles; DPs of the outer ring within r_e
    ((40, 33), True, 0.25),    # periodic axes wrap the 9x9 window
])
def test_weights_9x9(mcd, shape, periodic, jitter):
    pb = inputs.jittered_box(shape, 2, seed=21, periodic=periodic, jitter=jitter)
    W = oracle9(pb, pb.mask)
    st = stencils9(mcd, pb)
    assert st.check()[0] == 0
    compare_weights(mcd, st, W, pb.mesh.N, 81, 5)


def test_weights_9x9_with_neumann_body(mcd):
    pb, pos, m, normal, _cyl, _c = cylinder_state(48)
    pb.pos = pos
    W = oracle9(pb, m, normal, pb.bc_kind)
    st = stencils9(mcd, pb, mask=m, normal=normal, bc=pb.bc_kind)
    assert st.check()[0] == 0
    compare_weights(mcd, st, W, pb.mesh.N, 81, 5)
    ql = st.array(mcd.ARR_QL64).cpu().numpy().reshape(81, -1)
    qs = np.abs(W["row"]).max(axis=0) + 1e-300
    assert (np.abs(ql - W["QL"]).max(axis=0) <= WEIGHT_TOL * qs).all()
    qd = st.array(mcd.ARR_QD64).cpu().numpy().reshape(5, 81, -1)
    assert np.abs(qd - W["QD"]).max() <= WEIGHT_TOL * np.abs(W["D"]).max()


def test_spmv_and_rhs_9x9(mcd):
    pb, pos, m, normal, _cyl, _c = cylinder_state(40)
    pb.pos = pos
    W = oracle9(pb, m, normal, pb.bc_kind)
    A = solve.assemble(pb.mesh, W["row"])
    st = stencils9(mcd, pb, mask=m, normal=normal, bc=pb.bc_kind, want_derivs=False)
    rng = np.random.default_rng(3)
    x = rng.normal(size=pb.mesh.N)
    want = A @ x
    y64 = st.apply(dev(x)).cpu().numpy()
    assert np.abs(y64 - want).max() <= 1e-12 * np.abs(A).max() * np.abs(x).max() * 81
    y32 = st.apply(dev(x.astype(np.float32))).cpu().numpy()
    assert np.abs(y32 - want).max() <= 1e-5 * np.abs(A).max() * np.abs(x).max() * 3
    rhs = rng.normal(size=pb.mesh.N)
    bnd = rng.normal(size=pb.mesh.N)
    b = st.assemble_rhs(dev(rhs), dev(bnd)).cpu().numpy()
    bw = solve.form_rhs(pb.mesh, W["kind"], W["QL"], rhs, bnd, W["rscale"])
    assert np.allclose(b, bw, rtol=1e-12, atol=1e-12 * np.abs(bw).max())


@pytest.mark.parametrize("mode", [0, 1])
def test_solve_9x9_manufactured(mcd, mode):
    pb = inputs.manufactured_box(64, 2, seed=0)
    W = oracle9(pb, pb.mask)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], pb.rhs, pb.bnd, W["rscale"])
    x = solve.direct_solve(A, b)
    st = stencils9(mcd, pb, want_derivs=False)
    tol = 1e-11 if mode == 0 else 1e-10
    p, info = st.solve(dev(pb.rhs), dev(pb.bnd), tol=tol, mode=mode)
    got = p.cpu().numpy()
    assert info["rel_res"] <= tol
    assert np.linalg.norm(got - x) / np.linalg.norm(x) <= (1e-8 if mode == 0 else 1e-6)
    assert np.linalg.norm(b - A @ got) <= 1.01 * tol * np.linalg.norm(b)


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("support", [1, 4])
def test_solve_cylinder_array(mcd, mode, support):
    """The 25-cylinder array of Sec. 4.1 (Neumann cylinders, Dirichlet walls)
    on both stencils; masks and DPs from the oracle's multi-body update."""
    pb = inputs.cylinder_array_box(64, 6)
    bodies = pb.meta["bodies"]
    pos, m, _ = omask.update_dps_bodies(pb.mesh, pb.pos, pb.mask, bodies, n_relax=6, band=0.0)
    normal = omask.bodies_normals(pos, m, bodies)
    pb.pos = pos
    l0 = pb.mesh.l0
    if support == 4:
        W = oracle9(pb, m, normal, pb.bc_kind)
        st = stencils9(mcd, pb, mask=m, normal=normal, bc=pb.bc_kind, want_derivs=False)
    else:
        W = mls.build_weights(pb.mesh, pos, m, normal, pb.bc_kind, 1, 2.5 * l0)
        st = mcd.Stencils(pb.mesh, dev(pos.ravel()), dev(m), dev(normal.ravel()), bc_kind=pb.bc_kind,
                          weight_kind=1, r_e=2.5 * l0, want_derivs=False)
    assert st.check()[0] == 0
    rhs = np.where(m == -1, pb.rhs, 0.0)
    bnd = np.zeros(pb.mesh.N)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], rhs, bnd, W["rscale"])
    x = solve.direct_solve(A, b)
    tol = 1e-10
    p, info = st.solve(dev(rhs), dev(bnd), tol=tol, mode=mode)
    got = p.cpu().numpy()
    assert np.linalg.norm(got - x) / np.linalg.norm(x) <= (1e-7 if mode == 0 else 1e-6)
    assert np.linalg.norm(b - A @ got) <= 1.01 * tol * np.linalg.norm(b)


def test_wide_stencil_limits(mcd):
    # a periodic axis shorter than the 9x9 window is rejected on the host
    pb = inputs.jittered_box(8, 2, seed=1, periodic=True)
    with pytest.raises(mcd.McdError):
        stencils9(mcd, pb)
    # the flow driver runs on 3x3 stencils only
    pb = inputs.jittered_box(16, 2, seed=1)
    st = stencils9(mcd, pb, want_derivs=True)
    u = dev(np.zeros(pb.mesh.N))
    with pytest.raises(mcd.McdError):
        st.flow_predict(u, u, u, u, 0.01, 1e-3)
