"""GPU parity of the fractional-step driver (Sec. 3.3, Eqs. (20)-(22)).

Compares mcd_flow_predict / mcd_flow_project and a full Taylor-Green step
(predict, mixed or FP64 pressure solve, projection) with the oracle.
Tolerances: driver outputs 1e-10 relative to the field scale (FP64 on both
sides, different summation orders); a full step with the mixed solve 1e-6
relative L2 (the pressure tolerance of the mixed mode).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import flow, mls  # noqa: E402
from paper_2404_17542_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


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


def smooth_fields(pos):
    x, y = pos
    u = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y) + 0.3 * x * y
    v = -np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y) + 0.1 * x
    return u, v


@pytest.mark.parametrize("periodic", [False, True])
def test_predict_parity(mcd, periodic):
    pb = inputs.jittered_box((40, 33), 2, seed=4, periodic=periodic)
    u, v = smooth_fields(pb.pos)
    ubc, vbc = 0.5 * u, 0.5 * v
    nu, dt = 0.01, 0.2 * pb.mesh.l0
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    want_us, want_vs, want_src = flow.predict(pb.mesh, W, u, v, ubc, vbc, nu, dt, pb.mask)
    st = mcd.Stencils(pb.mesh, dev(pb.pos.ravel()), dev(pb.mask), precision=mcd.FP64, want_derivs=True)
    us, vs, src = st.flow_predict(dev(u), dev(v), dev(ubc), dev(vbc), nu, dt)
    for got, want in ((us, want_us), (vs, want_vs), (src, want_src)):
        got = got.cpu().numpy()
        assert np.abs(got - want).max() <= 1e-10 * np.abs(want).max()


def test_project_parity_with_neumann_body(mcd):
    from oracle import mask as omask
    pb = inputs.cylinder_box(48)
    cyl = pb.meta["cylinder"]
    c = cyl.centre(0.0)
    pos, m, _ = omask.update_dps(pb.mesh, pb.pos, pb.mask, c, cyl.radius, band=0.0, n_relax=6)
    normal = omask.circle_normals(pos, m, c, cyl.body_id)
    rng = np.random.default_rng(5)
    P = np.sin(3 * pos[0]) * np.cos(2 * pos[1])
    bnd = np.where(m == cyl.body_id, rng.normal(size=pb.mesh.N), 0.0)
    us, vs = smooth_fields(pos)
    ubc, vbc = np.full(pb.mesh.N, 0.2), np.full(pb.mesh.N, -0.1)
    dt = 0.01
    W = mls.build_weights(pb.mesh, pos, m, normal, pb.bc_kind)
    want_u, want_v = flow.project(pb.mesh, W, P, bnd, us, vs, ubc, vbc, dt, m)
    st = mcd.Stencils(pb.mesh, dev(pos.ravel()), dev(m), dev(normal.ravel()), bc_kind=pb.bc_kind,
                      precision=mcd.FP64, want_derivs=True)
    u, v = st.flow_project(dev(P), dev(bnd), dev(us), dev(vs), dev(ubc), dev(vbc), dt)
    assert np.abs(u.cpu().numpy() - want_u).max() <= 1e-10 * np.abs(want_u).max()
    assert np.abs(v.cpu().numpy() - want_v).max() <= 1e-10 * np.abs(want_v).max()


@pytest.mark.parametrize("mode", [0, 1])
def test_taylor_green_steps_match_oracle(mcd, mode):
    n, steps = 32, 3
    pb = inputs.tgv_box(n, seed=1)
    nu = pb.meta["nu"]
    dt = 0.2 * pb.mesh.l0
    u_o, v_o = pb.meta["u"].copy(), pb.meta["v"].copy()
    st = mcd.Stencils(pb.mesh, dev(pb.pos.ravel()), dev(pb.mask), precision=mcd.MIXED,
                      want_derivs=True)
    u_g, v_g = dev(u_o), dev(v_o)
    P_g = torch.zeros(pb.mesh.N, dtype=torch.float64, device="cuda")
    t = 0.0
    for _ in range(steps):
        t += dt
        ue, ve, pe = inputs.tgv_fields(pb.pos, t, nu)
        u_o, v_o, P_o = flow.step(pb.mesh, pb.pos, pb.mask, u_o, v_o, ue, ve, pe, nu, dt)
        us, vs, src = st.flow_predict(u_g, v_g, dev(ue), dev(ve), nu, dt)
        st.solve(src, dev(pe), p=P_g, tol=1e-11 if mode == 0 else 1e-10, mode=mode)
        u_g, v_g = st.flow_project(P_g, dev(pe), us, vs, dev(ue), dev(ve), dt)
    for got, want in ((u_g, u_o), (v_g, v_o), (P_g, P_o)):
        got = got.cpu().numpy()
        assert np.linalg.norm(got - want) <= 1e-6 * np.linalg.norm(want)
