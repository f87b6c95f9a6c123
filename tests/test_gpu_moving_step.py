"""GPU parity of the full moving-boundary step (Sec. 3.3 order: DP update,
ALE interpolation, stencils, predict, PPE with the body's Neumann datum,
projection, fluid force): mcd.AleFlow, one mcd_flow_step call per step,
against oracle.ale.moving_step over two steps of a translating cylinder.

Masks bit-exact; positions 1e-10 l0; with the FP64 solve (tol 1e-12) P, u, v
within 1e-7 of their scale and the force within 1e-6 relative after two
steps; with the mixed solve (tol 1e-10) 1e-6, and P within 1e-6 in
relative L2 over the fluid DPs.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ale  # noqa: E402
from oracle import mls  # noqa: E402
from oracle import mask as omask  # noqa: E402
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


@pytest.mark.parametrize("mode,tol,rtol", [(0, 1e-12, 1e-7), (1, 1e-10, 1e-6)])
def test_moving_steps_match_oracle(mcd, mode, tol, rtol):
    n = 48
    cyl = inputs.Cylinder(radius=0.15)
    pb = inputs.cylinder_box(n, cyl)
    mesh, l0 = pb.mesh, pb.mesh.l0
    dt = 0.3 * l0 / abs(cyl.velocity(0.0)[0])
    nu = 0.01

    def bodies_at(t):
        return [(cyl.body_id, cyl.centre(t), cyl.radius)], [cyl.velocity(t)]

    flow = mcd.AleFlow(mesh, dev(pb.pos.ravel()), dev(pb.mask), bodies_at, nu, dt,
                       precision=mcd.MIXED if mode == 1 else mcd.FP64, mode=mode, tol=tol)
    geo0, _V0 = bodies_at(0.0)
    pos, mask, _ = omask.update_dps_bodies(mesh, pb.pos, pb.mask, geo0, band=0.0)
    assert np.array_equal(flow.mask.cpu().numpy(), mask)
    u = np.zeros(mesh.N)
    v = np.zeros(mesh.N)
    Wv = mls.build_weights(mesh, pos, mask)
    t = 0.0
    for _step in range(2):
        gk, Vk = bodies_at(t)
        g1, V1 = bodies_at(t + dt)
        o = ale.moving_step(mesh, pos, mask, u, v, Wv, gk, g1, Vk, V1, dt, nu)
        info = flow.step()
        assert np.array_equal(flow.mask.cpu().numpy(), o["mask"])
        assert np.abs(flow.pos.cpu().numpy().reshape(2, -1) - o["pos"]).max() <= 1e-10 * l0
        assert info["fallbacks"] == o["fallbacks"]
        P = flow.P.cpu().numpy()
        fluid = o["mask"] != 0
        assert np.abs(P[fluid] - o["P"][fluid]).max() <= rtol * np.abs(o["P"]).max()
        assert np.linalg.norm(P[fluid] - o["P"][fluid]) <= rtol * np.linalg.norm(o["P"][fluid])
        scale = max(np.abs(o["u"]).max(), np.abs(o["v"]).max())
        assert np.abs(flow.u.cpu().numpy() - o["u"]).max() <= rtol * scale
        assert np.abs(flow.v.cpu().numpy() - o["v"]).max() <= rtol * scale
        (Fg, perim_g, sk_g) = info["forces"][cyl.body_id]
        Fo, perim_o, sk_o = o["F"][cyl.body_id]
        assert sk_g == sk_o
        assert abs(perim_g - perim_o) <= 1e-12 * perim_o
        assert np.abs(np.array(Fg) - Fo).max() <= 10 * rtol * np.abs(Fo).max()
        pos, mask, u, v, Wv = o["pos"], o["mask"], o["u"], o["v"], o["Wv"]
        t += dt
    # the body moved and the flow is not trivial
    assert np.abs(u).max() > 0.1 and np.abs(Fo).max() > 0.0


def test_rotating_sdf_body_steps_match_oracle(mcd):
    """A translating, rotating ellipse given by a discrete SDF (Sec. 2.5):
    the rigid-body velocity and the Neumann datum carry the rotation terms
    (Eqs. (24)-(29)), omega and d omega / dt both nonzero."""
    import math

    from oracle import sdf as osdf
    n = 64
    pb = inputs.jittered_box(n, 2, seed=2, jitter=0.0)
    mesh, l0 = pb.mesh, pb.mesh.l0
    ax, by = 0.2, 0.08
    h = l0 / 2
    org = (-(ax + 0.15), -(by + 0.15))
    ng = (int(math.ceil(2 * (ax + 0.15) / h)) + 1, int(math.ceil(2 * (by + 0.15) / h)) + 1)
    grid = inputs.sample_sdf_grid(inputs.ellipse_sdf(ax, by), org, h, ng)
    grid_d = dev(grid)
    dt = 0.25 * l0
    nu = 0.01
    bid = 2

    def kin(t):
        c = (0.5 + 0.05 * math.sin(2 * math.pi * t), 0.5)
        v = (0.1 * math.pi * math.cos(2 * math.pi * t), 0.0)
        th = 0.3 + math.sin(3.0 * t)
        om = 3.0 * math.cos(3.0 * t)
        return c, v, th, om

    def gpu_bodies(t):
        c, v, th, om = kin(t)
        return [mcd.SdfBody(bid, c, th, grid_d, org, h, omega=om)], [v]

    def oracle_bodies(t):
        c, v, th, om = kin(t)
        return [osdf.SdfBody(bid, c, th, grid, org, h, omega=om)], [v]

    t = 0.4
    flow = mcd.AleFlow(mesh, dev(pb.pos.ravel()), dev(pb.mask), gpu_bodies, nu, dt, t0=t,
                       precision=mcd.FP64, mode=0, tol=1e-12)
    g0, _v = oracle_bodies(t)
    pos, mask, _ = omask.update_dps_bodies(mesh, pb.pos, pb.mask, g0, band=0.0)
    assert np.array_equal(flow.mask.cpu().numpy(), mask)
    u = np.zeros(mesh.N)
    v = np.zeros(mesh.N)
    Wv = mls.build_weights(mesh, pos, mask)
    for _step in range(2):
        gk, Vk = oracle_bodies(t)
        g1, V1 = oracle_bodies(t + dt)
        o = ale.moving_step(mesh, pos, mask, u, v, Wv, gk, g1, Vk, V1, dt, nu)
        info = flow.step()
        assert np.array_equal(flow.mask.cpu().numpy(), o["mask"])
        assert np.abs(flow.pos.cpu().numpy().reshape(2, -1) - o["pos"]).max() <= 1e-10 * l0
        P = flow.P.cpu().numpy()
        fluid = o["mask"] != 0
        assert np.abs(P[fluid] - o["P"][fluid]).max() <= 1e-7 * np.abs(o["P"]).max()
        scale = max(np.abs(o["u"]).max(), np.abs(o["v"]).max())
        assert np.abs(flow.u.cpu().numpy() - o["u"]).max() <= 1e-7 * scale
        assert np.abs(flow.v.cpu().numpy() - o["v"]).max() <= 1e-7 * scale
        Fg = np.array(info["forces"][bid][0])
        Fo = o["F"][bid][0]
        assert np.abs(Fg - Fo).max() <= 1e-6 * np.abs(Fo).max()
        pos, mask, u, v, Wv = o["pos"], o["mask"], o["u"], o["v"], o["Wv"]
        t += dt
    # the rotation shows in the boundary velocity: the tangential part is not zero
    assert np.abs(v).max() > 0.05
