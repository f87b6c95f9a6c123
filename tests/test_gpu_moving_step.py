"""GPU parity of the full moving-boundary step (Sec. 3.3 order: DP update,
ALE interpolation, stencils, predict, PPE with the body's Neumann datum,
projection, fluid force): mcd.AleFlow, built from C-ABI calls, against
oracle.ale.moving_step over two steps of a translating cylinder.

Masks bit-exact; positions 1e-10 l0; with the FP64 solve (tol 1e-12) P, u, v
within 1e-7 of their scale and the force within 1e-6 relative after two
steps; with the mixed solve (tol 1e-9) 1e-5.
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


@pytest.mark.parametrize("mode,tol,rtol", [(0, 1e-12, 1e-7), (1, 1e-9, 1e-5)])
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
