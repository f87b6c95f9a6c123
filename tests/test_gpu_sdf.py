"""GPU parity of bodies given by a discrete SDF with posture angle (Sec. 2.5):
the DP update, boundary data with rotation (Eqs. (24)-(29)) and the ALE
shift, CUDA through the C ABI against the oracle.

The interpolated psi decides the vertex test, so masks agree except where a
vertex lies within rounding of the boundary (both classifications are then
valid): such cells must have a vertex with |psi| < 1e-10 l0.  Positions
1e-9 l0; normals and boundary data 1e-12.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ale  # noqa: E402
from oracle import mask as omask  # noqa: E402
from oracle import mls  # noqa: E402
from oracle import sdf  # noqa: E402
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


def ellipse_pair(mcd, theta, c=(0.51, 0.47), bid=2, omega=0.0, omega_dot=0.0):
    a, b, h, org = 0.25, 0.12, 1.0 / 256, (-0.4, -0.4)
    n = int(round(0.8 / h)) + 1
    grid = inputs.sample_sdf_grid(inputs.ellipse_sdf(a, b), org, h, (n, n))
    ob = sdf.SdfBody(bid, c, theta, grid, org, h)
    gb = mcd.SdfBody(bid, c, theta, dev(grid), org, h, omega=omega, omega_dot=omega_dot)
    return ob, gb


def check_masks(mesh, got, want, bodies):
    diff = np.nonzero(got != want)[0]
    nx = mesh.n[0]
    for k in diff:
        i, j = k % nx, k // nx
        psis = [abs(omask.nearest_body(bodies, (i + di) * mesh.l0, (j + dj) * mesh.l0)[1])
                for di in (0, 1) for dj in (0, 1)]
        assert min(psis) < 1e-10 * mesh.l0
    return len(diff)


@pytest.mark.parametrize("theta,alpha", [(0.6, 0.0), (-1.1, 0.03)])
def test_sdf_update_matches_oracle(mcd, theta, alpha):
    pb = inputs.jittered_box(96, 2, seed=4)
    ob, gb = ellipse_pair(mcd, theta)
    pos_o, m_o, _ = omask.update_dps_bodies(pb.mesh, pb.pos, pb.mask, [ob], n_relax=5, band=0.0, alpha=alpha)
    pos_g, m_g = dev(pb.pos.ravel()), dev(pb.mask)
    prev = torch.empty_like(m_g)
    mcd.update_dps_bodies(pb.mesh, [gb], pos_g, m_g, prev, n_relax=5, band=0.0, alpha=alpha)
    mg = m_g.cpu().numpy()
    assert check_masks(pb.mesh, mg, m_o, [ob]) <= 2
    same = mg == m_o
    pg = pos_g.cpu().numpy().reshape(2, -1)
    assert np.abs(pg[:, same] - pos_o[:, same]).max() <= 1e-9 * pb.mesh.l0
    assert (m_o == 2).sum() > 50


def test_mixed_circles_and_sdf_array(mcd):
    pb = inputs.cylinder_array_box(96, 6)
    bodies = pb.meta["bodies"]
    ob_list, gb_list = [], []
    for k, (bid, c, R) in enumerate(bodies):
        if k % 2 == 0:
            ob_list.append((bid, c, R))
            gb_list.append((bid, c, R))
            continue
        h, org = pb.mesh.l0 / 4, (-2 * R, -2 * R)
        n = int(round(4 * R / h)) + 1
        grid = inputs.sample_sdf_grid(inputs.circle_sdf(R), org, h, (n, n))
        ob_list.append(sdf.SdfBody(bid, c, 0.3 * k, grid, org, h))
        gb_list.append(mcd.SdfBody(bid, c, 0.3 * k, dev(grid), org, h))
    pos_o, m_o, _ = omask.update_dps_bodies(pb.mesh, pb.pos, pb.mask, ob_list, n_relax=4, band=0.0)
    pos_g, m_g = dev(pb.pos.ravel()), dev(pb.mask)
    mcd.update_dps_bodies(pb.mesh, gb_list, pos_g, m_g, torch.empty_like(m_g), n_relax=4, band=0.0)
    mg = m_g.cpu().numpy()
    assert check_masks(pb.mesh, mg, m_o, ob_list) <= 4
    same = mg == m_o
    assert np.abs(pos_g.cpu().numpy().reshape(2, -1)[:, same] - pos_o[:, same]).max() <= 1e-9 * pb.mesh.l0
    assert set(int(v) for v in np.unique(m_o) if v >= 2) == {b[0] for b in bodies}


def test_sdf_boundary_data_with_rotation(mcd):
    pb = inputs.jittered_box(96, 2, seed=4)
    om, omd, acc, vel = 1.7, -0.9, (0.4, -0.25), (0.3, 0.8)
    ob, gb = ellipse_pair(mcd, 0.6, omega=om, omega_dot=omd)
    pos, m, _ = omask.update_dps_bodies(pb.mesh, pb.pos, pb.mask, [ob], n_relax=5, band=0.0)
    normal = omask.bodies_normals(pos, m, [ob])
    ng, fg = mcd.bodies_boundary(pb.mesh, [gb], dev(pos.ravel()), dev(m), accs=[acc])
    assert np.abs(ng.cpu().numpy().reshape(2, -1) - normal).max() <= 1e-12
    sel = m == 2
    rx, ry = pos[0] - ob.centre[0], pos[1] - ob.centre[1]
    ax = acc[0] - omd * ry - om * om * rx          # dV/dt of a rigid body (Eqs. (26)-(29))
    ay = acc[1] + omd * rx - om * om * ry
    want = np.where(sel, -(ax * normal[0] + ay * normal[1]), 0.0)
    assert np.abs(fg.cpu().numpy() - want).max() <= 1e-12 * max(1.0, np.abs(want).max())
    ug, vg = mcd.bodies_velocity(pb.mesh, [gb], [vel], dev(pos.ravel()), dev(m))
    assert np.abs(ug.cpu().numpy() - np.where(sel, vel[0] - om * ry, 0.0)).max() <= 1e-14
    assert np.abs(vg.cpu().numpy() - np.where(sel, vel[1] + om * rx, 0.0)).max() <= 1e-14


def test_sdf_ale_matches_oracle(mcd):
    """The Appendix A shift follows the sign of the SDF body's gradient."""
    pb = inputs.jittered_box(96, 2, seed=4)
    ob0, gb0 = ellipse_pair(mcd, 0.6)
    ob1, gb1 = ellipse_pair(mcd, 0.64, c=(0.517, 0.466))
    pos_k, m_k, _ = omask.update_dps_bodies(pb.mesh, pb.pos, pb.mask, [ob0], n_relax=4, band=0.0)
    pos_1, m_1, _ = omask.update_dps_bodies(pb.mesh, pos_k, m_k, [ob1], n_relax=4)
    W = mls.build_weights(pb.mesh, pos_k, m_k)
    u = np.sin(3 * pos_k[0]) * np.cos(2 * pos_k[1])
    uo, fbo = ale.ale_interpolate(pb.mesh, pos_k, pos_1, m_k, m_1, u, W, [ob0])
    vel = mcd.Stencils(pb.mesh, dev(pos_k.ravel()), dev(m_k), want_derivs=True, precision=mcd.FP64)
    ug, _vg, fb = mcd.ale_interpolate(vel, [gb0], dev(pos_k.ravel()), dev(pos_1.ravel()), dev(m_k), dev(m_1),
                                      dev(u), dev(u))
    assert fb == fbo
    assert np.abs(ug.cpu().numpy() - uo).max() <= 1e-12 * np.abs(u).max()
    assert ((m_1 == -1) & (m_k != -1)).sum() > 5
