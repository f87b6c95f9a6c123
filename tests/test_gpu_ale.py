"""GPU parity of the ALE interpolation (Eq. (19), Appendix A) and of the fluid
force (Sec. 3.4, Eqs. (30)-(31)): the CUDA path through the C ABI against the
oracle.

Tolerances: interpolated velocities 1e-12 of the field scale (FP64 on both
sides, fused multiply-adds on the device); forces 1e-10 relative, the
perimeter 1e-12 relative (the neighbour choice is rounded as in the oracle);
fallback and skipped counts exact.
"""
import math
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import ale  # noqa: E402
from oracle import mask as omask  # noqa: E402
from oracle import mls  # noqa: E402
from paper_2404_17542_gb300 import inputs  # noqa: E402

sys.path.insert(0, os.path.dirname(__file__))
from test_oracle_ale import body_state, moving_step, quad  # noqa: E402

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


def smooth(x, y, a):
    return np.sin(a * x + 0.3) * np.cos(0.7 * a * y) + 0.2 * x * y


def ale_case(mcd, pb, pos_k, mask_k, pos_k1, mask_k1, bodies, fields):
    W = mls.build_weights(pb.mesh, pos_k, mask_k)
    vel = mcd.Stencils(pb.mesh, dev(pos_k.ravel()), dev(mask_k), want_derivs=True, precision=mcd.FP64)
    u, v = fields
    ug, vg, fb = mcd.ale_interpolate(vel, bodies, dev(pos_k.ravel()), dev(pos_k1.ravel()), dev(mask_k),
                                     dev(mask_k1), dev(u), dev(v))
    uo, fbo = ale.ale_interpolate(pb.mesh, pos_k, pos_k1, mask_k, mask_k1, u, W, bodies)
    vo, _ = ale.ale_interpolate(pb.mesh, pos_k, pos_k1, mask_k, mask_k1, v, W, bodies)
    return ug.cpu().numpy(), vg.cpu().numpy(), fb, uo, vo, fbo


def test_ale_matches_oracle_moving_cylinder(mcd):
    pb, pos_k, mask_k, pos_k1, mask_k1, bodies = moving_step()
    u = smooth(pos_k[0], pos_k[1], 5.0)
    v = smooth(pos_k[1], pos_k[0], 3.0)
    ug, vg, fb, uo, vo, fbo = ale_case(mcd, pb, pos_k, mask_k, pos_k1, mask_k1, bodies, (u, v))
    assert fb == fbo == 0
    assert np.abs(ug - uo).max() <= 1e-12 * np.abs(u).max()
    assert np.abs(vg - vo).max() <= 1e-12 * np.abs(v).max()
    # exact for quadratics on the device too, role-changed DPs included
    c = (0.3, -0.7, 0.4, 1.3, -0.9, 0.6)
    q = quad(pos_k[0], pos_k[1], c)
    ug, _vg, _fb, _uo, _vo, _ = ale_case(mcd, pb, pos_k, mask_k, pos_k1, mask_k1, bodies, (q, q))
    inner1 = mask_k1 == -1
    assert np.abs(ug[inner1] - quad(pos_k1[0], pos_k1[1], c)[inner1]).max() <= 1e-11
    assert (inner1 & (mask_k != -1)).sum() >= 5


def test_ale_matches_oracle_cylinder_array(mcd):
    """Several bodies: the shift follows the nearest body's normal."""
    pb = inputs.cylinder_array_box(96, 4)
    bodies = pb.meta["bodies"]
    l0 = pb.mesh.l0
    pos_k, mask_k, _ = omask.update_dps_bodies(pb.mesh, pb.pos, pb.mask, bodies, n_relax=4, band=0.0)
    moved = [(b, (c[0] + 0.55 * l0, c[1] - 0.35 * l0), R) for b, c, R in bodies]
    pos_k1, mask_k1, _ = omask.update_dps_bodies(pb.mesh, pos_k, mask_k, moved, n_relax=4)
    u = smooth(pos_k[0], pos_k[1], 4.0)
    v = smooth(pos_k[1], pos_k[0], 2.0)
    ug, vg, fb, uo, vo, fbo = ale_case(mcd, pb, pos_k, mask_k, pos_k1, mask_k1, bodies, (u, v))
    assert fb == fbo
    assert np.abs(ug - uo).max() <= 1e-12 * np.abs(u).max()
    assert np.abs(vg - vo).max() <= 1e-12 * np.abs(v).max()
    assert ((mask_k1 == -1) & (mask_k != -1)).sum() > 25


@pytest.mark.parametrize("n", [48, 96])
def test_fluid_force_matches_oracle(mcd, n):
    mesh, pos, mask, normal, R = body_state(n)
    bc = inputs.default_bc_kind(neumann_ids=(2,))
    Wp = mls.build_weights(mesh, pos, mask, normal, bc)
    Wv = mls.build_weights(mesh, pos, mask)
    x, y = pos
    P = smooth(x, y, 3.0)
    u = smooth(x, y, 4.0)
    v = smooth(y, x, 2.5)
    bnd = np.where(mask == 2, 0.4 * normal[0] - 0.3 * normal[1], np.where(mask == 1, P, 0.0))
    mu = 0.05
    Fo, perim_o, sk_o = ale.fluid_force(mesh, pos, mask, 2, normal, P, bnd, u, v, mu, Wp, Wv)
    pres = mcd.Stencils(mesh, dev(pos.ravel()), dev(mask), dev(normal.ravel()), bc_kind=bc, want_derivs=True,
                        precision=mcd.FP64)
    vel = mcd.Stencils(mesh, dev(pos.ravel()), dev(mask), want_derivs=True, precision=mcd.FP64)
    Fg, perim_g, sk_g = mcd.fluid_force(pres, vel, 2, dev(pos.ravel()), dev(mask), dev(normal.ravel()),
                                        dev(P), dev(bnd), dev(u), dev(v), mu)
    assert sk_g == sk_o == 0
    assert abs(perim_g - perim_o) <= 1e-12 * perim_o
    assert np.abs(np.array(Fg) - Fo).max() <= 1e-10 * np.abs(Fo).max()
    # the closed form for a linear pressure holds on the device as well
    a = (0.7, -0.4)
    Pl = 0.3 + a[0] * x + a[1] * y
    bl = np.where(mask == 2, a[0] * normal[0] + a[1] * normal[1], np.where(mask == 1, Pl, 0.0))
    z = np.zeros(mesh.N)
    Fl, _p, _s = mcd.fluid_force(pres, vel, 2, dev(pos.ravel()), dev(mask), dev(normal.ravel()), dev(Pl),
                                 dev(bl), dev(z), dev(z), 0.0)
    want = -np.array(a) * math.pi * R * R
    assert np.abs(np.array(Fl) - want).max() <= 2e-3 * np.abs(want).max()
