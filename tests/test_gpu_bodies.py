"""GPU parity of the DP update with several bodies (Sec. 2.2-2.5): the CUDA
path through the C ABI against the oracle on the 25-cylinder array.

Masks and previous masks bit-exact; positions within 1e-10 l0 (FP64 on both
sides, fused multiply-adds on the device).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def shifted(bodies, dx, dy):
    return [(bid, (c[0] + dx, c[1] + dy), R) for bid, c, R in bodies]


@pytest.mark.parametrize("gap_cells,alpha", [(12, 0.0), (2, 0.03)])
def test_array_update_matches_oracle(mcd, gap_cells, alpha):
    pb = inputs.cylinder_array_box(96, gap_cells)
    bodies = pb.meta["bodies"]
    l0 = pb.mesh.l0
    pos_o, m_o = pb.pos.copy(), pb.mask.copy()
    pos_g, m_g = dev(pb.pos.ravel()), dev(pb.mask)
    prev_g = torch.empty_like(m_g)
    # initial arrangement over every cell, then two band updates of a moved array
    for step, (dx, dy) in enumerate([(0.0, 0.0), (0.37 * l0, -0.21 * l0), (0.81 * l0, 0.12 * l0)]):
        bl = shifted(bodies, dx, dy)
        band = 0.0 if step == 0 else 5 * l0
        pos_o, m_new, prev_o = omask.update_dps_bodies(pb.mesh, pos_o, m_o, bl, n_relax=6, band=band,
                                                       alpha=alpha)
        mcd.update_dps_bodies(pb.mesh, bl, pos_g, m_g, prev_g, kappa=0.2, n_relax=6, band=band,
                              alpha=alpha)
        assert np.array_equal(m_g.cpu().numpy(), m_new)
        assert np.array_equal(prev_g.cpu().numpy(), m_o)
        pg = pos_g.cpu().numpy().reshape(2, -1)
        assert np.abs(pg - pos_o).max() <= 1e-10 * l0
        m_o = m_new
        pos_g.copy_(dev(pos_o.ravel()))
    ids = set(int(v) for v in np.unique(m_o) if v >= 2)
    assert ids == {b[0] for b in bodies}


def test_bodies_boundary_data(mcd):
    pb = inputs.cylinder_array_box(64, 6)
    bodies = pb.meta["bodies"]
    pos, m, _ = omask.update_dps_bodies(pb.mesh, pb.pos, pb.mask, bodies, n_relax=3, band=0.0)
    rng = np.random.default_rng(3)
    accs = [tuple(rng.uniform(-2, 2, size=2)) for _ in bodies]
    ng, fg = mcd.bodies_boundary(pb.mesh, bodies, dev(pos.ravel()), dev(m), accs=accs)
    normal = omask.bodies_normals(pos, m, bodies)
    assert np.allclose(ng.cpu().numpy().reshape(2, -1), normal, rtol=0, atol=1e-14)
    want = np.zeros(pb.mesh.N)
    for (bid, _c, _R), a in zip(bodies, accs):
        sel = m == bid
        want[sel] = -(a[0] * normal[0, sel] + a[1] * normal[1, sel])
    assert np.allclose(fg.cpu().numpy(), want, rtol=0, atol=1e-13)


def test_bad_body_lists_are_rejected(mcd):
    pb = inputs.cylinder_array_box(32, 6)
    pos_g, m_g = dev(pb.pos.ravel()), dev(pb.mask)
    prev_g = torch.empty_like(m_g)
    b = pb.meta["bodies"]
    with pytest.raises(mcd.McdError):
        mcd.update_dps_bodies(pb.mesh, [b[0], (b[0][0], b[1][1], b[1][2])], pos_g, m_g, prev_g)
    many = [(2 + k % 100, (0.5, 0.5), 0.01) for k in range(65)]
    with pytest.raises(mcd.McdError):
        mcd.update_dps_bodies(pb.mesh, many, pos_g, m_g, prev_g)
    assert np.array_equal(m_g.cpu().numpy(), pb.mask)   # nothing ran
