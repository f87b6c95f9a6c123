"""GPU parity at the benchmark's full size: the 1024 x 1024 oscillating-
cylinder system, in the launch configuration of the benchmark's first step.
That is the DP update with 30 relaxation sweeps, band 0, the Neumann
cylinder, the stencil build and the persistent mixed solve to 1e-8.

Each output is checked against the oracle at this size, or through a
property that holds at any size:
- masks: every cell, bit-exact, against the oracle's role rule (Eq. (1),
  Sec. 2.4).
- positions: sampled DPs on and next to the cylinder, against the
  oracle's update run on a 66 x 66 window around each one, to 1e-10 l0.
  The relaxation is a Jacobi sweep over the 3 x 3 neighbours.  After 30
  sweeps a DP depends only on cells at most 30 away, so the window's edge,
  32 or more cells away, cannot reach it.
- every DP stays in its closed cell.
- normals of the sampled body DPs, against the oracle's normal.
- PPE rows: sampled DPs (inner, Dirichlet wall, Neumann body) against
  the oracle's per-DP fit, from the GPU's positions and masks, within
  the weight tolerance of the parity tests.
- the solve: its FP64 residual, recomputed with the FP64 SpMV (a separate
  kernel), is at most the tolerance.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mask as omask  # noqa: E402
from oracle import mls  # noqa: E402
from paper_2404_17542_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

N_SIDE = 1024
N_RELAX = 30
WINDOW = 66
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


def window_update(pb, k, centre, radius, body_id):
    """The oracle's DP update on the WINDOW x WINDOW cells around cell k;
    returns the position and mask it gives DP k."""
    mesh, W = pb.mesh, WINDOW
    nx, l0 = mesh.n[0], mesh.l0
    i0, j0 = k % nx - W // 2, k // nx - W // 2
    wm = dataclasses.replace(mesh, n=(W, W, 1),
                             origin=(mesh.origin[0] + i0 * l0, mesh.origin[1] + j0 * l0, 0.0))
    ii, jj = np.meshgrid(np.arange(i0, i0 + W), np.arange(j0, j0 + W), indexing="xy")
    cells = (ii + nx * jj).ravel()          # window cell a + W b <- mesh cell
    p, m, _ = omask.update_dps(wm, pb.pos[:, cells].copy(), pb.mask[cells].copy(), centre, radius,
                               body_id=body_id, kappa=0.2, n_relax=N_RELAX, band=0.0)
    kc = W // 2 + W * (W // 2)
    return p[:, kc], m[kc]


def test_cylinder_system_full_size(mcd):
    pb = inputs.cylinder_box(N_SIDE)
    mesh, N, l0 = pb.mesh, pb.mesh.N, pb.mesh.l0
    cyl = pb.meta["cylinder"]
    c, R, bid = cyl.centre(0.0), cyl.radius, cyl.body_id
    pos, mask = dev(pb.pos.ravel()), dev(pb.mask)
    prev = torch.empty_like(mask)
    mcd.update_dps(mesh, c, R, bid, pos, mask, prev, kappa=0.2, n_relax=N_RELAX, band=0.0)
    normal = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    neu = torch.zeros(N, dtype=torch.float64, device="cuda")
    mcd.body_boundary(mesh, c, R, bid, pos, mask, acc=cyl.acceleration(0.0), normal=normal, neumann=neu)
    P = pos.cpu().numpy().reshape(2, N)
    M = mask.cpu().numpy()

    # masks, every cell
    assert np.array_equal(M, omask.remask(mesh, pb.mask, c, R, bid, 0.0))
    assert (M == bid).sum() > 100

    # positions: in the closed cell; sampled DPs against the windowed oracle
    ij = np.stack([np.arange(N) % mesh.n[0], np.arange(N) // mesh.n[0]])
    assert ((P >= ij * l0 - 1e-12 * l0) & (P <= (ij + 1) * l0 + 1e-12 * l0)).all()
    rng = np.random.default_rng(7)
    body = np.nonzero(M == bid)[0]
    d = np.hypot(pb.pos[0] - c[0], pb.pos[1] - c[1]) - R
    near_inner = np.nonzero((M == -1) & (d > 0) & (d < 3 * l0))[0]
    sample = list(rng.choice(body, 4, replace=False)) + list(rng.choice(near_inner, 1))
    Nrm = omask.circle_normals(P, M, c, bid)
    G = normal.cpu().numpy().reshape(2, N)
    for k in sample:
        p_o, m_o = window_update(pb, int(k), c, R, bid)
        assert m_o == M[k], k
        assert np.abs(P[:, k] - p_o).max() <= 1e-10 * l0, (k, P[:, k], p_o)
        assert np.abs(G[:, k] - Nrm[:, k]).max() <= 1e-12, k

    # PPE rows of sampled DPs against the oracle's per-DP fit
    st = mcd.Stencils(mesh, pos, mask, normal, bc_kind=pb.bc_kind, precision=mcd.MIXED)
    rows = st.array(mcd.ARR_ROW64).cpu().numpy().reshape(9, N)
    walls = np.nonzero(M == 1)[0]
    inner = np.nonzero(M == -1)[0]
    rows_sample = (list(rng.choice(inner, 30, replace=False)) + list(rng.choice(walls, 5, replace=False))
                   + list(rng.choice(body, 15, replace=False)) + list(near_inner[:5]))
    for i in rows_sample:
        f = mls.dp_fit(mesh, P, M, Nrm, pb.bc_kind, int(i))
        scale = np.abs(f["row"]).max()
        assert np.abs(rows[:, i] - f["row"]).max() <= WEIGHT_TOL * scale, i

    # the solve: FP64 residual of the returned field
    rhs = dev(inputs.ppe_source(pb.pos, 0.0))
    p, info = st.solve(rhs, neu, tol=1e-8, mode=mcd.MIXED)
    assert info["status"] == 0 and info["rel_res"] <= 1e-8
    b = st.assemble_rhs(rhs, neu)
    r = b - st.apply(p)
    assert float(r.norm() / b.norm()) <= 1.01e-8
