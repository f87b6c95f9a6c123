"""Parity of the benchmark's own path at 512^2 (the headline's path at a size
the oracle solves in about a minute): full moving-boundary steps of the
oscillating cylinder through mcd_flow_step (DP update, ALE interpolation of
u, v and of the pressure guess, stencils, predict, PPE, projection), the
learned warm start trained on the run's first steps, and the mixed solve
(TMA-staged FP32 recursion, FP64 true residual).  512 tiles of 32 x 16 over
the persistent grid: blocks own one or two tiles.

After the learned steps the pressure is compared element by element with
oracle.solve.direct_solve of the same step's system, assembled by the oracle
from the step's DP positions, masks, normals, Neumann data and PPE source
(the GPU's DP update is checked bit-exact against the oracle elsewhere):
within 1e-6 relative L2 over the non-void DPs at tol 1e-10, the mixed
mode's pressure tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import mls, solve  # noqa: E402
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


def test_learned_mixed_flow_steps_match_oracle(mcd):
    n = 512
    cyl = inputs.Cylinder()
    pb = inputs.cylinder_box(n, cyl)
    mesh = pb.mesh
    nu = 2 * cyl.radius / 100.0
    dt = min(0.2 * mesh.l0, 0.2 * mesh.l0 ** 2 / nu)

    def bodies_at(t):
        return [(cyl.body_id, cyl.centre(t), cyl.radius)], [cyl.velocity(t)]

    flow = mcd.AleFlow(mesh, torch.from_numpy(pb.pos.ravel().copy()).cuda(),
                       torch.from_numpy(pb.mask.copy()).cuda(), bodies_at, nu, dt, precision=mcd.MIXED,
                       mode=mcd.MIXED, tol=1e-10, ale_pressure=True)
    net = mcd.Net(inputs.cnn_flatten(*inputs.cnn_weights_extrapolating(3)))
    samples = []
    dprev = torch.zeros(mesh.N, dtype=torch.float64, device="cuda")
    for k in range(12):
        flow.step()
        st = flow.stencils(mcd.FLOW_PRESSURE)
        b = flow.array(mcd.FLOW_B)
        guess = flow.array(mcd.FLOW_GUESS)
        if k >= 2:
            samples.append(net.features(st, b, guess, dprev, flow.P))
        dprev = flow.P - guess
    for _ep in range(3):
        for x, tg, wt in samples:
            net.train_step(x, tg, wt, n, n, 1e-3)
    for _step in range(2):
        info = flow.step(net=net, dprev=dprev)
        solve_info = info["solve"]
        assert solve_info["rel_res"] <= 1e-10
        assert solve_info["rel_res_guess"] > 0.0 and solve_info["rel_res_start"] <= solve_info["rel_res_guess"]
    # the oracle's exact PPE solution of the last step's system
    pos = flow.pos.cpu().numpy().reshape(2, -1)
    m = flow.mask.cpu().numpy()
    normal = flow.array(mcd.FLOW_NORMAL).cpu().numpy().reshape(2, -1)
    bnd = flow.array(mcd.FLOW_BND).cpu().numpy()
    src = flow.array(mcd.FLOW_SRC).cpu().numpy()
    W = mls.build_weights(mesh, pos, m, normal, pb.bc_kind)
    A = solve.assemble(mesh, W["row"])
    b = solve.form_rhs(mesh, W["kind"], W["QL"], src, bnd, W["rscale"])
    want = solve.direct_solve(A, b)
    got = flow.P.cpu().numpy()
    fluid = m != 0
    err = np.linalg.norm(got[fluid] - want[fluid]) / np.linalg.norm(want[fluid])
    assert err <= 1e-6, err
    # and the assembled right-hand side the library used is the oracle's
    b_gpu = flow.array(mcd.FLOW_B).cpu().numpy()
    assert np.abs(b_gpu - b).max() <= 1e-10 * np.abs(b).max()
    flow.close()
