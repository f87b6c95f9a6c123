"""The network as a preconditioner of the mixed solve's refinement
(mcd_solve_params.precond).  At every update that restarts the FP32
recursion the solve hands the FP64 residual to the network, adds its
correction along the residual-minimising step (the warm start's line search)
and relaunches from the corrected iterate; a correction that cuts the
residual by less than 10 % ends the network's part for the rest of the solve.

System: the cylinder box at 128^2 after the DP update (Neumann body with an
accelerating datum), source sin(pi x) sin(pi y) on the inner DPs, every
solve from p = 0.  The oracle fixes which branch each network takes: its
first correction (oracle.cnn features, the bf16 forward pass, warm_start)
brings the residual to about 0.59 of ||r0|| for a network that returns its
residual channel (a Richardson step with the optimal step length), and
leaves it within 1e-8 of ||r0|| for a He-normal network.

* He-normal network: exactly one correction, after which the solve is the
  plain mixed solve from the corrected guess.  It therefore equals, bit for
  bit, the solve that takes the same network as its warm start (whose
  correction test_gpu_cnn checks against the oracle).
* Richardson network: a correction at the first update and again at the
  next restarting update; the pressure matches oracle.solve.direct_solve to
  1e-6 relative L2 at tol 1e-10 (the mixed mode's tolerance).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cnn, mls, solve  # noqa: E402
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


NETS = {"richardson": lambda: inputs.cnn_weights_extrapolating(5, scale=0.0, channel=0),
        "he": lambda: inputs.cnn_weights(5)}


@pytest.fixture(scope="module")
def system():
    """The oracle's system, its exact solution and each network's first
    correction ratio ||b - A q|| / ||b - A p0||."""
    n = 128
    pb = inputs.cylinder_box(n)
    cyl = pb.meta["cylinder"]
    c = cyl.centre(0.0)
    pos, m, _ = omask.update_dps(pb.mesh, pb.pos, pb.mask, c, cyl.radius, band=0.0, n_relax=4)
    normal = omask.circle_normals(pos, m, c, cyl.body_id)
    W = mls.build_weights(pb.mesh, pos, m, normal, pb.bc_kind)
    X, Y = pos
    rhs = np.where(m == -1, np.sin(np.pi * X) * np.sin(np.pi * Y), 0.0)
    a = cyl.acceleration(0.05)
    bnd = np.where(m == cyl.body_id, -(a[0] * normal[0] + a[1] * normal[1]), 0.0)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], rhs, bnd, W["rscale"])
    unknown = (W["kind"] == 1) | (W["kind"] == 3)
    p0 = np.where(unknown, 0.0, b / np.where(W["rscale"] != 0, W["rscale"], 1.0))
    p0 = np.where(W["kind"] == 0, 0.0, p0)
    r0 = b - A @ p0
    ratio = {}
    for name, make in NETS.items():
        ws, bs = make()
        x, (_s_r, _s_d, s_out) = cnn.features(pb.mesh, r0, m, pos, None)
        y = cnn.forward([cnn.bf16_round(w) for w in ws], bs, cnn.bf16_round(x)[:7],
                        rnd=cnn.bf16_round)[-1][0].ravel()
        q, _s = cnn.warm_start(A, b, p0, np.where(unknown, y * s_out, 0.0))
        ratio[name] = np.linalg.norm(b - A @ q) / np.linalg.norm(r0)
    return dict(pb=pb, pos=pos, m=m, normal=normal, rhs=rhs, bnd=bnd, want=solve.direct_solve(A, b),
                ratio=ratio)


def stencils(mcd, s):
    pb = s["pb"]
    return mcd.Stencils(pb.mesh, dev(s["pos"].ravel()), dev(s["m"]), dev(s["normal"].ravel()),
                        bc_kind=pb.bc_kind, precision=mcd.MIXED)


def net_of(mcd, name):
    return mcd.Net(inputs.cnn_flatten(*NETS[name]()))


@pytest.mark.parametrize("update_restart", [0, 1])
def test_failed_correction_leaves_the_plain_solve(mcd, system, update_restart):
    assert system["ratio"]["he"] > 1.0 - 1e-8
    st = stencils(mcd, system)
    net = net_of(mcd, "he")
    rhs, bnd = dev(system["rhs"]), dev(system["bnd"])
    kw = dict(tol=1e-10, mode=mcd.MIXED, update_restart=update_restart)
    p_pre, info_pre = st.solve(rhs, bnd, precond=net, **kw)
    p_ws, info_ws = st.solve(rhs, bnd, net=net, **kw)
    assert info_pre["net_corrections"] == 1
    assert info_ws["net_corrections"] == 0
    assert torch.equal(p_pre, p_ws)
    assert info_pre["iters"] == info_ws["iters"]
    assert info_pre["rel_res"] == info_ws["rel_res"] and info_pre["rel_res"] <= 1e-10
    st.close()


def test_corrections_at_restarts_converge_to_the_oracle(mcd, system):
    assert system["ratio"]["richardson"] < 0.8
    st = stencils(mcd, system)
    net = net_of(mcd, "richardson")
    p, info = st.solve(dev(system["rhs"]), dev(system["bnd"]), tol=1e-10, mode=mcd.MIXED,
                       update_restart=1, precond=net)
    assert info["net_corrections"] >= 2
    assert info["rel_res"] <= 1e-10
    want = system["want"]
    got = p.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) <= 1e-6
    # the same system without the network, for the record of the two paths
    p0, info0 = st.solve(dev(system["rhs"]), dev(system["bnd"]), tol=1e-10, mode=mcd.MIXED,
                         update_restart=1)
    assert np.linalg.norm(p0.cpu().numpy() - want) / np.linalg.norm(want) <= 1e-6
    assert info0["net_corrections"] == 0
    st.close()
