"""GPU parity of the batched solve (independent systems in one persistent
launch, CUDA graph replay, autotuned tiling).

Every system of a batch must match the oracle's direct solve of the same
system (oracle/mls.py weights, oracle/solve.py sparse LU): 1e-6 relative L2
for the mixed mode at tol 1e-10 (the single-system mixed bar) and 1e-9 for
FP64 at tol 1e-12.  Graph replays and other tilings reproduce the direct
launch to the solver tolerance (the per-system dot products are summed with
atomics, so results agree to rounding, not bit for bit).  At the full size
of the log-uniform 32^2 .. 512^2 workload every system must converge to its
tolerance (FP64 residual) and the smallest ones are checked against the
oracle.
"""
import os

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def make_batch(mcd, problems, precision):
    bt = mcd.Batch([pb.mesh for pb in problems], precision=precision)
    pos = dev(bt.pack_positions([pb.pos for pb in problems]))
    mask = dev(np.concatenate([pb.mask for pb in problems]))
    rhs = dev(np.concatenate([pb.rhs for pb in problems]))
    bnd = dev(np.concatenate([pb.bnd for pb in problems]))
    bt.build(pos, mask)
    return bt, rhs, bnd


def oracle_solution(pb):
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], pb.rhs, pb.bnd, W["rscale"])
    return solve.direct_solve(A, b)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def small_batch():
    sizes = inputs.batched_sizes(4, count=14, lo=5, hi=48)
    sizes[0], sizes[1] = 1, 2         # degenerate systems: every DP on the wall
    probs = [inputs.poly4_box(int(n), seed=100 + i) for i, n in enumerate(sizes)]
    return probs, [oracle_solution(pb) for pb in probs]


@pytest.mark.parametrize("mode,tol,bar", [(1, 1e-10, 1e-6), (0, 1e-12, 1e-9)])
def test_batch_matches_oracle(mcd, small_batch, mode, tol, bar):
    probs, want = small_batch
    bt, rhs, bnd = make_batch(mcd, probs, mcd.MIXED)
    p, res = bt.solve(rhs, bnd, tol=tol, mode=mode)
    got = p.cpu().numpy()
    assert np.all(res["status"] == 0)
    assert np.all(res["rel_res"] <= tol)
    for i, pb in enumerate(probs):
        gi = got[bt.offsets[i]:bt.offsets[i + 1]]
        assert rel(gi, want[i]) <= bar, (i, pb.mesh.n)


def test_batch_tilings_and_graph_agree(mcd, small_batch):
    probs, want = small_batch
    bt, rhs, bnd = make_batch(mcd, probs, mcd.MIXED)
    ref, _ = bt.solve(rhs, bnd, tol=1e-10)
    ref = ref.cpu().numpy()
    for rows in (1, 2, 4):
        for cps in (1, 2, 4):   # 4: the 64-register builds (FP32 1-2 rows) at full occupancy
            bt.set_tuning(rows, cps)
            p, res = bt.solve(rhs, bnd, tol=1e-10, graph=(rows == 2))
            assert np.all(res["status"] == 0)
            assert rel(p.cpu().numpy(), ref) <= 1e-8
    # replay of the captured graph with the same arguments
    bt.set_tuning(2, 1)
    p = torch.zeros(bt.N, dtype=torch.float64, device="cuda")
    for _ in range(3):
        p.zero_()
        p, res = bt.solve(rhs, bnd, p=p, tol=1e-10, graph=True)
        assert np.all(res["status"] == 0)
        assert rel(p.cpu().numpy(), ref) <= 1e-8


def test_batch_autotune_cache(mcd, small_batch, tmp_path):
    probs, _ = small_batch
    bt, rhs, bnd = make_batch(mcd, probs, mcd.MIXED)
    p = torch.zeros(bt.N, dtype=torch.float64, device="cuda")
    cache = tmp_path / "tune.txt"
    ms = bt.autotune(rhs, bnd, p, sweeps=20, cache_path=cache)
    assert ms > 0
    choice = bt.tuning()
    assert choice[0] in (1, 2, 4) and 1 <= choice[1] <= 4
    lines = cache.read_text().strip().splitlines()
    assert len(lines) == 1 and " | " in lines[0]
    bt.set_tuning(1, 1)
    ms2 = bt.autotune(rhs, bnd, p, sweeps=20, cache_path=cache)   # read from the cache
    assert bt.tuning() == choice and ms2 == pytest.approx(ms, rel=1e-5)
    assert len(cache.read_text().strip().splitlines()) == 1
    p.zero_()
    p, res = bt.solve(rhs, bnd, p=p, tol=1e-10)
    assert np.all(res["status"] == 0)


def test_batch_rejects_neumann_and_3d(mcd):
    pb = inputs.poly4_box(8, seed=1)
    with pytest.raises(mcd.McdError):
        mcd.Batch([pb.mesh], bc_kind=inputs.default_bc_kind(neumann_ids=(2,)))
    pb3 = inputs.manufactured_box(4, 3, seed=0)
    with pytest.raises(mcd.McdError):
        mcd.Batch([pb3.mesh])


@pytest.mark.slow
def test_full_batched_workload(mcd):
    """256 systems of log-uniform size 32^2 .. 512^2 (seed 4)."""
    probs = inputs.batched_poly4(4)
    bt, rhs, bnd = make_batch(mcd, probs, mcd.MIXED)
    for rows, cps in ((2, 2), (4, 2)):
        bt.set_tuning(rows, cps)
        p, res = bt.solve(rhs, bnd, tol=1e-8, graph=True)
        print(f"tiling {rows}x{cps}: FP64 finishes {int(res['fallback'].sum())}, "
              f"iterations max {res['iters'].max()}")
        assert np.all(res["status"] == 0)
    assert np.all(res["rel_res"] <= 1e-8)
    got = p.cpu().numpy()
    order = np.argsort([pb.mesh.N for pb in probs])[:3]
    for i in order:
        want = oracle_solution(probs[i])
        gi = got[bt.offsets[i]:bt.offsets[i + 1]]
        assert rel(gi, want) <= 1e-6, (i, probs[i].mesh.n)


def test_system_views_at_odd_offsets(mcd):
    """System i of a batch as a stencil handle (mcd_batch_stencils): its rows
    start at DP offset off_i inside the batch's arrays, odd here (the systems
    before it have odd cell counts), so the SpMV takes its scalar path.  The
    product matches the oracle's matrix of that system; the learned warm
    start runs per system inside the batched solve, never raises a system's
    residual, and every system still converges to the oracle's solution."""
    sizes = [33, 35, 40, 37, 44]
    probs = [inputs.poly4_box(n, seed=300 + i) for i, n in enumerate(sizes)]
    bt, rhs, bnd = make_batch(mcd, probs, mcd.MIXED)
    offs = bt.offsets
    assert offs[1] % 2 == 1 and offs[2] % 2 == 0 and offs[3] % 2 == 0 and offs[4] % 2 == 1
    rng = np.random.default_rng(5)
    for i, pb in enumerate(probs):
        st = bt.stencils(i)
        W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
        A = solve.assemble(pb.mesh, W["row"])
        x = rng.normal(size=pb.mesh.N)
        # x and y start at the system's offset too (slices of batch-sized arrays)
        big = torch.zeros(int(offs[-1]), dtype=torch.float64, device="cuda")
        big[offs[i]:offs[i + 1]] = dev(x)
        out = torch.zeros_like(big)
        st.apply(big[offs[i]:offs[i + 1]], out[offs[i]:offs[i + 1]])
        want = A @ x
        scale = np.abs(A).multiply(np.abs(x)[None, :]).sum(axis=1).A.ravel()
        got = out[offs[i]:offs[i + 1]].cpu().numpy()
        assert np.all(np.abs(got - want) <= 1e-13 * scale + 1e-300), i
    net = mcd.Net(inputs.cnn_flatten(*inputs.cnn_weights(7)))
    p, res = bt.solve(rhs, bnd, tol=1e-10, mode=mcd.MIXED, net=net)
    assert (res["status"] == 0).all()
    got = p.cpu().numpy()
    for i, pb in enumerate(probs):
        assert rel(got[offs[i]:offs[i + 1]], oracle_solution(pb)) <= 1e-6, i
