"""GPU tests of the persistent solver's grid barriers (Sec. 3.3 solve).

- Every schedule matches the oracle's direct solve, in FP64 and mixed mode,
  within the parity tests' tolerances: two grid barriers per iteration (the
  default), one (mixed, non-periodic 2D 3x3 meshes) and three.  The
  one-barrier schedule is Bi-CGSTAB with its reductions merged (omega and
  beta from dot-product polynomials in alpha, t from the recurrence
  u - alpha q); in FP32 those recurrences round differently, and its
  iteration count stays within 25 % of the two-barrier count.
- Results are deterministic.  Block 0 adds the blocks' partial sums in
  block order, so two solves of the same system give bit-identical fields
  and iteration counts.
- The bounded wait of the barriers gives up with MCD_ETIMEOUT when nothing
  sets the polled word (a flag that no one sets, no GPU fault), and the
  context stays usable for a solve afterwards.
- The barrier-stage stamps of the trace are causally ordered, per barrier:
  - block 0 enters, publishes its partials, has every partial and updates
    the scalars, in that order;
  - the last block publishes its partials before block 0 has them all;
  - every released block wakes after block 0's scalar update.
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def small():
    # 160 x 160 cells: 5 x 10 tiles of 32 x 16, one per block
    pb = inputs.manufactured_box(160, 2, seed=3)
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    A = solve.assemble(pb.mesh, W["row"])
    b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], pb.rhs, pb.bnd, W["rscale"])
    return pb, solve.direct_solve(A, b)


@pytest.fixture(scope="module")
def large():
    # 400 x 400 cells: 13 x 25 tiles (a ragged column) over at most 304
    # blocks, so some blocks own two tiles
    return inputs.manufactured_box(400, 2, seed=5)


def stencils(mcd, pb):
    return mcd.Stencils(pb.mesh, dev(pb.pos.ravel()), dev(pb.mask), want_derivs=False)


# (FP64 / mixed, barriers: 0 default (two), 1 (mixed: one), 3)
SCHEDULES = [(0, 0), (1, 0), (1, 1), (0, 3), (1, 3)]


@pytest.mark.parametrize("mode,barriers", SCHEDULES)
def test_schedules_match_oracle(mcd, small, mode, barriers):
    pb, x = small
    tol = 1e-11 if mode == 0 else 1e-10
    p, info = stencils(mcd, pb).solve(dev(pb.rhs), dev(pb.bnd), tol=tol, mode=mode, barriers=barriers)
    assert info["rel_res"] <= tol
    got = p.cpu().numpy()
    assert np.linalg.norm(got - x) / np.linalg.norm(x) <= (1e-8 if mode == 0 else 1e-6)


@pytest.mark.parametrize("mode,barriers", SCHEDULES)
def test_solves_are_bit_identical(mcd, large, mode, barriers):
    st = stencils(mcd, large)
    tol = 1e-11 if mode == 0 else 1e-10
    runs = [st.solve(dev(large.rhs), dev(large.bnd), tol=tol, mode=mode, barriers=barriers) for _ in range(2)]
    (p1, i1), (p2, i2) = runs
    assert i1["rel_res"] <= tol
    assert i1["iters"] == i2["iters"] and i1["fallback"] == i2["fallback"]
    assert torch.equal(p1, p2)


def test_barrier_trace_is_causally_ordered(mcd, large):
    st = stencils(mcd, large)
    mcd.trace_enable(True)
    try:
        _p, info = st.solve(dev(large.rhs), dev(large.bnd), tol=1e-10, mode=mcd.MIXED)
        _ph, _end, _sm, _start, bar = mcd.trace_read()
    finally:
        mcd.trace_enable(False)
    bar = bar.astype(np.int64)
    epochs = [e for e in range(1, 256) if (bar[e] > 0).all()]
    assert len(epochs) >= min(100, info["iters"])
    for e in epochs:
        t = bar[e]
        assert t[0] <= t[1] <= t[2] <= t[3] <= t[4] <= t[5], (e, t)
        assert t[6] <= t[2], (e, t)   # the last arrival precedes "every partial seen"
        assert t[7] >= t[4], (e, t)   # wake-ups follow the scalar update


def test_bounded_wait_reports_timeout_and_context_survives(mcd, small):
    assert mcd.selftest_bounded_wait(True) == mcd.OK
    assert mcd.selftest_bounded_wait(False, polls=2048) == mcd.ETIMEOUT
    assert b"gave up" in mcd.lib().mcd_last_error()
    pb, x = small
    p, info = stencils(mcd, pb).solve(dev(pb.rhs), dev(pb.bnd), tol=1e-10, mode=mcd.MIXED)
    assert info["rel_res"] <= 1e-10
    assert np.linalg.norm(p.cpu().numpy() - x) / np.linalg.norm(x) <= 1e-6


@pytest.mark.parametrize("shape", [(1000, 700), (404, 397)])
def test_staged_operands_match_direct_loads(mcd, shape):
    """The FP32 two-barrier solve with each tile's operands staged by TMA
    (the default on non-periodic 2D 3x3 meshes) and with direct loads runs
    the same arithmetic in the same order: the same iterations and the same
    bits.  1000 x 700 gives blocks several tiles (the two-stage pipeline
    turns over); 404 x 397 leaves ragged tiles in x and y, where the copies
    reach past the mesh.  The solution also meets the oracle."""
    pb = inputs.manufactured_box(shape, 2, seed=9)
    st = mcd.Stencils(pb.mesh, dev(pb.pos.ravel()), dev(pb.mask), precision=mcd.MIXED)
    out = {}
    try:
        for staged in (True, False):
            mcd.solver_set_staging(staged)
            p, info = st.solve(dev(pb.rhs), dev(pb.bnd), tol=1e-10, mode=mcd.MIXED)
            out[staged] = (p.clone(), info)
    finally:
        mcd.solver_set_staging(True)
    (p1, i1), (p0, i0) = out[True], out[False]
    assert i1["iters"] == i0["iters"] and i1["refinements"] == i0["refinements"]
    assert torch.equal(p1, p0)
    assert i1["rel_res"] <= 1e-10 and i1["fallback"] == 0
    if shape[0] * shape[1] <= 404 * 397:
        W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
        A = solve.assemble(pb.mesh, W["row"])
        b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], pb.rhs, pb.bnd, W["rscale"])
        x = solve.direct_solve(A, b)
        got = p1.cpu().numpy()
        assert np.linalg.norm(got - x) <= 1e-6 * np.linalg.norm(x)


@pytest.mark.parametrize("shape", [(1000, 700), (404, 397)])
def test_one_barrier_schedule(mcd, shape):
    """The one-barrier schedule against the two-barrier default on the same
    system: both meet tol and the oracle, and the iteration counts agree
    within 25 % (4667 against 4003 at 1000 x 700).  Repeat solves are
    bit-identical.  1000 x 700: blocks own several tiles; 404 x 397: ragged
    tiles, where the two-cell halo copies reach past the mesh."""
    pb = inputs.manufactured_box(shape, 2, seed=9)
    st = mcd.Stencils(pb.mesh, dev(pb.pos.ravel()), dev(pb.mask), precision=mcd.MIXED)
    p1, i1 = st.solve(dev(pb.rhs), dev(pb.bnd), tol=1e-10, mode=mcd.MIXED, barriers=1)
    p1b, i1b = st.solve(dev(pb.rhs), dev(pb.bnd), tol=1e-10, mode=mcd.MIXED, barriers=1)
    p2, i2 = st.solve(dev(pb.rhs), dev(pb.bnd), tol=1e-10, mode=mcd.MIXED)
    assert torch.equal(p1, p1b) and i1["iters"] == i1b["iters"]
    assert i1["rel_res"] <= 1e-10 and i2["rel_res"] <= 1e-10
    assert i1["fallback"] == 0
    assert abs(i1["iters"] - i2["iters"]) <= 0.25 * i2["iters"], (i1["iters"], i2["iters"])
    assert np.linalg.norm((p1 - p2).cpu().numpy()) <= 1e-6 * np.linalg.norm(p2.cpu().numpy())
    if shape[0] * shape[1] <= 404 * 397:
        W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
        A = solve.assemble(pb.mesh, W["row"])
        b = solve.form_rhs(pb.mesh, W["kind"], W["QL"], pb.rhs, pb.bnd, W["rscale"])
        x = solve.direct_solve(A, b)
        assert np.linalg.norm(p1.cpu().numpy() - x) / np.linalg.norm(x) <= 1e-6
