"""GPU parity of the matrix-free stencil SpMV (mcd_apply_laplacian, the rows
of Eq. (21)) on the layouts that select each kernel: non-periodic meshes with
n0 a multiple of 4 (FP32: TMA-streamed tiles; FP64: shared-memory tiles with
16-byte loads), periodic meshes (shared-memory tiles), n0 not a multiple of 4
(scalar tiles); sizes with ragged tiles in x and y; and sampled rows at the
full 4096^2 size.

FP64: the oracle's CSR product to 1e-13 of sum |c_s x_j|.  FP32: the exact
value of the FP32 difference-form row applied to the FP32 vector (computed
in FP64 here) within the rounding of the differences x_j - x_i
(2^-24 sum |c_s (x_j - x_i)|) plus 2 ulp of the result: the kernel splits
every product exactly and sums with TwoSum.
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


def neighbours(mesh, k):
    """Cell index of each of the 9 slots of DP k (slot s = (di+1) + 3 (dj+1));
    a missing neighbour of a non-periodic axis maps onto the cell itself."""
    n0, n1 = mesh.n[0], mesh.n[1]
    i, j = k % n0, k // n0
    out = np.empty((9,) + np.shape(k), dtype=np.int64)
    for s in range(9):
        di, dj = s % 3 - 1, s // 3 - 1
        ii, jj = i + di, j + dj
        if mesh.periodic[0]:
            ii = ii % n0
        else:
            ii = np.where((ii < 0) | (ii >= n0), i, ii)
        if mesh.periodic[1]:
            jj = jj % n1
        else:
            jj = np.where((jj < 0) | (jj >= n1), j, jj)
        out[s] = ii + n0 * jj
    return out


def check_fp32(r32k, x32, y32k, nb, k):
    """y32k (the results of DPs k) against their FP32 difference-form rows
    r32k [9][len(k)] applied exactly to x32."""
    xi = x32[k].astype(np.float64)
    w = r32k.astype(np.float64)
    d = (x32[nb].astype(np.float64) - xi[None, :]).astype(np.float32).astype(np.float64)
    terms = w * d
    terms[4] = w[4] * xi
    exact = terms.sum(axis=0)
    bound = 2.0 ** -24 * np.abs(w * (x32[nb] - xi[None, :])).sum(axis=0) \
        + 2 * np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64) + 1e-30
    err = np.abs(y32k.astype(np.float64) - exact)
    assert np.all(err <= bound), (err / bound).max()


@pytest.mark.parametrize("shape,periodic", [((300, 37), False), ((301, 37), False), ((300, 37), True),
                                            ((64, 8), False), ((128, 129), False)])
def test_spmv_matches_oracle(mcd, shape, periodic):
    pb = inputs.jittered_box(shape, 2, seed=5, periodic=periodic)
    W = mls.build_weights(pb.mesh, pb.pos, pb.mask)
    A = solve.assemble(pb.mesh, W["row"])
    st = mcd.Stencils(pb.mesh, dev(pb.pos.ravel()), dev(pb.mask), precision=mcd.MIXED)
    N = pb.mesh.N
    rng = np.random.default_rng(7)
    x = rng.normal(size=N)
    want = A @ x
    scale = np.abs(A).multiply(np.abs(x)[None, :]).sum(axis=1).A.ravel()
    y64 = st.apply(dev(x)).cpu().numpy()
    assert np.all(np.abs(y64 - want) <= 1e-13 * scale + 1e-300)
    x32 = x.astype(np.float32)
    y32 = st.apply(dev(x32)).cpu().numpy()
    row32 = st.array(mcd.ARR_ROW32).cpu().numpy().reshape(9, N)
    k = np.arange(N)
    check_fp32(row32, x32, y32, neighbours(pb.mesh, k), k)
    # two calls in a row give the same bits (nothing carried between calls)
    assert torch.equal(st.apply(dev(x32)), st.apply(dev(x32)))
    st.close()


def test_spmv_full_size_sampled_rows(mcd):
    """The 4096^2 box of the SpMV benchmark, the launch it times: 8192 sampled
    rows recomputed here from the handle's own rows (FP64 and FP32)."""
    n = 4096
    pb = inputs.manufactured_box(n, 2, seed=0)
    mesh, N = pb.mesh, pb.mesh.N
    st = mcd.Stencils(mesh, dev(pb.pos.ravel()), dev(pb.mask), precision=mcd.MIXED)
    del pb
    g = torch.Generator(device="cuda").manual_seed(0)
    x = torch.rand(N, generator=g, device="cuda", dtype=torch.float64)
    rng = np.random.default_rng(1)
    k = np.unique(np.concatenate([rng.integers(0, N, 8192), [0, n - 1, N - n, N - 1, n * 17 + 127, n * 17 + 128]]))
    kk = torch.from_numpy(k).cuda()
    nb = neighbours(mesh, k)
    y64 = st.apply(x)
    r64 = st.array(mcd.ARR_ROW64).view(9, N)[:, kk].cpu().numpy()
    xs = x.cpu().numpy()
    want = (r64 * xs[nb]).sum(axis=0)
    scale = np.abs(r64 * xs[nb]).sum(axis=0)
    assert np.all(np.abs(y64[kk].cpu().numpy() - want) <= 1e-13 * scale)
    x32 = x.to(torch.float32)
    y32 = st.apply(x32)
    r32 = st.array(mcd.ARR_ROW32).view(9, N)[:, kk].cpu().numpy()
    check_fp32(r32, x32.cpu().numpy(), y32[kk].cpu().numpy(), nb, k)
    st.close()
