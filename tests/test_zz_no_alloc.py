"""The allocation-free DP update against the regular one.

mcd_update_dps_static keeps its Jacobi scratch in a fixed array inside the
library, for callers that must not allocate GPU memory while they step.  It
must give the same masks (bit for bit) and positions as mcd_update_dps, also
when called twice in a row (the second call sees the scratch the first one
left behind).  This file is collected last on purpose.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

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


def test_static_update_matches_regular_update_twice(mcd):
    n = 96
    pb = inputs.cylinder_box(n)
    cyl = pb.meta["cylinder"]
    pos_a = torch.from_numpy(pb.pos.ravel().copy()).cuda()
    mask_a = torch.from_numpy(pb.mask.copy()).cuda()
    prev_a = torch.empty_like(mask_a)
    pos_b, mask_b, prev_b = pos_a.clone(), mask_a.clone(), prev_a.clone()
    for step, (t, band, n_relax) in enumerate([(0.0, 0.0, 7), (0.006, 5 * pb.mesh.l0, 10)]):
        c = cyl.centre(t)
        mcd.update_dps(pb.mesh, c, cyl.radius, cyl.body_id, pos_a, mask_a, prev_a,
                       n_relax=n_relax, band=band)
        mcd.update_dps_static(pb.mesh, c, cyl.radius, cyl.body_id, pos_b, mask_b, prev_b,
                              n_relax=n_relax, band=band)
        torch.cuda.synchronize()
        assert torch.equal(mask_a, mask_b), f"masks differ at call {step}"
        assert torch.equal(prev_a, prev_b)
        err = (pos_a - pos_b).abs().max().item()
        assert err <= 1e-12 * pb.mesh.l0, err


def test_static_update_rejects_meshes_beyond_the_fixed_scratch(mcd):
    n = 1025
    mesh = inputs.Mesh(dim=2, n=(n, n, 1), l0=1.0 / n)
    N = n * n
    pos = torch.zeros(2 * N, dtype=torch.float64, device="cuda")
    mask = torch.full((N,), -1, dtype=torch.int8, device="cuda")
    prev = torch.empty_like(mask)
    with pytest.raises(mcd.McdError) as e:
        mcd.update_dps_static(mesh, (0.5, 0.5), 0.05, 2, pos, mask, prev)
    assert e.value.status == mcd.EINVAL
    assert "MCD_NOALLOC_MAX_DPS" in str(e.value)
