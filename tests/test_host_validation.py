"""Host-side argument checks of the C ABI (no GPU needed).

Every call here is rejected by the library's host code before any device
work: bad body lists and SDF grids, stencil options (support radius, weight
kind, periodic axes too short for the 9x9 window, the batch on wide
stencils), and NULL arguments of the ALE and force entry points (the flow
driver's refusal of wide stencils needs a built handle: a GPU test).  Pointers are placeholders that the rejected calls never touch.
"""
import ctypes as C

import pytest


@pytest.fixture(scope="module")
def mcd():
    from paper_2404_17542_gb300 import build
    build.build()
    from paper_2404_17542_gb300 import mcd as m
    m.lib()
    return m


PH = C.c_void_p(0x1000)   # placeholder, never dereferenced by a rejected call


def mesh2d(mcd, n=16, periodic=False):
    m = mcd.c_mesh()
    m.dim = 2
    m.n[0], m.n[1], m.n[2] = n, n, 1
    m.l0 = 1.0 / n
    if periodic:
        m.periodic[0] = m.periodic[1] = 1
    return m


def update(mcd, mesh, bodies, n):
    return mcd.lib().mcd_update_dps(C.byref(mesh), bodies, n, PH, PH, PH, 0.2, 4, 0.1, 0.0, None)


def circle(mcd, bid, r=0.1):
    return mcd.make_body((0.5, 0.5), r, bid)


def test_body_lists_rejected(mcd):
    m = mesh2d(mcd)
    one = (mcd.c_body * 1)(circle(mcd, 2))
    assert update(mcd, m, one, 0) == mcd.EINVAL                      # no body
    many = (mcd.c_body * 65)(*[circle(mcd, 2 + k) for k in range(65)])
    assert update(mcd, m, many, 65) == mcd.EINVAL                    # more than MCD_MAX_BODIES
    dup = (mcd.c_body * 2)(circle(mcd, 3), circle(mcd, 3))
    assert update(mcd, m, dup, 2) == mcd.EINVAL                      # repeated id
    wall = (mcd.c_body * 1)(circle(mcd, 1))
    assert update(mcd, m, wall, 1) == mcd.EINVAL                     # id 1 is the wall
    flat = (mcd.c_body * 1)(circle(mcd, 2, r=0.0))
    assert update(mcd, m, flat, 1) == mcd.EINVAL                     # circle without radius
    m3 = mesh2d(mcd)
    m3.dim, m3.n[2] = 3, 16
    assert update(mcd, m3, one, 1) == mcd.ENOTSUP                    # 2D only


def test_sdf_grids_rejected(mcd):
    m = mesh2d(mcd)
    b = circle(mcd, 2)
    b.sdf_dev = 0x2000
    b.sdf_n[0], b.sdf_n[1] = 2, 10
    b.sdf_h = 0.01
    assert update(mcd, m, (mcd.c_body * 1)(b), 1) == mcd.EINVAL      # grid narrower than 3 points
    b.sdf_n[0] = 10
    b.sdf_h = 0.0
    assert update(mcd, m, (mcd.c_body * 1)(b), 1) == mcd.EINVAL      # no spacing
    arr = (mcd.c_body * 1)(circle(mcd, 2))
    assert mcd.lib().mcd_bodies_boundary(C.byref(m), arr, 0, PH, PH, PH, None, None) == mcd.EINVAL
    assert mcd.lib().mcd_bodies_velocity(C.byref(m), arr, 0, PH, PH, PH, PH, None) == mcd.EINVAL


def params(mcd, support=1, weight_kind=0):
    p = mcd.c_mls_params()
    p.weight_kind = weight_kind
    p.r_e = p.r_s = 1.0 / 16
    p.precision = mcd.MIXED
    p.support = support
    return p


def build(mcd, mesh, prm):
    h = C.c_void_p(None)
    return mcd.lib().mcd_build_stencils(C.byref(mesh), PH, PH, None, C.byref(prm), C.byref(h), None)


def test_stencil_options_rejected(mcd):
    m = mesh2d(mcd)
    assert build(mcd, m, params(mcd, support=2)) == mcd.EINVAL       # only 3x3 or 9x9
    assert build(mcd, m, params(mcd, weight_kind=3)) == mcd.EINVAL   # unknown weight
    assert build(mcd, mesh2d(mcd, n=8, periodic=True), params(mcd, support=4)) == mcd.EINVAL
    m3 = mesh2d(mcd)
    m3.dim, m3.n[2] = 3, 16
    assert build(mcd, m3, params(mcd, support=4)) == mcd.EINVAL      # 9x9 is 2D only
    meshes = (mcd.c_mesh * 1)(mesh2d(mcd))
    bt = C.c_void_p(None)
    assert mcd.lib().mcd_batch_create(meshes, 1, C.byref(params(mcd, support=4)), C.byref(bt)) == mcd.ENOTSUP


def test_ale_and_force_null_arguments(mcd):
    arr = (mcd.c_body * 1)(circle(mcd, 2))
    L = mcd.lib()
    assert L.mcd_ale_interpolate(None, arr, 1, PH, PH, PH, PH, PH, PH, PH, PH, None, None) == mcd.EINVAL
    out = (C.c_double * 4)()
    assert L.mcd_fluid_force(None, None, 2, PH, PH, PH, PH, PH, PH, PH, 0.01, out, None) == mcd.EINVAL


def test_bounded_wait_selftest_limits(mcd):
    L = mcd.lib()
    assert L.mcd_selftest_bounded_wait(0, 0, None) == mcd.EINVAL           # no polls
    assert L.mcd_selftest_bounded_wait(0, (1 << 20) + 1, None) == mcd.EINVAL   # over about a second
