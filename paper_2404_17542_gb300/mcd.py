"""Thin ctypes binding of libmcd (include/mcd.h).

Argument marshalling only: every step of the hot path runs in the CUDA
library.  torch supplies device memory and the current stream.  If the
library is missing or no GPU is present the calls raise; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libmcd.so")

# status codes
OK, EINVAL, ENOMEM, ECUDA, ESINGULAR, ENOCONV, EBREAKDOWN, ENONFINITE, ETIMEOUT, ENOTSUP = range(10)
STATUS_NAMES = {0: "MCD_OK", 1: "MCD_EINVAL", 2: "MCD_ENOMEM", 3: "MCD_ECUDA", 4: "MCD_ESINGULAR",
                5: "MCD_ENOCONV", 6: "MCD_EBREAKDOWN", 7: "MCD_ENONFINITE", 8: "MCD_ETIMEOUT",
                9: "MCD_ENOTSUP"}
FP64, MIXED = 0, 1
DT_F64, DT_F32 = 0, 1
W_GAUSS, W_COS2, W_LSMPS = 0, 1, 2
BC_DIRICHLET, BC_NEUMANN = 0, 1
ARR_ROW64, ARR_ROW32, ARR_QL64, ARR_D64, ARR_QD64, ARR_RSCALE, ARR_KIND = range(7)


class McdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class c_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n", C.c_int * 3), ("l0", C.c_double),
                ("origin", C.c_double * 3), ("periodic", C.c_int * 3)]


class c_mls_params(C.Structure):
    _fields_ = [("weight_kind", C.c_int), ("r_e", C.c_double), ("r_s", C.c_double),
                ("precision", C.c_int), ("want_derivs", C.c_int), ("bc_kind", C.c_uint8 * 128),
                ("support", C.c_int)]


class c_solve_params(C.Structure):
    _fields_ = [("tol", C.c_double), ("max_iter", C.c_int), ("mode", C.c_int),
                ("inner_tol", C.c_double), ("max_refine", C.c_int), ("net", C.c_void_p),
                ("check_every", C.c_int), ("update_restart", C.c_int), ("net_dprev", C.c_void_p),
                ("barriers", C.c_int), ("precond", C.c_void_p)]


class c_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int), ("refinements", C.c_int), ("restarts", C.c_int),
                ("rel_res", C.c_double), ("b_norm", C.c_double), ("unknowns", C.c_int64),
                ("rel_res_guess", C.c_double), ("rel_res_start", C.c_double), ("fallback", C.c_int),
                ("net_corrections", C.c_int), ("discarded", C.c_int)]


class c_batch_tuning(C.Structure):
    _fields_ = [("rows", C.c_int), ("ctas_per_sm", C.c_int)]


class c_batch_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int), ("updates", C.c_int), ("rel_res", C.c_double),
                ("fallback", C.c_int), ("discarded", C.c_int)]


class c_body(C.Structure):
    _fields_ = [("id", C.c_int), ("c", C.c_double * 3), ("radius", C.c_double),
                ("vel", C.c_double * 3), ("acc", C.c_double * 3), ("theta", C.c_double),
                ("omega", C.c_double), ("omega_dot", C.c_double), ("sdf_dev", C.c_void_p),
                ("sdf_n", C.c_int * 2), ("sdf_origin", C.c_double * 2), ("sdf_h", C.c_double)]


class c_flow_params(C.Structure):
    _fields_ = [("nu", C.c_double), ("weight_kind", C.c_int), ("r_e", C.c_double), ("precision", C.c_int),
                ("kappa", C.c_double), ("n_relax", C.c_int), ("band", C.c_double), ("alpha", C.c_double),
                ("ale_pressure", C.c_int), ("forces", C.c_int)]


MAX_BODIES = 64


class c_flow_info(C.Structure):
    _fields_ = [("solve", c_solve_info), ("ale_fallbacks", C.c_int), ("ale_fallbacks_p", C.c_int),
                ("nbodies", C.c_int), ("force", (C.c_double * 2) * MAX_BODIES),
                ("perimeter", C.c_double * MAX_BODIES), ("skipped", C.c_int * MAX_BODIES)]


_lib = None

# name -> (restype, argtypes)
_SIGS = {
    "mcd_build_stencils": (C.c_int, [C.POINTER(c_mesh), C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(c_mls_params), C.POINTER(C.c_void_p), C.c_void_p]),
    "mcd_stencils_check": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    "mcd_stencils_destroy": (None, [C.c_void_p]),
    "mcd_stencils_array": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
    "mcd_stencils_copy": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mcd_apply_laplacian": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "mcd_assemble_rhs": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mcd_solve_pressure": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.POINTER(c_solve_params), C.POINTER(c_solve_info), C.c_void_p]),
    "mcd_update_dps": (C.c_int, [C.POINTER(c_mesh), C.POINTER(c_body), C.c_int, C.c_void_p, C.c_void_p,
                                 C.c_void_p, C.c_double, C.c_int, C.c_double, C.c_double, C.c_void_p]),
    "mcd_update_dps_static": (C.c_int, [C.POINTER(c_mesh), C.POINTER(c_body), C.c_int, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_double,
                                        C.c_double, C.c_void_p]),
    "mcd_body_boundary": (C.c_int, [C.POINTER(c_mesh), C.POINTER(c_body), C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_void_p]),
    "mcd_bodies_boundary": (C.c_int, [C.POINTER(c_mesh), C.POINTER(c_body), C.c_int, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mcd_bodies_velocity": (C.c_int, [C.POINTER(c_mesh), C.POINTER(c_body), C.c_int, C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mcd_ale_interpolate": (C.c_int, [C.c_void_p, C.POINTER(c_body), C.c_int] + [C.c_void_p] * 10),
    "mcd_fluid_force": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int] + [C.c_void_p] * 7
                        + [C.c_double, C.POINTER(C.c_double), C.c_void_p]),
    "mcd_flow_predict": (C.c_int, [C.c_void_p] + [C.c_void_p] * 4 + [C.c_double, C.c_double]
                         + [C.c_void_p] * 3 + [C.c_void_p]),
    "mcd_flow_project": (C.c_int, [C.c_void_p] + [C.c_void_p] * 6 + [C.c_double]
                         + [C.c_void_p] * 2 + [C.c_void_p]),
    "mcd_net_param_count": (C.c_int64, [C.c_int, C.c_int, C.c_int]),
    "mcd_net_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int64, C.POINTER(C.c_void_p)]),
    "mcd_net_destroy": (None, [C.c_void_p]),
    "mcd_net_read": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int64]),
    "mcd_net_features": (C.c_int, [C.c_void_p] * 9 + [C.c_void_p]),
    "mcd_net_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "mcd_net_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int,
                                     C.c_float, C.c_void_p, C.c_void_p]),
    "mcd_net_warm_start": (C.c_int, [C.c_void_p] * 6 + [C.c_void_p]),
    "mcd_batch_create": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(c_mls_params), C.POINTER(C.c_void_p)]),
    "mcd_batch_destroy": (None, [C.c_void_p]),
    "mcd_batch_offset": (C.c_int64, [C.c_void_p, C.c_int]),
    "mcd_batch_build": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mcd_batch_check": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.c_void_p]),
    "mcd_batch_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(c_solve_params),
                                  C.c_int, C.c_void_p, C.c_void_p]),
    "mcd_batch_stencils": (C.c_void_p, [C.c_void_p, C.c_int]),
    "mcd_batch_set_tuning": (C.c_int, [C.c_void_p, C.POINTER(c_batch_tuning)]),
    "mcd_batch_get_tuning": (C.c_int, [C.c_void_p, C.POINTER(c_batch_tuning)]),
    "mcd_batch_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(c_solve_params),
                                     C.c_int, C.c_char_p, C.POINTER(C.c_double), C.c_void_p]),
    "mcd_flow_create": (C.c_int, [C.POINTER(c_mesh), C.POINTER(c_flow_params), C.c_void_p, C.c_int,
                                  C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p), C.c_void_p]),
    "mcd_flow_destroy": (None, [C.c_void_p]),
    "mcd_flow_restart": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "mcd_flow_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                C.POINTER(c_solve_params)] + [C.c_void_p] * 5
                      + [C.POINTER(c_flow_info), C.c_void_p]),
    "mcd_flow_stencils": (C.c_void_p, [C.c_void_p, C.c_int]),
    "mcd_flow_copy": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "mcd_timing_enable": (C.c_int, [C.c_int]),
    "mcd_timing_read": (C.c_int, [C.c_int, C.POINTER(C.c_int64), C.POINTER(C.c_double)]),
    "mcd_launch_count": (C.c_int64, []),
    "mcd_solver_set_staging": (C.c_int, [C.c_int]),
    "mcd_selftest_bounded_wait": (C.c_int, [C.c_int, C.c_int64, C.c_void_p]),
    "mcd_trace_enable": (C.c_int, [C.c_int]),
    "mcd_trace_read": (C.c_int, [C.POINTER(C.c_uint64)]),
    "mcd_last_error": (C.c_char_p, []),
    "mcd_version": (C.c_char_p, []),
}


def exported_symbols():
    """Names the binding expects the library to export."""
    return sorted(_SIGS)


def lib():
    """Load libmcd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2404_17542_gb300.build` (there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise McdError(status, lib().mcd_last_error().decode())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor, dtype=None, numel=None):
    if not t.is_cuda:
        raise ValueError("tensor must live on a CUDA device")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"expected {numel} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def make_mesh(mesh) -> c_mesh:
    """c_mesh from any object with dim, n, l0, origin, periodic."""
    m = c_mesh()
    m.dim = int(mesh.dim)
    for d in range(3):
        m.n[d] = int(mesh.n[d]) if d < len(mesh.n) else 1
        m.origin[d] = float(mesh.origin[d]) if d < len(mesh.origin) else 0.0
        m.periodic[d] = int(mesh.periodic[d]) if d < len(mesh.periodic) else 0
    m.l0 = float(mesh.l0)
    return m


class Stencils:
    """Owner of an mcd_stencils handle (MLS weights + PPE rows)."""

    def __init__(self, mesh, pos, mask, normal=None, bc_kind=None, weight_kind=W_GAUSS,
                 r_e=None, r_s=None, precision=MIXED, want_derivs=False, support=1):
        self.mesh = mesh
        self.cmesh = make_mesh(mesh)
        self.N = int(np.prod([mesh.n[d] for d in range(mesh.dim)]))
        self.dim = mesh.dim
        self.support = int(support)
        self.S = (2 * self.support + 1) ** mesh.dim
        self.nb = 5 if mesh.dim == 2 else 9
        p = c_mls_params()
        p.weight_kind = int(weight_kind)
        p.r_e = float(mesh.l0 if r_e is None else r_e)
        p.r_s = float(mesh.l0 if r_s is None else r_s)
        p.precision = int(precision)
        p.want_derivs = int(bool(want_derivs))
        bc = np.zeros(128, dtype=np.uint8) if bc_kind is None else np.asarray(bc_kind, dtype=np.uint8)
        for i in range(128):
            p.bc_kind[i] = int(bc[i])
        p.support = self.support
        self.prm = p
        self.handle = C.c_void_p(None)
        self.rebuild(pos, mask, normal)

    def rebuild(self, pos, mask, normal=None):
        npos = _ptr(pos, torch.float64, self.dim * self.N)
        nmask = _ptr(mask, torch.int8, self.N)
        nn = _ptr(normal, torch.float64, self.dim * self.N) if normal is not None else C.c_void_p(None)
        _check(lib().mcd_build_stencils(C.byref(self.cmesh), npos, nmask, nn, C.byref(self.prm),
                                        C.byref(self.handle), _stream()))

    def check(self):
        bad = C.c_int64(-1)
        st = lib().mcd_stencils_check(self.handle, C.byref(bad), _stream())
        return st, bad.value

    def array(self, which):
        """Copy of a device array of the handle as a torch tensor."""
        ptr = C.c_void_p()
        cnt = C.c_int64()
        _check(lib().mcd_stencils_array(self.handle, which, C.byref(ptr), C.byref(cnt)))
        if cnt.value == 0:
            return None
        dt = {ARR_ROW32: torch.float32, ARR_KIND: torch.int8}.get(which, torch.float64)
        out = torch.empty(cnt.value, dtype=dt, device="cuda")
        _check(lib().mcd_stencils_copy(self.handle, which, _ptr(out), _stream()))
        return out

    def apply(self, x: torch.Tensor, out: torch.Tensor | None = None):
        dt = DT_F64 if x.dtype == torch.float64 else DT_F32
        y = torch.empty_like(x) if out is None else out
        _check(lib().mcd_apply_laplacian(self.handle, _ptr(x, numel=self.N), _ptr(y, x.dtype, self.N),
                                         dt, _stream()))
        return y

    def assemble_rhs(self, rhs: torch.Tensor, bnd: torch.Tensor, out=None):
        b = torch.empty(self.N, dtype=torch.float64, device=rhs.device) if out is None else out
        _check(lib().mcd_assemble_rhs(self.handle, _ptr(rhs, torch.float64, self.N),
                                      _ptr(bnd, torch.float64, self.N), _ptr(b, torch.float64, self.N),
                                      _stream()))
        return b

    def solve(self, rhs, bnd, p=None, tol=1e-8, mode=MIXED, max_iter=200000, inner_tol=0.3,
              max_refine=60, check_every=64, update_restart=0, raise_on_error=True, net=None,
              dprev=None, barriers=0, precond=None):
        """Solve the PPE; returns (p, info dict).  p is updated in place if given.
        net (a Net) adds its warm-start correction to p first; dprev (or
        None) is the last pressure increment it reads, and is overwritten
        with this solve's increment p(out) - p(in) when the solve converges."""
        if p is None:
            p = torch.zeros(self.N, dtype=torch.float64, device=rhs.device)
        sp = c_solve_params(tol=tol, max_iter=max_iter, mode=mode, inner_tol=inner_tol,
                            max_refine=max_refine, net=None if net is None else net.handle,
                            check_every=check_every, update_restart=int(update_restart),
                            net_dprev=None if dprev is None else _ptr(dprev, torch.float64, self.N),
                            barriers=int(barriers), precond=None if precond is None else precond.handle)
        info = c_solve_info()
        st = lib().mcd_solve_pressure(self.handle, _ptr(rhs, torch.float64, self.N),
                                      _ptr(bnd, torch.float64, self.N), _ptr(p, torch.float64, self.N),
                                      C.byref(sp), C.byref(info), _stream())
        d = dict(status=st, iters=info.iters, refinements=info.refinements, restarts=info.restarts,
                 rel_res=info.rel_res, b_norm=info.b_norm, unknowns=info.unknowns,
                 rel_res_guess=info.rel_res_guess, rel_res_start=info.rel_res_start,
                 fallback=info.fallback, net_corrections=info.net_corrections, discarded=info.discarded)
        if st != OK and raise_on_error:
            raise McdError(st, lib().mcd_last_error().decode())
        return p, d

    def flow_predict(self, u, v, ubc, vbc, nu, dt, us=None, vs=None, src=None):
        """u*, v* and (1/dt) div u* (Eqs. (20)-(21)); needs want_derivs=True."""
        us = torch.empty_like(u) if us is None else us
        vs = torch.empty_like(v) if vs is None else vs
        src = torch.empty_like(u) if src is None else src
        f64 = torch.float64
        _check(lib().mcd_flow_predict(self.handle, _ptr(u, f64, self.N), _ptr(v, f64, self.N),
                                      _ptr(ubc, f64, self.N), _ptr(vbc, f64, self.N), float(nu),
                                      float(dt), _ptr(us, f64, self.N), _ptr(vs, f64, self.N),
                                      _ptr(src, f64, self.N), _stream()))
        return us, vs, src

    def flow_project(self, P, bnd, us, vs, ubc, vbc, dt, u=None, v=None):
        """u = u* - dt grad P (Eq. (22)) with this handle's gradient weights."""
        u = torch.empty_like(us) if u is None else u
        v = torch.empty_like(vs) if v is None else v
        f64 = torch.float64
        _check(lib().mcd_flow_project(self.handle, _ptr(P, f64, self.N), _ptr(bnd, f64, self.N),
                                      _ptr(us, f64, self.N), _ptr(vs, f64, self.N),
                                      _ptr(ubc, f64, self.N), _ptr(vbc, f64, self.N), float(dt),
                                      _ptr(u, f64, self.N), _ptr(v, f64, self.N), _stream()))
        return u, v

    def close(self):
        if self.handle and self.handle.value:
            lib().mcd_stencils_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StencilsView(Stencils):
    """A stencil handle owned by the library (e.g. a flow run's pressure
    stencils): the array and solve helpers of Stencils, nothing to free."""

    def __init__(self, handle, mesh, support=1):
        self.mesh = mesh
        self.cmesh = make_mesh(mesh)
        self.N = int(np.prod([mesh.n[d] for d in range(mesh.dim)]))
        self.dim = mesh.dim
        self.support = support
        self.S = (2 * support + 1) ** mesh.dim
        self.nb = 5 if mesh.dim == 2 else 9
        self.handle = C.c_void_p(handle)

    def rebuild(self, pos, mask, normal=None):
        raise RuntimeError("a library-owned stencil handle is rebuilt by its owner")

    def close(self):
        self.handle = C.c_void_p(None)


class Batch:
    """Owner of an mcd_batch handle: independent 2D systems stored back to
    back (system i owns DPs offsets[i] .. offsets[i+1] of every per-DP array;
    its positions are the [2][N_i] block at 2 offsets[i]).  r_e and r_s are
    multiples of each system's l0."""

    def __init__(self, meshes, weight_kind=W_GAUSS, r_e=1.0, r_s=1.0, precision=MIXED, bc_kind=None):
        self.meshes = list(meshes)
        n = len(self.meshes)
        arr = (c_mesh * n)(*[make_mesh(m) for m in self.meshes])
        p = c_mls_params()
        p.weight_kind = int(weight_kind)
        p.r_e = float(r_e)
        p.r_s = float(r_s)
        p.precision = int(precision)
        p.want_derivs = 0
        bc = np.zeros(128, dtype=np.uint8) if bc_kind is None else np.asarray(bc_kind, dtype=np.uint8)
        for i in range(128):
            p.bc_kind[i] = int(bc[i])
        self.prm = p
        self.handle = C.c_void_p(None)
        _check(lib().mcd_batch_create(C.cast(arr, C.c_void_p), n, C.byref(p), C.byref(self.handle)))
        self.offsets = np.array([lib().mcd_batch_offset(self.handle, i) for i in range(n + 1)], dtype=np.int64)
        self.N = int(self.offsets[-1])

    @staticmethod
    def pack_positions(pos_list):
        """Host array of the per-system [2][N_i] position blocks, back to back."""
        return np.concatenate([np.asarray(p, np.float64).reshape(2, -1).ravel() for p in pos_list])

    def build(self, pos, mask):
        _check(lib().mcd_batch_build(self.handle, _ptr(pos, torch.float64, 2 * self.N),
                                     _ptr(mask, torch.int8, self.N), _stream()))

    def check(self):
        bad = C.c_int64(-1)
        st = lib().mcd_batch_check(self.handle, C.byref(bad), _stream())
        return st, bad.value

    def solve(self, rhs, bnd, p=None, tol=1e-8, mode=MIXED, max_iter=200000, inner_tol=0.3, graph=False,
              raise_on_error=True, update_restart=0, net=None):
        """Solve every system; returns (p, dict of per-system arrays status,
        iters, updates, rel_res)."""
        if p is None:
            p = torch.zeros(self.N, dtype=torch.float64, device=rhs.device)
        sp = c_solve_params(tol=tol, max_iter=max_iter, mode=mode, inner_tol=inner_tol, max_refine=0,
                            net=None if net is None else net.handle, check_every=0,
                            update_restart=int(update_restart), net_dprev=None)
        n = len(self.meshes)
        res = (c_batch_result * n)()
        f64 = torch.float64
        st = lib().mcd_batch_solve(self.handle, _ptr(rhs, f64, self.N), _ptr(bnd, f64, self.N),
                                   _ptr(p, f64, self.N), C.byref(sp), 1 if graph else 0,
                                   C.cast(res, C.c_void_p), _stream())
        out = {k: np.array([getattr(r, k) for r in res])
               for k in ("status", "iters", "updates", "rel_res", "fallback", "discarded")}
        out["return"] = st
        if st != OK and raise_on_error:
            raise McdError(st, lib().mcd_last_error().decode())
        return p, out

    def stencils(self, i):
        """System i as a (library-owned) stencil handle."""
        h = lib().mcd_batch_stencils(self.handle, int(i))
        if not h:
            raise McdError(EINVAL, f"no system {i}")
        return StencilsView(h, self.meshes[i])

    def set_tuning(self, rows, ctas_per_sm):
        t = c_batch_tuning(rows=int(rows), ctas_per_sm=int(ctas_per_sm))
        _check(lib().mcd_batch_set_tuning(self.handle, C.byref(t)))

    def tuning(self):
        t = c_batch_tuning()
        _check(lib().mcd_batch_get_tuning(self.handle, C.byref(t)))
        return t.rows, t.ctas_per_sm

    def autotune(self, rhs, bnd, p, tol=1e-8, mode=MIXED, sweeps=40, cache_path=None):
        """Pick the fastest tiling; returns ms per sweep of the choice."""
        sp = c_solve_params(tol=tol, max_iter=200000, mode=mode, inner_tol=0.3, max_refine=0, net=None,
                            check_every=0, update_restart=1, net_dprev=None)
        ms = C.c_double(0.0)
        f64 = torch.float64
        _check(lib().mcd_batch_autotune(self.handle, _ptr(rhs, f64, self.N), _ptr(bnd, f64, self.N),
                                        _ptr(p, f64, self.N), C.byref(sp), int(sweeps),
                                        None if cache_path is None else str(cache_path).encode(),
                                        C.byref(ms), _stream()))
        return ms.value

    def close(self):
        if self.handle and self.handle.value:
            lib().mcd_batch_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


NET_PARAMS, NET_GRADS, NET_ADAM_M, NET_ADAM_V = range(4)
N_CHANNELS = 8


class Net:
    """Owner of an mcd_net handle: the learned warm start (conv network)."""

    def __init__(self, params, c_in=7, width=32, layers=4):
        flat = np.ascontiguousarray(params, dtype=np.float32)
        self.c_in, self.width, self.layers = c_in, width, layers
        self.n_params = int(lib().mcd_net_param_count(c_in, width, layers))
        if self.n_params < 0:
            raise McdError(ENOTSUP, "unsupported network shape")
        self.handle = C.c_void_p(None)
        _check(lib().mcd_net_create(c_in, width, layers, flat.ctypes.data_as(C.c_void_p),
                                    flat.size, C.byref(self.handle)))

    def read(self, which=NET_PARAMS):
        out = np.empty(self.n_params, dtype=np.float32)
        _check(lib().mcd_net_read(self.handle, int(which), out.ctypes.data_as(C.c_void_p), out.size))
        return out

    def features(self, st: Stencils, b, p, dprev=None, p_true=None):
        """bf16 features [N][8] (int16 storage of the bf16 bits); with p_true
        also (target, weight) float32 [N]."""
        N = st.N
        f64 = torch.float64
        x = torch.empty((N, N_CHANNELS), dtype=torch.int16, device=b.device)
        tgt = wt = None
        if p_true is not None:
            tgt = torch.empty(N, dtype=torch.float32, device=b.device)
            wt = torch.empty(N, dtype=torch.float32, device=b.device)
        _check(lib().mcd_net_features(
            self.handle, st.handle, _ptr(b, f64, N), _ptr(p, f64, N),
            None if dprev is None else _ptr(dprev, f64, N),
            None if p_true is None else _ptr(p_true, f64, N), _ptr(x),
            None if tgt is None else _ptr(tgt), None if wt is None else _ptr(wt), _stream()))
        return x if p_true is None else (x, tgt, wt)

    def forward(self, x, nx, ny, y=None):
        y = torch.empty(nx * ny, dtype=torch.float32, device=x.device) if y is None else y
        _check(lib().mcd_net_forward(self.handle, _ptr(x, torch.int16, nx * ny * N_CHANNELS), int(nx),
                                     int(ny), _ptr(y, torch.float32, nx * ny), _stream()))
        return y

    def train_step(self, x, target, weight, nx, ny, lr, loss=None):
        """One Adam step; loss (float64 [1] on the device) receives the loss."""
        N = nx * ny
        _check(lib().mcd_net_train_step(self.handle, _ptr(x, torch.int16, N * N_CHANNELS),
                                        _ptr(target, torch.float32, N), _ptr(weight, torch.float32, N),
                                        int(nx), int(ny), float(lr),
                                        None if loss is None else _ptr(loss, torch.float64, 1),
                                        _stream()))

    def warm_start(self, st: Stencils, b, p, dprev=None):
        """p <- p + s e in place; returns (rel. residual before, after, s)."""
        stats = (C.c_double * 3)()
        f64 = torch.float64
        _check(lib().mcd_net_warm_start(self.handle, st.handle, _ptr(b, f64, st.N),
                                        None if dprev is None else _ptr(dprev, f64, st.N),
                                        _ptr(p, f64, st.N), stats, _stream()))
        return stats[0], stats[1], stats[2]

    def close(self):
        if self.handle and self.handle.value:
            lib().mcd_net_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bf16_bits_to_float(x: torch.Tensor) -> torch.Tensor:
    """float32 values of bf16 bit patterns held in an int16 tensor."""
    return (x.to(torch.int32) << 16).view(torch.float32)


def make_body(centre, radius, body_id, vel=(0.0, 0.0), acc=(0.0, 0.0)) -> c_body:
    b = c_body()
    b.id = int(body_id)
    b.c[0], b.c[1], b.c[2] = float(centre[0]), float(centre[1]), 0.0
    b.radius = float(radius)
    b.vel[0], b.vel[1], b.vel[2] = float(vel[0]), float(vel[1]), 0.0
    b.acc[0], b.acc[1], b.acc[2] = float(acc[0]), float(acc[1]), 0.0
    return b


class SdfBody:
    """A body given by SDF samples on a grid in its local frame (Sec. 2.5):
    grid is a contiguous device float64 tensor [n_y][n_x] of psi (> 0 in the
    fluid) at origin + (i, j) h; the body sits at `centre` with posture angle
    `theta` and turns at `omega` (angular acceleration `omega_dot`)."""

    def __init__(self, body_id, centre, theta, grid, origin, h, omega=0.0, omega_dot=0.0):
        self.id = int(body_id)
        self.centre = (float(centre[0]), float(centre[1]))
        self.theta = float(theta)
        if not (grid.is_cuda and grid.dtype == torch.float64 and grid.is_contiguous() and grid.dim() == 2):
            raise ValueError("grid must be a contiguous 2D float64 CUDA tensor")
        self.grid = grid
        self.origin = (float(origin[0]), float(origin[1]))
        self.h = float(h)
        self.omega = float(omega)
        self.omega_dot = float(omega_dot)


def make_bodies(bodies, accs=None, vels=None):
    """C array of bodies from circles (id, centre, radius) and SdfBody
    objects (and per-body accelerations and velocities)."""
    arr = (c_body * len(bodies))()
    for b, body in enumerate(bodies):
        vel = (0.0, 0.0) if vels is None else vels[b]
        acc = (0.0, 0.0) if accs is None else accs[b]
        if isinstance(body, SdfBody):
            cb = make_body(body.centre, 0.0, body.id, vel=vel, acc=acc)
            cb.theta, cb.omega, cb.omega_dot = body.theta, body.omega, body.omega_dot
            cb.sdf_dev = body.grid.data_ptr()
            cb.sdf_n[0], cb.sdf_n[1] = body.grid.shape[1], body.grid.shape[0]
            cb.sdf_origin[0], cb.sdf_origin[1] = body.origin
            cb.sdf_h = body.h
            arr[b] = cb
        else:
            bid, c, R = body
            arr[b] = make_body(c, R, bid, vel=vel, acc=acc)
    return arr


def body_id(body):
    return body.id if isinstance(body, SdfBody) else body[0]


def bodies_velocity(mesh, bodies, vels, pos, mask, ubc=None, vbc=None):
    """Boundary velocity of every DP: its rigid body's velocity at the DP,
    0 elsewhere."""
    cm = make_mesh(mesh)
    arr = make_bodies(bodies, vels=vels)
    N = mesh.n[0] * mesh.n[1]
    ubc = torch.empty(N, dtype=torch.float64, device=mask.device) if ubc is None else ubc
    vbc = torch.empty(N, dtype=torch.float64, device=mask.device) if vbc is None else vbc
    _check(lib().mcd_bodies_velocity(C.byref(cm), arr, len(bodies), _ptr(pos, torch.float64, 2 * N),
                                     _ptr(mask, torch.int8, N), _ptr(ubc, torch.float64, N),
                                     _ptr(vbc, torch.float64, N), _stream()))
    return ubc, vbc


def update_dps_bodies(mesh, bodies, pos, mask, mask_prev, kappa=0.2, n_relax=10, band=None,
                      alpha=0.0):
    """One DP update (Sec. 2.2-2.4, nearest SDF of Sec. 2.5) for the bodies
    [(id, centre, radius)], in place on pos/mask."""
    cm = make_mesh(mesh)
    arr = make_bodies(bodies)
    N = mesh.n[0] * mesh.n[1]
    band = 5.0 * mesh.l0 if band is None else band
    _check(lib().mcd_update_dps(C.byref(cm), arr, len(bodies), _ptr(pos, torch.float64, 2 * N),
                                _ptr(mask, torch.int8, N), _ptr(mask_prev, torch.int8, N),
                                float(kappa), int(n_relax), float(band), float(alpha), _stream()))


def bodies_boundary(mesh, bodies, pos, mask, accs=None, normal=None, neumann=None):
    """Normals of every body's DPs and the Neumann data -acc . n (Eq. (23))."""
    cm = make_mesh(mesh)
    arr = make_bodies(bodies, accs)
    N = mesh.n[0] * mesh.n[1]
    n = torch.empty(2 * N, dtype=torch.float64, device=pos.device) if normal is None else normal
    f = torch.empty(N, dtype=torch.float64, device=pos.device) if neumann is None else neumann
    _check(lib().mcd_bodies_boundary(C.byref(cm), arr, len(bodies), _ptr(pos, torch.float64, 2 * N),
                                     _ptr(mask, torch.int8, N), _ptr(n, torch.float64, 2 * N),
                                     _ptr(f, torch.float64, N), _stream()))
    return n, f


def ale_interpolate(vel_k, bodies_k, pos_k, pos_k1, mask_k, mask_k1, u, v):
    """Step-k velocity at the step-(k+1) positions (Eq. (19), Appendix A).
    Returns (u~, v~, number of fallbacks)."""
    N = vel_k.N
    uo = torch.empty_like(u)
    vo = torch.empty_like(v)
    fb = torch.zeros(1, dtype=torch.int32, device=u.device)
    arr = make_bodies(bodies_k)
    _check(lib().mcd_ale_interpolate(vel_k.handle, arr, len(bodies_k), _ptr(pos_k, torch.float64, 2 * N),
                                     _ptr(pos_k1, torch.float64, 2 * N), _ptr(mask_k, torch.int8, N),
                                     _ptr(mask_k1, torch.int8, N), _ptr(u, torch.float64, N),
                                     _ptr(v, torch.float64, N), _ptr(uo, torch.float64, N),
                                     _ptr(vo, torch.float64, N), _ptr(fb, torch.int32, 1), _stream()))
    return uo, vo, int(fb.item())


def fluid_force(pres, vel, body_id, pos, mask, normal, P, bnd, u, v, mu):
    """Force of the fluid on body `body_id` (Eqs. (30)-(31)).
    Returns ((F_x, F_y), sum dGamma, skipped DPs)."""
    N = pres.N
    out = (C.c_double * 4)()
    _check(lib().mcd_fluid_force(pres.handle, vel.handle, int(body_id), _ptr(pos, torch.float64, 2 * N),
                                 _ptr(mask, torch.int8, N), _ptr(normal, torch.float64, 2 * N),
                                 _ptr(P, torch.float64, N),
                                 _ptr(bnd, torch.float64, N) if bnd is not None else C.c_void_p(None),
                                 _ptr(u, torch.float64, N), _ptr(v, torch.float64, N), float(mu), out,
                                 _stream()))
    return (out[0], out[1]), out[2], int(out[3])


def update_dps(mesh, centre, radius, body_id, pos, mask, mask_prev, kappa=0.2, n_relax=10,
               band=None, alpha=0.0):
    """One moving-boundary DP update (Sec. 2.2-2.4) in place on pos/mask."""
    cm = make_mesh(mesh)
    b = make_body(centre, radius, body_id)
    N = mesh.n[0] * mesh.n[1]
    band = 5.0 * mesh.l0 if band is None else band
    _check(lib().mcd_update_dps(C.byref(cm), C.byref(b), 1, _ptr(pos, torch.float64, 2 * N),
                                _ptr(mask, torch.int8, N), _ptr(mask_prev, torch.int8, N),
                                float(kappa), int(n_relax), float(band), float(alpha), _stream()))


def update_dps_static(mesh, centre, radius, body_id, pos, mask, mask_prev, kappa=0.2, n_relax=10,
                      band=None, alpha=0.0):
    """update_dps through the allocation-free entry point (fixed scratch of
    MCD_NOALLOC_MAX_DPS cells inside the library; see include/mcd.h)."""
    cm = make_mesh(mesh)
    b = make_body(centre, radius, body_id)
    N = mesh.n[0] * mesh.n[1]
    band = 5.0 * mesh.l0 if band is None else band
    _check(lib().mcd_update_dps_static(C.byref(cm), C.byref(b), 1, _ptr(pos, torch.float64, 2 * N),
                                       _ptr(mask, torch.int8, N), _ptr(mask_prev, torch.int8, N),
                                       float(kappa), int(n_relax), float(band), float(alpha), _stream()))


def body_boundary(mesh, centre, radius, body_id, pos, mask, acc=(0.0, 0.0), normal=None, neumann=None):
    """Normals of the body DPs and the Neumann datum -acc . n (Eq. (23))."""
    cm = make_mesh(mesh)
    b = make_body(centre, radius, body_id, acc=acc)
    N = mesh.n[0] * mesh.n[1]
    n = torch.empty(2 * N, dtype=torch.float64, device=pos.device) if normal is None else normal
    f = torch.empty(N, dtype=torch.float64, device=pos.device) if neumann is None else neumann
    _check(lib().mcd_body_boundary(C.byref(cm), C.byref(b), _ptr(pos, torch.float64, 2 * N),
                                   _ptr(mask, torch.int8, N), _ptr(n, torch.float64, 2 * N),
                                   _ptr(f, torch.float64, N), _stream()))
    return n, f


K_BICG_A, K_BICG_B, K_BICG_C, K_RESIDUAL, K_BUILD, K_UPDATE, K_OTHER, K_SOLVE, K_CNN, K_BATCH = range(10)
KERNEL_NAMES = ["bicg_ka", "bicg_kb", "bicg_kc", "residual64", "build_kernel", "update", "other",
                "bicg_persistent", "cnn", "bicg_batch"]


def timing_enable(sample_every: int):
    _check(lib().mcd_timing_enable(int(sample_every)))


def timing_read(kernel: int):
    """(sampled launches, summed device ms) of a kernel class."""
    n = C.c_int64()
    ms = C.c_double()
    _check(lib().mcd_timing_read(int(kernel), C.byref(n), C.byref(ms)))
    return n.value, ms.value


def trace_enable(on: bool):
    _check(lib().mcd_trace_enable(1 if on else 0))


def trace_read():
    """Phase timestamps (64, 8) of block 0; for iteration 10 the per-block end
    of the first phase, SM ids and iteration start times; and the grid
    barriers' stage stamps (256 epochs, 8 stages), from the last persistent
    launch."""
    buf = (C.c_uint64 * (512 + 6144 + 2048))()
    _check(lib().mcd_trace_read(buf))
    a = np.array(buf, dtype=np.uint64)
    return (a[:512].reshape(64, 8), a[512:512 + 2048], a[512 + 2048:512 + 4096], a[512 + 4096:512 + 6144],
            a[6656:].reshape(256, 8))


def selftest_bounded_wait(set_flag: bool, polls: int = 4096) -> int:
    """Status of the bounded-wait self-test (MCD_OK when the polled word is
    set, MCD_ETIMEOUT when nothing sets it); no exception either way."""
    return int(lib().mcd_selftest_bounded_wait(1 if set_flag else 0, int(polls), None))


def solver_set_staging(on: bool):
    """Stage the persistent solve's tile operands with TMA (default) or not."""
    _check(lib().mcd_solver_set_staging(1 if on else 0))


def launch_count() -> int:
    return int(lib().mcd_launch_count())


def version():
    return lib().mcd_version().decode()


FLOW_B, FLOW_GUESS, FLOW_BND, FLOW_SRC, FLOW_NORMAL = range(5)
FLOW_VELOCITY, FLOW_PRESSURE = 0, 1


class AleFlow:
    """Moving-boundary fractional steps (Sec. 3.3) through mcd_flow_step:
    one library call per step does the DP update, the ALE interpolation,
    the stencils, predict, the PPE, the projection and the forces, and forms
    the bodies' dV/dt and d omega/dt by the differences of Eq. (29).

    bodies_at(t) -> ([bodies], [(vx, vy)]): the bodies at time t (circles
    (id, centre, radius) or SdfBody objects with their posture angle and
    angular velocity) and their translational velocities.  The state (DP
    positions and masks, u, v, P) lives in device tensors.  With
    ale_pressure the PPE starts from the step-k pressure carried to the new
    positions (Eq. (19), Appendix A), else from the step-k pressure.
    """

    def __init__(self, mesh, pos, mask, bodies_at, nu, dt, t0=0.0, weight_kind=W_GAUSS, r_e=None,
                 precision=MIXED, mode=MIXED, tol=1e-8, kappa=0.2, n_relax=10, band=None,
                 ale_pressure=True, forces=True):
        self.mesh, self.bodies_at, self.nu, self.dt, self.t = mesh, bodies_at, nu, dt, t0
        self.mode, self.tol = mode, tol
        self.N = mesh.n[0] * mesh.n[1]
        dev = pos.device
        self.pos, self.mask = pos, mask
        self.cmesh = make_mesh(mesh)
        self.prm = c_flow_params(nu=float(nu), weight_kind=int(weight_kind),
                                 r_e=float(0.0 if r_e is None else r_e), precision=int(precision),
                                 kappa=float(kappa), n_relax=int(n_relax),
                                 band=float(0.0 if band is None else band), alpha=0.0,
                                 ale_pressure=int(bool(ale_pressure)), forces=int(bool(forces)))
        geo, vel = bodies_at(t0)
        self.ids = [body_id(b) for b in geo]
        arr = make_bodies(geo, vels=vel)
        self.handle = C.c_void_p(None)
        _check(lib().mcd_flow_create(C.byref(self.cmesh), C.byref(self.prm), arr, len(geo),
                                     _ptr(pos, torch.float64, 2 * self.N), _ptr(mask, torch.int8, self.N),
                                     C.byref(self.handle), _stream()))
        z = lambda: torch.zeros(self.N, dtype=torch.float64, device=dev)  # noqa: E731
        self.u, self.v, self.P = z(), z(), z()
        self.info = {}

    def step(self, mode=None, net=None, dprev=None, tol=None, raise_on_error=True, precond=None,
             update_restart=1, inner_tol=0.3):
        """One step; returns {solve, fallbacks, fallbacks_p, forces}.  net /
        dprev: the learned warm start of the solve, precond: the network that
        preconditions its refinement (as in Stencils.solve)."""
        geo_k, V_k = self.bodies_at(self.t)
        geo_1, V_1 = self.bodies_at(self.t + self.dt)
        bk = make_bodies(geo_k, vels=V_k)
        b1 = make_bodies(geo_1, vels=V_1)
        sp = c_solve_params(tol=float(self.tol if tol is None else tol),
                            max_iter=200000, mode=int(self.mode if mode is None else mode),
                            inner_tol=float(inner_tol),
                            max_refine=60, net=None if net is None else net.handle, check_every=64,
                            update_restart=int(update_restart),
                            net_dprev=None if dprev is None else _ptr(dprev, torch.float64, self.N),
                            barriers=0, precond=None if precond is None else precond.handle)
        fi = c_flow_info()
        f64 = torch.float64
        st = lib().mcd_flow_step(self.handle, bk, b1, len(geo_k), float(self.dt), C.byref(sp),
                                 _ptr(self.pos, f64, 2 * self.N), _ptr(self.mask, torch.int8, self.N),
                                 _ptr(self.u, f64, self.N), _ptr(self.v, f64, self.N), _ptr(self.P, f64, self.N),
                                 C.byref(fi), _stream())
        si = fi.solve
        solve = dict(status=st, iters=si.iters, refinements=si.refinements, restarts=si.restarts,
                     rel_res=si.rel_res, b_norm=si.b_norm, unknowns=si.unknowns,
                     rel_res_guess=si.rel_res_guess, rel_res_start=si.rel_res_start, fallback=si.fallback,
                     net_corrections=si.net_corrections, discarded=si.discarded)
        if st != OK and raise_on_error:
            raise McdError(st, lib().mcd_last_error().decode())
        forces = {bid: ((fi.force[b][0], fi.force[b][1]), fi.perimeter[b], fi.skipped[b])
                  for b, bid in enumerate(self.ids)}
        self.t += self.dt
        self.info = dict(solve=solve, fallbacks=fi.ale_fallbacks, fallbacks_p=fi.ale_fallbacks_p, forces=forces)
        return self.info

    def snapshot(self):
        """Copies of the run's state (cloud, fields, time)."""
        return (self.pos.clone(), self.mask.clone(), self.u.clone(), self.v.clone(), self.P.clone(), self.t)

    def restore(self, snap):
        """Continue from a snapshot: its state, and the velocity stencils of
        its cloud rebuilt for the next step's ALE interpolation."""
        pos, mask, u, v, P, t = snap
        for dst, src in ((self.pos, pos), (self.mask, mask), (self.u, u), (self.v, v), (self.P, P)):
            dst.copy_(src)
        self.t = t
        _check(lib().mcd_flow_restart(self.handle, _ptr(self.pos, torch.float64, 2 * self.N),
                                      _ptr(self.mask, torch.int8, self.N), _stream()))

    def stencils(self, which=FLOW_PRESSURE):
        """The run's current velocity or pressure stencils (library-owned)."""
        h = lib().mcd_flow_stencils(self.handle, int(which))
        return StencilsView(h, self.mesh)

    def array(self, which, out=None):
        """Copy of an array of the last step (FLOW_B, FLOW_GUESS, FLOW_BND,
        FLOW_SRC: [N]; FLOW_NORMAL: [2][N])."""
        n = 2 * self.N if which == FLOW_NORMAL else self.N
        out = torch.empty(n, dtype=torch.float64, device=self.u.device) if out is None else out
        _check(lib().mcd_flow_copy(self.handle, int(which), _ptr(out, torch.float64, n), _stream()))
        return out

    @property
    def normal(self):
        return self.array(FLOW_NORMAL)

    @property
    def bnd(self):
        return self.array(FLOW_BND)

    def close(self):
        if self.handle and self.handle.value:
            lib().mcd_flow_destroy(self.handle)
            self.handle = C.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
