"""Oracle: chi=1 quadratic MLS stencil weights, one DP at a time (FP64).

TEST INFRASTRUCTURE (see the package header): only tests, smoke() and the
bench's CPU-baseline leg may use it.

Restates Sec. 3.2 of arXiv 2404.17542:
  * approximation  phi^h(X) = phi_c + p(X) . Phi_c,  X = (x - x_c) / r_s   (Eq. (12))
  * 2D quadratic basis p = (X, Y, X^2/2, XY, Y^2/2)                         (Eq. (13))
    3D reading: p = (X, Y, Z, X^2/2, Y^2/2, Z^2/2, XY, YZ, XZ)
  * Phi_c holds the scaled first and second derivatives at x_c              (Eq. (14))
  * objective J: weighted residuals over Lambda_c (inner + Dirichlet DPs),
    the Neumann term over Lambda^N_c, and the chi_c Lagrange constraint     (Eq. (15), (16))
  * weight w = cos^2(pi r / (2 r_e)) for r <= r_e, else 0                   (Eq. (17))
    plus the Gaussian w = exp(-(r / r_e)^2) used by the synthetic workloads
    and the least-squares MPS weight w = (1 - r / r_e)^2 for r < r_e, else 0
    (Tamai and Koshizuka, 2014), the scheme the paper pairs with its
    expanded 9x9 stencil, r_e = 3.5 l0                                    (Sec. 4.1)
  * only chi_c = 1 with x_c = x_i and phi_c = phi_i is used (end of Sec. 3.2)

With chi_c = 1 the constraint fixes phi_c = phi_i, and dJ/dPhi = 0 gives the
normal equations
    M Phi = sum_{j in Lambda_c} w_j p_j (phi_j - phi_i)
          + sum_{j in Lambda^N_c} w_j p^N_j r_s f_j,
    M     = sum_{j in Lambda_c} w_j p_j p_j^T + sum_{j in Lambda^N_c} w_j p^N_j p^N_j^T,
with p^N_j = n_j . grad_X p(X_j).  The oracle solves M by Cholesky (a library
primitive) and returns, per DP, the weights that turn neighbour values (and
Neumann data) into each physical derivative.

Readings where the paper is silent:
  * compact support D_c = the 3x3 (3x3x3) background cells around the DP's
    own cell (Sec. 2.3, Sec. 3.2); periodic axes wrap with the minimum image;
  * the expanded stencil of Sec. 4.1 is the same fit over the (2R+1)^dim
    cells around the DP's cell with R = 4 (9x9), `support` = R below; the
    paper names its influence radius (3.5 l0) and the least-squares MPS
    type-A scheme, whose weight is taken as (1 - r/r_e)^2; every other rule
    (roles, Neumann terms, row scaling) is that of the 3x3 stencil;
  * a Neumann DP's own gradient comes from a linear chi=1 fit,
    p = (X, Y[, Z]), over all its non-void neighbours (no Neumann terms):
    a boundary DP can have as few as 4 non-void neighbours, too few for the
    5-term quadratic fit (the paper shifts the support for boundary
    derivatives for this reason, Sec. 3.4); a Dirichlet DP's value is
    prescribed, so it gets an identity row and no derivative weights;
  * PPE rows: inner DP -> MLS Laplacian with Neumann neighbours moved to the
    right-hand side; Neumann DP -> n . grad P = f from its own value fit,
    scaled so that its diagonal is -1/r_s^2 (a row equilibration that leaves
    the solution unchanged; unscaled, those rows have diagonals of either
    sign and size 1/l0 and slow Bi-CGSTAB by more than an order of
    magnitude); Dirichlet DP and void DP -> identity row.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

INNER, VOID = -1, 0


class SingularStencil(Exception):
    """The moment matrix of DP `dp` is not positive definite."""

    def __init__(self, dp):
        super().__init__(f"singular MLS moment matrix at DP {dp}")
        self.dp = dp


def basis(X):
    """p(X) of Eq. (13) (2D) and its 3D analogue; X is a length-dim vector."""
    if len(X) == 2:
        x, y = X
        return np.array([x, y, 0.5 * x * x, x * y, 0.5 * y * y])
    x, y, z = X
    return np.array([x, y, z, 0.5 * x * x, 0.5 * y * y, 0.5 * z * z,
                     x * y, y * z, x * z])


def basis_normal(X, n):
    """p^N = n . grad_X p(X): the normal-derivative basis of Eq. (15)."""
    if len(X) == 2:
        x, y = X
        nx, ny = n
        return np.array([nx, ny, nx * x, nx * y + ny * x, ny * y])
    x, y, z = X
    nx, ny, nz = n
    return np.array([nx, ny, nz, nx * x, ny * y, nz * z,
                     nx * y + ny * x, ny * z + nz * y, nx * z + nz * x])


def basis_orders(dim):
    """Derivative order of each Phi component (1 = gradient, 2 = Hessian)."""
    return [1, 1, 2, 2, 2] if dim == 2 else [1, 1, 1, 2, 2, 2, 2, 2, 2]


def laplacian_components(dim):
    """Indices of the pure second derivatives in Phi (their sum is lap)."""
    return [2, 4] if dim == 2 else [3, 4, 5]


def weight(r, kind, r_e):
    """Eq. (17) (kind 1, cos^2 with cut-off r_e), the Gaussian (kind 0) or
    the least-squares MPS weight (kind 2, (1 - r/r_e)^2 below r_e)."""
    if kind == 1:
        if r <= r_e:
            return math.cos(math.pi * r / (2.0 * r_e)) ** 2
        return 0.0
    if kind == 2:
        if r < r_e:
            return (1.0 - r / r_e) ** 2
        return 0.0
    return math.exp(-(r / r_e) ** 2)


def cell_coords(mesh, k):
    """(i, j[, l]) of cell k with k = i + n_x (j + n_y l)."""
    i = k % mesh.n[0]
    rest = k // mesh.n[0]
    if mesh.dim == 2:
        return (i, rest)
    return (i, rest % mesh.n[1], rest // mesh.n[1])


def support_of(mesh, S):
    """Support radius R of a stencil with S = (2R+1)^dim slots."""
    W = round(S ** (1.0 / mesh.dim))
    assert W ** mesh.dim == S and W % 2 == 1, "slot count is not an odd power"
    return W // 2


def stencil_slots(mesh, k, support=1):
    """Neighbour cells of cell k in slot order (first offset fastest).

    Returns a list of (slot, neighbour index or None, offset tuple).  With
    W = 2 support + 1, slot s of a 2D stencil is (di+R) + W (dj+R); in 3D add
    W^2 (dl+R).  Cells outside a non-periodic domain give None; periodic axes
    wrap.
    """
    c = cell_coords(mesh, k)
    dim = mesh.dim
    out = []
    rng = tuple(range(-support, support + 1))
    offsets = ([(di, dj) for dj in rng for di in rng] if dim == 2 else
               [(di, dj, dl) for dl in rng for dj in rng for di in rng])
    for s, off in enumerate(offsets):
        idx = []
        ok = True
        for d in range(dim):
            v = c[d] + off[d]
            if v < 0 or v >= mesh.n[d]:
                if mesh.periodic[d]:
                    v %= mesh.n[d]
                else:
                    ok = False
                    break
            idx.append(v)
        if not ok:
            out.append((s, None, off))
            continue
        kk = idx[0] + mesh.n[0] * (idx[1] + (mesh.n[1] * idx[2] if dim == 3 else 0))
        out.append((s, kk, off))
    return out


def rel_offset(mesh, pos, i, j):
    """x_j - x_i with the periodic minimum image on periodic axes."""
    dx = pos[:, j] - pos[:, i]
    for d in range(mesh.dim):
        if mesh.periodic[d]:
            L = mesh.n[d] * mesh.l0
            dx[d] -= L * round(dx[d] / L)
    return dx


def dp_fit(mesh, pos, mask, normal, bc_kind, i, weight_kind=0, r_e=None,
           r_s=None, support=1):
    """Weights of DP i over the (2 support + 1)^dim cells around its cell.

    Returns a dict with
      kind  'void' | 'inner' | 'dirichlet' | 'neumann'
      D     (nb, S) value weights: derivative_k(x_i) = sum_s D[k, s] phi_s
            (a Neumann DP has gradient rows only)
            (the centre slot holds -sum of the others, from phi_j - phi_i);
            derivatives are physical (Phi_k / r_s^order_k)
      QD    (nb, S) Neumann weights: derivative_k gains sum_s QD[k, s] f_s
      row   (S,) PPE matrix row;  QL (S,) Neumann weights of the PPE row
      rscale  factor applied to the boundary datum in the right-hand side
    """
    dim = mesh.dim
    S = (2 * support + 1) ** dim
    centre = S // 2
    nb = 5 if dim == 2 else 9
    r_e = mesh.l0 if r_e is None else r_e
    r_s = mesh.l0 if r_s is None else r_s
    orders = basis_orders(dim)
    lapc = laplacian_components(dim)

    out = dict(D=np.zeros((nb, S)), QD=np.zeros((nb, S)),
               row=np.zeros(S), QL=np.zeros(S), rscale=1.0)
    mi = int(mask[i])
    if mi == VOID:
        out["kind"] = "void"
        out["row"][centre] = 1.0
        return out
    is_bnd = mi >= 1
    if is_bnd:
        out["kind"] = "neumann" if bc_kind[mi] == 1 else "dirichlet"
    else:
        out["kind"] = "inner"
    if out["kind"] == "dirichlet":
        # prescribed value: identity row, no derivative weights are formed
        out["row"][centre] = 1.0
        return out

    value_js, neu_js = [], []
    for s, j, _off in stencil_slots(mesh, i, support):
        if j is None or j == i:
            continue
        mj = int(mask[j])
        if mj == VOID:
            continue
        if is_bnd:
            value_js.append((s, j))          # own fit: all non-void values
        elif mj >= 1 and bc_kind[mj] == 1:
            neu_js.append((s, j))            # Lambda^N_c (Eq. (16))
        else:
            value_js.append((s, j))          # Lambda_c (Eq. (16))

    # a Neumann DP's own row needs only its gradient: linear chi=1 fit
    nf = dim if out["kind"] == "neumann" else nb
    M = np.zeros((nf, nf))
    Pv = np.zeros((nf, S))   # columns w_j p_j
    Pn = np.zeros((nf, S))   # columns w_j p^N_j r_s
    for s, j in value_js:
        dx = rel_offset(mesh, pos, i, j)
        w = weight(float(np.linalg.norm(dx)), weight_kind, r_e)
        p = basis(dx / r_s)[:nf]
        M += w * np.outer(p, p)
        Pv[:, s] = w * p
    for s, j in neu_js:
        dx = rel_offset(mesh, pos, i, j)
        w = weight(float(np.linalg.norm(dx)), weight_kind, r_e)
        pn = basis_normal(dx / r_s, normal[:, j])
        M += w * np.outer(pn, pn)
        Pn[:, s] = w * pn * r_s

    try:
        cf = scipy.linalg.cho_factor(M, lower=True)
    except np.linalg.LinAlgError as exc:
        raise SingularStencil(i) from exc
    Zv = scipy.linalg.cho_solve(cf, Pv)
    Zn = scipy.linalg.cho_solve(cf, Pn)
    scale = np.array([r_s ** o for o in orders[:nf]])[:, None]
    D = np.zeros((nb, S))
    QD = np.zeros((nb, S))
    D[:nf] = Zv / scale
    D[:, centre] = -D.sum(axis=1)
    QD[:nf] = Zn / scale
    out["D"], out["QD"] = D, QD

    if out["kind"] == "inner":
        out["row"] = D[lapc].sum(axis=0)
        out["QL"] = QD[lapc].sum(axis=0)
    elif out["kind"] == "neumann":
        n = normal[:, i]
        row = sum(n[d] * D[d] for d in range(dim))
        diag = row[centre]
        if diag == 0.0:
            raise SingularStencil(i)
        # row equilibration: scale n . grad P = f so that its diagonal is
        # -1/r_s^2 (the solution is unchanged; the right-hand side is scaled
        # by the same factor)
        sigma = -1.0 / (r_s * r_s * diag)
        out["row"] = sigma * row
        out["rscale"] = sigma
    return out


KIND_CODE = {"void": 0, "inner": 1, "dirichlet": 2, "neumann": 3}


def build_weights(mesh, pos, mask, normal=None, bc_kind=None, weight_kind=0,
                  r_e=None, r_s=None, dps=None, support=1):
    """Weights of every DP (or of the listed `dps`), slot-major SoA, over the
    (2 support + 1)^dim cells around each DP's cell.

    Returns dict(row (S,N), QL (S,N), D (nb,S,N), QD (nb,S,N), kind (N,) int,
    rscale (N,)).
    Raises SingularStencil for the first DP whose moment matrix fails.
    """
    N = mesh.N
    dim = mesh.dim
    S = (2 * support + 1) ** dim
    nb = 5 if dim == 2 else 9
    if bc_kind is None:
        bc_kind = np.zeros(128, dtype=np.uint8)
    if normal is None:
        normal = np.zeros((dim, N))
    idx = range(N) if dps is None else dps
    res = dict(row=np.zeros((S, N)), QL=np.zeros((S, N)),
               D=np.zeros((nb, S, N)), QD=np.zeros((nb, S, N)),
               kind=np.zeros(N, dtype=np.int64), rscale=np.ones(N))
    for i in idx:
        f = dp_fit(mesh, pos, mask, normal, bc_kind, i, weight_kind, r_e, r_s, support)
        res["row"][:, i] = f["row"]
        res["QL"][:, i] = f["QL"]
        res["D"][:, :, i] = f["D"]
        res["QD"][:, :, i] = f["QD"]
        res["kind"][i] = KIND_CODE[f["kind"]]
        res["rscale"][i] = f["rscale"]
    return res
