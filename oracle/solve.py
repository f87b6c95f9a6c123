"""Oracle: the pressure-Poisson system and its Krylov solve (FP64).

TEST INFRASTRUCTURE (see the package header): only tests, smoke() and the
bench's CPU-baseline leg may use it.

Restates Sec. 3.3 of arXiv 2404.17542: the MLS discretisation of
lap P = (1/dt) div u* (Eq. (21)) with the Neumann condition of Eq. (23) on
moving bodies gives a sparse, nonsymmetric linear system that the paper
solves with Bi-CGSTAB.  The oracle
  * assembles that system as a scipy CSR matrix from the per-DP rows of
    `oracle.mls` (one row per DP, columns = its 3x3 / 3x3x3 cells);
  * forms the right-hand side: inner DP b = f - (Neumann data terms moved
    from the MLS fit), Dirichlet DP b = g, Neumann DP b = f, void DP b = 0;
  * solves it exactly with a sparse direct factorisation (the plain
    definition x = A^-1 b; a library primitive), and
  * restates textbook Bi-CGSTAB (van der Vorst, 1992) step by step.

Reading: convergence is judged on ||b - A x||_2 / ||b||_2 (for x0 = 0 this
is the paper's "relative to the initial norm", Sec. 4.2).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse
import scipy.sparse.linalg

from .mls import stencil_slots, support_of


def assemble(mesh, row):
    """CSR matrix with A[i, j_s] = row[s, i] over the stencil slots s of DP i
    (3x3 or expanded support, from the slot count)."""
    S, N = row.shape
    R = support_of(mesh, S)
    rows, cols, vals = [], [], []
    for i in range(N):
        for s, j, _off in stencil_slots(mesh, i, R):
            if j is None:
                continue
            v = row[s, i]
            if v != 0.0:
                rows.append(i)
                cols.append(j)
                vals.append(v)
    return scipy.sparse.csr_matrix((vals, (rows, cols)), shape=(N, N))


def form_rhs(mesh, kind, QL, rhs, bnd, rscale=None):
    """Right-hand side of the PPE system (kind codes from oracle.mls).

    Boundary rows take their datum times `rscale` (the Neumann row
    equilibration factor of oracle.mls; 1 for Dirichlet rows).
    """
    N = mesh.N
    R = support_of(mesh, QL.shape[0])
    b = np.zeros(N)
    for i in range(N):
        k = kind[i]
        if k == 1:        # inner: f_i minus the Neumann data moved to the RHS
            acc = rhs[i]
            for s, j, _off in stencil_slots(mesh, i, R):
                if j is not None and QL[s, i] != 0.0:
                    acc -= QL[s, i] * bnd[j]
            b[i] = acc
        elif k in (2, 3):  # Dirichlet value g or Neumann datum f
            b[i] = bnd[i] * (1.0 if rscale is None else rscale[i])
    return b


def direct_solve(A, b):
    """x = A^-1 b by sparse LU (SuperLU)."""
    return scipy.sparse.linalg.spsolve(A.tocsc(), b)


class Breakdown(Exception):
    pass


def bicgstab(A, b, x0=None, tol=1e-10, max_iter=100000):
    """Textbook unpreconditioned Bi-CGSTAB.  Returns (x, iterations, rel_res).

    The shadow residual is r^ = r0; when |r^ . r| <= 1e-14 |r^| |r| the
    recurrence restarts with r^ = r.  Iterations stop when the updated
    residual satisfies ||r|| <= tol ||b||; the returned rel_res is the true
    ||b - A x|| / ||b||.
    """
    x = np.zeros_like(b) if x0 is None else x0.astype(np.float64).copy()
    r = b - A @ x
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return np.zeros_like(b), 0, 0.0
    rhat = r.copy()
    rho = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    it = 0
    if np.linalg.norm(r) <= tol * bnorm:
        return x, 0, np.linalg.norm(r) / bnorm
    restarts = 0
    while it < max_iter:
        it += 1
        rho_new = rhat @ r
        if abs(rho_new) <= 1e-14 * np.linalg.norm(rhat) * np.linalg.norm(r):
            # breakdown of the Lanczos recurrence: restart with r^ = r
            restarts += 1
            if restarts > 50:
                raise Breakdown("repeated rho breakdown")
            rhat = r.copy()
            rho = alpha = omega = 1.0
            v = np.zeros_like(b)
            p = np.zeros_like(b)
            rho_new = rhat @ r
        beta = (rho_new / rho) * (alpha / omega)
        rho = rho_new
        p = r + beta * (p - omega * v)
        v = A @ p
        alpha = rho / (rhat @ v)
        s = r - alpha * v
        if np.linalg.norm(s) <= tol * bnorm:
            x = x + alpha * p
            break
        t = A @ s
        tt = t @ t
        if tt == 0.0:
            raise Breakdown("t = 0")
        omega = (t @ s) / tt
        x = x + alpha * p + omega * s
        r = s - omega * t
        if np.linalg.norm(r) <= tol * bnorm:
            break
        if omega == 0.0:
            raise Breakdown("omega = 0")
    rel = np.linalg.norm(b - A @ x) / bnorm
    return x, it, rel
