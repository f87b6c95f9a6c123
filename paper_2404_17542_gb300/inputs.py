"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and
the bench.

This module builds problem *data* only: background meshes, discrete-point (DP)
clouds, boundary ids, manufactured fields and their analytic derivatives.  It
holds none of the method's arithmetic (no masking, arrangement, MLS fit or
solve).  Every generator takes an explicit seed and uses numpy's PCG64, so the
same arrays reach both sides of every parity test.

Conventions (shared with the C-ABI):
  * cell / DP index  k = i + n_x * (j + n_y * l)  (one DP per cell, Sec. 2.2);
  * positions are SoA float64 arrays of shape (dim, N);
  * mask is int8: -1 inner, 0 void, >= 1 boundary id (Sec. 2.2, Eq. (1));
  * boundary id 1 is the domain wall, ids >= 2 are moving bodies.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

INNER = -1
VOID = 0
WALL_ID = 1
BODY_ID = 2

BC_DIRICHLET = 0
BC_NEUMANN = 1


@dataclass
class Mesh:
    """Uniform Cartesian background mesh of width l0 (Sec. 2.1-2.2)."""

    dim: int
    n: tuple
    l0: float
    origin: tuple = (0.0, 0.0, 0.0)
    periodic: tuple = (0, 0, 0)

    @property
    def N(self) -> int:
        out = 1
        for d in range(self.dim):
            out *= self.n[d]
        return out

    def cell_ijk(self):
        """Integer cell coordinates, shape (dim, N), in index order."""
        axes = [np.arange(self.n[d]) for d in range(self.dim)]
        grids = np.meshgrid(*axes, indexing="ij")
        # index k = i + n_x*(j + n_y*l): i varies fastest -> ravel in Fortran order
        return np.stack([g.ravel(order="F") for g in grids])

    def centroids(self):
        ijk = self.cell_ijk().astype(np.float64)
        org = np.array(self.origin[: self.dim], dtype=np.float64)[:, None]
        return org + (ijk + 0.5) * self.l0


@dataclass
class Problem:
    mesh: Mesh
    pos: np.ndarray            # (dim, N) float64
    mask: np.ndarray           # (N,) int8
    rhs: np.ndarray = None     # (N,) float64, interior right-hand side f
    bnd: np.ndarray = None     # (N,) float64, Dirichlet g / Neumann data
    exact: np.ndarray = None   # (N,) float64, manufactured solution (if any)
    normal: np.ndarray = None  # (dim, N) float64 boundary normals (or None)
    bc_kind: np.ndarray = field(default_factory=lambda: default_bc_kind())
    meta: dict = field(default_factory=dict)


def default_bc_kind(neumann_ids=()):
    """Per boundary id: 0 Dirichlet, 1 Neumann (128 entries, id 0 unused)."""
    bc = np.zeros(128, dtype=np.uint8)
    for i in neumann_ids:
        bc[i] = BC_NEUMANN
    return bc


def wall_cells(mesh: Mesh):
    """Boolean (N,) marking cells with a face on a non-periodic domain wall."""
    ijk = mesh.cell_ijk()
    on = np.zeros(mesh.N, dtype=bool)
    for d in range(mesh.dim):
        if mesh.periodic[d]:
            continue
        on |= (ijk[d] == 0) | (ijk[d] == mesh.n[d] - 1)
    return on


def snap_wall_dps(mesh: Mesh, pos: np.ndarray) -> np.ndarray:
    """DP cloud convention for box walls: a wall cell's DP lies on the wall.

    Each coordinate of a cell touching the lower (upper) wall of a
    non-periodic axis is set to that wall; corner cells go to the corner.
    This defines where the synthetic problem's boundary DPs sit; it is input
    construction, not part of the arrangement algorithm.
    """
    ijk = mesh.cell_ijk()
    out = pos.copy()
    for d in range(mesh.dim):
        if mesh.periodic[d]:
            continue
        lo = mesh.origin[d]
        hi = mesh.origin[d] + mesh.n[d] * mesh.l0
        out[d, ijk[d] == 0] = lo
        out[d, ijk[d] == mesh.n[d] - 1] = hi
    return out


def jittered_box(n: int, dim: int, seed: int, jitter: float = 0.25,
                 periodic: bool = False, length: float = 1.0) -> Problem:
    """Box of side `length` along x, one DP per cell at the centroid +
    U[-jitter*l0, jitter*l0]^dim.  `n` is the cell count per axis (an int, or
    a tuple for a non-cubic box with the same l0).

    Non-periodic boxes get Dirichlet wall DPs (id 1) snapped onto the walls.
    """
    ns = tuple(n) if isinstance(n, (tuple, list)) else tuple([n] * dim)
    l0 = length / ns[0]
    per = (1, 1, 1) if periodic else (0, 0, 0)
    mesh = Mesh(dim=dim, n=tuple(list(ns) + [1] * (3 - dim)), l0=l0,
                origin=(0.0, 0.0, 0.0), periodic=per)
    rng = np.random.default_rng(seed)
    pos = mesh.centroids() + rng.uniform(-jitter * l0, jitter * l0,
                                         size=(dim, mesh.N))
    mask = np.full(mesh.N, INNER, dtype=np.int8)
    if not periodic:
        pos = snap_wall_dps(mesh, pos)
        mask[wall_cells(mesh)] = WALL_ID
    return Problem(mesh=mesh, pos=pos, mask=mask)


def sin_product(pos: np.ndarray):
    """u = prod_d sin(pi x_d) and its Laplacian f = -dim pi^2 u."""
    dim = pos.shape[0]
    u = np.ones(pos.shape[1])
    for d in range(dim):
        u = u * np.sin(math.pi * pos[d])
    return u, -dim * math.pi ** 2 * u


def manufactured_box(n: int, dim: int, seed: int, jitter: float = 0.25) -> Problem:
    """Poisson problem lap u = f with u = prod sin(pi x), Dirichlet g = u on walls."""
    pb = jittered_box(n, dim, seed, jitter)
    u, f = sin_product(pb.pos)
    pb.rhs = f
    pb.bnd = np.where(pb.mask >= 1, u, 0.0)
    pb.exact = u
    return pb


def poly4_coeffs(rng):
    """Random coefficients c[a, b] (a + b <= 4) of a 2D degree-4 polynomial."""
    c = np.zeros((5, 5))
    for a in range(5):
        for b in range(5 - a):
            c[a, b] = rng.uniform(-1.0, 1.0)
    return c


def poly4_eval(c, x, y):
    """u = sum c_ab x^a y^b and its analytic Laplacian."""
    u = np.zeros_like(x)
    lap = np.zeros_like(x)
    for a in range(5):
        for b in range(5 - a):
            u += c[a, b] * x ** a * y ** b
            if a >= 2:
                lap += c[a, b] * a * (a - 1) * x ** (a - 2) * y ** b
            if b >= 2:
                lap += c[a, b] * b * (b - 1) * x ** a * y ** (b - 2)
    return u, lap


def poly4_box(n: int, seed: int, jitter: float = 0.25) -> Problem:
    """2D Poisson instance with a random degree-4 polynomial solution."""
    rng = np.random.default_rng(seed)
    c = poly4_coeffs(rng)
    pb = jittered_box(n, 2, int(rng.integers(0, 2**31 - 1)), jitter)
    u, lap = poly4_eval(c, pb.pos[0], pb.pos[1])
    pb.rhs = lap
    pb.bnd = np.where(pb.mask >= 1, u, 0.0)
    pb.exact = u
    pb.meta["coeffs"] = c
    return pb


def batched_sizes(seed: int, count: int = 256, lo: int = 32, hi: int = 512):
    """Mesh widths n_k = floor(exp(U(ln lo, ln hi))) for `count` instances."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(math.log(lo), math.log(hi), size=count)
    return np.floor(np.exp(u)).astype(np.int64)


def batched_poly4(seed: int, count: int = 256, lo: int = 32, hi: int = 512):
    """Independent degree-4 polynomial Poisson instances of log-uniform size."""
    sizes = batched_sizes(seed, count, lo, hi)
    rng = np.random.default_rng(seed + 7919)
    seeds = rng.integers(0, 2**31 - 1, size=count)
    return [poly4_box(int(n), int(s)) for n, s in zip(sizes, seeds)]


@dataclass
class Cylinder:
    """Rigid circular body oscillating along x: x_c(t) = x0 - A sin(2 pi f t)."""

    x0: float = 0.5
    y0: float = 0.5
    radius: float = 0.05
    amp: float = 5 * 0.1 / (2 * math.pi)
    freq: float = 2.0
    body_id: int = BODY_ID

    def centre(self, t: float):
        return (self.x0 - self.amp * math.sin(2 * math.pi * self.freq * t), self.y0)

    def velocity(self, t: float):
        w = 2 * math.pi * self.freq
        return (-self.amp * w * math.cos(w * t), 0.0)

    def acceleration(self, t: float):
        w = 2 * math.pi * self.freq
        return (self.amp * w * w * math.sin(w * t), 0.0)


def cylinder_box(n: int, cyl: Cylinder | None = None) -> Problem:
    """Unit box for the oscillating-cylinder workload before any DP update.

    DPs start at the cell centroids (Sec. 2.3 step (i)); wall cells carry the
    Dirichlet wall id with their DPs on the wall; every other cell starts as
    inner until the masking of the DP update runs.
    """
    cyl = cyl or Cylinder()
    l0 = 1.0 / n
    mesh = Mesh(dim=2, n=(n, n, 1), l0=l0)
    pos = snap_wall_dps(mesh, mesh.centroids())
    mask = np.full(mesh.N, INNER, dtype=np.int8)
    mask[wall_cells(mesh)] = WALL_ID
    pb = Problem(mesh=mesh, pos=pos, mask=mask,
                 bc_kind=default_bc_kind(neumann_ids=(cyl.body_id,)))
    pb.meta["cylinder"] = cyl
    return pb


def cylinder_array(n: int, gap: float, count: int = 5, side: float = 2.0):
    """Stationary cylinder array of the multiple-cylinder flow (Sec. 4.1):
    count x count equal circles on a square lattice of pitch side / count
    filling the square [0, side]^2, diameter pitch - gap, on an n x n
    background mesh (l0 = side / n; the paper's case is side 2 with l0 = 1/64,
    n = 128).  `gap` is the surface-to-surface distance of neighbouring
    cylinders.  Returns [(id, (cx, cy), radius)] with ids 2, 3, ... row by
    row."""
    pitch = side / count
    radius = 0.5 * (pitch - gap)
    if radius <= 0.0:
        raise ValueError("gap must be smaller than the pitch")
    out = []
    for j in range(count):
        for i in range(count):
            out.append((BODY_ID + i + count * j, ((i + 0.5) * pitch, (j + 0.5) * pitch), radius))
    return out


def cylinder_array_box(n: int, gap_cells: float, count: int = 5, side: float = 2.0) -> Problem:
    """Square box of side `side` (n x n cells) for the cylinder array of
    Sec. 4.1 before any DP update: DPs at the cell centroids, Dirichlet wall
    cells with their DPs on the wall, every other cell inner.  The gap is
    gap_cells * (1/64), the paper's l0, whatever n is, so that finer meshes
    resolve the same geometry.  Every cylinder id is a Neumann boundary; the
    right-hand side is ppe_source at t = 0."""
    l0 = side / n
    mesh = Mesh(dim=2, n=(n, n, 1), l0=l0)
    pos = snap_wall_dps(mesh, mesh.centroids())
    mask = np.full(mesh.N, INNER, dtype=np.int8)
    mask[wall_cells(mesh)] = WALL_ID
    bodies = cylinder_array(n, gap_cells / 64.0, count, side)
    pb = Problem(mesh=mesh, pos=pos, mask=mask,
                 bc_kind=default_bc_kind(neumann_ids=[b[0] for b in bodies]))
    pb.rhs = ppe_source(pos / side, 0.0)
    pb.meta["bodies"] = bodies
    return pb


def sample_sdf_grid(psi_local, origin, h: float, n):
    """SDF samples of a body in its own frame: grid[j, i] = psi_local(x, y)
    at (x, y) = origin + (i, j) h, n = (n_x, n_y) points (data for a body
    described by a discrete SDF, psi > 0 in the fluid)."""
    nx, ny = n
    xs = origin[0] + h * np.arange(nx)
    ys = origin[1] + h * np.arange(ny)
    X, Y = np.meshgrid(xs, ys)
    return np.ascontiguousarray(psi_local(X, Y), dtype=np.float64)


def circle_sdf(radius: float):
    """psi(x, y) = |x| - R of a circle centred at the local origin."""
    return lambda x, y: np.sqrt(x * x + y * y) - radius


def ellipse_sdf(a: float, b: float):
    """A signed distance-like function of the ellipse (x/a)^2 + (y/b)^2 = 1
    (local frame): the level-set function scaled to unit gradient on the
    ellipse, (r - 1) / |grad r| with r = sqrt((x/a)^2 + (y/b)^2); exact on
    the boundary, a smooth approximation off it."""
    def psi(x, y):
        r = np.sqrt((x / a) ** 2 + (y / b) ** 2)
        g = np.sqrt((x / (a * a)) ** 2 + (y / (b * b)) ** 2) / np.maximum(r, 1e-300)
        return (r - 1.0) / np.maximum(g, 1e-300)
    return psi


@dataclass
class PassingCylinders:
    """Two cylinders passing each other (the configuration of Sec. 4.4):
    D = 1 in a closed box of H = 16 D by L = 32 D, lower cylinder at
    (L_c, 0), upper at (L - L_c, H_s) at t = 0 (L_c = 8 D, H_s = 1.5 D);
    both oscillate along x with amplitude A = 1 / (2 pi f), f = 1 / T,
    T = 8, for two periods, then move at U = 2 pi f A = 1, the lower one
    towards +x and the upper one towards -x.  Ids 2 (lower) and 3 (upper).
    The box spans y in [-7.25, 8.75] (centred between the cylinders)."""

    D: float = 1.0
    L: float = 32.0
    H: float = 16.0
    Lc: float = 8.0
    Hs: float = 1.5
    T: float = 8.0

    @property
    def f(self):
        return 1.0 / self.T

    @property
    def A(self):
        return 1.0 / (2 * math.pi * self.f)

    @property
    def U(self):
        return 2 * math.pi * self.f * self.A

    def x_offset(self, t):
        """Displacement and velocity of the lower cylinder (the upper one
        moves by the opposite)."""
        if t <= 2 * self.T:
            w = 2 * math.pi * self.f
            return self.A * math.sin(w * t), self.A * w * math.cos(w * t)
        return self.U * (t - 2 * self.T), self.U

    def bodies(self, t):
        """[(id, centre, radius)] and [(vx, vy)] at time t."""
        dx, v = self.x_offset(t)
        R = 0.5 * self.D
        return ([(2, (self.Lc + dx, 0.0), R), (3, (self.L - self.Lc - dx, self.Hs), R)],
                [(v, 0.0), (-v, 0.0)])


def passing_cylinders_box(l0: float = 2.55e-2, cfg: PassingCylinders | None = None) -> Problem:
    """The closed box of the two passing cylinders on cells of width l0 (the
    paper's 2.55e-2 gives 1255 x 627 cells): DPs at the centroids, Dirichlet
    wall cells with their DPs on the walls, every other cell inner."""
    cfg = cfg or PassingCylinders()
    nx = int(round(cfg.L / l0))
    ny = int(round(cfg.H / l0))
    y0 = 0.5 * cfg.Hs - 0.5 * cfg.H
    mesh = Mesh(dim=2, n=(nx, ny, 1), l0=cfg.L / nx, origin=(0.0, y0, 0.0))
    pos = snap_wall_dps(mesh, mesh.centroids())
    mask = np.full(mesh.N, INNER, dtype=np.int8)
    mask[wall_cells(mesh)] = WALL_ID
    pb = Problem(mesh=mesh, pos=pos, mask=mask, bc_kind=default_bc_kind(neumann_ids=(2, 3)))
    pb.meta["passing"] = cfg
    return pb


@dataclass
class FlappingWing:
    """The hovering elliptic wing (the configuration of Sec. 4.6): chord
    c = 1, aspect ratio e = 4, in a closed 16 c x 16 c box whose upper and
    right walls are H0 = L0 = 6 c from the origin; stroke plane at
    beta = pi / 3; a(t) = a0 / 2 (1 + cos(2 t / a0)) along it and attack
    angle theta(t) = theta0 (1 - sin(2 t / a0 + phi)), a0 = 5 / 2,
    theta0 = pi / 4, phi = 0; period T = pi a0.  Reading: the wing's
    centre is a(t) (cos beta, sin beta) and its chord makes the angle
    beta - theta(t) with the x axis.  Body id 2."""

    c: float = 1.0
    e: float = 4.0
    L: float = 16.0
    H0: float = 6.0
    beta: float = math.pi / 3
    a0: float = 2.5
    theta0: float = math.pi / 4
    phi: float = 0.0
    body_id: int = BODY_ID

    @property
    def T(self):
        return math.pi * self.a0

    def a(self, t):
        return 0.5 * self.a0 * (1.0 + math.cos(2.0 * t / self.a0))

    def a_dot(self, t):
        return -math.sin(2.0 * t / self.a0)

    def theta(self, t):
        return self.theta0 * (1.0 - math.sin(2.0 * t / self.a0 + self.phi))

    def posture(self, t):
        return self.beta - self.theta(t)

    def omega(self, t):
        """d posture / dt = -d theta / dt."""
        return self.theta0 * (2.0 / self.a0) * math.cos(2.0 * t / self.a0 + self.phi)

    def centre(self, t):
        return (self.a(t) * math.cos(self.beta), self.a(t) * math.sin(self.beta))

    def velocity(self, t):
        return (self.a_dot(t) * math.cos(self.beta), self.a_dot(t) * math.sin(self.beta))

    def sdf_grid(self, h):
        """The wing's SDF (ellipse_sdf) sampled in its own frame, with a
        margin of 0.3 c around it; returns (grid, origin)."""
        ax, by = 0.5 * self.c, 0.5 * self.c / self.e
        m = 0.3 * self.c
        org = (-(ax + m), -(by + m))
        n = (int(math.ceil(2 * (ax + m) / h)) + 1, int(math.ceil(2 * (by + m) / h)) + 1)
        return sample_sdf_grid(ellipse_sdf(ax, by), org, h, n), org


def flapping_wing_box(l0: float = 51.0 / 1600.0, cfg: FlappingWing | None = None) -> Problem:
    """The closed box of the flapping wing on cells of width about l0 (the
    paper's 51/1600 gives 502 x 502 cells): DPs at the centroids,
    Dirichlet wall cells with their DPs on the walls, every other cell
    inner."""
    cfg = cfg or FlappingWing()
    n = int(round(cfg.L / l0))
    lo = cfg.H0 - cfg.L
    mesh = Mesh(dim=2, n=(n, n, 1), l0=cfg.L / n, origin=(lo, lo, 0.0))
    pos = snap_wall_dps(mesh, mesh.centroids())
    mask = np.full(mesh.N, INNER, dtype=np.int8)
    mask[wall_cells(mesh)] = WALL_ID
    pb = Problem(mesh=mesh, pos=pos, mask=mask, bc_kind=default_bc_kind(neumann_ids=(cfg.body_id,)))
    pb.meta["wing"] = cfg
    return pb


def ppe_source(pos: np.ndarray, t: float):
    """Smooth synthetic interior source for the pressure Poisson equation,
    standing in for div(u*)/dt of a flow step: O(1) amplitude, a few
    wavelengths across the unit box."""
    x, y = pos[0], pos[1]
    tp = 2.0 * math.pi
    return (np.sin(tp * x) * np.sin(tp * y) + 0.5 * np.cos(3 * tp * x) * np.sin(tp * y)) * \
        math.cos(tp * t)


def tgv_fields(pos: np.ndarray, t: float, nu: float):
    """Closed-form 2D Taylor-Green vortex on the periodic unit square."""
    x, y = pos[0], pos[1]
    F = math.exp(-8.0 * math.pi ** 2 * nu * t)
    tp = 2.0 * math.pi
    u = np.sin(tp * x) * np.cos(tp * y) * F
    v = -np.cos(tp * x) * np.sin(tp * y) * F
    p = 0.25 * (np.cos(2 * tp * x) + np.cos(2 * tp * y)) * F * F
    return u, v, p


def tgv_box(n: int, seed: int, jitter: float = 0.25, re: float = 100.0) -> Problem:
    """Periodic TGV at t = 0 on a jittered periodic DP cloud.

    DP 0 carries the Dirichlet id so that its pressure is pinned to the
    closed form (the periodic pressure system is otherwise singular).
    """
    pb = jittered_box(n, 2, seed, jitter, periodic=True)
    nu = 1.0 / re
    u, v, p = tgv_fields(pb.pos, 0.0, nu)
    pb.mask[0] = WALL_ID
    pb.meta.update(nu=nu, u=u, v=v, p=p)
    return pb


def cnn_weights(seed: int, c_in: int = 7, width: int = 32, layers: int = 4,
                c_out: int = 1):
    """He-initialised 3x3 conv weights [(c_out, c_in, 3, 3)] and zero biases,
    rounded to float32 (the precision of the network's master copy)."""
    rng = np.random.default_rng(seed)
    chans = [c_in] + [width] * (layers - 1) + [c_out]
    ws, bs = [], []
    for a, b in zip(chans[:-1], chans[1:]):
        std = math.sqrt(2.0 / (9 * a))
        ws.append(rng.normal(0.0, std, size=(b, a, 3, 3)).astype(np.float32).astype(np.float64))
        bs.append(np.zeros(b))
    return ws, bs


def cnn_weights_extrapolating(seed: int, scale: float = 0.1, c_in: int = 7, width: int = 32,
                              layers: int = 4, channel: int = 6):
    """Initial weights whose network already computes y = x[channel] (the
    input's increment channel) exactly, plus He-normal weights times `scale`
    everywhere else: two hidden channels carry relu(x) and relu(-x) through
    the centre taps, the last layer takes their difference (weights +-1 and
    0, exact in bf16).  Training starts from that map instead of from noise."""
    ws, bs = cnn_weights(seed, c_in, width, layers)
    for w in ws:
        w *= scale
    ws[0][0, :, :, :] = 0.0
    ws[0][1, :, :, :] = 0.0
    ws[0][0, channel, 1, 1] = 1.0
    ws[0][1, channel, 1, 1] = -1.0
    for w in ws[1:-1]:
        w[0:2, :, :, :] = 0.0
        w[:, 0:2, :, :] = 0.0
        w[0, 0, 1, 1] = 1.0
        w[1, 1, 1, 1] = 1.0
    ws[-1][:, 0:2, :, :] = 0.0
    ws[-1][0, 0, 1, 1] = 1.0
    ws[-1][0, 1, 1, 1] = -1.0
    return ws, bs


def cnn_flatten(ws, bs):
    """Flat float32 parameter vector: per layer W[o][c][dj][di], then b[o]."""
    parts = []
    for w, b in zip(ws, bs):
        parts += [np.asarray(w, np.float32).ravel(), np.asarray(b, np.float32).ravel()]
    return np.concatenate(parts)


def cnn_unflatten(flat, c_in: int = 7, width: int = 32, layers: int = 4, c_out: int = 1):
    """Inverse of cnn_flatten (float64 arrays)."""
    chans = [c_in] + [width] * (layers - 1) + [c_out]
    ws, bs, at = [], [], 0
    for a, b in zip(chans[:-1], chans[1:]):
        n = b * a * 9
        ws.append(np.asarray(flat[at:at + n], np.float64).reshape(b, a, 3, 3))
        at += n
        bs.append(np.asarray(flat[at:at + b], np.float64))
        at += b
    return ws, bs
