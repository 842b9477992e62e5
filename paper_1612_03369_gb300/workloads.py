"""Seeded synthetic inputs for the particle hot path.

This module only builds INPUTS: mesh vertex coordinates, Q2 nodal velocity
values, time steps and regression targets.  It holds none of the method's
arithmetic (no cell map, no inverse map, no basis evaluation, no integrator,
no location, no sorting), so both the CUDA path and the CPU oracle can take
their inputs from here without sharing any of the computation under test.

Workloads (the method is Sec. 2.3-2.7 of Gassmoeller et al., arXiv 1612.03369;
the paper's own experiments need a Stokes solver and datasets, so these seeded
fields stand in for its spherical-shell circular flow and convection runs):

  c1  2D unit square, 32x32 uniform quads, rigid rotation about (1/2, 1/2),
      16 particles per cell, one property (= x0), RK2, dt at CFL 0.5, 10 steps
  c2  3D unit cube, 64^3 hexes with interior vertices jittered by up to 0.1 h,
      velocity = curl of 8 random-phase sinusoidal vector potentials with zero
      wall-normal flow, 20 particles per cell, 3 properties, RK4, 50 steps
  c3  as c2 at 128^3 (precision form), RK4, 20 steps
  c4  as c2 at 32^3 with 32 particles per cell (adjoint), RK4, 20 steps
  c5  64 independent 2D problems, 64^2..512^2 jittered quads, stream-function
      velocity, log-normal particles per cell (median 8, max 128), RK4, 10 steps

Random sub-streams (numpy PCG64 keyed on [seed, sub-stream]): 0 vertex
jitter, 1 field phases, 2 particles (the seed handed to the library), 3
regression targets, 4 ensemble sizes.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SUB_JITTER, SUB_FIELD, SUB_PARTICLES, SUB_TARGETS, SUB_ENSEMBLE = 0, 1, 2, 3, 4


def rng(seed: int, sub: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(sub)])


def particle_seed(seed: int) -> int:
    """64-bit seed handed to the library's counter-based particle generator."""
    return int(rng(seed, SUB_PARTICLES).integers(0, 2**63 - 1))


# --------------------------------------------------------------------- mesh


def uniform_vertices(n: tuple[int, ...]) -> np.ndarray:
    """Vertex coordinates [dim][nverts] of the uniform grid on the unit box.

    Vertex (i, j[, k]) sits at (i/nx, j/ny[, k/nz]) and has flat index
    i + (nx+1)*(j + (ny+1)*k).
    """
    dim = len(n)
    axes = [np.arange(m + 1, dtype=np.float64) / m for m in n]
    grids = np.meshgrid(*axes, indexing="ij")  # grids[a][i,j,k]
    # flat index runs fastest in i: transpose to (k, j, i) then ravel
    return np.stack([g.transpose(tuple(range(dim))[::-1]).ravel() for g in grids])


def jittered_vertices(n: tuple[int, ...], seed: int, frac: float = 0.1) -> np.ndarray:
    """Uniform grid with every coordinate of every interior vertex moved by
    U(-frac*h, frac*h) on its own axis; boundary vertices stay put so the
    walls remain flat."""
    X = uniform_vertices(n)
    dim = len(n)
    g = rng(seed, SUB_JITTER)
    nv = [m + 1 for m in n]
    idx = np.indices(nv[::-1]).reshape(dim, -1)[::-1]  # idx[a][flat] = index along axis a
    interior = np.ones(X.shape[1], dtype=bool)
    for a in range(dim):
        interior &= (idx[a] > 0) & (idx[a] < n[a])
    for a in range(dim):
        h = 1.0 / n[a]
        off = g.uniform(-frac * h, frac * h, size=X.shape[1])
        X[a] = np.where(interior, X[a] + off, X[a])
    return X


def q2_node_coords(n: tuple[int, ...], X: np.ndarray) -> np.ndarray:
    """Physical coordinates [dim][nnodes] of the Q2 nodes of a (bi/tri)linear
    mesh: an even node index along an axis sits on a vertex line, an odd one
    halfway between the two neighbouring vertex lines, so nodes are vertices,
    edge midpoints, face centres and cell centres (averages of 1, 2, 4 or 8
    vertices).  Node (I, J[, K]) has flat index I + (2nx+1)*(J + (2ny+1)*K)."""
    dim = len(n)
    nv = [m + 1 for m in n]
    nq = [2 * m + 1 for m in n]
    nnodes = int(np.prod(nq))
    flat = np.arange(nnodes)
    I = []  # node index along each axis
    rem = flat
    for a in range(dim):
        I.append(rem % nq[a])
        rem = rem // nq[a]
    stride = [1, nv[0], nv[0] * nv[1]]
    out = np.zeros((dim, nnodes))
    for corner in np.ndindex(*(2,) * dim):
        v = np.zeros(nnodes, dtype=np.int64)
        for a in range(dim):
            v += (I[a] // 2 + np.where(I[a] % 2 == 1, corner[a], 0)) * stride[a]
        out += X[:, v]
    return out / float(2**dim)


# ------------------------------------------------------------------- fields


def rotation_field(P: np.ndarray) -> np.ndarray:
    """Rigid rotation about (1/2, 1/2): u = (-(y - 1/2), x - 1/2)."""
    return np.stack([-(P[1] - 0.5), P[0] - 0.5])


def curl_potential_field(P: np.ndarray, seed: int, n_modes: int = 8) -> tuple[np.ndarray, dict]:
    """u = curl A with A = (g1 sin(pi y) sin(pi z), g2 sin(pi x) sin(pi z),
    g3 sin(pi x) sin(pi y)), g_i = sum_m cos(pi k_m . x + phi_{m,i}),
    k_m in {1,2,3}^3, phi uniform in [0, 2 pi).  Every wall-normal component
    carries a factor sin(pi x_n), so the normal flow vanishes on the walls."""
    g = rng(seed, SUB_FIELD)
    k = g.integers(1, 4, size=(n_modes, 3)).astype(np.float64)
    phi = g.uniform(0.0, 2.0 * math.pi, size=(n_modes, 3))
    x, y, z = P
    pi = math.pi
    sx, sy, sz = np.sin(pi * x), np.sin(pi * y), np.sin(pi * z)
    cx, cy, cz = np.cos(pi * x), np.cos(pi * y), np.cos(pi * z)
    gv = np.zeros((3,) + x.shape)
    dg = np.zeros((3, 3) + x.shape)  # dg[i][j] = d g_i / d x_j
    for m in range(n_modes):
        arg = pi * (k[m, 0] * x + k[m, 1] * y + k[m, 2] * z)
        for i in range(3):
            gv[i] += np.cos(arg + phi[m, i])
            s = np.sin(arg + phi[m, i])
            for j in range(3):
                dg[i, j] -= pi * k[m, j] * s
    g1, g2, g3 = gv
    ux = sx * (dg[2, 1] * sy + g3 * pi * cy - dg[1, 2] * sz - g2 * pi * cz)
    uy = sy * (dg[0, 2] * sz + g1 * pi * cz - dg[2, 0] * sx - g3 * pi * cx)
    uz = sz * (dg[1, 0] * sx + g2 * pi * cx - dg[0, 1] * sy - g1 * pi * cy)
    return np.stack([ux, uy, uz]), {"k": k, "phi": phi}


def stream_function_field(P: np.ndarray, seed: int, n_modes: int = 8) -> np.ndarray:
    """2D u = (d psi/dy, -d psi/dx) with psi = sin(pi x) sin(pi y) *
    sum_m cos(pi k_m . x + phi_m); the sin factors make psi vanish on the walls,
    so the normal flow is zero there."""
    g = rng(seed, SUB_FIELD)
    k = g.integers(1, 4, size=(n_modes, 2)).astype(np.float64)
    phi = g.uniform(0.0, 2.0 * math.pi, size=n_modes)
    x, y = P
    pi = math.pi
    sx, sy, cx, cy = np.sin(pi * x), np.sin(pi * y), np.cos(pi * x), np.cos(pi * y)
    G = np.zeros_like(x)
    Gx = np.zeros_like(x)
    Gy = np.zeros_like(x)
    for m in range(n_modes):
        arg = pi * (k[m, 0] * x + k[m, 1] * y) + phi[m]
        G += np.cos(arg)
        Gx -= pi * k[m, 0] * np.sin(arg)
        Gy -= pi * k[m, 1] * np.sin(arg)
    dpsi_dx = pi * cx * sy * G + sx * sy * Gx
    dpsi_dy = pi * sx * cy * G + sx * sy * Gy
    return np.stack([dpsi_dy, -dpsi_dx])


def zero_wall_normal(n: tuple[int, ...], U: np.ndarray) -> np.ndarray:
    """Set the wall-normal component of every boundary node exactly to 0."""
    dim = len(n)
    nq = [2 * m + 1 for m in n]
    idx = np.indices(nq[::-1]).reshape(dim, -1)[::-1]
    U = U.copy()
    for a in range(dim):
        wall = (idx[a] == 0) | (idx[a] == nq[a] - 1)
        U[a, wall] = 0.0
    return U


def normalise_max(U: np.ndarray) -> np.ndarray:
    """Scale so that the largest nodal speed is 1."""
    s = np.sqrt((U * U).sum(axis=0)).max()
    return U / s if s > 0 else U


def cfl_dt(n: tuple[int, ...], X: np.ndarray, U: np.ndarray, cfl: float) -> float:
    """R8: dt = CFL * h_min / max_nodes |U|, h_min the shortest cell edge."""
    dim = len(n)
    nv = [m + 1 for m in n]
    Xg = X.reshape((dim,) + tuple(nv[::-1]))
    hmin = math.inf
    for a in range(dim):
        ax = dim - 1 - a  # array axis of mesh axis a
        d = np.diff(Xg, axis=ax + 1)  # edges along mesh axis a
        hmin = min(hmin, float(np.sqrt((d * d).sum(axis=0)).min()))
    umax = float(np.sqrt((U * U).sum(axis=0)).max())
    return cfl * hmin / umax


# ------------------------------------------------------------------ configs


@dataclass
class Workload:
    name: str
    dim: int
    n: tuple
    X: np.ndarray  # [dim][nverts]
    U: np.ndarray  # [dim][nnodes]
    ppc: int | None  # uniform particles per cell, or None with per_cell
    per_cell: np.ndarray | None
    n_props: int
    integrator: int  # 1 Euler, 2 RK2, 4 RK4
    dt: float
    n_steps: int
    seed: int
    pseed: int  # particle seed for the counter-based generator
    first_id: int = 0
    meta: dict = field(default_factory=dict)

    @property
    def ncells(self) -> int:
        return int(np.prod(self.n))

    @property
    def n_particles(self) -> int:
        if self.per_cell is not None:
            return int(self.per_cell.sum())
        return self.ncells * int(self.ppc)


def c1(n: int = 32, ppc: int = 16, n_steps: int = 10, seed: int = 1) -> Workload:
    dims = (n, n)
    X = uniform_vertices(dims)
    U = rotation_field(q2_node_coords(dims, X))
    dt = cfl_dt(dims, X, U, 0.5)
    return Workload("c1_2d_rotation_%d^2" % n, 2, dims, X, U, ppc, None, 1, 2, dt, n_steps, seed, particle_seed(seed))


def curl_cube(n: int, ppc: int, n_steps: int, seed: int, integrator: int = 4, n_props: int = 3,
              name: str = "3d_curl") -> Workload:
    dims = (n, n, n)
    X = jittered_vertices(dims, seed)
    U, meta = curl_potential_field(q2_node_coords(dims, X), seed)
    U = zero_wall_normal(dims, normalise_max(U))
    dt = cfl_dt(dims, X, U, 0.5)
    return Workload("%s_%d^3" % (name, n), 3, dims, X, U, ppc, None, n_props, integrator, dt, n_steps, seed,
                    particle_seed(seed), meta=meta)


def c2(n: int = 64, ppc: int = 20, n_steps: int = 50, seed: int = 2) -> Workload:
    return curl_cube(n, ppc, n_steps, seed, name="c2_3d_curl")


def c3(n: int = 128, ppc: int = 20, n_steps: int = 20, seed: int = 2) -> Workload:
    return curl_cube(n, ppc, n_steps, seed, name="c3_3d_curl_fp32basis")


def c4(n: int = 32, ppc: int = 32, n_steps: int = 20, seed: int = 4) -> Workload:
    return curl_cube(n, ppc, n_steps, seed, name="c4_3d_adjoint")


def member_per_cell(side: int, seed: int, sigma: float = 1.0, median: float = 8.0, max_ppc: int = 128) -> np.ndarray:
    """Particles per cell of one ensemble member (log-normal, R13)."""
    z = rng(seed, SUB_ENSEMBLE).standard_normal(side * side)
    return np.minimum(max_ppc, np.rint(np.exp(math.log(median) + sigma * z))).astype(np.uint32)


def c5_member_seed(p: int, seed: int = 5) -> int:
    return seed * 1000 + p


def c5_member(side: int, seed: int, sigma: float = 1.0, median: float = 8.0, max_ppc: int = 128,
              n_steps: int = 10) -> Workload:
    """One ensemble member: jittered side^2 quads, stream-function field,
    particles per cell min(max_ppc, round(exp(ln(median) + sigma Z))) (R13)."""
    dims = (side, side)
    X = jittered_vertices(dims, seed)
    U = zero_wall_normal(dims, normalise_max(stream_function_field(q2_node_coords(dims, X), seed)))
    per_cell = member_per_cell(side, seed, sigma, median, max_ppc)
    dt = cfl_dt(dims, X, U, 0.5)
    return Workload("c5_member_%d^2" % side, 2, dims, X, U, None, per_cell, 1, 4, dt, n_steps, seed,
                    particle_seed(seed))


def c5_sides(n_problems: int = 64, seed: int = 5) -> list[int]:
    """n = round(2^(6 + 3U)) per side, log-uniform in 64..512."""
    u = rng(seed, SUB_ENSEMBLE).uniform(0.0, 1.0, size=n_problems)
    return [int(round(2.0 ** (6.0 + 3.0 * v))) for v in u]


def c5(n_problems: int = 64, seed: int = 5, scale: float = 1.0) -> list[Workload]:
    sides = c5_sides(n_problems, seed)
    out = []
    for p, s in enumerate(sides):
        s = max(2, int(round(s * scale)))
        out.append(c5_member(s, c5_member_seed(p, seed)))
    return out


def adjoint_targets(x_final: np.ndarray, h: float, seed: int) -> np.ndarray:
    """Regression targets: final positions plus N(0, h^2) noise."""
    return x_final + h * rng(seed, SUB_TARGETS).standard_normal(x_final.shape)
