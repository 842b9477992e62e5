"""ctypes front end of the CPU oracle (oracle/pic_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg use this module; the library under test never imports it.

The oracle is a plain, slow, FP64, -ffp-contract=off restatement of the
paper's particle steps (Gassmoeller et al., arXiv 1612.03369, Sec. 2.2-2.7).
Every function here only marshals numpy arrays into the C code.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pic_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp.%d" % os.getpid()
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB)
    P = C.c_void_p
    i64, u64, u32, f64 = C.c_int64, C.c_uint64, C.c_uint32, C.c_double
    lib.orc_mesh_create.restype = P
    lib.orc_mesh_create.argtypes = [C.c_int, P, P]
    lib.orc_mesh_set_velocity.argtypes = [P, P]
    lib.orc_mesh_set_velocity_next.argtypes = [P, P]
    lib.orc_mesh_destroy.argtypes = [P]
    lib.orc_phi.argtypes = [P, i64, P, P]
    lib.orc_newton.restype = C.c_int
    lib.orc_newton.argtypes = [P, i64, P, P, P, P]
    lib.orc_inside.restype = C.c_int
    lib.orc_inside.argtypes = [P, i64, P, P]
    lib.orc_owner.restype = i64
    lib.orc_owner.argtypes = [P, P, P]
    lib.orc_owner_brute.restype = i64
    lib.orc_owner_brute.argtypes = [P, P, P]
    lib.orc_q2_eval.argtypes = [P, i64, P, P]
    lib.orc_splitmix64.restype = u64
    lib.orc_splitmix64.argtypes = [u64, u64]
    lib.orc_seed.restype = i64
    lib.orc_seed.argtypes = [P, P, u32, u64, u64, P, P, P, P]
    lib.orc_advect.restype = i64
    lib.orc_advect.argtypes = [P, i64, P, P, P, P, P, C.c_int, f64, C.c_int, C.c_int, P]
    lib.orc_locate_points.argtypes = [P, i64, P, P, P, C.c_int]
    lib.orc_cell_average.argtypes = [i64, i64, P, P, f64, P, P]
    lib.orc_cell_average_kind.argtypes = [i64, i64, P, P, C.c_int, f64, P, P]
    lib.orc_advect_adjoint.restype = f64
    lib.orc_advect_adjoint.argtypes = [P, i64, P, P, P, f64, C.c_int, C.c_int, P, P]
    lib.orc_advect_properties.restype = i64
    lib.orc_advect_properties.argtypes = [P, i64, P, P, P, P, P, C.c_int, f64, C.c_int, C.c_int, C.c_int, f64, f64,
                                          C.c_int, P]
    lib.orc_vertex_average.argtypes = [P, i64, P, P, P, f64, P, P]
    lib.orc_cell_lsq_linear.argtypes = [P, i64, P, P, P, f64, P, P]
    lib.orc_cell_weights.argtypes = [P, P, P]
    lib.orc_draw_cell_counts.argtypes = [i64, P, i64, u64, P]
    lib.orc_seed_mh.restype = i64
    lib.orc_seed_mh.argtypes = [P, P, P, u32, u64, u64, P, P, P, P]
    lib.orc_import.restype = i64
    lib.orc_import.argtypes = [P, i64, P, u64, P, P, P, P]
    lib.orc_advect_tangent.restype = None
    lib.orc_advect_tangent.argtypes = [P, i64, P, P, P, f64, C.c_int, C.c_int, P, P, P]
    lib.orc_advect_loss.restype = f64
    lib.orc_advect_loss.argtypes = [P, i64, P, P, P, f64, C.c_int, C.c_int, P]
    _lib = lib
    return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class Mesh:
    """Structured mesh of (bi/tri)linear cells with a Q2 nodal velocity."""

    def __init__(self, n, X, U=None):
        lib = _load()
        self.dim = len(n)
        self.n = tuple(int(v) for v in n)
        nn = np.array(list(self.n) + [1] * (3 - self.dim), dtype=np.int64)
        self.X = np.ascontiguousarray(X, dtype=np.float64)
        assert self.X.shape == (self.dim, int(np.prod([v + 1 for v in self.n])))
        self._h = lib.orc_mesh_create(self.dim, _p(nn), _p(self.X))
        self.ncells = int(np.prod(self.n))
        if U is not None:
            self.set_velocity(U)

    def set_velocity(self, U):
        self.U = np.ascontiguousarray(U, dtype=np.float64)
        assert self.U.shape == (self.dim, int(np.prod([2 * v + 1 for v in self.n])))
        _load().orc_mesh_set_velocity(self._h, _p(self.U))

    def set_velocity_next(self, Un=None):
        """Field at the end of every step (time interpolation), or None."""
        if Un is None:
            self.Unext = None
            _load().orc_mesh_set_velocity_next(self._h, None)
            return
        self.Unext = np.ascontiguousarray(Un, dtype=np.float64)
        assert self.Unext.shape == self.U.shape
        _load().orc_mesh_set_velocity_next(self._h, _p(self.Unext))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_mesh_destroy(self._h)
            self._h = None

    # single-point primitives --------------------------------------------
    def phi(self, K: int, xhat) -> np.ndarray:
        t = np.ascontiguousarray(xhat, dtype=np.float64)
        out = np.zeros(self.dim)
        _load().orc_phi(self._h, int(K), _p(t), _p(out))
        return out

    def newton(self, K: int, x, start=None):
        x = np.ascontiguousarray(x, dtype=np.float64)
        s = np.full(self.dim, 0.5) if start is None else np.ascontiguousarray(start, dtype=np.float64)
        t = np.zeros(self.dim)
        it = C.c_int(0)
        conv = _load().orc_newton(self._h, int(K), _p(x), _p(s), _p(t), C.byref(it))
        return bool(conv), t, int(it.value)

    def inside(self, K: int, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        t = np.zeros(self.dim)
        r = _load().orc_inside(self._h, int(K), _p(x), _p(t))
        return bool(r), t

    def owner(self, x, brute: bool = False):
        x = np.ascontiguousarray(x, dtype=np.float64)
        t = np.zeros(self.dim)
        f = _load().orc_owner_brute if brute else _load().orc_owner
        K = f(self._h, _p(x), _p(t))
        return int(K), t

    def q2(self, K: int, xhat) -> np.ndarray:
        t = np.ascontiguousarray(xhat, dtype=np.float64)
        out = np.zeros(self.dim)
        _load().orc_q2_eval(self._h, int(K), _p(t), _p(out))
        return out

    # batched ----------------------------------------------------------------
    def locate(self, x, brute: bool = False):
        """x [n][dim] -> (cell [n] int64, -1 = outside; xhat [n][dim])."""
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, self.dim)
        n = x.shape[0]
        cell = np.zeros(n, dtype=np.int64)
        xh = np.zeros((n, self.dim))
        _load().orc_locate_points(self._h, n, _p(x), _p(cell), _p(xh), int(brute))
        return cell, xh


def splitmix64(seed: int, n: int) -> int:
    return int(_load().orc_splitmix64(C.c_uint64(seed & (2**64 - 1)), C.c_uint64(n)))


class Particles:
    """Particle-major arrays in (cell, id) order."""

    def __init__(self, x, xhat, cell, id, props):
        self.x = np.ascontiguousarray(x, dtype=np.float64)
        self.xhat = np.ascontiguousarray(xhat, dtype=np.float64)
        self.cell = np.ascontiguousarray(cell, dtype=np.int64)
        self.id = np.ascontiguousarray(id, dtype=np.uint64)
        self.props = np.ascontiguousarray(props, dtype=np.float64)
        self.n_lost = 0

    @property
    def n(self) -> int:
        return int(self.cell.shape[0])

    def copy(self) -> "Particles":
        p = Particles(self.x.copy(), self.xhat.copy(), self.cell.copy(), self.id.copy(), self.props.copy())
        p.n_lost = self.n_lost
        return p

    def subset(self, mask) -> "Particles":
        return Particles(self.x[mask], self.xhat[mask], self.cell[mask], self.id[mask], self.props[mask])


def seed_particles(mesh: Mesh, per_cell=None, uniform_count: int = 0, seed: int = 0, first_id: int = 0,
                   n_props: int = 0) -> Particles:
    """Local-coordinate generation, ids in creation order (R11)."""
    if per_cell is not None:
        pc = np.ascontiguousarray(per_cell, dtype=np.uint32)
        N = int(pc.sum())
        pcp = _p(pc)
    else:
        pc = None
        N = mesh.ncells * int(uniform_count)
        pcp = None
    d = mesh.dim
    x = np.zeros((N, d))
    xh = np.zeros((N, d))
    cell = np.zeros(N, dtype=np.int64)
    ids = np.zeros(N, dtype=np.uint64)
    n = _load().orc_seed(mesh._h, pcp, int(uniform_count), C.c_uint64(seed & (2**64 - 1)), C.c_uint64(first_id),
                         _p(x), _p(xh), _p(cell), _p(ids))
    assert n == N
    return Particles(x, xh, cell, ids, np.zeros((N, n_props)))


def cell_weights(mesh: Mesh, rho) -> np.ndarray:
    """Sec. 2.2: w_K = int_K rho_h dx for a (bi/tri)linear density given at the vertices."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    assert rho.shape == (mesh.X.shape[1],)
    w = np.zeros(mesh.ncells)
    _load().orc_cell_weights(mesh._h, _p(rho), _p(w))
    return w


def draw_cell_counts(w, n_particles: int, seed: int) -> np.ndarray:
    """Sec. 2.2 listing: n_particles draws over the accumulated weights (R19)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    counts = np.zeros(w.shape[0], dtype=np.int64)
    _load().orc_draw_cell_counts(int(w.shape[0]), _p(w), int(n_particles), C.c_uint64(seed & (2**64 - 1)),
                                 _p(counts))
    return counts


def seed_particles_mh(mesh: Mesh, per_cell, rho, thinning: int, seed: int, first_id: int = 0,
                      n_props: int = 0) -> Particles:
    """Sec. 2.2 in-cell Metropolis-Hastings generation with density rho (R20)."""
    pc = np.ascontiguousarray(per_cell, dtype=np.uint32)
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    N = int(pc.sum())
    d = mesh.dim
    x, xh = np.zeros((N, d)), np.zeros((N, d))
    cell, ids = np.zeros(N, dtype=np.int64), np.zeros(N, dtype=np.uint64)
    n = _load().orc_seed_mh(mesh._h, _p(pc), _p(rho), int(thinning), C.c_uint64(seed & (2**64 - 1)),
                            C.c_uint64(first_id), _p(x), _p(xh), _p(cell), _p(ids))
    assert n == N
    return Particles(x, xh, cell, ids, np.zeros((N, n_props)))


def import_points(mesh: Mesh, x, first_id: int = 0, n_props: int = 0) -> Particles:
    """Sec. 2.2 prescribed locations: owner search for every point, ids in input order."""
    x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1, mesh.dim)
    n, d = x.shape
    xo, xh = np.zeros((n, d)), np.zeros((n, d))
    cell, ids = np.zeros(n, dtype=np.int64), np.zeros(n, dtype=np.uint64)
    c = _load().orc_import(mesh._h, n, _p(x), C.c_uint64(first_id), _p(xo), _p(xh), _p(cell), _p(ids))
    return Particles(xo[:c], xh[:c], cell[:c], ids[:c], np.zeros((c, n_props)))


def advect(mesh: Mesh, parts: Particles, dt: float, integrator: int, n_steps: int) -> Particles:
    """n_steps of (advance all particles with stage locates; drop lost; sort
    by (cell, id)).  Returns a new Particles."""
    p = parts.copy()
    d = mesh.dim
    nprops = p.props.shape[1] if p.props.ndim == 2 else 0
    lost = C.c_int64(0)
    n = _load().orc_advect(mesh._h, p.n, _p(p.x), _p(p.xhat), _p(p.cell), _p(p.id), _p(p.props), nprops,
                           float(dt), int(integrator), int(n_steps), C.byref(lost))
    out = Particles(p.x[:n], p.xhat[:n], p.cell[:n], p.id[:n], p.props[:n])
    out.n_lost = parts.n_lost + int(lost.value)
    return out


def advect_properties(mesh: Mesh, parts: Particles, dt: float, integrator: int, n_steps: int, damage: int = -1,
                      alpha: float = 0.0, beta: float = 0.0, defgrad: int = -1) -> Particles:
    """advect() with the Sec. 2.6 property ODEs integrated along the paths:
    property `damage` holds d (d' = alpha |sym grad u| - beta d), properties
    defgrad .. defgrad + dim^2 - 1 hold F row-major (F' = grad u F); -1 = off."""
    p = parts.copy()
    d = mesh.dim
    nprops = p.props.shape[1] if p.props.ndim == 2 else 0
    lost = C.c_int64(0)
    n = _load().orc_advect_properties(mesh._h, p.n, _p(p.x), _p(p.xhat), _p(p.cell), _p(p.id), _p(p.props), nprops,
                                      float(dt), int(integrator), int(n_steps), int(damage), float(alpha),
                                      float(beta), int(defgrad), C.byref(lost))
    if n < 0:
        raise ValueError("advect_properties: the steady field only")
    out = Particles(p.x[:n], p.xhat[:n], p.cell[:n], p.id[:n], p.props[:n])
    out.n_lost = parts.n_lost + int(lost.value)
    return out


def cell_average(ncells: int, cell, value, empty_fill: float = 0.0, kind: int = 0):
    """Per-cell average (Sec. 2.7 (ii)): kind 0 arithmetic, 1 geometric,
    2 harmonic; left folds in store order."""
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    value = np.ascontiguousarray(value, dtype=np.float64)
    avg = np.zeros(ncells)
    cnt = np.zeros(ncells, dtype=np.int64)
    _load().orc_cell_average_kind(int(ncells), int(cell.shape[0]), _p(cell), _p(value), int(kind), float(empty_fill),
                                  _p(avg), _p(cnt))
    return avg, cnt


def vertex_average(mesh: Mesh, cell, xhat, value, empty_fill: float = 0.0):
    """Sec. 2.7 (iv): shape-function-weighted average at the mesh vertices
    (R17).  Returns (avg [nverts], weight sum [nverts])."""
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    xhat = np.ascontiguousarray(xhat, dtype=np.float64)
    value = np.ascontiguousarray(value, dtype=np.float64)
    nv = mesh.X.shape[1]
    avg, w = np.zeros(nv), np.zeros(nv)
    _load().orc_vertex_average(mesh._h, int(cell.shape[0]), _p(cell), _p(xhat), _p(value), float(empty_fill), _p(avg),
                               _p(w))
    return avg, w


def cell_lsq_linear(mesh: Mesh, cell, xhat, value, empty_fill: float = 0.0):
    """Sec. 2.7 (v): per-cell linear least squares in reference coordinates
    (R18).  Returns (coef [ncells][dim+1], count [ncells])."""
    cell = np.ascontiguousarray(cell, dtype=np.int64)
    xhat = np.ascontiguousarray(xhat, dtype=np.float64)
    value = np.ascontiguousarray(value, dtype=np.float64)
    coef = np.zeros((mesh.ncells, mesh.dim + 1))
    cnt = np.zeros(mesh.ncells, dtype=np.int64)
    _load().orc_cell_lsq_linear(mesh._h, int(cell.shape[0]), _p(cell), _p(xhat), _p(value), float(empty_fill),
                                _p(coef), _p(cnt))
    return coef, cnt


def advect_adjoint(mesh: Mesh, parts: Particles, dt: float, integrator: int, n_steps: int, targets):
    """(loss, dL/dU [dim][nnodes]) for L = sum over survivors of |x_final - target|^2;
    targets [N][dim] in the order of `parts`."""
    t = np.ascontiguousarray(targets, dtype=np.float64)
    g = np.zeros((mesh.dim, mesh.U.shape[1]))
    L = _load().orc_advect_adjoint(mesh._h, parts.n, _p(parts.x), _p(parts.xhat), _p(parts.cell), float(dt),
                                   int(integrator), int(n_steps), _p(t), _p(g))
    return float(L), g


def advect_tangent(mesh: Mesh, parts: Particles, dt: float, integrator: int, n_steps: int, V):
    """(dx [N][dim], alive [N]): the derivative of each particle's final
    position in the direction V ([dim][nnodes]) of the nodal velocities, by
    forward (tangent-linear) mode; 0 for particles lost on the way."""
    Vc = np.ascontiguousarray(V, dtype=np.float64)
    dx = np.zeros((parts.n, mesh.dim))
    alive = np.zeros(parts.n, dtype=np.int32)
    _load().orc_advect_tangent(mesh._h, parts.n, _p(parts.x), _p(parts.xhat), _p(parts.cell), float(dt),
                               int(integrator), int(n_steps), _p(Vc), _p(dx), _p(alive))
    return dx, alive.astype(bool)


def advect_loss(mesh: Mesh, parts: Particles, dt: float, integrator: int, n_steps: int, targets) -> float:
    t = np.ascontiguousarray(targets, dtype=np.float64)
    return float(_load().orc_advect_loss(mesh._h, parts.n, _p(parts.x), _p(parts.xhat), _p(parts.cell), float(dt),
                                         int(integrator), int(n_steps), _p(t)))
