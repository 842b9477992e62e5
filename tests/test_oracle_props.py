"""Pins of the oracle's property ODEs (Sec. 2.6: damage d' = alpha |eps-dot| - beta d,
deformation gradient F' = grad u F) against closed forms and against the
derivative of the oracle's own position map.

- In a field linear in x, Q2 on (bi/tri)linear cells is exact and
  grad u_h = A everywhere.  The classical RK methods are affine-equivariant,
  so n steps give F_n = R(dt A)^n F_0 and d_n - d* = R(-beta dt)^n (d_0 - d*),
  with R the method's stability polynomial and d* = alpha |sym A|_F / beta.
  A random F_0 that does not commute with A also tells G F from F G.
- F integrated along a path by the same RK as the position is the derivative
  of the discrete position map x_0 -> x_n.  With a quadratic field on an
  affine mesh grad u_h is continuous, the map is smooth, and central
  differences of the positions alone must reproduce F.
"""
import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W


def _rk_poly(Z, integrator):
    I = np.eye(Z.shape[0])
    if integrator == 1:
        return I + Z
    if integrator == 2:
        return I + Z + Z @ Z / 2
    Z2 = Z @ Z
    return I + Z + Z2 / 2 + Z2 @ Z / 6 + Z2 @ Z2 / 24


def _A(dim):
    if dim == 2:
        return np.array([[0.2, -1.0], [0.7, -0.3]])
    return np.array([[0.3, -1.0, 0.2], [0.8, -0.1, 0.4], [-0.5, 0.6, -0.2]])


@pytest.mark.parametrize("dim,integrator", [(2, 1), (2, 2), (2, 4), (3, 2), (3, 4)])
def test_linear_field_closed_forms(oracle_mod, dim, integrator):
    O = oracle_mod
    n = (8, 8) if dim == 2 else (5, 5, 5)
    X = W.jittered_vertices(n, 41)
    P = W.q2_node_coords(n, X)
    A = _A(dim)
    c = np.full(dim, 0.5)
    m = O.Mesh(n, X, A @ (P - c[:, None]))
    p0 = O.seed_particles(m, uniform_count=3, seed=8, n_props=2 + dim * dim)
    g = np.random.default_rng(12)
    N = p0.n
    p0.props[:, 0] = g.uniform(0.0, 2.0, N)                  # d_0
    F0 = g.uniform(-1.0, 1.0, (N, dim, dim)) + 2 * np.eye(dim)
    p0.props[:, 1:1 + dim * dim] = F0.reshape(N, -1)         # F_0, row-major
    p0.props[:, -1] = g.uniform(-5, 5, N)                    # rides along
    alpha, beta, dt, steps = 0.7, 1.3, 0.03, 5
    p = O.advect_properties(m, p0, dt, integrator, steps, damage=0, alpha=alpha, beta=beta, defgrad=1)
    assert p.n > 0.5 * N
    Rn = np.linalg.matrix_power(_rk_poly(dt * A, integrator), steps)
    sym = 0.5 * (A + A.T)
    dstar = alpha * np.sqrt((sym * sym).sum()) / beta
    rd = _rk_poly(np.array([[-beta * dt]]), integrator)[0, 0] ** steps
    start = {int(i): k for k, i in enumerate(p0.id)}
    for i, x, pr in zip(p.id, p.x, p.props):
        k = start[int(i)]
        np.testing.assert_allclose(x, c + Rn @ (p0.x[k] - c), rtol=0, atol=1e-13)
        np.testing.assert_allclose(pr[1:1 + dim * dim].reshape(dim, dim), Rn @ F0[k], rtol=0, atol=5e-13)
        assert abs(pr[0] - (dstar + rd * (p0.props[k, 0] - dstar))) < 5e-14
        assert pr[-1] == p0.props[k, -1]
    # the position part is the plain advection, bit for bit
    q = O.advect(m, p0, dt, integrator, steps)
    np.testing.assert_array_equal(q.id, p.id)
    np.testing.assert_array_equal(q.x, p.x)
    np.testing.assert_array_equal(q.cell, p.cell)


def test_rigid_rotation_no_strain(oracle_mod):
    """A rigid rotation has eps-dot = 0: damage only heals, d_n = R(-beta dt)^n d_0,
    and F stays the RK approximation of a rotation."""
    O = oracle_mod
    n = (8, 8)
    X = W.jittered_vertices(n, 43)
    P = W.q2_node_coords(n, X)
    A = np.array([[0.0, -1.0], [1.0, 0.0]])
    m = O.Mesh(n, X, A @ (P - 0.5))
    p0 = O.seed_particles(m, uniform_count=2, seed=9, n_props=5)
    p0.props[:, 0] = 1.0
    p0.props[:, 1:5] = np.eye(2).reshape(-1)
    dt, steps, beta = 0.05, 8, 0.9
    p = O.advect_properties(m, p0, dt, 4, steps, damage=0, alpha=3.0, beta=beta, defgrad=1)
    rd = _rk_poly(np.array([[-beta * dt]]), 4)[0, 0] ** steps
    np.testing.assert_allclose(p.props[:, 0], rd, rtol=0, atol=2e-14)
    Rn = np.linalg.matrix_power(_rk_poly(dt * A, 4), steps)
    np.testing.assert_allclose(p.props[:, 1:5], np.tile(Rn.reshape(-1), (p.n, 1)), rtol=0, atol=2e-14)


@pytest.mark.parametrize("integrator", [2, 4])
def test_defgrad_is_derivative_of_position_map(oracle_mod, integrator):
    O = oracle_mod
    n = (4, 4, 4)
    X = W.uniform_vertices(n)
    P = W.q2_node_coords(n, X)

    def f(p):
        x, y, z = p
        return 0.3 * np.stack([x * x - 2 * y * z + 0.5, y * y + x * z - z, 3 * x * y + z * z - x - 0.4])

    m = O.Mesh(n, X, f(P))
    g = np.random.default_rng(5)
    x0 = g.uniform(0.35, 0.65, (6, 3))
    cell, xh = m.locate(x0)
    N = len(x0)
    base = O.Particles(x0, xh, cell, np.arange(N, dtype=np.uint64), np.tile(np.eye(3).reshape(-1), (N, 1)))
    dt, steps, h = 0.02, 5, 1e-5
    p = O.advect_properties(m, base, dt, integrator, steps, defgrad=0)
    assert p.n == N
    F = {int(i): pr.reshape(3, 3) for i, pr in zip(p.id, p.props)}
    for k in range(N):
        fd = np.zeros((3, 3))
        for j in range(3):
            ends = []
            for sgn in (1.0, -1.0):
                xs = x0[k].copy()
                xs[j] += sgn * h
                c1, t1 = m.locate(xs[None])
                q = O.advect(m, O.Particles(xs[None], t1, c1, np.zeros(1, np.uint64), np.zeros((1, 0))), dt,
                             integrator, steps)
                assert q.n == 1
                ends.append(q.x[0])
            fd[:, j] = (ends[0] - ends[1]) / (2 * h)
        np.testing.assert_allclose(F[k], fd, rtol=0, atol=1e-8)
        # and F is not its transpose here (the check above can tell them apart)
        assert np.abs(F[k] - F[k].T).max() > 1e-4


def test_odes_off_is_plain_advection(oracle_mod):
    O = oracle_mod
    wl = W.curl_cube(4, 3, 3, seed=3)
    m = O.Mesh(wl.n, wl.X, wl.U)
    p0 = O.seed_particles(m, uniform_count=3, seed=4, n_props=2)
    p0.props[:] = np.random.default_rng(1).uniform(size=p0.props.shape)
    a = O.advect(m, p0, wl.dt, 4, 3)
    b = O.advect_properties(m, p0, wl.dt, 4, 3)
    np.testing.assert_array_equal(a.x, b.x)
    np.testing.assert_array_equal(a.xhat, b.xhat)
    np.testing.assert_array_equal(a.props, b.props)


def test_two_fields_refused(oracle_mod):
    O = oracle_mod
    n = (2, 2)
    X = W.uniform_vertices(n)
    U = np.zeros((2, 25))
    m = O.Mesh(n, X, U)
    m.set_velocity_next(U)
    p0 = O.seed_particles(m, uniform_count=1, seed=1, n_props=1)
    with pytest.raises(ValueError):
        O.advect_properties(m, p0, 0.1, 4, 1, damage=0)
