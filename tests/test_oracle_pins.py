"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here compares the oracle with itself: every expected value is a
closed form (exact transport, matrix powers of the RK stability function,
exact rotations), a brute-force search, a published generator output, or an
invariant of the method (Sec. 2.1 each particle in exactly one cell, unique
ids, sorted by cell; Sec. 2.4 only out-of-domain particles are dropped).
"""
import math
import os

import numpy as np
import pytest

from paper_1612_03369_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mesh(O, n, X, U=None):
    return O.Mesh(n, X, U)


def _const_U(n, c):
    nq = int(np.prod([2 * m + 1 for m in n]))
    return np.stack([np.full(nq, float(v)) for v in c])


# ------------------------------------------------------------ generator --


def test_splitmix64_published_vector(oracle_mod):
    want = [int(l) for l in open(os.path.join(GOLDEN, "splitmix64_seed1234567.txt")) if l.strip() and l[0] != "#"]
    got = [oracle_mod.splitmix64(1234567, i) for i in range(len(want))]
    assert got == want


def test_seed_local_coordinates(oracle_mod):
    n = (3, 2, 2)
    X = W.jittered_vertices(n, 7)
    m = _mesh(oracle_mod, n, X)
    per = np.array([0, 3, 1, 5, 2, 0, 4, 1, 1, 0, 7, 2], dtype=np.uint32)
    p = oracle_mod.seed_particles(m, per_cell=per, seed=99, first_id=1000, n_props=2)
    assert p.n == per.sum()
    np.testing.assert_array_equal(p.id, 1000 + np.arange(p.n, dtype=np.uint64))
    np.testing.assert_array_equal(p.cell, np.repeat(np.arange(12), per))
    assert (p.xhat >= 0).all() and (p.xhat < 1).all()
    # x-hat_j of particle g is the top 53 bits of output g*dim+j
    for g in (0, 5, p.n - 1):
        for j in range(3):
            r = oracle_mod.splitmix64(99, g * 3 + j)
            assert p.xhat[g, j] == (r >> 11) * 2.0**-53
    # each particle lies in its seeding cell
    for g in range(p.n):
        ok, t = m.inside(int(p.cell[g]), p.x[g])
        assert ok
        np.testing.assert_allclose(t, p.xhat[g], atol=1e-13)


# ---------------------------------------------------- map and inverse --


def test_affine_cell_inverse_closed_form(oracle_mod):
    # one cell, Phi(xh) = (2 xi, eta): the inverse is explicit and Newton
    # is exact after one step (second step observes a zero update)
    X = np.array([[0.0, 2.0, 0.0, 2.0], [0.0, 0.0, 1.0, 1.0]])
    m = _mesh(oracle_mod, (1, 1), X)
    conv, t, it = m.newton(0, [1.5, 0.25])
    assert conv and it <= 2
    np.testing.assert_array_equal(t, [0.75, 0.25])
    np.testing.assert_array_equal(m.phi(0, [0.75, 0.25]), [1.5, 0.25])


@pytest.mark.parametrize("n", [(4, 3), (3, 3, 3)])
def test_newton_round_trip(oracle_mod, n):
    X = W.jittered_vertices(n, 11)
    m = _mesh(oracle_mod, n, X)
    g = np.random.default_rng(3)
    h = 1.0 / max(n)
    C = int(np.prod(n))
    for K in range(C):
        for _ in range(5):
            xh = g.uniform(-0.2, 1.2, size=len(n))
            x = m.phi(K, xh)
            conv, t, it = m.newton(K, x)
            assert conv
            np.testing.assert_allclose(t, xh, atol=1e-13)
            np.testing.assert_allclose(m.phi(K, t), x, atol=1e-14 * h * 10)


def test_newton_affine_one_step(oracle_mod):
    # a sheared parallelogram mesh is affine per cell
    n = (3, 2)
    X = W.uniform_vertices(n)
    X[0] = X[0] + 0.3 * X[1]
    m = _mesh(oracle_mod, n, X)
    for K in range(6):
        conv, t, it = m.newton(K, m.phi(K, [0.3, 0.9]))
        assert conv and it <= 2
        np.testing.assert_allclose(t, [0.3, 0.9], atol=1e-15)


# --------------------------------------------------------------- owner --


def test_owner_hand_cases(oracle_mod):
    m = _mesh(oracle_mod, (2, 2), W.uniform_vertices((2, 2)))
    cases = {
        (0.25, 0.25): 0, (0.75, 0.25): 1, (0.25, 0.75): 2, (0.75, 0.75): 3,
        (0.5, 0.5): 0,    # vertex shared by all four: lowest index
        (0.5, 0.25): 0,   # face between 0 and 1
        (0.75, 0.5): 1,   # face between 1 and 3
        (0.5, 0.75): 2,   # face between 2 and 3
        (1.0, 1.0): 3, (0.0, 0.0): 0,
        (1.0 + 1e-12, 0.5): 1,   # inside the eps band of R3
        (1.0 + 1e-6, 0.5): -1,   # outside the domain: lost
        (-0.1, 0.2): -1,
    }
    for x, K in cases.items():
        assert m.owner(x)[0] == K, x
        assert m.owner(x, brute=True)[0] == K, x


@pytest.mark.parametrize("n", [(2, 2), (3, 3), (3, 3, 3)])
def test_owner_binned_equals_bruteforce(oracle_mod, n):
    X = W.jittered_vertices(n, 5)
    m = _mesh(oracle_mod, n, X)
    dim = len(n)
    g = np.random.default_rng(1)
    pts = [g.uniform(-0.05, 1.05, size=(400, dim))]
    # points on shared faces, edges and vertices: Phi_K at reference points
    # with coordinates in {0, 1/2, 1}
    C = int(np.prod(n))
    ref = np.array(list(np.ndindex(*(3,) * dim))) / 2.0
    on = [m.phi(K, r) for K in range(C) for r in ref]
    pts.append(np.array(on))
    P = np.concatenate(pts)
    cb, tb = m.locate(P, brute=True)
    cf, tf = m.locate(P, brute=False)
    np.testing.assert_array_equal(cf, cb)
    np.testing.assert_array_equal(tf, tb)
    # every located point is inside its owner and no lower-index cell holds it
    for x, K in zip(P, cb):
        if K < 0:
            continue  # brute force already tried every cell
        assert m.inside(int(K), x)[0]
        for Kp in range(int(K)):
            assert not m.inside(Kp, x)[0]


def test_vertices_owned_by_lowest_cell(oracle_mod):
    n = (3, 3, 3)
    m = _mesh(oracle_mod, n, W.jittered_vertices(n, 8))
    # interior vertex (1,1,1) is shared by cells (0..1)^3; the lowest is 0
    K, _ = m.owner(m.phi(0, [1.0, 1.0, 1.0]))
    assert K == 0
    # vertex (2,1,1) is shared by cells i in {1,2}, j,k in {0,1}: lowest = 1
    K, _ = m.owner(m.phi(1, [1.0, 1.0, 1.0]))
    assert K == 1


# ------------------------------------------------------------ Q2 field --


def test_q2_partition_of_unity_and_nodes(oracle_mod):
    n = (2, 2, 2)
    X = W.jittered_vertices(n, 2)
    nq = 125
    m = _mesh(oracle_mod, n, X)
    # Kronecker property: a field that is 1 at one node and 0 elsewhere
    for node in (0, 31, 62, 124):
        U = np.zeros((3, nq))
        U[:, node] = [1.0, 2.0, -3.0]
        m.set_velocity(U)
        I, J, Kk = node % 5, (node // 5) % 5, node // 25
        for K in range(8):
            i, j, k = K % 2, (K // 2) % 2, K // 4
            a, b, c = I - 2 * i, J - 2 * j, Kk - 2 * k
            for aa in range(3):
                for bb in range(3):
                    for cc in range(3):
                        u = m.q2(K, [aa / 2, bb / 2, cc / 2])
                        hit = (aa, bb, cc) == (a, b, c)
                        np.testing.assert_allclose(u, [1.0, 2.0, -3.0] if hit else [0, 0, 0], atol=1e-15)
    m.set_velocity(_const_U(n, (0.7, -0.2, 1.5)))
    g = np.random.default_rng(0)
    for K in range(8):
        for _ in range(20):
            np.testing.assert_allclose(m.q2(K, g.uniform(0, 1, 3)), [0.7, -0.2, 1.5], rtol=0, atol=4e-16 * 27)


def test_q2_reproduces_quadratics_on_affine_mesh(oracle_mod):
    n = (3, 2, 2)
    X = W.uniform_vertices(n)
    X[0] = X[0] * 1.3 + 0.2 * X[2]
    P = W.q2_node_coords(n, X)

    def f(p):
        x, y, z = p
        return np.stack([x * x - 2 * y * z + 0.5, y * y + x * z - z, 3 * x * y + z * z - x])

    m = _mesh(oracle_mod, n, X, f(P))
    g = np.random.default_rng(4)
    for K in range(12):
        for _ in range(10):
            t = g.uniform(0, 1, 3)
            np.testing.assert_allclose(m.q2(K, t), f(m.phi(K, t)), atol=2e-14)


# ---------------------------------------------------------- integrators --


def _seed(O, m, ppc, seed=3, n_props=0):
    return O.seed_particles(m, uniform_count=ppc, seed=seed, n_props=n_props)


@pytest.mark.parametrize("integrator", [1, 2, 4])
def test_constant_field_exact_transport(oracle_mod, integrator):
    n = (4, 3, 3)
    X = W.jittered_vertices(n, 21)
    c = np.array([0.31, -0.17, 0.23])
    m = _mesh(oracle_mod, n, X, _const_U(n, c))
    p0 = _seed(oracle_mod, m, 6)
    dt, steps = 0.01, 4
    p = oracle_mod.advect(m, p0, dt, integrator, steps)
    want = {int(i): x + steps * dt * c for i, x in zip(p0.id, p0.x)}
    for i, x in zip(p.id, p.x):
        np.testing.assert_allclose(x, want[int(i)], rtol=0, atol=4 * steps * 2.3e-16 * 4)
    # exactly the particles whose straight path leaves the unit cube are lost
    kept = set(int(i) for i in p.id)
    for i, x0 in zip(p0.id, p0.x):
        xe = x0 + steps * dt * c
        out = (xe < -1e-9).any() or (xe > 1 + 1e-9).any()
        inn = (xe > 1e-9).all() and (xe < 1 - 1e-9).all()
        if out:
            assert int(i) not in kept
        if inn:
            assert int(i) in kept
    assert p.n + p.n_lost == p0.n


def _rk_matrix(Z, integrator):
    I = np.eye(Z.shape[0])
    if integrator == 1:
        return I + Z
    if integrator == 2:
        return I + Z + Z @ Z / 2
    Z2 = Z @ Z
    return I + Z + Z2 / 2 + Z2 @ Z / 6 + Z2 @ Z2 / 24


@pytest.mark.parametrize("dim,integrator", [(2, 2), (2, 4), (3, 4), (3, 2)])
def test_linear_field_closed_form(oracle_mod, dim, integrator):
    """Rigid rotation is linear in x, so Q2 on (bi/tri)linear cells carries it
    exactly and n RK steps are x_n - c = R(dt A)^n (x_0 - c)."""
    n = (8, 8) if dim == 2 else (5, 5, 5)
    X = W.jittered_vertices(n, 31)
    P = W.q2_node_coords(n, X)
    A = np.zeros((dim, dim))
    A[0, 1], A[1, 0] = -1.0, 1.0
    c = np.full(dim, 0.5)
    U = A @ (P - c[:, None])
    m = _mesh(oracle_mod, n, X, U)
    p0 = _seed(oracle_mod, m, 4)
    dt, steps = 0.05, 6
    p = oracle_mod.advect(m, p0, dt, integrator, steps)
    Rn = np.linalg.matrix_power(_rk_matrix(dt * A, integrator), steps)
    want = {int(i): c + Rn @ (x - c) for i, x in zip(p0.id, p0.x)}
    assert p.n > 0.5 * p0.n
    for i, x in zip(p.id, p.x):
        np.testing.assert_allclose(x, want[int(i)], rtol=0, atol=1e-13)
    # lost == some stage or end point left the domain (closed form, margins)
    R1 = _rk_matrix(dt * A, integrator)
    kept = set(int(i) for i in p.id)
    for i, x0 in zip(p0.id, p0.x):
        pts, x = [], x0.copy()
        for _ in range(steps):
            y = x - c
            k1 = dt * (A @ y)
            if integrator == 2:
                pts.append(x + k1 / 2)
            if integrator == 4:
                k2 = dt * (A @ (y + k1 / 2))
                k3 = dt * (A @ (y + k2 / 2))
                pts += [x + k1 / 2, x + k2 / 2, x + k3]
            x = c + R1 @ y
            pts.append(x)
        pts = np.array(pts)
        if (pts < -1e-9).any() or (pts > 1 + 1e-9).any():
            assert int(i) not in kept
        elif (pts > 1e-9).all() and (pts < 1 - 1e-9).all():
            assert int(i) in kept


def test_rk_reading_discriminates():
    """RK4 as printed (k2, k3 carrying dt/2, weights 1/6, 1/3, 1/3, 1/6) moves
    a particle by 2/3 of dt*u in a constant field; the classical reading
    moves it by dt*u.  The exact-transport pin above therefore rejects the
    printed form.  This checks that arithmetic."""
    u, dt = 1.0, 1.0
    k1 = dt * u
    k2 = dt / 2 * u
    k3 = dt / 2 * u
    k4 = dt * u
    assert k1 / 6 + k2 / 3 + k3 / 3 + k4 / 6 == pytest.approx(2.0 / 3.0)


@pytest.mark.parametrize("integrator,order", [(2, 2), (4, 4)])
def test_convergence_order_rotation(oracle_mod, integrator, order):
    """Remark on convergence: against the exact trajectory of a field that Q2
    represents exactly, the error falls like dt^q."""
    n = (8, 8)
    X = W.jittered_vertices(n, 13)
    P = W.q2_node_coords(n, X)
    U = W.rotation_field(P)
    m = _mesh(oracle_mod, n, X, U)
    x0 = np.array([[0.6, 0.55], [0.45, 0.3], [0.52, 0.71]])
    cell, xh = m.locate(x0)
    p0 = oracle_mod.Particles(x0, xh, cell, np.arange(3, dtype=np.uint64), np.zeros((3, 0)))
    T = 1.0
    errs = []
    for steps in (10, 20, 40):
        p = oracle_mod.advect(m, p0, T / steps, integrator, steps)
        order_idx = np.argsort(p.id)
        xs = p.x[order_idx]
        th = T
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        exact = 0.5 + (x0 - 0.5) @ R.T
        errs.append(np.abs(xs - exact).max())
    for a, b in zip(errs, errs[1:]):
        assert a / b == pytest.approx(2**order, rel=0.1)


@pytest.mark.parametrize("integrator", [2, 4])
def test_convergence_on_piecewise_q2_field(oracle_mod, integrator):
    """Against a 256-step solution of the same u_h (a curl field on jittered
    hexes), the error at fixed T falls by about 4 per halving of dt for both
    RK2 and RK4: u_h is only continuous across faces, its gradient jumps, and
    a step whose stages straddle a face loses the higher orders.  A stage
    located in the wrong cell, or a stage point formed from the wrong k,
    breaks the convergence altogether."""
    wl = W.curl_cube(4, 2, 1, 5, n_props=0)
    m = _mesh(oracle_mod, wl.n, wl.X, wl.U)
    p0 = oracle_mod.seed_particles(m, uniform_count=2, seed=3)
    T = 8 * wl.dt

    def final(steps):
        p = oracle_mod.advect(m, p0.copy(), T / steps, integrator, steps)
        return {int(i): x for i, x in zip(p.id, p.x)}

    ref = final(256)
    errs = []
    for steps in (8, 16, 32):
        r = final(steps)
        common = [i for i in r if i in ref]
        assert len(common) >= 0.9 * p0.n
        errs.append(max(np.abs(r[i] - ref[i]).max() for i in common))
    for a, b in zip(errs, errs[1:]):
        assert 3.0 < a / b < 6.0, errs


# ------------------------------------------------ rebin and conservation --


def test_conservation_and_sorted(oracle_mod):
    wl = W.c1(n=16, ppc=8, n_steps=8)
    m = _mesh(oracle_mod, wl.n, wl.X, wl.U)
    p0 = oracle_mod.seed_particles(m, uniform_count=wl.ppc, seed=wl.pseed, n_props=1)
    p = oracle_mod.advect(m, p0, 4 * wl.dt, wl.integrator, wl.n_steps)
    assert p.n_lost > 0
    assert p.n + p.n_lost == p0.n
    assert len(set(p.id.tolist())) == p.n
    assert set(p.id.tolist()) <= set(p0.id.tolist())
    key = p.cell.astype(np.int64) * (2**40) + p.id.astype(np.int64)
    assert (np.diff(key) > 0).all()
    # stored x-hat is the inverse map of x in the stored cell
    for K, x, t in zip(p.cell[:200], p.x[:200], p.xhat[:200]):
        np.testing.assert_allclose(m.phi(int(K), t), x, atol=1e-15)
        assert m.owner(x)[0] == K


# ------------------------------------------------------------- averages --


def test_cell_average_pins(oracle_mod):
    C = 7
    cell = np.array([0, 0, 0, 2, 2, 3, 5, 5, 5, 5, 6], dtype=np.int64)
    for v in (0.5, 3.0, -2.25):
        avg, cnt = oracle_mod.cell_average(C, cell, np.full(cell.shape, v), empty_fill=-7.0)
        np.testing.assert_array_equal(cnt, [3, 0, 2, 1, 0, 4, 1])
        np.testing.assert_array_equal(avg, [v, -7.0, v, v, -7.0, v, v])
    g = np.random.default_rng(9)
    vals = g.uniform(-1, 1, cell.shape)
    avg, cnt = oracle_mod.cell_average(C, cell, vals)
    for K in range(C):
        sel = vals[cell == K]
        if len(sel):
            exact = math.fsum(sel) / len(sel)
            assert abs(avg[K] - exact) <= len(sel) * 2.0**-53 * np.abs(sel).max()
        else:
            assert avg[K] == 0.0 and cnt[K] == 0


def test_geometric_and_harmonic_average_pins(oracle_mod):
    """Sec. 2.7 (ii): geometric exp(mean log v) and harmonic n / sum(1/v)."""
    cell = np.array([0, 0, 1, 1, 1, 3, 3], dtype=np.int64)
    v = np.array([2.0, 8.0, 1.0, 3.0, 9.0, 0.5, 4.0])
    g, cnt = oracle_mod.cell_average(4, cell, v, empty_fill=-1.0, kind=1)
    h, _ = oracle_mod.cell_average(4, cell, v, empty_fill=-1.0, kind=2)
    a, _ = oracle_mod.cell_average(4, cell, v, empty_fill=-1.0, kind=0)
    np.testing.assert_allclose(g, [4.0, 3.0, -1.0, math.sqrt(2.0)], rtol=4e-16)     # sqrt(16), cbrt(27), sqrt(2)
    np.testing.assert_allclose(h, [3.2, 27.0 / 13.0, -1.0, 8.0 / 9.0], rtol=4e-16)  # 2ab/(a+b), 3/(1+1/3+1/9)
    assert (a[[0, 1, 3]] >= g[[0, 1, 3]]).all() and (g[[0, 1, 3]] >= h[[0, 1, 3]]).all()  # AM >= GM >= HM
    # a constant cell averages to the constant; a non-positive value gives NaN
    g2, _ = oracle_mod.cell_average(2, np.array([0, 0, 0, 1, 1]), np.array([7.5, 7.5, 7.5, 2.0, -1.0]), kind=1)
    assert abs(g2[0] - 7.5) <= 2 * np.spacing(7.5) and math.isnan(g2[1])
    h2, _ = oracle_mod.cell_average(1, np.array([0, 0]), np.array([0.0, 2.0]), kind=2)
    assert math.isnan(h2[0])


@pytest.mark.parametrize("integrator", [1, 2, 4])
def test_time_interpolated_field(oracle_mod, integrator):
    """Sec. 2.3: u-tilde_h interpolates u_h^n and u_h^{n+1} linearly in time
    (reading R6).  (a) U^{n+1} = U^n gives the steady result bit for bit;
    (b) spatially uniform fields c0 -> c1 move every particle by exactly
    dt (c0 + c1) / 2 per step (RK2 and RK4 integrate a linear-in-time
    velocity exactly), forward Euler by dt c0."""
    n = (3, 3, 3)
    X = W.jittered_vertices(n, 17)
    U = W.curl_potential_field(W.q2_node_coords(n, X), 5)[0]
    m = oracle_mod.Mesh(n, X, U)
    p0 = oracle_mod.seed_particles(m, uniform_count=4, seed=2)
    steady = oracle_mod.advect(m, p0, 0.02, integrator, 3)
    m.set_velocity_next(U)
    same = oracle_mod.advect(m, p0, 0.02, integrator, 3)
    np.testing.assert_array_equal(same.x, steady.x)
    np.testing.assert_array_equal(same.id, steady.id)
    c0, c1 = np.array([0.2, -0.1, 0.3]), np.array([-0.3, 0.25, 0.1])
    m.set_velocity(_const_U(n, c0))
    m.set_velocity_next(_const_U(n, c1))
    dt, steps = 0.01, 3
    p = oracle_mod.advect(m, p0, dt, integrator, steps)
    per = dt * c0 if integrator == 1 else dt * 0.5 * (c0 + c1)
    want = {int(i): x + steps * per for i, x in zip(p0.id, p0.x)}
    assert p.n > p0.n // 2
    for i, x in zip(p.id, p.x):
        np.testing.assert_allclose(x, want[int(i)], rtol=0, atol=1e-15)
